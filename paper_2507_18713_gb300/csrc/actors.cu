// actors.cu -- ray casting with dynamic actors (Sec. IV-A).
//
// Every actor is a scene of its own, built in the actor's canonical frame,
// and placed in the world by a pose that moves over the sensor's exposure
// (linear translation, geodesic rotation: the same interpolation as the
// sensor's).  Per ray:
//  1. the actor boxes the ray meets, as entry-sorted [t_in, t_out] intervals
//     (a bounding-sphere test, then a slab test against the actor's tight box
//     in its frame);
//  2. the static walk and one actor walk at a time (actor boxes are disjoint,
//     so their intervals are too) advance together, one structure step per
//     lane per warp-wide round; the hit with the smaller entry is composited
//     first (the static one on ties), by Eq. 3-4 with early termination;
//  3. an actor hit's field uses the ray moved into the actor's frame: local
//     coordinates and the SH view direction of the canonical frame.
// A rigid map keeps distances along the ray, so both walks' t are metres
// from the same origin.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "traverse.cuh"

using namespace salf;

namespace {

#ifndef SALF_ACTOR_MIN_BLOCKS
#define SALF_ACTOR_MIN_BLOCKS 1  // resident merge blocks per SM the register budget must allow
#endif
// The same for the lean merge variant (static pinhole cameras without
// intensity).  Without the other sensors' ray generation and the intensity
// field it fits 128 registers: 4 resident blocks per SM measured faster (1080p
// camera with 24 actors 0.834 -> 0.754 ms).  5 blocks (96 registers, 64 bytes
// of spills) were faster again (0.717 -> 0.689 ms), and 6 no better.  Merge
// blocks hold most of an SM's registers while they run, so the ray kernel
// beside them gets few slots; the merge kernel's total warp time sets the frame.
#ifndef SALF_ACTOR_MIN_BLOCKS_LEAN
#define SALF_ACTOR_MIN_BLOCKS_LEAN 5
#endif

constexpr int kActorWarps = 4;  // warps per block
constexpr int kMaxIntervals = 8;
constexpr int kMaskWords = SALF_MAX_ACTORS / 32;  // per-tile candidate actors (bits)

__device__ __forceinline__ void rotate_about(const float k[3], float sa, float omc, float v[3]) {
  // Rodrigues: v + sin(a) (k x v) + (1 - cos(a)) k x (k x v)
  const float cx = k[1] * v[2] - k[2] * v[1], cy = k[2] * v[0] - k[0] * v[2],
              cz = k[0] * v[1] - k[1] * v[0];
  const float ccx = k[1] * cz - k[2] * cy, ccy = k[2] * cx - k[0] * cz, ccz = k[0] * cy - k[1] * cx;
  v[0] = fmaf(omc, ccx, fmaf(sa, cx, v[0]));
  v[1] = fmaf(omc, ccy, fmaf(sa, cy, v[1]));
  v[2] = fmaf(omc, ccz, fmaf(sa, cz, v[2]));
}

// The ray (sensor origin, world direction d, time fraction s) in actor A's
// canonical frame: origin relative to the actor's pose translation, rotated
// back by R(s)^T = R0^T rot(axis, -s angle).
__device__ __forceinline__ void actor_frame(const ActorDev& A, float s, const float d[3],
                                            float oc[3], float dc[3]) {
  float rel[3], dw[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    rel[a] = fmaf(s, A.orel1[a] - A.orel0[a], A.orel0[a]);
    dw[a] = d[a];
  }
  if (s > 0.f && A.angle != 0.f) {
    float sh, ch;
    sincosf(-0.5f * s * A.angle, &sh, &ch);
    const float sa = 2.f * sh * ch, omc = 2.f * sh * sh;
    rotate_about(A.axis, sa, omc, rel);
    rotate_about(A.axis, sa, omc, dw);
  }
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    oc[c] = A.R0[c] * rel[0] + A.R0[3 + c] * rel[1] + A.R0[6 + c] * rel[2];
    dc[c] = A.R0[c] * dw[0] + A.R0[3 + c] * dw[1] + A.R0[6 + c] * dw[2];
  }
}

// Conservative test: may the ray (direction d from the sensor origin at time
// fraction s, over [tn, tf]) meet actor A's box?  Its bounding sphere.
__device__ __forceinline__ bool may_meet(const ActorDev& A, const Ray& r) {
  float c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) c[a] = fmaf(r.s, A.cc1[a] - A.cc0[a], A.cc0[a]);
  const float tca = c[0] * r.d[0] + c[1] * r.d[1] + c[2] * r.d[2];
  const float d2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2] - tca * tca;
  return !(d2 > A.radius * A.radius || tca + A.radius < r.tn || tca - A.radius > r.tf);
}

// Exact test: the ray's [t_in, t_out] with actor A's tight box (in its frame),
// clipped to the ray's [tn, tf]; false if empty.
__device__ __forceinline__ bool box_interval(const ActorDev& A, const Ray& r, float* t_in) {
  float oc[3], dc[3];
  actor_frame(A, r.s, r.d, oc, dc);
  float a0 = r.tn, a1 = r.tf;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float inv = 1.f / (fabsf(dc[a]) < 1e-20f ? 1e-20f : dc[a]);
    const float p = (A.box_lo[a] - oc[a]) * inv, q = (A.box_hi[a] - oc[a]) * inv;
    a0 = fmaxf(a0, fminf(p, q));
    a1 = fminf(a1, fmaxf(p, q));
  }
  *t_in = a0;
  return a1 > a0;
}

// Split the request's tiles into those whose rays may meet an actor (list 1,
// rendered by the merge kernel) and the rest (list 0, rendered by the plain
// ray kernel).  One warp per tile, tiles taken in launch order.
__global__ void __launch_bounds__(128) k_classify_tiles(const __grid_constant__ LaunchParams P,
                                                        const ActorDev* __restrict__ actors,
                                                        int n_actors, int* __restrict__ lists,
                                                        int* __restrict__ counts,
                                                        unsigned* __restrict__ masks) {
  const int tile = blockIdx.x * 4 + (threadIdx.x >> 5);
  if (tile >= P.req[0].n_tiles) return;
  const int lane = threadIdx.x & 31;
  const ReqDev& Q = P.req[0];
  int u0, v0;
  tile_origin(Q, tile, &u0, &v0);
  const int u = u0 + lane % Q.tile_w, v = v0 + lane / Q.tile_w;
  // the warp's rays as a cone: mean direction, cosine of the widest ray, the
  // range of time fractions and of t_near / t_far
  Ray r;
  r.s = 0.f;
  r.valid = false;
  r.d[0] = r.d[1] = r.d[2] = 0.f;
  r.tn = 0.f;
  r.tf = 0.f;
  const bool in_img = u < Q.W && v < Q.H;
  if (in_img) gen_ray(Q, P.S, u, v, v * Q.W + u, r);
  const bool ok = in_img && r.valid;
  float m[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float x = ok ? r.d[a] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    m[a] = x;
  }
  const float mn = sqrtf(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
  bool any = false;
  if (__any_sync(0xffffffffu, ok) && mn > 0.f) {
    const float inv = 1.f / mn;
#pragma unroll
    for (int a = 0; a < 3; ++a) m[a] *= inv;
    float cmin = ok ? m[0] * r.d[0] + m[1] * r.d[1] + m[2] * r.d[2] : 1.f;
    float smin = ok ? r.s : 1.f, smax = ok ? r.s : 0.f, tn = ok ? r.tn : 3.4e38f, tf = ok ? r.tf : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      cmin = fminf(cmin, __shfl_xor_sync(0xffffffffu, cmin, o));
      smin = fminf(smin, __shfl_xor_sync(0xffffffffu, smin, o));
      smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, o));
      tn = fminf(tn, __shfl_xor_sync(0xffffffffu, tn, o));
      tf = fmaxf(tf, __shfl_xor_sync(0xffffffffu, tf, o));
    }
    // widen by FP32 slack; a cone wider than 90 degrees accepts everything
    const float half = acosf(fminf(fmaxf(cmin, -1.f), 1.f)) + 1e-4f;
    // each lane tests actors lane, lane + 32, ...: the sphere (centre moving
    // linearly over [smin, smax]: its segment's bounding sphere) against the cone
    for (int k0 = 0; k0 < n_actors; k0 += 32) {
      const int k = k0 + lane;
      bool meet = false;
      if (k < n_actors) {
      const ActorDev& A = actors[k];
      float c0[3], c1[3], c[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        c0[a] = fmaf(smin, A.cc1[a] - A.cc0[a], A.cc0[a]);
        c1[a] = fmaf(smax, A.cc1[a] - A.cc0[a], A.cc0[a]);
        c[a] = 0.5f * (c0[a] + c1[a]);
      }
      const float dx = c1[0] - c0[0], dy = c1[1] - c0[1], dz = c1[2] - c0[2];
      const float rad = A.radius + 0.5f * sqrtf(dx * dx + dy * dy + dz * dz);
      const float dist = sqrtf(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
      if (dist <= rad) {
        meet = true;  // the sensor is inside the sphere
      } else if (half >= 1.5707963f) {
        meet = true;
      } else {
        // angle between the cone axis and the centre, less the sphere's angular radius
        const float ca = fminf(fmaxf((m[0] * c[0] + m[1] * c[1] + m[2] * c[2]) / dist, -1.f), 1.f);
        const float ang = acosf(ca) - asinf(fminf(rad / dist, 1.f));
        meet = ang <= half && dist - rad <= tf && dist + rad >= tn;
      }
      }
      // the cone's candidates, then each lane's own ray against each candidate box
      unsigned cand = __ballot_sync(0xffffffffu, meet), hit = 0u;
      while (cand) {
        const int j = __ffs(cand) - 1;
        cand &= cand - 1u;
        float tin;
        const bool mine = ok && may_meet(actors[k0 + j], r) && box_interval(actors[k0 + j], r, &tin);
        if (__any_sync(0xffffffffu, mine)) hit |= 1u << j;
      }
      if (lane == 0) masks[(size_t)tile * kMaskWords + (k0 >> 5)] = hit;
      any = any || hit != 0u;
    }
  }
  if (lane == 0) {
    const int which = any ? 1 : 0;
    const int slot = atomicAdd(&counts[which], 1);
    lists[which * Q.n_tiles + slot] = tile;
  }
}

// Start actor A's walk for the ray (frame conversion to its grid cells).
__device__ __forceinline__ void actor_walk(const ActorDev& A, const Ray& r, Walk& w,
                                           float gam[4]) {
  float oc[3], dc[3];
  actor_frame(A, r.s, r.d, oc, dc);
  Ray ra;
  ra.valid = true;
  ra.tn = r.tn;
  ra.tf = r.tf;
  ra.s = r.s;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float g = (oc[a] - A.origin[a]) * A.inv_sfin;
    const float f = floorf(g);
    ra.Oi[a] = (int)f;
    ra.Of[a] = g - f;
    ra.d[a] = dc[a];
  }
  walk_init(A.S, ra, w);
  sh_basis(dc, gam);
}

// LEAN: every ray comes from a pinhole camera with one pose for the frame and
// no intensity is asked for (that ray generation only, no intensity field).
template <int DT, int MODE, bool DUMP, bool LEAN>
__global__ void __launch_bounds__(32 * kActorWarps,
                                  LEAN ? SALF_ACTOR_MIN_BLOCKS_LEAN : SALF_ACTOR_MIN_BLOCKS)
    k_forward_actors(
    const __grid_constant__ LaunchParams P, const ActorDev* __restrict__ actors, int n_actors,
    const unsigned* __restrict__ masks) {
  const int warp = blockIdx.x * kActorWarps + (threadIdx.x >> 5);
  if (warp >= P.total_tiles) return;
  const int lane = threadIdx.x & 31;
  const ReqDev& Q = P.req[0];
  const DevScene& S = P.S;
  int tile = warp - Q.tile_begin;
  if (Q.tile_list) {
    if (tile >= __ldg(Q.tile_count)) return;
    tile = __ldg(&Q.tile_list[tile]);
  }
  int u0, v0;
  tile_origin(Q, tile, &u0, &v0);
  const int u = u0 + lane % Q.tile_w;
  const int v = v0 + lane / Q.tile_w;
  const bool in_img = (u < Q.W) && (v < Q.H);
  const int ray = v * Q.W + u;

  Ray r;
  Walk ws;
  ws.alive = false;
  r.valid = false;
  r.s = 0.f;
  r.d[0] = r.d[1] = r.d[2] = 0.f;
  if (in_img) {
    if (LEAN)
      gen_ray_pinhole(Q, u, v, r);
    else
      gen_ray(Q, S, u, v, ray, r);
    walk_init(S, r, ws);
  }
  float gam_s[4];
  sh_basis(r.d, gam_s);

  // 1. entry-sorted actor intervals along the ray
  float iv_in[kMaxIntervals];
  int iv_k[kMaxIntervals];
  int ni = 0;
  if (in_img && r.valid) {
    // candidates: the actors the tile's cone may meet
    for (int wd = 0; wd * 32 < n_actors; ++wd) {
      unsigned bits = __ldg(&masks[(size_t)tile * kMaskWords + wd]);
      while (bits) {
        const int k = wd * 32 + __ffs(bits) - 1;
        bits &= bits - 1u;
        const ActorDev& A = actors[k];
        float a0;
        if (!may_meet(A, r) || !box_interval(A, r, &a0)) continue;
        // insertion into the sorted list (the farthest is dropped when full)
        int pos = ni < kMaxIntervals ? ni : kMaxIntervals - 1;
        if (ni == kMaxIntervals) {
          atomicOr(S.status, SALF_DEVERR_ACTOR_CAP);
          if (a0 >= iv_in[pos]) continue;
        } else {
          ++ni;
        }
        while (pos > 0 && iv_in[pos - 1] > a0) {
          iv_in[pos] = iv_in[pos - 1];
          iv_k[pos] = iv_k[pos - 1];
          --pos;
        }
        iv_in[pos] = a0;
        iv_k[pos] = k;
      }
    }
  }

  // 2. merge the static walk with one actor walk at a time, in warp-wide
  // rounds: per round a lane takes at most one structure step (of the static
  // or the actor walk), then composites the next hit once both walks have
  // resolved theirs
  const bool want_int = !LEAN && Q.want_int != 0;
  const float tmin = Q.t_min;
  Accum acc{1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0};
  Hit hs, ha;
  bool hs_ok = false, ha_ok = false;
  Walk wa;
  wa.alive = false;
  float gam_a[4] = {0.f, 0.f, 0.f, 0.f};
  int cur = -1, nxt = 0;
  float nxt_in = ni > 0 ? iv_in[0] : 0.f;  // entry of interval nxt (the list is in local memory)
  bool live = in_img && r.valid;
  for (;;) {
    if (!__any_sync(0xffffffffu, live)) break;
    if (!live) continue;
    if (cur >= 0 && !ha_ok && !wa.alive) cur = -1;  // the open actor is exhausted
    // the next actor box starts before the pending static hit (a little early
    // is harmless: hits are composited by entry)
    const bool start_next =
        cur < 0 && nxt < ni && (!hs_ok || nxt_in <= hs.tin + 1e-5f * fmaxf(1.f, fabsf(hs.tin)));
    if (!hs_ok && ws.alive) {
      hs_ok = next_hit(S, ws, hs);
    } else if (start_next) {
      cur = iv_k[nxt++];
      nxt_in = nxt < ni ? iv_in[nxt] : 0.f;
      actor_walk(actors[cur], r, wa, gam_a);
      ha_ok = false;
    } else if (cur >= 0 && !ha_ok && wa.alive) {
      ha_ok = next_hit(actors[cur].S, wa, ha);
    }
    // an actor walk that ended this round (or opened empty) leaves the next
    // interval to be weighed against the pending static hit
    if (cur >= 0 && !ha_ok && !wa.alive) cur = -1;
    const bool s_res = hs_ok || !ws.alive;
    const bool a_res = cur < 0 ? !(nxt < ni && (!hs_ok || nxt_in <= hs.tin + 1e-5f * fmaxf(1.f, fabsf(hs.tin))))
                               : (ha_ok || !wa.alive);
    if (!(s_res && a_res)) continue;
    if (ha_ok && (!hs_ok || ha.tin < hs.tin)) {
      const ActorDev& A = actors[cur];
      const GlobalRec src{reinterpret_cast<const float4*>(A.S.params) +
                          (size_t)ha.vox * RecordLayout<DT>::kChunks};
      composite_hit<DT, MODE>(wa, ha, src, want_int, gam_a, acc);
      if (DUMP && acc.nvis < Q.vcap)
        Q.visits[(size_t)ray * Q.vcap + acc.nvis] = A.id_base + __ldg(&A.S.order[ha.vox]);
      ha_ok = false;
    } else if (hs_ok) {
      const GlobalRec src{reinterpret_cast<const float4*>(S.params) +
                          (size_t)hs.vox * RecordLayout<DT>::kChunks};
      composite_hit<DT, MODE>(ws, hs, src, want_int, gam_s, acc);
      if (DUMP && acc.nvis < Q.vcap)
        Q.visits[(size_t)ray * Q.vcap + acc.nvis] = __ldg(&S.order[hs.vox]);
      hs_ok = false;
    } else {
      // both walks exhausted and no actor left to open
      if (cur < 0 && nxt >= ni) live = false;
      continue;
    }
    ++acc.nvis;
    if (acc.T < tmin) live = false;
  }
  if (!in_img) return;
  write_outputs(Q, ray, r.valid, acc);
  if (DUMP && Q.vcap > 0) {
    Q.vcount[ray] = acc.nvis;
    for (int k = acc.nvis; k < Q.vcap; ++k) Q.visits[(size_t)ray * Q.vcap + k] = -1;
  }
}

// Adjoint of one hit, composited in the merge order: with the ray's saved
// totals (gQ = g . Q), the prefix sum Pk of w g.q and T in front of the hit,
//   dL/dtau = T_next (g . q) - (gQ - Pk) - T_end (g_rgb . background),
// chained through the hit's field in its own frame (Eq. 1-2, 5-6), then
// added to the record's gradient row (16-byte atomics).  Returns T_next.
template <int DT, int MODE>
__device__ __forceinline__ float adjoint_hit(const Walk& w, const Hit& h, const float4* rec,
                                             const int* order, int n, float* dparams,
                                             int* status, bool want_int, const float gam[4],
                                             const float g[6], float gQ, float Tend, float gbg,
                                             float T, float* Pk) {
  if (h.vox < 0 || h.vox >= n) {  // never expected: record it and skip the hit
    atomicOr(status, SALF_DEVERR_BOUNDS);
    return T;
  }
  const float tm = 0.5f * (h.tin + h.tout);
  const float dl = h.tout - h.tin;
  float x[3];
  local_coords(w, h, tm, x);
  Field f;
  const GlobalRec src{rec + (size_t)h.vox * RecordLayout<DT>::kChunks};
  field_eval_src<DT, MODE>(src, want_int, x, gam, f);
  const float e = __expf(-f.sig * dl);
  const float wgt = T * (1.f - e);
  const float gq = g[0] * f.c[0] + g[1] * f.c[1] + g[2] * f.c[2] + g[3] * tm + g[4] + g[5] * f.io;
  *Pk = fmaf(wgt, gq, *Pk);
  const float Tn = T * e;
  if (!dparams) return Tn;
  const float dtau = Tn * gq - (gQ - *Pk) - Tend * gbg;
  const float dsig = dtau * dl;
  float gr[32];
  const float xh[4] = {x[0], x[1], x[2], 1.f};
  float gs;  // dL/d(geometry value W . [x, 1])
  gr[25] = gr[26] = 0.f;
  if (MODE == SALF_FIELD_EXP) {
    gs = dsig * f.sig;
  } else {
    const float ex = __expf(-fabsf(f.lin) / f.b);
    gs = dsig * (f.a / (2.f * f.b)) * ex;
    gr[25] = dsig * f.sig / f.a;
    gr[26] = -dsig * f.a * f.lin * ex / (2.f * f.b * f.b);
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) gr[q] = gs * xh[q];
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    const float dz = wgt * g[ch] * f.c[ch] * (1.f - f.c[ch]);
#pragma unroll
    for (int a = 0; a < 3; ++a) gr[4 + 3 * ch + a] = dz * xh[a];
#pragma unroll
    for (int b = 0; b < 4; ++b) gr[13 + 4 * ch + b] = dz * gam[b];
  }
  const float di = want_int ? wgt * g[5] * f.io * (1.f - f.io) : 0.f;
#pragma unroll
  for (int q = 0; q < 4; ++q) gr[27 + q] = di * xh[q];
  gr[31] = 0.f;
  const int key = __ldg(&order[h.vox]);
  if (key < 0 || key >= n) {
    atomicOr(status, SALF_DEVERR_BOUNDS);
    return Tn;
  }
  float4* dst = reinterpret_cast<float4*>(dparams) + (size_t)key * 8;
#pragma unroll
  for (int q = 0; q < 8; ++q)
    if (q < 7 || want_int)
      atomicAdd(dst + q, make_float4(gr[4 * q], gr[4 * q + 1], gr[4 * q + 2], gr[4 * q + 3]));
  return Tn;
}

// Adjoint of k_forward_actors on the tiles whose rays may meet an actor: the
// same merge walk (the same hits in the same order, the first n_visits of
// them, n_visits from the saved totals), each hit's gradient row going to the
// static scene's buffer or its actor's.
template <int DT, int MODE>
__global__ void __launch_bounds__(32 * kActorWarps, SALF_ACTOR_MIN_BLOCKS) k_backward_actors(
    const __grid_constant__ LaunchParams P, const ActorDev* __restrict__ actors, int n_actors,
    const unsigned* __restrict__ masks) {
  const int warp = blockIdx.x * kActorWarps + (threadIdx.x >> 5);
  if (warp >= P.total_tiles) return;
  const int lane = threadIdx.x & 31;
  const ReqDev& Q = P.req[0];
  const DevScene& S = P.S;
  int tile = warp - Q.tile_begin;
  if (Q.tile_list) {
    if (tile >= __ldg(Q.tile_count)) return;
    tile = __ldg(&Q.tile_list[tile]);
  }
  if (tile < 0 || tile >= Q.n_tiles) {  // never expected: record it and skip the tile
    if (lane == 0) atomicOr(S.status, SALF_DEVERR_BOUNDS);
    return;
  }
  int u0, v0;
  tile_origin(Q, tile, &u0, &v0);
  const int u = u0 + lane % Q.tile_w;
  const int v = v0 + lane / Q.tile_w;
  const bool in_img = (u >= 0) && (v >= 0) && (u < Q.W) && (v < Q.H);
  const int ray = v * Q.W + u;

  Ray r;
  Walk ws;
  ws.alive = false;
  r.valid = false;
  r.s = 0.f;
  r.d[0] = r.d[1] = r.d[2] = 0.f;
  float g[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float gQ = 0.f, Tend = 1.f;
  int nv = 0;
  if (in_img) {
    gen_ray(Q, S, u, v, ray, r);
    walk_init(S, r, ws);
    const float4* sp = reinterpret_cast<const float4*>(Q.bsaved) + 2 * (size_t)ray;
    const float4 s0 = __ldg(sp), s1 = __ldg(sp + 1);
    if (Q.g_rgb) {
      g[0] = __ldg(Q.g_rgb + 3 * (size_t)ray);
      g[1] = __ldg(Q.g_rgb + 3 * (size_t)ray + 1);
      g[2] = __ldg(Q.g_rgb + 3 * (size_t)ray + 2);
    }
    if (Q.g_depth) g[3] = __ldg(Q.g_depth + ray);
    if (Q.g_opacity) g[4] = __ldg(Q.g_opacity + ray);
    if (Q.g_int && Q.want_int) g[5] = __ldg(Q.g_int + ray);
    gQ = g[0] * s0.x + g[1] * s0.y + g[2] * s0.z + g[3] * s0.w + g[4] * s1.x + g[5] * s1.y;
    Tend = s1.z;
    nv = r.valid ? (int)s1.w : 0;
  }
  float gam_s[4];
  sh_basis(r.d, gam_s);
  const float gbg = g[0] * Q.bg[0] + g[1] * Q.bg[1] + g[2] * Q.bg[2];

  // 1. entry-sorted actor intervals along the ray (as in the forward)
  float iv_in[kMaxIntervals];
  int iv_k[kMaxIntervals];
  int ni = 0;
  if (in_img && r.valid) {
    for (int wd = 0; wd * 32 < n_actors; ++wd) {
      unsigned bits = __ldg(&masks[(size_t)tile * kMaskWords + wd]);
      while (bits) {
        const int k = wd * 32 + __ffs(bits) - 1;
        bits &= bits - 1u;
        const ActorDev& A = actors[k];
        float a0;
        if (!may_meet(A, r) || !box_interval(A, r, &a0)) continue;
        int pos = ni < kMaxIntervals ? ni : kMaxIntervals - 1;
        if (ni == kMaxIntervals) {
          atomicOr(S.status, SALF_DEVERR_ACTOR_CAP);
          if (a0 >= iv_in[pos]) continue;
        } else {
          ++ni;
        }
        while (pos > 0 && iv_in[pos - 1] > a0) {
          iv_in[pos] = iv_in[pos - 1];
          iv_k[pos] = iv_k[pos - 1];
          --pos;
        }
        iv_in[pos] = a0;
        iv_k[pos] = k;
      }
    }
  }

  // 2. the forward's merge walk, with the adjoint of each composited hit
  const bool want_int = Q.want_int != 0;
  float T = 1.f, Pk = 0.f;
  int done = 0;
  Hit hs, ha;
  bool hs_ok = false, ha_ok = false;
  Walk wa;
  wa.alive = false;
  float gam_a[4] = {0.f, 0.f, 0.f, 0.f};
  int cur = -1, nxt = 0;
  float nxt_in = ni > 0 ? iv_in[0] : 0.f;  // entry of interval nxt (the list is in local memory)
  bool live = in_img && r.valid && nv > 0;
  for (;;) {
    if (!__any_sync(0xffffffffu, live)) break;
    if (!live) continue;
    if (cur >= 0 && !ha_ok && !wa.alive) cur = -1;
    const bool start_next =
        cur < 0 && nxt < ni && (!hs_ok || nxt_in <= hs.tin + 1e-5f * fmaxf(1.f, fabsf(hs.tin)));
    if (!hs_ok && ws.alive) {
      hs_ok = next_hit(S, ws, hs);
    } else if (start_next) {
      cur = iv_k[nxt++];
      nxt_in = nxt < ni ? iv_in[nxt] : 0.f;
      if (cur < 0 || cur >= n_actors) {  // never expected: record it and stop the ray
        atomicOr(S.status, SALF_DEVERR_BOUNDS);
        live = false;
        continue;
      }
      actor_walk(actors[cur], r, wa, gam_a);
      ha_ok = false;
    } else if (cur >= 0 && !ha_ok && wa.alive) {
      ha_ok = next_hit(actors[cur].S, wa, ha);
    }
    // an actor walk that ended this round (or opened empty) leaves the next
    // interval to be weighed against the pending static hit
    if (cur >= 0 && !ha_ok && !wa.alive) cur = -1;
    const bool s_res = hs_ok || !ws.alive;
    const bool a_res = cur < 0 ? !(nxt < ni && (!hs_ok || nxt_in <= hs.tin + 1e-5f * fmaxf(1.f, fabsf(hs.tin))))
                               : (ha_ok || !wa.alive);
    if (!(s_res && a_res)) continue;
    if (ha_ok && (!hs_ok || ha.tin < hs.tin)) {
      const ActorDev& A = actors[cur];
      T = adjoint_hit<DT, MODE>(wa, ha, reinterpret_cast<const float4*>(A.S.params), A.S.order,
                                A.S.n, A.dparams, S.status, want_int, gam_a, g, gQ, Tend, gbg,
                                T, &Pk);
      ha_ok = false;
    } else if (hs_ok) {
      T = adjoint_hit<DT, MODE>(ws, hs, reinterpret_cast<const float4*>(S.params), S.order,
                                S.n, Q.d_params, S.status, want_int, gam_s, g, gQ, Tend, gbg,
                                T, &Pk);
      hs_ok = false;
    } else {
      if (cur < 0 && nxt >= ni) live = false;
      continue;
    }
    if (++done >= nv) live = false;  // the forward composited exactly nv hits
  }
}

template <int DT, int MODE>
void launch_actors(const LaunchParams& P, const ActorDev* actors, int n, const unsigned* masks,
                   bool dump, cudaStream_t st) {
  const int blocks = (P.total_tiles + kActorWarps - 1) / kActorWarps;
  if (blocks == 0) return;
  const ReqDev& q = P.req[0];
  if (dump)
    k_forward_actors<DT, MODE, true, false><<<blocks, 32 * kActorWarps, 0, st>>>(P, actors, n, masks);
  else if (q.kind == SALF_PINHOLE && !q.moving && !q.want_int)
    k_forward_actors<DT, MODE, false, true><<<blocks, 32 * kActorWarps, 0, st>>>(P, actors, n, masks);
  else
    k_forward_actors<DT, MODE, false, false><<<blocks, 32 * kActorWarps, 0, st>>>(P, actors, n, masks);
}

}  // namespace

cudaError_t salf_launch_backward_actors(const LaunchParams& P, const ActorDev* actors,
                                        int n_actors, const unsigned* masks, cudaStream_t st) {
  const int blocks = (P.total_tiles + kActorWarps - 1) / kActorWarps;
  if (blocks == 0) return cudaSuccess;
  const int dt = P.S.dtype, md = P.S.mode;
  if (dt == SALF_F32 && md == SALF_FIELD_EXP)
    k_backward_actors<SALF_F32, SALF_FIELD_EXP><<<blocks, 32 * kActorWarps, 0, st>>>(P, actors, n_actors, masks);
  else if (dt == SALF_F32)
    k_backward_actors<SALF_F32, SALF_FIELD_SDF><<<blocks, 32 * kActorWarps, 0, st>>>(P, actors, n_actors, masks);
  else if (md == SALF_FIELD_EXP)
    k_backward_actors<SALF_BF16, SALF_FIELD_EXP><<<blocks, 32 * kActorWarps, 0, st>>>(P, actors, n_actors, masks);
  else
    k_backward_actors<SALF_BF16, SALF_FIELD_SDF><<<blocks, 32 * kActorWarps, 0, st>>>(P, actors, n_actors, masks);
  return cudaGetLastError();
}

cudaError_t salf_launch_classify(const LaunchParams& P, const ActorDev* actors, int n_actors,
                                 int* lists, int* counts, unsigned* masks, cudaStream_t st) {
  const int blocks = (P.req[0].n_tiles + 3) / 4;
  if (blocks > 0)
    k_classify_tiles<<<blocks, 128, 0, st>>>(P, actors, n_actors, lists, counts, masks);
  return cudaGetLastError();
}

cudaError_t salf_launch_actors(const LaunchParams& P, const ActorDev* actors, int n_actors,
                               const unsigned* masks, cudaStream_t st) {
  const bool dump = P.req[0].vcap > 0;
  const int dt = P.S.dtype, md = P.S.mode;
  if (dt == SALF_F32 && md == SALF_FIELD_EXP)
    launch_actors<SALF_F32, SALF_FIELD_EXP>(P, actors, n_actors, masks, dump, st);
  else if (dt == SALF_F32)
    launch_actors<SALF_F32, SALF_FIELD_SDF>(P, actors, n_actors, masks, dump, st);
  else if (md == SALF_FIELD_EXP)
    launch_actors<SALF_BF16, SALF_FIELD_EXP>(P, actors, n_actors, masks, dump, st);
  else
    launch_actors<SALF_BF16, SALF_FIELD_SDF>(P, actors, n_actors, masks, dump, st);
  return cudaGetLastError();
}
