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
//     so their intervals are too) advance together; the hit with the smaller
//     entry is composited first (the static one on ties), by Eq. 3-4 with
//     early termination;
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

constexpr int kActorWarps = 4;  // warps per block
constexpr int kMaxIntervals = 8;

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

template <int DT, int MODE, bool DUMP>
__global__ void __launch_bounds__(32 * kActorWarps) k_forward_actors(
    const __grid_constant__ LaunchParams P, const ActorDev* __restrict__ actors, int n_actors) {
  const int warp = blockIdx.x * kActorWarps + (threadIdx.x >> 5);
  if (warp >= P.total_tiles) return;
  const int lane = threadIdx.x & 31;
  const ReqDev& Q = P.req[0];
  const DevScene& S = P.S;
  int u0, v0;
  tile_origin(Q, warp - Q.tile_begin, &u0, &v0);
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
    const float tf = r.tf;
    for (int k = 0; k < n_actors; ++k) {
      const ActorDev& A = actors[k];
      float c[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) c[a] = fmaf(r.s, A.cc1[a] - A.cc0[a], A.cc0[a]);
      const float tca = c[0] * r.d[0] + c[1] * r.d[1] + c[2] * r.d[2];
      const float d2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2] - tca * tca;
      if (d2 > A.radius * A.radius || tca + A.radius < r.tn || tca - A.radius > tf) continue;
      float oc[3], dc[3];
      actor_frame(A, r.s, r.d, oc, dc);
      float a0 = r.tn, a1 = tf;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float inv = 1.f / (fabsf(dc[a]) < 1e-20f ? 1e-20f : dc[a]);
        const float p = (A.box_lo[a] - oc[a]) * inv, q = (A.box_hi[a] - oc[a]) * inv;
        a0 = fmaxf(a0, fminf(p, q));
        a1 = fminf(a1, fmaxf(p, q));
      }
      if (!(a1 > a0)) continue;
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

  // 2. merge the static walk with one actor walk at a time
  const bool want_int = Q.want_int != 0;
  const float tmin = Q.t_min;
  Accum acc{1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0};
  Hit hs, ha;
  bool hs_ok = false, ha_ok = false;
  Walk wa;
  wa.alive = false;
  float gam_a[4] = {0.f, 0.f, 0.f, 0.f};
  int cur = -1, nxt = 0;
  const int unlimited = 1 << 30;
  bool done = !(in_img && r.valid);
  while (!done) {
    if (!hs_ok && ws.alive) hs_ok = next_hit(S, ws, hs, unlimited);
    // an actor whose box the ray enters before the pending static hit starts
    // now (a little early is harmless: the merge orders hits by entry)
    if (cur < 0 && nxt < ni &&
        (!hs_ok || iv_in[nxt] <= hs.tin + 1e-5f * fmaxf(1.f, fabsf(hs.tin)))) {
      cur = iv_k[nxt++];
      actor_walk(actors[cur], r, wa, gam_a);
      ha_ok = false;
    }
    if (cur >= 0 && !ha_ok) {
      if (wa.alive) ha_ok = next_hit(actors[cur].S, wa, ha, unlimited);
      if (!ha_ok && !wa.alive) {
        cur = -1;
        continue;
      }
    }
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
      // nothing pending: finished unless an actor is still to start
      if (cur < 0 && nxt >= ni && !ws.alive) break;
      continue;
    }
    ++acc.nvis;
    if (acc.T < tmin) done = true;
  }
  if (!in_img) return;
  write_outputs(Q, ray, r.valid, acc);
  if (DUMP && Q.vcap > 0) {
    Q.vcount[ray] = acc.nvis;
    for (int k = acc.nvis; k < Q.vcap; ++k) Q.visits[(size_t)ray * Q.vcap + k] = -1;
  }
}

template <int DT, int MODE>
void launch_actors(const LaunchParams& P, const ActorDev* actors, int n, bool dump,
                   cudaStream_t st) {
  const int blocks = (P.total_tiles + kActorWarps - 1) / kActorWarps;
  if (blocks == 0) return;
  if (dump)
    k_forward_actors<DT, MODE, true><<<blocks, 32 * kActorWarps, 0, st>>>(P, actors, n);
  else
    k_forward_actors<DT, MODE, false><<<blocks, 32 * kActorWarps, 0, st>>>(P, actors, n);
}

}  // namespace

cudaError_t salf_launch_actors(const LaunchParams& P, const ActorDev* actors, int n_actors,
                               cudaStream_t st) {
  const bool dump = P.req[0].vcap > 0;
  const int dt = P.S.dtype, md = P.S.mode;
  if (dt == SALF_F32 && md == SALF_FIELD_EXP)
    launch_actors<SALF_F32, SALF_FIELD_EXP>(P, actors, n_actors, dump, st);
  else if (dt == SALF_F32)
    launch_actors<SALF_F32, SALF_FIELD_SDF>(P, actors, n_actors, dump, st);
  else if (md == SALF_FIELD_EXP)
    launch_actors<SALF_BF16, SALF_FIELD_EXP>(P, actors, n_actors, dump, st);
  else
    launch_actors<SALF_BF16, SALF_FIELD_SDF>(P, actors, n_actors, dump, st);
  return cudaGetLastError();
}
