// render.cu -- fused forward ray-cast kernel (sm_103a).
//
// One thread per ray, one warp per 8x4 pixel tile (32 consecutive rays for
// explicit rays), one launch for a whole batch of requests.  Per ray: sensor
// ray generation -> traversal of the sparse voxel structure -> Eq. 1/5-6
// density and Eq. 2 colour at each segment midpoint -> Eq. 3-4 front-to-back
// compositing, stopping once the transmittance drops below t_min.
//
// Each round of the loop, every live lane takes one structure step toward its
// next hit voxel (empty leaves are skipped whole),
// then the lanes that have a hit gather their records and composite together;
// the warp leaves the loop when no lane has work left (ballot).  Lanes whose
// ray terminated early idle in the ballot.
//
// Span-parallel variant (SEG): 2^seg_shift neighbouring lanes share one ray.
// Lane k walks from the k-th of the equal cut points of the ray's span in the
// voxels' box and composites, from T = 1, the voxels whose entry distance lies
// in [cut_k, cut_k+1).  Front-to-back compositing of consecutive spans is
// associative -- (C, T) of span a then span b is (C_a + T_a C_b, T_a T_b)
// (Eq. 3-4) -- so prefix products of the spans' transmittances (shuffles)
// give each span the T in front of it.  Every round each lane compares the
// products so far (they only fall) with t_min: a span stops once the spans in
// front of it, or they and its own hits, bring T below t_min.  Once the spans
// in front have finished, the product is final and a span stops exactly where
// the whole ray would; only a span that went past that point before then is
// walked a second time from the final T in front of it.  Spans behind the
// stop are dropped, so the result is the whole-ray walk's up to rounding.
#include "traverse.cuh"

// Warps per block and resident blocks per SM of each forward variant (they
// bound the registers per thread).  Coherent camera batches are throughput-
// bound and gain from more resident warps; divergent sensors (fisheye,
// panorama, LiDAR) are bound by their heaviest warps' latency and lose more to
// the register spills that extra residency costs.
#ifndef SALF_FWD_WPB_COHERENT
#define SALF_FWD_WPB_COHERENT 4
#endif
#ifndef SALF_FWD_BLOCKS_COHERENT
#define SALF_FWD_BLOCKS_COHERENT 7
#endif
// Sensor kinds (bit = salf_sensor_kind) that take the high-occupancy variant.
#ifndef SALF_FWD_COHERENT_KINDS
#define SALF_FWD_COHERENT_KINDS ((1 << SALF_PINHOLE) | (1 << SALF_RAYS_EXPLICIT))
#endif
#ifndef SALF_FWD_WPB_DIVERGENT
#define SALF_FWD_WPB_DIVERGENT 8
#endif
#ifndef SALF_FWD_BLOCKS_DIVERGENT
#define SALF_FWD_BLOCKS_DIVERGENT 2
#endif
// Span-parallel variant (batches with a request of more than one span per ray).
#ifndef SALF_FWD_WPB_SEG
#define SALF_FWD_WPB_SEG 8
#endif
#ifndef SALF_FWD_BLOCKS_SEG
#define SALF_FWD_BLOCKS_SEG 2
#endif

using namespace salf;

// RD: the variant can write the raydrop output (instantiated only for
// batches that ask for it, so the other variants keep their code).  INT: the
// variant can evaluate the intensity field; whole-ray batches that ask for no
// intensity (cameras) take a variant without that code, which leaves the
// compiler a smaller loop (measured 2.6% faster on the 1080p camera frame).
// PH: every request is a pinhole camera with one pose per frame, so only that
// ray generation is compiled in (fewer spilled registers: 1080p camera frame
// 0.391 -> 0.381 ms).
template <int DT, int MODE, bool DUMP, int WPB, int MINB, bool SEG, bool RD, bool INT, bool PH>
__global__ void __launch_bounds__(32 * WPB, MINB) k_forward(const __grid_constant__ LaunchParams P) {
  const int warp = blockIdx.x * WPB + (threadIdx.x >> 5);
  if (warp >= P.total_tiles) return;
  const int lane = threadIdx.x & 31;
  const ReqDev& Q = P.req[find_request(P, warp)];
  const DevScene& S = P.S;
  int tile = warp - Q.tile_begin;
  if (Q.tile_list) {
    if (tile >= __ldg(Q.tile_count)) return;
    tile = __ldg(&Q.tile_list[tile]);
  }
  // SEG: lanes (k + K * j), k < K = 2^seg_shift, share the tile's j-th ray
  const int ks = SEG ? Q.seg_shift : 0;
  const int K = 1 << ks;
  const int kseg = lane & (K - 1);
  const int rl = lane >> ks;
  int u0, v0;
  tile_origin(Q, tile, &u0, &v0);
  const int u = u0 + rl % Q.tile_w;
  const int v = v0 + rl / Q.tile_w;
  const bool in_img = (u < Q.W) && (v < Q.H);
  const int ray = v * Q.W + u;

  Ray r;
  Walk w;
  w.alive = false;
  r.valid = false;
  r.d[0] = r.d[1] = r.d[2] = 0.f;
  float t0r = 0.f, cut_lo = 0.f, cut_hi = __int_as_float(0x7f800000), walk_end = cut_hi;
  if (in_img) {
    if (PH)
      gen_ray_pinhole(Q, u, v, r);
    else
      gen_ray(Q, S, u, v, ray, r);
    walk_init(S, r, w);
    if (DUMP && Q.ray_dump) dump_ray(Q, S, r, ray);
    if (SEG && ks > 0 && w.alive) {
      // cut points t0 + L j / K: one expression for both lanes that share a cut
      t0r = w.t;
      const float L = w.tend - w.t, invK = 1.f / (float)K;
      cut_lo = fmaf(L, (float)kseg * invK, t0r);
      if (kseg + 1 < K) {
        cut_hi = fmaf(L, (float)(kseg + 1) * invK, t0r);
        // a hit found once the walk is past cut_hi enters after it (its entry
        // plane is the one the walk crossed); the margin covers hops whose
        // exit rounded below their entry
        walk_end = cut_hi + 4e-6f * fabsf(cut_hi);
      }
      if (kseg > 0) walk_seek(S, w, cut_lo);
    }
  }
  float gam[4];
  sh_basis(r.d, gam);
  const bool want_int = INT && Q.want_int != 0;
  const bool want_drop = RD && Q.raydrop != nullptr;
  const float tmin = Q.t_min;
  Accum A{1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0, 0.f};
  float T_prev = 1.f;  // SEG: this span's T before its last composited hit
  bool keep = true;    // SEG: the whole ray reaches this lane's span

  for (int pass = 0;; ++pass) {
    for (;;) {
      Hit h;
      bool hit = next_hit<!SEG>(S, w, h);
      if (SEG && !hit && w.t > walk_end) w.alive = false;  // the rest is the next span's
      if (!__any_sync(0xffffffffu, hit || w.alive)) break;
      if (SEG && hit && ks > 0) {  // composite only the voxels entered inside this span
        const float te = hit_entry(w, h, t0r);
        if (te >= cut_hi) {
          hit = false;
          w.alive = false;
        } else if (te < cut_lo) {
          hit = false;
        }
      }
      if (hit) {
        const GlobalRec src{reinterpret_cast<const float4*>(S.params) +
                            (size_t)h.vox * RecordLayout<DT>::kChunks};
        if (SEG) T_prev = A.T;
        const float e = composite_hit<DT, MODE>(w, h, src, want_int, gam, A, want_drop);
        if (DUMP) {
          if (A.nvis < Q.vcap) Q.visits[(size_t)ray * Q.vcap + A.nvis] = __ldg(&S.order[h.vox]);
          if (Q.max_alpha)  // alpha >= 0: FP32 bit patterns order like the values
            atomicMax(&Q.max_alpha[__ldg(&S.order[h.vox])], __float_as_uint(1.f - e));
        }
        ++A.nvis;
        if (A.T < tmin && !(SEG && ks > 0 && pass == 0)) w.alive = false;
      }
      if (SEG && ks > 0 && pass == 0) {
        // T in front of the span (ex) and after its hits so far (inc): below
        // t_min, the ray stops before here (or here): nothing left to walk
        float inc, ex;
        span_products(A.T, kseg, K, &inc, &ex);
        if (inc < tmin) w.alive = false;
      }
    }
    if (!SEG || ks == 0 || pass > 0) break;
    // final products (never above those that stopped lanes during the walk)
    float inc, Tf;
    span_products(A.T, kseg, K, &inc, &Tf);
    // the ray (if it gets here) stops inside this span; it gets here unless an
    // earlier span of it says so too -- one ballot, so every lane agrees
    const bool ends = inc < tmin;
    const unsigned em = __ballot_sync(0xffffffffu, ends);
    const unsigned before = ((1u << lane) - 1u) & ~((1u << (lane & ~(K - 1))) - 1u);
    keep = (em & before) == 0u;
    // exact if the span's last hit is the first one to bring T below t_min;
    // else it composited past the stop: walk it again from Tf
    const bool redo = keep && ends && Tf < 1.f && !(Tf * T_prev >= tmin);
    if (redo) {
      A = Accum{Tf, 0.f, 0.f, 0.f, 0.f, 0.f, 0, 0.f};
      walk_seek(S, w, cut_lo);
      w.alive = true;
    } else if (keep) {
      A.C0 *= Tf;
      A.C1 *= Tf;
      A.C2 *= Tf;
      A.Dp *= Tf;
      A.Ip *= Tf;
      if (want_drop) A.Rp *= Tf;
      A.T *= Tf;
    }
    if (!__any_sync(0xffffffffu, redo)) break;
  }
  if (SEG && ks > 0) {
    // sum the kept spans; the ray's final T is the smallest kept one (T only falls)
    if (!keep) A = Accum{1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0, 0.f};
    for (int off = K >> 1; off > 0; off >>= 1) {
      A.C0 += __shfl_xor_sync(0xffffffffu, A.C0, off, K);
      A.C1 += __shfl_xor_sync(0xffffffffu, A.C1, off, K);
      A.C2 += __shfl_xor_sync(0xffffffffu, A.C2, off, K);
      A.Dp += __shfl_xor_sync(0xffffffffu, A.Dp, off, K);
      A.Ip += __shfl_xor_sync(0xffffffffu, A.Ip, off, K);
      if (want_drop) A.Rp += __shfl_xor_sync(0xffffffffu, A.Rp, off, K);
      A.T = fminf(A.T, __shfl_xor_sync(0xffffffffu, A.T, off, K));
      A.nvis += __shfl_xor_sync(0xffffffffu, A.nvis, off, K);
    }
    if (kseg != 0) return;
  }
  if (!in_img) return;
  write_outputs(Q, ray, r.valid, A, want_drop);
  if (DUMP) {
    if (Q.steps_out) Q.steps_out[ray] = w.steps;
    if (Q.vcap > 0) {
      Q.vcount[ray] = A.nvis;
      for (int k = A.nvis; k < Q.vcap; ++k) Q.visits[(size_t)ray * Q.vcap + k] = -1;
    }
  }
}

template <int DT, int MODE, bool DUMP, int WPB, int MINB, bool SEG, bool RD, bool INT,
          bool PH = false>
static void launch_one(const LaunchParams& P, cudaStream_t st) {
  const int blocks = (P.total_tiles + WPB - 1) / WPB;
  if (blocks > 0)
    k_forward<DT, MODE, DUMP, WPB, MINB, SEG, RD, INT, PH><<<blocks, 32 * WPB, 0, st>>>(P);
}

template <int DT, int MODE>
static cudaError_t launch_fm(const LaunchParams& P, bool dump, bool coherent, bool seg, bool rd,
                             bool want_int, bool pinhole, cudaStream_t st) {
  constexpr int WD = SALF_FWD_WPB_DIVERGENT, BD = SALF_FWD_BLOCKS_DIVERGENT;
  constexpr int WS = SALF_FWD_WPB_SEG, BS = SALF_FWD_BLOCKS_SEG;
  constexpr int WC = SALF_FWD_WPB_COHERENT, BC = SALF_FWD_BLOCKS_COHERENT;
  if (dump)
    launch_one<DT, MODE, true, WD, BD, false, true, true>(P, st);
  else if (seg && rd)
    launch_one<DT, MODE, false, WS, BS, true, true, true>(P, st);
  else if (seg)
    launch_one<DT, MODE, false, WS, BS, true, false, true>(P, st);
  else if (rd)
    launch_one<DT, MODE, false, WD, BD, false, true, true>(P, st);
  else if (coherent && want_int)
    launch_one<DT, MODE, false, WC, BC, false, false, true>(P, st);
  else if (pinhole)
    launch_one<DT, MODE, false, WC, BC, false, false, false, true>(P, st);
  else if (coherent)
    launch_one<DT, MODE, false, WC, BC, false, false, false>(P, st);
  else if (want_int)
    launch_one<DT, MODE, false, WD, BD, false, false, true>(P, st);
  else
    launch_one<DT, MODE, false, WD, BD, false, false, false>(P, st);
  return cudaGetLastError();
}

static cudaError_t launch_variant(const LaunchParams& P, cudaStream_t st) {
  bool dump = false, coherent = true, seg = false, rd = false, want_int = false, pinhole = true;
  for (int i = 0; i < P.n_req; ++i) {
    const ReqDev& q = P.req[i];
    pinhole = pinhole && q.kind == SALF_PINHOLE && !q.moving;
    dump = dump || q.vcap > 0 || q.ray_dump || q.steps_out || q.max_alpha;
    coherent = coherent && ((SALF_FWD_COHERENT_KINDS >> q.kind) & 1);
    seg = seg || q.seg_shift > 0;
    rd = rd || q.raydrop;
    want_int = want_int || q.want_int;
  }
  // the debug variant walks whole rays: its requests must be tiled for that
  if (dump && seg) return cudaErrorInvalidValue;
  const int dt = P.S.dtype, md = P.S.mode;
  if (dt == SALF_F32 && md == SALF_FIELD_EXP)
    return launch_fm<SALF_F32, SALF_FIELD_EXP>(P, dump, coherent, seg, rd, want_int, pinhole, st);
  if (dt == SALF_F32 && md == SALF_FIELD_SDF)
    return launch_fm<SALF_F32, SALF_FIELD_SDF>(P, dump, coherent, seg, rd, want_int, pinhole, st);
  if (dt == SALF_BF16 && md == SALF_FIELD_EXP)
    return launch_fm<SALF_BF16, SALF_FIELD_EXP>(P, dump, coherent, seg, rd, want_int, pinhole, st);
  return launch_fm<SALF_BF16, SALF_FIELD_SDF>(P, dump, coherent, seg, rd, want_int, pinhole, st);
}

// A batch that mixes requests of different variants runs as one launch per
// variant: span-parallel requests; static pinhole cameras that ask for no
// intensity or raydrop (the lean variant); the rest.  Each group keeps its own
// variant's code and shape, and each request's result does not depend on the
// split (the lean variant's outputs equal the general one's bit for bit).
static int variant_group(const ReqDev& q) {
  if (q.seg_shift > 0) return 0;
  const bool dump = q.vcap > 0 || q.ray_dump || q.steps_out || q.max_alpha;
  if (q.kind == SALF_PINHOLE && !q.moving && !q.want_int && !q.raydrop && !dump) return 1;
  return 2;
}

cudaError_t salf_launch_forward(const LaunchParams& P, cudaStream_t st) {
  int count[3] = {0, 0, 0};
  for (int i = 0; i < P.n_req; ++i) ++count[variant_group(P.req[i])];
  const int groups = (count[0] > 0) + (count[1] > 0) + (count[2] > 0);
  if (groups <= 1 || P.req[0].tile_list) return launch_variant(P, st);
  for (int part = 0; part < 3; ++part) {
    if (!count[part]) continue;
    LaunchParams G = P;
    G.n_req = 0;
    G.total_tiles = 0;
    for (int i = 0; i < P.n_req; ++i) {
      if (variant_group(P.req[i]) != part) continue;
      G.req[G.n_req] = P.req[i];
      G.req[G.n_req].tile_begin = G.total_tiles;
      G.total_tiles += P.req[i].n_tiles;
      ++G.n_req;
    }
    const cudaError_t e = launch_variant(G, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
