// backward.cu -- hand-written adjoint of the forward ray-cast kernel.
//
// For L with per-ray gradients g = dL/d(rgb, depth, opacity, intensity) the
// kernel re-traverses each ray, recomputes the transmittance front to back
// (nothing per voxel is stored by the forward pass), and uses the saved
// per-ray totals Q = (C, D, O, I) for the suffix sums:
//   w_k = T_k alpha_k,  q_k = (c_k, t_mid,k, 1, iota_k),
//   dL/dtau_k = T_{k+1} (g . q_k) - (g . Q - sum_{j<=k} w_j g . q_j)
//               - T_end (g_rgb . background),     tau_k = sigma_k delta_k,
// then chains through Eq. 1 (d sigma / d W = sigma [x, 1]) or Eq. 5-6
// (d sigma / d s = a e^{-|s|/b} / (2b), d sigma / d a = sigma / a,
//  d sigma / d b = -a s e^{-|s|/b} / (2 b^2)) and Eq. 2 (d c / d z = c (1 - c),
// d z / d W_c = x, d z / d W_sh = gamma).  The raydrop output adds
// q_k = sigmoid(rho_k) and a background of 1 (T_end), and d/d rho_k =
// w_k s (1 - s).  Each round, the lanes with a hit walk their rays in order
// (T, the suffix sums and dL/dtau need it) and queue the hit's coefficients
// in a per-warp ring in shared memory; whenever 32 are queued, the whole warp
// builds their 32-scalar gradient rows and adds them to the caller's
// input-order FP32 buffer with 16-byte vector atomics.  Rows of one voxel in
// a batch are staged in shared memory and summed first, each lane adding some
// of the 16-byte chunks, so a voxel takes one set of atomics per batch.
#include "traverse.cuh"

// warps per block and resident blocks per SM asked of the compiler
#ifndef SALF_BWD_WARPS
#define SALF_BWD_WARPS 4
#endif
#ifndef SALF_BWD_MIN_BLOCKS
#define SALF_BWD_MIN_BLOCKS 5  // 96 registers, 20 warps per SM: measured faster than 4 (111) and 6 (spills)
#endif

using namespace salf;

// LEAN: every request is a pinhole camera with one pose for the frame and
// asks for neither intensity nor raydrop gradients: only that ray generation
// and no intensity or raydrop terms are compiled in (8-camera training
// adjoint measured 1.5% faster).
template <int DT, int MODE, bool LEAN>
__global__ void __launch_bounds__(32 * SALF_BWD_WARPS, SALF_BWD_MIN_BLOCKS)
    k_backward(const __grid_constant__ LaunchParams P) {
  const int warp = blockIdx.x * SALF_BWD_WARPS + (threadIdx.x >> 5);
  if (warp >= P.total_tiles) return;
  const int lane = threadIdx.x & 31;
  const ReqDev& Q = P.req[find_request(P, warp)];
  const DevScene& S = P.S;
  int tile = warp - Q.tile_begin;
  if (Q.tile_list) {  // a subset of the tiles (the actor adjoint takes the rest)
    if (tile >= __ldg(Q.tile_count)) return;
    tile = __ldg(&Q.tile_list[tile]);
    if (tile < 0 || tile >= Q.n_tiles) {  // never expected: record it and skip the tile
      if (lane == 0) atomicOr(S.status, SALF_DEVERR_BOUNDS);
      return;
    }
  }
  int u0, v0;
  tile_origin(Q, tile, &u0, &v0);
  const int u = u0 + lane % Q.tile_w;
  const int v = v0 + lane / Q.tile_w;
  const bool in_img = (u < Q.W) && (v < Q.H);
  const int ray = v * Q.W + u;

  Ray r;
  Walk w;
  w.alive = false;
  r.valid = false;
  r.d[0] = r.d[1] = r.d[2] = 0.f;
  float g[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  float gQ = 0.f, Tend = 1.f, gp = 0.f;
  int nv = 0;
  if (in_img) {
    if (LEAN)
      gen_ray_pinhole(Q, u, v, r);
    else
      gen_ray(Q, S, u, v, ray, r);
    walk_init(S, r, w);
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
    if (Q.g_raydrop) {  // composited part of the raydrop output: raydrop - T_end
      gp = __ldg(Q.g_raydrop + ray);
      gQ = fmaf(gp, __ldg(Q.b_raydrop + ray) - Tend, gQ);
    }
    nv = (int)s1.w;
    if (!r.valid) nv = 0;
    if (nv == 0) w.alive = false;
  }
  float gam[4];
  sh_basis(r.d, gam);
  const bool want_int = !LEAN && Q.want_int != 0;
  const bool want_drop = !LEAN && Q.g_raydrop != nullptr;
  const float gbg = g[0] * Q.bg[0] + g[1] * Q.bg[1] + g[2] * Q.bg[2] + gp;
  float T = 1.f, Pk = 0.f;
  int k = 0;
  __shared__ float s_rows[SALF_BWD_WARPS][32][33];  // padded: conflict-free columns
  float(*rows)[33] = s_rows[threadIdx.x >> 5];
  // per-warp ring of pending hits (16 words each, padded to 17): each round's
  // hits are queued, and the gradient rows and their atomics run 32 at a time
  // on the whole warp
  constexpr int QN = 64, QW = 17;
  __shared__ float s_queue[SALF_BWD_WARPS][QN * QW];
  float* queue = s_queue[threadIdx.x >> 5];
  int head = 0, tail = 0;  // warp-uniform
  const int nq = (want_int || want_drop) ? 8 : 7;

  // gradient rows of n queued hits (n <= 32), summed per voxel, added to d_params
  auto flush = [&](int n) {
    const bool act = lane < n;
    float gr[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) gr[q] = 0.f;
    int key = 0;
    if (act) {
      const float* it = queue + ((head + lane) & (QN - 1)) * QW;
      key = __float_as_int(it[0]);
      const float xh[4] = {it[1], it[2], it[3], 1.f};
      const float gm[4] = {kSH0, it[13], it[14], it[15]};  // gamma_0 is a constant
#pragma unroll
      for (int q = 0; q < 4; ++q) gr[q] = it[4] * xh[q];
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const float dz = it[7 + ch];
#pragma unroll
        for (int a = 0; a < 3; ++a) gr[4 + 3 * ch + a] = dz * xh[a];
#pragma unroll
        for (int b = 0; b < 4; ++b) gr[13 + 4 * ch + b] = dz * gm[b];
      }
      gr[25] = MODE == SALF_FIELD_EXP ? 0.f : it[5];  // SDF a, b (not queued in EXP mode)
      gr[26] = MODE == SALF_FIELD_EXP ? 0.f : it[6];
      const float di = want_int ? it[10] : 0.f, dr = want_drop ? it[11] : 0.f;
#pragma unroll
      for (int q = 0; q < 4; ++q) gr[27 + q] = di * xh[q];
      gr[31] = dr;
    }
    __syncwarp();
    const unsigned act_lanes = __ballot_sync(0xffffffffu, act);
    if (act) {
      const unsigned peers = __match_any_sync(act_lanes, key);
      float4* dst = reinterpret_cast<float4*>(Q.d_params) + (size_t)key * 8;
      if (peers == (1u << lane)) {
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q < nq)
            atomicAdd(dst + q, make_float4(gr[4 * q], gr[4 * q + 1], gr[4 * q + 2], gr[4 * q + 3]));
      } else {
        // several rows of one voxel: each lane sums some 16-byte chunks over them
#pragma unroll
        for (int q = 0; q < 32; ++q) rows[lane][q] = gr[q];
        __syncwarp(peers);
        const int gn = __popc(peers), rank = __popc(peers & ((1u << lane) - 1u));
        for (int c = rank; c < nq; c += gn) {
          float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
          unsigned m = peers;
          while (m) {
            const int l2 = __ffs(m) - 1;
            m &= m - 1u;
            sum.x += rows[l2][4 * c];
            sum.y += rows[l2][4 * c + 1];
            sum.z += rows[l2][4 * c + 2];
            sum.w += rows[l2][4 * c + 3];
          }
          atomicAdd(dst + c, sum);
        }
        __syncwarp(peers);
      }
    }
    head += n;
    __syncwarp();
  };

  for (;;) {
    Hit h;
    const bool hit = next_hit(S, w, h);
    if (!__any_sync(0xffffffffu, hit || w.alive)) break;
    const unsigned hit_lanes = __ballot_sync(0xffffffffu, hit);
    if (hit) {
      const float tm = 0.5f * (h.tin + h.tout);
      const float dl = h.tout - h.tin;
      float x[3];
      local_coords(w, h, tm, x);
      Field f;
      field_eval<DT, MODE>(S, h.vox, want_int, x, gam, f, want_drop);
      const float sig = f.sig, lin = f.lin, io = f.io;
      const float* c = f.c;
      const float e = __expf(-sig * dl);
      const float wgt = T * (1.f - e);
      // the intensity and raydrop terms only when asked for (a product with a zero
      // factor is not dropped by the compiler)
      float gq = g[0] * c[0] + g[1] * c[1] + g[2] * c[2] + g[3] * tm + g[4];
      if (want_int) gq += g[5] * io;
      if (want_drop) gq += gp * f.dr;
      Pk = fmaf(wgt, gq, Pk);
      const float Tn = T * e;
      const float dtau = Tn * gq - (gQ - Pk) - Tend * gbg;
      const float dsig = dtau * dl;
      // the hit's coefficients: the gradient row is built from them later
      float* it = queue + ((tail + __popc(hit_lanes & ((1u << lane) - 1u))) & (QN - 1)) * QW;
      it[0] = __int_as_float(__ldg(&S.order[h.vox]));
      it[1] = x[0];
      it[2] = x[1];
      it[3] = x[2];
      if (MODE == SALF_FIELD_EXP) {
        it[4] = dsig * sig;
      } else {
        const float a = f.a, b = f.b;
        const float ex = __expf(-fabsf(lin) / b);
        it[4] = dsig * (a / (2.f * b)) * ex;
        it[5] = dsig * sig / a;
        it[6] = -dsig * a * lin * ex / (2.f * b * b);
      }
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) it[7 + ch] = wgt * g[ch] * c[ch] * (1.f - c[ch]);
      if (want_int) it[10] = wgt * g[5] * io * (1.f - io);
      if (want_drop) it[11] = wgt * gp * f.dr * (1.f - f.dr);
      it[13] = gam[1];
      it[14] = gam[2];
      it[15] = gam[3];
      T = Tn;
      if (++k >= nv) w.alive = false;
    }
    tail += __popc(hit_lanes);
    __syncwarp();
    if (tail - head >= 32) flush(32);
  }
  while (tail - head > 0) flush(min(32, tail - head));
}

template <int DT, int MODE>
static cudaError_t launch_bm(const LaunchParams& P, cudaStream_t st) {
  const int blocks = (P.total_tiles + SALF_BWD_WARPS - 1) / SALF_BWD_WARPS;
  if (blocks == 0) return cudaSuccess;
  bool lean = true;
  for (int i = 0; i < P.n_req; ++i) {
    const ReqDev& q = P.req[i];
    lean = lean && q.kind == SALF_PINHOLE && !q.moving && !q.want_int && !q.g_raydrop;
  }
  if (lean)
    k_backward<DT, MODE, true><<<blocks, 32 * SALF_BWD_WARPS, 0, st>>>(P);
  else
    k_backward<DT, MODE, false><<<blocks, 32 * SALF_BWD_WARPS, 0, st>>>(P);
  return cudaGetLastError();
}

cudaError_t salf_launch_backward(const LaunchParams& P, cudaStream_t st) {
  const int dt = P.S.dtype, md = P.S.mode;
  if (dt == SALF_F32 && md == SALF_FIELD_EXP) return launch_bm<SALF_F32, SALF_FIELD_EXP>(P, st);
  if (dt == SALF_F32 && md == SALF_FIELD_SDF) return launch_bm<SALF_F32, SALF_FIELD_SDF>(P, st);
  if (dt == SALF_BF16 && md == SALF_FIELD_EXP) return launch_bm<SALF_BF16, SALF_FIELD_EXP>(P, st);
  return launch_bm<SALF_BF16, SALF_FIELD_SDF>(P, st);
}
