// render.cu -- fused forward ray-cast kernel (sm_103a).
//
// One thread per ray, one warp per 8x4 pixel tile (32 consecutive rays for
// explicit rays), one launch for a whole batch of requests.  Per ray: sensor
// ray generation -> traversal of the sparse voxel structure -> Eq. 1/5-6
// density and Eq. 2 colour at each segment midpoint -> Eq. 3-4 front-to-back
// compositing, stopping once the transmittance drops below t_min.
//
// Each round of the loop, every live lane takes at most `step_budget`
// structure steps toward its next hit voxel (empty leaves are skipped whole),
// then the lanes that have a hit gather their records and composite together;
// the warp leaves the loop when no lane has work left (ballot).  Lanes whose
// ray terminated early idle in the ballot.
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

using namespace salf;

template <int DT, int MODE, bool DUMP, int WPB, int MINB>
__global__ void __launch_bounds__(32 * WPB, MINB) k_forward(const __grid_constant__ LaunchParams P) {
  const int warp = blockIdx.x * WPB + (threadIdx.x >> 5);
  if (warp >= P.total_tiles) return;
  const int lane = threadIdx.x & 31;
  const ReqDev& Q = P.req[find_request(P, warp)];
  const DevScene& S = P.S;
  int u0, v0;
  tile_origin(Q, warp - Q.tile_begin, &u0, &v0);
  const int u = u0 + lane % Q.tile_w;
  const int v = v0 + lane / Q.tile_w;
  const bool in_img = (u < Q.W) && (v < Q.H);
  const int ray = v * Q.W + u;

  Ray r;
  Walk w;
  w.alive = false;
  r.valid = false;
  r.d[0] = r.d[1] = r.d[2] = 0.f;
  if (in_img) {
    gen_ray(Q, S, u, v, ray, r);
    walk_init(S, r, w);
    if (DUMP && Q.ray_dump) dump_ray(Q, S, r, ray);
  }
  float gam[4];
  sh_basis(r.d, gam);
  const bool want_int = Q.want_int != 0;
  const float tmin = Q.t_min;
  float T = 1.f, C0 = 0.f, C1 = 0.f, C2 = 0.f, Dp = 0.f, Ip = 0.f;
  int nvis = 0;

  // composite one hit voxel (Eq. 3-4) with its field at the segment midpoint
  auto shade = [&](const Hit& h) {
    const float tm = 0.5f * (h.tin + h.tout);
    const float dl = h.tout - h.tin;
    float x[3];
    local_coords(w, h, tm, x);
    Field f;
    field_eval<DT, MODE>(S, h.vox, want_int, x, gam, f);
    const float sig = f.sig, io = f.io;
    const float* c = f.c;
    const float e = __expf(-sig * dl);   // 1 - alpha (Eq. 4)
    const float wgt = T * (1.f - e);     // T_i alpha_i (Eq. 3)
    C0 = fmaf(wgt, c[0], C0);
    C1 = fmaf(wgt, c[1], C1);
    C2 = fmaf(wgt, c[2], C2);
    Dp = fmaf(wgt, tm, Dp);
    Ip = fmaf(wgt, io, Ip);
    T *= e;
    if (DUMP) {
      if (nvis < Q.vcap) Q.visits[(size_t)ray * Q.vcap + nvis] = __ldg(&S.order[h.vox]);
    }
    ++nvis;
  };

  const int budget = P.step_budget > 0 ? P.step_budget : 1 << 30;
  for (;;) {
    Hit h;
    const bool hit = next_hit(S, w, h, budget);
    if (!__any_sync(0xffffffffu, hit || w.alive)) break;
    if (hit) {
      shade(h);
      if (T < tmin) w.alive = false;
    }
  }
  if (!in_img) return;
  const bool valid = r.valid;
  const float Op = 1.f - T;  // sum of T_i alpha_i telescopes to 1 - T_end (Eq. 3-4)
  if (Q.rgb) {
    float* o = Q.rgb + 3 * (size_t)ray;
    o[0] = valid ? fmaf(T, Q.bg[0], C0) : 0.f;
    o[1] = valid ? fmaf(T, Q.bg[1], C1) : 0.f;
    o[2] = valid ? fmaf(T, Q.bg[2], C2) : 0.f;
  }
  if (Q.depth) Q.depth[ray] = Dp;
  if (Q.opacity) Q.opacity[ray] = Op;
  if (Q.intensity) Q.intensity[ray] = Ip;
  if (Q.saved) {
    float4* s = reinterpret_cast<float4*>(Q.saved) + 2 * (size_t)ray;
    s[0] = make_float4(C0, C1, C2, Dp);
    s[1] = make_float4(Op, Ip, T, (float)nvis);
  }
  if (Q.valid) Q.valid[ray] = valid ? 1 : 0;
  if (DUMP) {
    if (Q.steps_out) Q.steps_out[ray] = w.steps;
    if (Q.vcap > 0) {
      Q.vcount[ray] = nvis;
      for (int k = nvis; k < Q.vcap; ++k) Q.visits[(size_t)ray * Q.vcap + k] = -1;
    }
  }
}

template <int DT, int MODE, bool DUMP, int WPB, int MINB>
static void launch_one(const LaunchParams& P, cudaStream_t st) {
  const int blocks = (P.total_tiles + WPB - 1) / WPB;
  if (blocks > 0) k_forward<DT, MODE, DUMP, WPB, MINB><<<blocks, 32 * WPB, 0, st>>>(P);
}

template <int DT, int MODE>
static cudaError_t launch_fm(const LaunchParams& P, bool dump, bool coherent, cudaStream_t st) {
  if (dump)
    launch_one<DT, MODE, true, SALF_FWD_WPB_DIVERGENT, SALF_FWD_BLOCKS_DIVERGENT>(P, st);
  else if (coherent)
    launch_one<DT, MODE, false, SALF_FWD_WPB_COHERENT, SALF_FWD_BLOCKS_COHERENT>(P, st);
  else
    launch_one<DT, MODE, false, SALF_FWD_WPB_DIVERGENT, SALF_FWD_BLOCKS_DIVERGENT>(P, st);
  return cudaGetLastError();
}

cudaError_t salf_launch_forward(const LaunchParams& P, cudaStream_t st) {
  bool dump = false, coherent = true;
  for (int i = 0; i < P.n_req; ++i) {
    const ReqDev& q = P.req[i];
    dump = dump || q.vcap > 0 || q.ray_dump || q.steps_out;
    coherent = coherent && ((SALF_FWD_COHERENT_KINDS >> q.kind) & 1);
  }
  const int dt = P.S.dtype, md = P.S.mode;
  if (dt == SALF_F32 && md == SALF_FIELD_EXP)
    return launch_fm<SALF_F32, SALF_FIELD_EXP>(P, dump, coherent, st);
  if (dt == SALF_F32 && md == SALF_FIELD_SDF)
    return launch_fm<SALF_F32, SALF_FIELD_SDF>(P, dump, coherent, st);
  if (dt == SALF_BF16 && md == SALF_FIELD_EXP)
    return launch_fm<SALF_BF16, SALF_FIELD_EXP>(P, dump, coherent, st);
  return launch_fm<SALF_BF16, SALF_FIELD_SDF>(P, dump, coherent, st);
}
