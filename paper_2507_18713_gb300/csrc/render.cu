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
  Accum A{1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0};

  const int budget = P.step_budget > 0 ? P.step_budget : 1 << 30;
  for (;;) {
    Hit h;
    const bool hit = next_hit(S, w, h, budget);
    if (!__any_sync(0xffffffffu, hit || w.alive)) break;
    if (hit) {
      const GlobalRec src{reinterpret_cast<const float4*>(S.params) +
                          (size_t)h.vox * RecordLayout<DT>::kChunks};
      const float e = composite_hit<DT, MODE>(w, h, src, want_int, gam, A);
      if (DUMP) {
        if (A.nvis < Q.vcap) Q.visits[(size_t)ray * Q.vcap + A.nvis] = __ldg(&S.order[h.vox]);
        if (Q.max_alpha)  // alpha >= 0: FP32 bit patterns order like the values
          atomicMax(&Q.max_alpha[__ldg(&S.order[h.vox])], __float_as_uint(1.f - e));
      }
      ++A.nvis;
      if (A.T < tmin) w.alive = false;
    }
  }
  if (!in_img) return;
  write_outputs(Q, ray, r.valid, A);
  if (DUMP) {
    if (Q.steps_out) Q.steps_out[ray] = w.steps;
    if (Q.vcap > 0) {
      Q.vcount[ray] = A.nvis;
      for (int k = A.nvis; k < Q.vcap; ++k) Q.visits[(size_t)ray * Q.vcap + k] = -1;
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
    dump = dump || q.vcap > 0 || q.ray_dump || q.steps_out || q.max_alpha;
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
