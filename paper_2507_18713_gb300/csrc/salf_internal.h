// salf_internal.h -- structures shared by the host runtime and the sm_103a
// kernels of libsalf.  Not part of the public ABI (include/salf.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/salf.h"

#define SALF_MAX_MASK_LEVELS 12
#define SALF_MAX_COL_LEVELS 16
#define SALF_MAX_BATCH 24
#ifndef SALF_TILE_W
#define SALF_TILE_W 8  // camera warp tile: SALF_TILE_W x (32 / SALF_TILE_W) pixels
#endif
#define SALF_TILE_H (32 / SALF_TILE_W)
#define SALF_WARPS_PER_BLOCK 8
// Spans per ray when the caller leaves the choice to the library (power of 2 <= 8).
#ifndef SALF_SEGMENTS_LIDAR
#define SALF_SEGMENTS_LIDAR 4
#endif
#ifndef SALF_SEGMENTS_FISHEYE
#define SALF_SEGMENTS_FISHEYE 1
#endif
#ifndef SALF_SEGMENTS_PANORAMA
#define SALF_SEGMENTS_PANORAMA 1
#endif
// Azimuths per warp tile of a LiDAR walked in spans (power of 2; the rest of
// the tile's rays are beams).
#ifndef SALF_SEG_LIDAR_TILE_W
#define SALF_SEG_LIDAR_TILE_W 8
#endif

// Device status-word bits.
#define SALF_DEVERR_STEP_CAP 1  // a traversal loop reached its iteration bound
#define SALF_DEVERR_SDF_AB 2    // an SDF record has a <= 0 or b <= 0
#define SALF_DEVERR_ACTOR_CAP 4 // a ray met more actor boxes than it can hold
#define SALF_DEVERR_BOUNDS 8    // an adjoint kernel met an index outside its buffers (skipped)

// Read-only view of a built scene, passed to kernels by value.
//
// Acceleration structure (replaces the paper's pointer octree, Sec. III-B):
//  * occupancy pyramid: mask level 0 has one 64-bit word per 4x4x4 block of
//    level-0 cells (bit = Morton index of the cell inside the block) plus the
//    rank offset of the block's first occupied cell in `cells` and, when
//    every occupied cell of the block is one level-0 voxel, the index of the
//    block's first voxel (voxels are numbered block by block, cells inside a
//    block in bit order), else all ones; mask level
//    m >= 1 has one word per 4x4x4 words of level m-1 (bit set iff that word
//    is non-zero).  An empty cell is skipped together with the largest empty
//    aligned pyramid cell that contains it (one slab exit per skip).
//  * cells[rank] = (e, cm) for each occupied level-0 cell.  cm == 0: e is a
//    voxel index (>= 0) or -2 - node for a subdivided cell; nodes hold 8
//    children with the same encoding (-1 = empty child).  cm != 0: the cell is
//    split once into voxels; cm is the occupancy of its 8 children (bit =
//    x | y << 1 | z << 2) and child c is voxel e + popcount(cm & ((1 << c) - 1)).
//  * column pyramid: for every footprint of 2^c x 2^c level-0 columns, a
//    128-bit mask of the z-layers (layer = layer_cells level-0 cells high)
//    that hold any voxel.  A ray in an empty layer of a footprint can jump to
//    the nearest occupied layer in its direction of travel, or to the
//    footprint's side, in one step.
//  * params: records in voxel order (block, cell inside the block, Morton
//    index of the min corner inside the cell), FP32 or BF16;
//    order[internal] = input index; vox_box[internal] = (min corner in finest
//    cells, log2 of the edge in finest cells), read by the rasteriser.
struct DevScene {
  const uint4* mask0;
  const unsigned long long* mask[SALF_MAX_MASK_LEVELS];
  int mdim[SALF_MAX_MASK_LEVELS][3];
  const int2* cells;
  const int* nodes;
  const uint4* col[SALF_MAX_COL_LEVELS];  // column masks per level: (lo64, hi64) as uint4
  int cdim[SALF_MAX_COL_LEVELS][2];
  int CL;           // column levels
  int layer_shift;  // log2(layer height in finest cells)
  int n_layers;     // <= 128
  const void* params;
  const int* order;
  const int4* vox_box;
  int* status;
  double origin[3];
  double inv_sfin;  // finest cells per metre
  int K;
  int M;
  int Gf[3];
  int bmin[3], bmax[3];  // tight box of all voxels, finest cells [bmin, bmax)
  int mode, dtype;
  int n;
};

// One render request as the kernels see it (prepared on the host in FP64).
struct ReqDev {
  int kind, W, H;
  int moving;          // 1: per-ray pose (rolling-shutter camera or LiDAR with t1 > t0)
  float inv_fx, inv_fy, cx, cy;
  float half_fov, elev_min, elev_max, elev_step;
  float R0[9];         // rotation at t0
  // R(t) = rotation by s * rel_angle about rel_axis (world frame) applied
  // after R0, s = (t - t0) / (t1 - t0): the slerp geodesic from R0 to R1
  float rel_axis[3];
  float rel_angle;
  int Oi[3];           // sensor origin at t0 in finest-cell units: Oi + Of
  float Of[3];
  float dO[3];         // origin(t1) - origin(t0), finest-cell units
  float t_near, t_far; // metres; t_far = +inf if unbounded
  float time0, time1;  // t0, t1 (only for the debug ray dump)
  const float* rays;   // explicit rays (device)
  // outputs
  float* rgb;
  float* depth;
  float* opacity;
  float* intensity;
  float* saved;
  unsigned char* valid;
  int* vcount;
  int* visits;
  int vcap;
  float* ray_dump;
  int* steps_out;
  unsigned* max_alpha;  // per voxel (input order): largest alpha, as FP32 bits (alpha >= 0)
  float* raydrop;       // sum T_i alpha_i sigmoid(rho_i) + T_end
  float t_min;
  float bg[3];
  int want_int;
  // tiling: tile rows are launched outward from first_row, alternating below
  // and above it (the most nearly horizontal rays, the longest ones, first)
  int tiles_x, tiles_y;
  int tile_w, tile_h;  // rays per warp tile: tile_w x tile_h = 32 >> seg_shift
  int tile_begin, n_tiles;
  int first_row;
  // each ray's span in the voxels' box is cut into 2^seg_shift equal parts,
  // walked by neighbouring lanes and composited in order (forward only)
  int seg_shift;
  // optional subset of the tiles (device): warp w of the request renders
  // tile tile_list[w] while w < *tile_count (null: every tile, in order)
  const int* tile_list;
  const int* tile_count;
  // backward inputs (unused by the forward kernel)
  const float* bsaved;
  const float* g_rgb;
  const float* g_depth;
  const float* g_opacity;
  const float* g_int;
  const float* b_raydrop;  // the forward's raydrop output
  const float* g_raydrop;
  float* d_params;
};

// One placed actor as the actor kernel sees it (prepared on the host in FP64
// for one request; frames: world = the static scene's, canonical = the
// actor scene's).
struct ActorDev {
  DevScene S;           // the actor's voxels (canonical frame)
  float R0[9];          // canonical -> world rotation at the sensor's t0
  float axis[3], angle; // R(s) = rot(axis, s * angle) R0
  float orel0[3], orel1[3];  // sensor origin minus actor position at t0, t1 (world m)
  float cc0[3], cc1[3];      // bounding-sphere centre minus sensor origin at t0, t1
  float radius;
  float origin[3];      // actor grid min corner (canonical m)
  float inv_sfin;       // actor finest cells per metre
  float box_lo[3], box_hi[3];  // tight box of the actor's voxels (canonical m)
  int id_base;          // visit ids of its voxels: id_base + input index
  float* dparams;       // adjoint: dL/d(record scalars) of its voxels (input order), or null
};

struct LaunchParams {
  DevScene S;
  int n_req;
  int total_tiles;
  ReqDev req[SALF_MAX_BATCH];
};

// ---------------------------------------------------------------- host side

struct salf_ctx {
  int device;
};

struct salf_scene {
  salf_ctx* ctx = nullptr;
  int device = 0;
  DevScene dev{};
  int64_t n = 0;
  int32_t mode = 0, dtype = 0, K = 0;
  int32_t dims[3] = {0, 0, 0};
  double origin[3] = {0, 0, 0};
  double s0 = 0, sfin = 0;
  int64_t n_cells0 = 0, n_nodes = 0, device_bytes = 0;
  std::vector<void*> allocations;  // every device buffer the scene owns
  // library-owned FP32 gradient buffer (n x 32, input order; salf_scene_params)
  std::mutex grads_mu;
  float* grads = nullptr;
  // staging for host-memory outputs / explicit rays (grown on demand)
  std::mutex staging_mu;
  void* staging = nullptr;
  size_t staging_bytes = 0;
  // rasteriser workspaces (grown on demand, guarded by raster_mu): per-voxel
  // arrays, per-pair arrays, and a pinned word for the pair count
  std::mutex raster_mu;
  void* raster_vox = nullptr;
  size_t raster_vox_bytes = 0;
  void* raster_pairs = nullptr;
  size_t raster_pairs_bytes = 0;
  unsigned long long* raster_count_host = nullptr;
  cudaEvent_t raster_done = nullptr;  // end of the last call's GPU work
  // per-call actor tables (grown on demand, guarded by actor_mu)
  std::mutex actor_mu;
  void* actor_buf = nullptr;
  size_t actor_buf_bytes = 0;
  cudaEvent_t actor_done = nullptr;
  // refinement plan workspace (guarded by refine_mu)
  std::mutex refine_mu;
  void* refine_ws = nullptr;
  size_t refine_ws_bytes = 0;
  unsigned long long* refine_host = nullptr;  // pinned: counts read back
  bool refine_planned = false;
  int64_t refine_n_new = 0;
  // the merge kernel runs on this stream beside the ray kernel (fork / join)
  cudaStream_t actor_aux = nullptr;
  cudaEvent_t actor_fork = nullptr, actor_join = nullptr;
  // the voxel keys in input order (device, scene-owned; salf_scene_save)
  const uint8_t* key_level = nullptr;
  const int32_t* key_ijk = nullptr;
};

// NVTX ranges around the library's calls (host side: the range holds the
// call's launches, so profilers attribute its kernels to it).  Header-only
// NVTX3; a range costs a few nanoseconds when no tool is attached.
#ifndef SALF_NVTX
#define SALF_NVTX 1
#endif
#if SALF_NVTX
#include <nvtx3/nvToolsExt.h>
struct SalfRange {
  explicit SalfRange(const char* name) { nvtxRangePushA(name); }
  ~SalfRange() { nvtxRangePop(); }
  SalfRange(const SalfRange&) = delete;
  SalfRange& operator=(const SalfRange&) = delete;
};
#else
struct SalfRange {
  explicit SalfRange(const char*) {}
};
#endif
#define SALF_RANGE(name) SalfRange salf_range_(name)

// Implemented in the .cu / .cpp files of the library.
void salf_set_error(const std::string& msg);
salf_status salf_cuda_fail(cudaError_t e, const char* what);
// Resolve the no-alloc entry point's staging array on `device` (current).
salf_status salf_noalloc_setup(int device);
salf_status salf_build_scene_impl(salf_ctx* ctx, const salf_scene_desc* d, salf_scene** out);
// The same build from device-resident level / ijk / params (validated by the caller).
salf_status salf_build_scene_gpu(salf_ctx* ctx, const salf_scene_desc* d, salf_scene** out);
// A device buffer owned (and freed) by the scene.
salf_status salf_scene_dalloc(salf_scene* s, size_t bytes, void** p);
// Keep a copy of the build's voxel keys in the scene (for salf_scene_save).
salf_status salf_scene_keep_keys(salf_scene* s, const salf_scene_desc* d);
salf_status salf_prepare_request(const salf_scene* sc, const salf_sensor* sen,
                                 const salf_render_opts* opts, ReqDev* r);
// Warp tiles of a request with 2^seg_shift lanes per ray (0: whole rays);
// callers whose kernels walk whole rays re-tile with 0.
void salf_request_tiling(ReqDev* r, const salf_sensor* s, int seg_shift);
int salf_auto_segments(int kind);
int64_t salf_request_rays(const salf_sensor* sen);
void salf_relative_rotation(const double* pose0, const double* pose1, float axis[3],
                            float* angle);
cudaError_t salf_launch_gather_params(const float* in, const int* order, void* out, int64_t n,
                                      int dtype, int mode, int* status, cudaStream_t st);
cudaError_t salf_launch_forward(const LaunchParams& P, cudaStream_t st);
// masks: per tile, SALF_MAX_ACTORS / 32 words of candidate actors (bits).
cudaError_t salf_launch_actors(const LaunchParams& P, const ActorDev* actors, int n_actors,
                               const unsigned* masks, cudaStream_t st);
// Tiles of request 0 whose rays may meet an actor -> lists[n_tiles + i],
// the others -> lists[i]; counts[1], counts[0] (zeroed by the caller); per
// tile the candidate actors -> masks.
cudaError_t salf_launch_classify(const LaunchParams& P, const ActorDev* actors, int n_actors,
                                 int* lists, int* counts, unsigned* masks, cudaStream_t st);
// Tile rasterisation of one pinhole request (r prepared by
// salf_prepare_request, outputs set); fills *stats when non-null.
salf_status salf_raster_run(salf_scene* sc, const ReqDev& r, double fx, double fy,
                            salf_raster_stats* stats, cudaStream_t st);
cudaError_t salf_launch_backward(const LaunchParams& P, cudaStream_t st);
// Adjoint of the actor frame on the tiles listed in P.req[0].tile_list (the
// merge walk of salf_launch_actors, gradients into d_params and each actor's
// dparams).
cudaError_t salf_launch_backward_actors(const LaunchParams& P, const ActorDev* actors,
                                        int n_actors, const unsigned* masks, cudaStream_t st);
