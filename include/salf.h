/*
 * salf.h -- C ABI of the GB300 (sm_103a) SaLF ray-cast renderer.
 *
 * SaLF (arXiv 2507.18713) represents a scene as a sparse set of disjoint,
 * axis-aligned cubic voxels on a multi-level grid (Sec. III-A), each holding a
 * small local field: a density (Eq. 1, or an SDF turned into a density by
 * Eq. 5-6) and a colour with l <= 1 spherical harmonics (Eq. 2).  A ray is
 * rendered by visiting the voxels it crosses front to back, sampling each
 * voxel's field at the midpoint of the ray-voxel segment and compositing by
 * Eq. 3-4 (Sec. III-A "Volume rendering", Sec. III-B "Ray-Casting with Octree
 * Acceleration").
 *
 * Conventions shared by every call:
 *   - Every call returns a salf_status; nothing aborts, throws or traps.  On
 *     failure salf_last_error() gives a thread-local message.
 *   - Render calls are asynchronous and ordered on the caller's CUDA stream
 *     (a cudaStream_t passed as void*; NULL = the legacy default stream),
 *     unless the outputs are host memory (salf_outputs.on_host = 1), in which
 *     case the call also copies the results back and returns after the stream
 *     has drained (on_host = 2: page-locked host outputs, asynchronous).
 *   - Output buffers are owned by the caller.  Contexts, scenes and servers
 *     are owned by the library (created/destroyed through this API).
 *   - World frame: metres, right-handed, z up.  Camera frame: x right, y down,
 *     z forward.  LiDAR frame: x forward, y left, z up.
 *   - Ray index of pixel (u, v) (or LiDAR azimuth column u, beam row v) is
 *     v * width + u.  Per-ray outputs are dense arrays over that index.
 */
#ifndef SALF_H
#define SALF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SALF_OK = 0,
  SALF_ERR_INVALID = 1,   /* bad argument (null pointer, size, enum, range) */
  SALF_ERR_OOM = 2,       /* device or host allocation failed */
  SALF_ERR_CUDA = 3,      /* a CUDA runtime call failed */
  SALF_ERR_OVERLAP = 4,   /* scene voxels overlap (Sec. III-D requires disjoint voxels) */
  SALF_ERR_AGAIN = 5,     /* serving: request not admitted yet */
  SALF_ERR_TIMEOUT = 6,   /* serving: wait ran out */
  SALF_ERR_NOT_FOUND = 7, /* serving: unknown or released ticket */
  SALF_ERR_SHUTDOWN = 8,  /* serving: server is shutting down */
  SALF_ERR_DEVICE = 9,    /* a kernel reported an internal error through its status word */
  SALF_ERR_IO = 10        /* a scene file could not be opened, read or written, or is malformed */
} salf_status;

typedef enum { SALF_FIELD_EXP = 0, SALF_FIELD_SDF = 1 } salf_field_mode;
typedef enum { SALF_F32 = 0, SALF_BF16 = 1 } salf_dtype;
typedef enum {
  SALF_PINHOLE = 0,
  SALF_FISHEYE_EQUIDIST = 1,
  SALF_PANO_EQUIRECT = 2,
  SALF_LIDAR_SPIN = 3,
  SALF_RAYS_EXPLICIT = 4
} salf_sensor_kind;

typedef struct salf_ctx salf_ctx;
typedef struct salf_scene salf_scene;
typedef struct salf_server salf_server;

/* Number of scalars in one voxel record (Sec. III-A learnable parameters). */
#define SALF_RECORD_SCALARS 32

/*
 * Scene input (Sec. III-A).  The root volume is a grid of dims[0..2] cubic
 * cells of edge s0 with min corner `origin`; a cell of level l has edge
 * s0 / 2^l and 0 <= level <= max_level (K, at most 10).  Voxel v is the cell
 * ijk[3v..3v+2] of level level[v].  Voxels must be disjoint (Sec. III-D): a
 * voxel whose ancestor is also present, or a duplicate, gives SALF_ERR_OVERLAP.
 * dims[a] << max_level must not exceed 2^21.
 *
 * Record layout (32 scalars per voxel, input order):
 *   [0:4]   W_sigma (Eq. 1) or W_s (Eq. 5): 3 slopes, then the bias
 *   [4:13]  W_c (Eq. 2), row-major 3x3 (rows r, g, b; columns x, y, z)
 *   [13:25] W_sh (Eq. 2), row-major 3x4 (rows r, g, b; SH basis
 *           gamma(w) = [C0, C1 w_y, C1 w_z, C1 w_x], C0 = 1/(2 sqrt(pi)),
 *           C1 = sqrt(3)/(2 sqrt(pi)), w = unit ray direction)
 *   [25] a, [26] b (Eq. 6; SDF mode requires a > 0 and b > 0)
 *   [27:31] W_int: intensity field sigmoid(W_int . [x, 1]), 3 slopes then bias
 *   [31]    rho: LiDAR raydrop logit, constant over the voxel (raydrop output)
 * `params` are FP32 (host memory, or device memory if params_on_device);
 * `dtype` selects how the scene stores them (FP32, or BF16 converted by
 * round-to-nearest; all arithmetic is FP32 either way).  level and ijk are
 * host memory, unless keys_on_device: then level, ijk and params are device
 * memory (params_on_device must be set) and the whole build runs on the GPU
 * (same structure, same errors).  Everything is copied: the caller may free
 * its arrays when salf_build_scene returns.
 */
typedef struct {
  int64_t n;
  double origin[3];
  double s0;
  int32_t dims[3];
  int32_t max_level;
  const uint8_t* level;
  const int32_t* ijk;
  int32_t mode;   /* salf_field_mode */
  int32_t dtype;  /* salf_dtype */
  const float* params;
  int32_t params_on_device;
  int32_t keys_on_device;
} salf_scene_desc;

/*
 * A sensor (Fig. 2; Sec. V-C rolling shutter).  width x height rays:
 *   PINHOLE: direction (( u+0.5-cx)/fx, (v+0.5-cy)/fy, 1), normalised.
 *   FISHEYE_EQUIDIST: theta = |((u+0.5-cx)/fx, (v+0.5-cy)/fy)| is the angle off
 *     the optical axis (image radius = f * theta); rays with theta > fov/2 are
 *     invalid (valid = 0, outputs 0).
 *   PANO_EQUIRECT: longitude 2 pi ((u+0.5)/width - 0.5) (0 = optical axis,
 *     increasing to the right), latitude from elev_max (top) to elev_min
 *     (bottom) at the pixel centres.
 *   LIDAR_SPIN: width azimuth columns (azimuth 2 pi u / width, counter-
 *     clockwise from sensor +x), height beams with elevations from elev_max
 *     (row 0) down to elev_min (last row), evenly spaced, inclusive.
 *   RAYS_EXPLICIT: width rays given as 8 floats (ox, oy, oz, dx, dy, dz,
 *     t_near, t_far) in `rays` (device memory; host memory only when the
 *     outputs are on the host); directions are normalised; t_far <= 0 means
 *     unbounded.
 * pose0 / pose1: sensor-to-world 3x4 row-major [R | t] at times t0 / t1.  Per-
 * ray time: LiDAR column u -> t0 + (u/width)(t1 - t0); camera row v ->
 * t0 + (v/(height-1))(t1 - t0) if rolling_shutter, else t0.  The pose at a
 * time is the linear interpolation of the translations and the spherical
 * linear interpolation of the rotations (pose0 exactly at t0).
 * Rays start at t_near (>= 0) and end at t_far (<= 0: unbounded), in metres
 * along the unit direction.
 */
typedef struct {
  int32_t kind;
  int32_t width, height;
  float fx, fy, cx, cy;
  float fov;
  float elev_min, elev_max;
  double pose0[12], pose1[12];
  double t0, t1;
  int32_t rolling_shutter;
  float t_near, t_far;
  const float* rays;
} salf_sensor;

/*
 * Render options.  t_min_transmittance: a ray stops after compositing the
 * voxel that brings its transmittance below this value (0 = never stop).
 * background is added as T_end * background to the (premultiplied) colour.
 * want_intensity: also evaluate the intensity field.  visits_cap > 0 records,
 * per ray, the first visits_cap composited voxels (input indices, -1 padded)
 * and the total count: a debugging aid that slows the kernel.
 * ray_segments: 1, 2, 4 or 8 splits each ray's span inside the voxels' box
 * into that many equal parts walked at the same time by neighbouring threads
 * and composited front to back in order (Eq. 3-4 are associative over
 * consecutive spans); a part in which the ray actually stopped is walked
 * again from the transmittance in front of it, so the outputs are those of
 * the whole-ray walk up to rounding.  It shortens the longest rays' serial
 * latency (LiDAR beams near the horizon).  0 = the library's choice per
 * sensor kind.  Renders that record visits, ray dumps, step counts or alpha
 * maxima, rasterised and actor renders and the backward pass walk whole rays.
 */
typedef struct {
  float t_min_transmittance;
  float background[3];
  int32_t want_intensity;
  int32_t visits_cap;
  int32_t ray_segments;
} salf_render_opts;

/*
 * Per-ray outputs (R = width * height entries each; NULL = not wanted):
 *   rgb       R x 3: sum_i T_i alpha_i c_i (Eq. 3) + T_end * background
 *   depth     R: sum_i T_i alpha_i t_mid,i (expected distance, unnormalised;
 *             LiDAR range)
 *   opacity   R: sum_i T_i alpha_i = 1 - T_end
 *   intensity R: sum_i T_i alpha_i iota_i
 *   saved     R x 8: (C_r, C_g, C_b, depth, opacity, intensity, T_end,
 *             visited count as float) -- the input salf_render_backward needs
 *   valid     R bytes: 1 if the ray exists (fisheye rays outside the FOV: 0)
 *   visit_count, visits: see salf_render_opts.visits_cap
 *   ray_dump  R x 8 (debugging aid): the generated ray as (ox, oy, oz, dx, dy,
 *             dz, time, valid) in world coordinates
 *   steps     R (debugging aid): structure leaves the traversal stepped through
 *   raydrop   R: sum_i T_i alpha_i sigmoid(rho_i) + T_end, the probability that
 *             the LiDAR return is dropped (a ray that leaves the scene returns
 *             nothing); Sec. V-C and Table III name raydrop without a form.
 *             salf_render_rays only (not rasterised, actor or no-alloc renders)
 * on_host = 0: device pointers; on_host = 1: host pointers, and the call
 * returns when they hold the results.  Page-locked buffers the device can
 * address (cudaHostAlloc / cudaHostRegister under unified addressing; saved
 * 16-byte aligned) are written by the kernel in place; otherwise the library
 * renders into its own device staging buffers and copies back.
 * on_host = 2 (salf_render_rays only): page-locked host pointers the device
 * can address, written by the kernel in place, and the call is asynchronous
 * like a device-output render: the buffers hold the results once `stream`
 * has drained (cudaStreamSynchronize, or an event recorded after the call).
 * A caller can so keep several frames in flight, each in its own buffers.
 * Any other host buffer is rejected (SALF_ERR_INVALID); nothing is staged.
 */
typedef struct {
  float* rgb;
  float* depth;
  float* opacity;
  float* intensity;
  float* saved;
  uint8_t* valid;
  int32_t* visit_count;
  int32_t* visits;
  float* ray_dump;
  int32_t* steps;
  int32_t on_host;
  float* max_alpha;  /* n (scene voxels, input order), device, salf_render_rays only:
                        max-accumulated with each voxel's largest composited alpha
                        (Eq. 4) over the rays; the caller zeroes it (pruning, Sec. III-C) */
  float* raydrop;
} salf_outputs;

typedef struct {
  int64_t n;
  int32_t mode, dtype;
  int32_t max_level;
  int32_t dims[3];
  int64_t n_level0_cells;   /* occupied level-0 cells */
  int64_t n_nodes;          /* subdivision nodes below level 0 */
  int64_t device_bytes;     /* device memory held by the scene */
  const void* dev_params;   /* records in the scene's internal voxel order */
  const int32_t* dev_order; /* internal index -> input index */
} salf_scene_info;

/* Create a context bound to CUDA device `device`. */
salf_status salf_create(int32_t device, salf_ctx** out);
void salf_destroy(salf_ctx* ctx);

/*
 * Build a scene (Sec. III-A representation, Sec. III-B acceleration
 * structure).  Voxels are sorted in Morton order of their min corner, checked
 * for overlaps, and indexed by an occupancy pyramid of 64-bit masks over 4^3
 * blocks (with rank offsets into the level-0 cell table) plus 8-way
 * subdivision nodes below level 0.  Synchronous.  Errors: INVALID (sizes,
 * ranges, SDF a or b <= 0), OVERLAP, OOM, CUDA.
 */
salf_status salf_build_scene(salf_ctx* ctx, const salf_scene_desc* desc, salf_scene** out);
void salf_scene_destroy(salf_scene* scene);
salf_status salf_scene_get_info(const salf_scene* scene, salf_scene_info* info);

/*
 * Replace the scene's records with `params` (n x 32 FP32, input order, host
 * or device), converting to the scene's storage dtype.  Ordered on `stream`;
 * host params are copied before the call returns.  The voxel set is unchanged.
 */
salf_status salf_scene_update_params(salf_scene* scene, const float* params,
                                     int32_t params_on_device, void* stream);

/*
 * Device views of a scene's learnable state (Sec. III-A records), for
 * wrapping as tensors.  *dev_params (if dev_params is not NULL): the scene's
 * records, n x 32 in its storage dtype (FP32 or BF16) and in its internal
 * voxel order (salf_scene_info.dev_order maps internal -> input index);
 * library-owned, valid until salf_scene_destroy, replaced in place by
 * salf_scene_update_params.  *dev_grads (if dev_grads is not NULL): the
 * scene's own FP32 gradient buffer, n x 32 in input order, 16-byte aligned,
 * created and zeroed by the first call that asks for it (synchronous
 * cudaMalloc + cudaMemset), freed by salf_scene_destroy; salf_render_backward
 * with d_params = NULL accumulates into it, and the caller zeroes it between
 * steps.  Errors: INVALID (null scene), OOM, CUDA.
 */
salf_status salf_scene_params(salf_scene* scene, void** dev_params, void** dev_grads);

/*
 * Render all rays of `sensor` (Eq. 1-6 along the voxels each ray crosses).
 * Errors: INVALID (sizes, kind, no output requested), CUDA, DEVICE.
 */
salf_status salf_render_rays(salf_scene* scene, const salf_sensor* sensor,
                             const salf_render_opts* opts, const salf_outputs* out,
                             void* stream);

/*
 * Render n sensors in one launch (n <= 24 per launch; more are split into
 * launches of 24), e.g. the cameras of one training step.  Each sensor's
 * outputs are those of a lone salf_render_rays call with the same options
 * (rays are independent); one launch lets the sensors' longest rays overlap
 * instead of paying their serial latency once per sensor.  sensors[i] and
 * outs[i] as for salf_render_rays; outputs must be device memory (on_host,
 * visits, ray_dump, steps and max_alpha are rejected).  `opts` applies to
 * every sensor.  Asynchronous on `stream`.  Errors: INVALID, CUDA.
 */
salf_status salf_render_rays_batch(salf_scene* scene, int32_t n, const salf_sensor* sensors,
                                   const salf_render_opts* opts, const salf_outputs* outs,
                                   void* stream);

/*
 * The adjoint of a salf_render_rays_batch call (or of n salf_render_rays
 * calls) in one launch: for sensor i, saved[i] is its R_i x 8 saved array and
 * d_rgb[i], d_depth[i], d_opacity[i], d_intensity[i] its dL/d(outputs) (the
 * arrays of pointers may be NULL, and so may their entries: zero).  d_params
 * (n_voxels x 32 FP32, input order, device, 16-byte aligned; NULL = the
 * scene's own gradient buffer) is ACCUMULATED (+=) with the sum over the
 * sensors.  Raydrop gradients are not supported here.  Asynchronous on
 * `stream`.  Errors: INVALID, CUDA.
 */
salf_status salf_render_backward_batch(salf_scene* scene, int32_t n, const salf_sensor* sensors,
                                       const salf_render_opts* opts, const float* const* saved,
                                       const float* const* d_rgb, const float* const* d_depth,
                                       const float* const* d_opacity,
                                       const float* const* d_intensity, float* d_params,
                                       void* stream);

/*
 * salf_render_rays for host output buffers, without any device allocation.
 * The paper has no counterpart: this serves callers that cannot let a library
 * allocate device memory -- real-time loops that cannot absorb an
 * allocation's latency and implicit synchronisation, applications whose
 * device memory is reserved up front by their own pooling allocator, and
 * plug-ins whose host forbids them to allocate.  (salf_render_rays with
 * on_host = 1 grows a staging buffer with cudaMalloc instead.)
 * Page-locked host buffers the device can address (cudaHostAlloc /
 * cudaHostRegister; saved 16-byte aligned) are written by the kernel in place.
 * Other buffers are staged in a fixed 48 MiB array compiled into the library;
 * requests whose outputs need more staging than that are rejected with
 * SALF_ERR_INVALID.  salf_create resolves the array on its device (with
 * lazy module loading, that is when the device allocates it), so the array
 * is resident from the first salf_create on a device until the process
 * exits: a caller that reserves device memory in its own pool does so after
 * salf_create.  `out` holds host pointers (on_host is ignored); the debug
 * outputs (visits, visit_count, ray_dump, steps), max_alpha and raydrop are
 * not supported (SALF_ERR_INVALID); explicit rays must be device memory.
 * Calls on one device share the array: two calls that overlap on the GPU
 * (e.g. from two host threads) race, so serialise them.  Synchronous:
 * returns after the outputs are in the host buffers.  Calls no cudaMalloc,
 * cudaFree or allocating routine.
 */
salf_status salf_render_rays_host_noalloc(salf_scene* scene, const salf_sensor* sensor,
                                          const salf_render_opts* opts,
                                          const salf_outputs* out, void* stream);

/*
 * Adjoint of salf_render_rays (gradients of Eq. 1-6 compositing, transmittance
 * recomputed front to back).  `saved` is the R x 8 array the forward call wrote
 * with the same scene, sensor and options.  d_rgb (R x 3), d_depth,
 * d_opacity, d_intensity, d_raydrop (R each; NULL = zero) are dL/d(outputs);
 * with d_raydrop, `raydrop` is the forward's raydrop output (R; its composited
 * part raydrop - T_end enters the suffix sums), else it may be NULL.  d_params
 * (n x 32 FP32, input order, device memory, 16-byte aligned; NULL = the
 * scene's own gradient buffer, see salf_scene_params) is ACCUMULATED (+=)
 * with dL/d(record scalars); scalars a field mode does not use receive no
 * gradient.  All pointers are device memory.  Asynchronous on `stream`.
 * The only forward outputs the adjoint reads are the per-ray totals in
 * `saved` (and the raydrop output with d_raydrop): transmittances and every
 * per-voxel quantity are recomputed by walking the rays again.
 */
salf_status salf_render_backward(salf_scene* scene, const salf_sensor* sensor,
                                 const salf_render_opts* opts, const float* saved,
                                 const float* d_rgb, const float* d_depth,
                                 const float* d_opacity, const float* d_intensity,
                                 const float* raydrop, const float* d_raydrop,
                                 float* d_params, void* stream);

/*
 * Tile rasterisation of a pinhole camera (Sec. III-B, "Tile-based
 * Splatting"): every voxel is projected onto the image and listed in each
 * 16 x 16-pixel tile its projection may cover; each tile's list is sorted
 * front to back and composited by one thread block, with the records staged
 * in shared memory.  Per pixel, a voxel's opacity comes from the exact length
 * of the pixel's ray inside it and its colour from the field at that
 * segment's midpoint (Eq. 1-6), as in salf_render_rays.
 * Sort order: level-0 cells by their L1 cell distance from the camera's
 * level-0 cell, then, inside a cell, octree children nearest-first relative
 * to the camera.  For a point camera this order agrees with the order along
 * every pixel ray, so the outputs equal salf_render_rays' for the same camera
 * (the paper's splatting is allowed to approximate; this one does not).
 * Sensor: SALF_PINHOLE with one pose for the frame (rolling_shutter = 0 or
 * t1 <= t0); other sensors are rejected with SALF_ERR_INVALID.  Outputs as
 * for salf_render_rays, device memory only (on_host, ray_dump and steps are
 * rejected; visits/visit_count are supported).  The tile lists live in a
 * scene-owned workspace that grows on demand (cudaMalloc); calls on one scene
 * are serialised by a lock.  The call waits on `stream` once, for the number
 * of (voxel, tile) pairs, then enqueues the sort and the tile kernel and
 * returns.  `stats` (optional) receives the frame's counts.  Errors: INVALID,
 * OOM, CUDA; INVALID also when the sort key (tile index and camera-order key)
 * would need more than 64 bits.
 */
typedef struct {
  int64_t visible_voxels;  /* voxels listed in at least one tile */
  int64_t pairs;           /* (voxel, tile) list entries */
  int32_t tiles;           /* 16 x 16 tiles of the image */
  int32_t key_bits;        /* bits of the sort key (8 per radix pass) */
  int32_t kernels;         /* kernel launches of the call */
  int32_t reserved;
} salf_raster_stats;

salf_status salf_render_raster(salf_scene* scene, const salf_sensor* sensor,
                               const salf_render_opts* opts, const salf_outputs* out,
                               salf_raster_stats* stats, void* stream);

/*
 * Dynamic actors (Sec. IV-A).  An actor is a voxel set in its own canonical
 * frame, built as a scene with salf_build_scene (same device, dtype and field
 * mode as the static scene).  A request places each actor by pose0 / pose1:
 * canonical -> world 3x4 row-major maps at the sensor's t0 / t1.  A ray at
 * time fraction s of the exposure sees the actor at the pose interpolated
 * like the sensor's (linear translation, geodesic rotation); for sensors
 * without per-ray time, s = 0.  Per ray, the static voxels' hits and every
 * actor's hits are composited together in order of entry (Eq. 3-4, early
 * termination; the static hit first on ties).  An actor hit's field (Eq. 1-2,
 * 5-6) uses the actor's canonical frame for its local coordinates and for the
 * SH view direction.  The boxes of the actors' voxels must be pairwise
 * disjoint at t0 and at t1 (SALF_ERR_OVERLAP otherwise), so along a ray at
 * most one actor is open at a time.  A ray keeps the 8 nearest actor boxes it
 * meets (more sets a device status bit, see salf_scene_check).
 * Outputs as for salf_render_rays, device memory only (visits report actor
 * voxels as id_base + the voxel's input index in its actor scene).  The actor
 * table travels in a scene-owned device buffer (grown on demand; calls on one
 * scene are ordered on the GPU).  Asynchronous on `stream`.  Errors: INVALID
 * (sizes, more than SALF_MAX_ACTORS actors, null or mismatched actor scenes),
 * OVERLAP, OOM, CUDA.
 */
#define SALF_MAX_ACTORS 256

typedef struct {
  const salf_scene* actor;      /* voxels in the actor's canonical frame */
  double pose0[12], pose1[12];  /* canonical -> world at the sensor's t0 / t1 */
  int32_t id_base;              /* visit id offset of this actor's voxels */
  int32_t reserved;
} salf_actor;

salf_status salf_render_rays_actors(salf_scene* scene, const salf_actor* actors,
                                    int32_t n_actors, const salf_sensor* sensor,
                                    const salf_render_opts* opts, const salf_outputs* out,
                                    void* stream);

/*
 * Adjoint of salf_render_rays_actors (actors are fitted together with the
 * static scene, Sec. IV-A): the gradients of the merged walk's compositing,
 * transmittance recomputed front to back as in salf_render_backward.  `saved`
 * is the R x 8 array that salf_render_rays_actors wrote with the same scene,
 * actors, poses, sensor and options; d_rgb, d_depth, d_opacity, d_intensity
 * are dL/d(outputs) as for salf_render_backward (raydrop is not part of the
 * actor render).  d_params (static scene, n x 32 FP32, input order, device;
 * NULL = the scene's own gradient buffer, see salf_scene_params) and
 * actor_d_params[k] (actor k's n_k x 32 FP32, input order of its voxels,
 * device; a NULL array or entry = no gradient for that actor) are
 * ACCUMULATED (+=); all 16-byte aligned.  The per-call actor table and tile
 * lists live in the scene-owned actor workspace (calls on one scene are
 * ordered on the GPU).  Asynchronous on `stream`.  Errors: INVALID, OVERLAP,
 * OOM, CUDA.
 */
salf_status salf_render_backward_actors(salf_scene* scene, const salf_actor* actors,
                                        int32_t n_actors, const salf_sensor* sensor,
                                        const salf_render_opts* opts, const float* saved,
                                        const float* d_rgb, const float* d_depth,
                                        const float* d_opacity, const float* d_intensity,
                                        float* d_params, float* const* actor_d_params,
                                        void* stream);

/*
 * Densification and pruning (Sec. III-C), in two calls.
 * salf_scene_refine_plan decides per voxel, from `grads` (n x 32 FP32,
 * dL/d(record scalars), input order, device, 16-byte aligned) and
 * `max_alpha` (n FP32, input order, device: e.g. salf_outputs.max_alpha of
 * the training renders):
 *   - prune if max_alpha < prune_alpha (the paper uses 0.001);
 *   - else split into 8 octree children if the voxel is above the finest
 *     level and the L1 norm of its colour-field gradient (record slots 4..12,
 *     W_c) exceeds split_threshold;
 *   - else keep.
 * It waits on `stream` and returns the counts (n_new = n_kept + 8 n_split).
 * salf_scene_refine_apply then writes the new voxel list, in input order with
 * children (order 0..7: bits x | y << 1 | z << 2 pick the upper halves) in
 * place of their parent: level_out (n_new), ijk_out (n_new x 3), params_out
 * (n_new x 32 FP32, 16-byte aligned), all device memory, from `params` (the
 * current n x 32 FP32 records, input order, device, 16-byte aligned).  A
 * child's record carries its parent's fields exactly (all fields are affine
 * in the local coordinates: slopes halve, offsets take W.o/2, the colour rows'
 * share goes to their SH DC term).  The result is a voxel set for
 * salf_build_scene (same grid).  Asynchronous on `stream`.  The plan lives in
 * a scene-owned workspace until the next plan.  Errors: INVALID (null or
 * misaligned pointers, apply without a plan), OOM, CUDA.
 */
typedef struct {
  int64_t n_new, n_kept, n_split, n_pruned;
} salf_refine_counts;

salf_status salf_scene_refine_plan(salf_scene* scene, const float* grads, const float* max_alpha,
                                   float split_threshold, float prune_alpha,
                                   salf_refine_counts* counts, void* stream);
salf_status salf_scene_refine_apply(salf_scene* scene, const float* params, uint8_t* level_out,
                                    int32_t* ijk_out, float* params_out, void* stream);

/*
 * L_reg of Eq. 7 over the face-adjacent voxel pairs of the scene, from the
 * records `params` (n x 32 FP32, input order, device, 16-byte aligned):
 *   sum over pairs (i, j) of lambda_s |s_i - s_j| + lambda_alpha |alpha_i -
 *   alpha_j| + lambda_n (1 - n_i . n_j),
 * where, at the centre of the shared face (the smaller voxel's face), s_k is
 * the geometry field W_k . [x_k, 1] (record slots 0..3: W_sigma or W_s),
 * alpha_k = 1 - exp(-sigma_k l) with sigma_k its density (Eq. 1 or Eq. 6) and
 * l the smaller voxel's edge in metres, and n_k = W_k[0:3] / |W_k[0:3]| (0 if
 * that is 0).  *loss (one float, device) and grads (n x 32 FP32, input order,
 * device) are ACCUMULATED (+=); |.| takes sign(0) = 0 as its slope.
 * Asynchronous on `stream`.  Errors: INVALID, CUDA.
 */
salf_status salf_scene_reg_loss(salf_scene* scene, const float* params, float lambda_s,
                                float lambda_alpha, float lambda_n, float* loss, float* grads,
                                void* stream);

/*
 * Secondary rays (Sec. V-C and Fig. 1 name refraction, reflection and
 * shadows among the effects ray casting through the voxels supports; the
 * paper gives no construction, this is the library's).  For primary ray i of `sensor` (the
 * sensor of an earlier salf_render_rays, same ray generation), with that
 * render's depth D_i = sum w t_m and opacity O_i = sum w (device, R floats):
 *   - no secondary ray (direction 0, an invalid explicit ray) unless the ray
 *     is valid and O_i >= min_opacity;
 *   - hit point X = o + (D_i / O_i) d, the expected termination distance;
 *   - no secondary ray unless X lies inside a voxel whose geometry slopes
 *     g = W[0:3] (record slots 0..2: W_sigma or W_s) are not all 0;
 *   - surface normal n = -g / |g| (the field grows into the surface for
 *     both Eq. 1 and Eq. 6), turned to face the incoming ray (n . d <= 0);
 *   - REFLECT: r = d - 2 (d . n) n, origin X + offset n;
 *     REFRACT (Snell, eta = n_incident / n_transmitted): with c = -d . n and
 *     k = 1 - eta^2 (1 - c^2), r = eta d + (eta c - sqrt(k)) n, origin
 *     X - offset n; k < 0 (total internal reflection) gives the reflection;
 *     SHADOW: r = light_dir / |light_dir| (toward a distant light), origin
 *     X + offset n.
 * rays_out (R x 8 FP32, device, 16-byte aligned) gets (origin, r, 0, t_far),
 * the salf_sensor explicit-ray layout: render them with SALF_RAYS_EXPLICIT
 * (their opacity is the shadow's occlusion; their colour the reflected or
 * refracted light).  Asynchronous on `stream`.  Errors: INVALID (null or
 * misaligned pointers, kind, eta <= 0, zero light direction, min_opacity
 * outside (0, 1], offset < 0), CUDA.
 */
typedef enum {
  SALF_SECONDARY_REFLECT = 0,
  SALF_SECONDARY_REFRACT = 1,
  SALF_SECONDARY_SHADOW = 2
} salf_secondary_kind;

typedef struct {
  int32_t kind;
  float eta;
  float light_dir[3];
  float min_opacity;
  float offset;  /* metres */
  float t_far;   /* secondary ray length; <= 0: unbounded */
} salf_secondary_opts;

salf_status salf_secondary_rays(salf_scene* scene, const salf_sensor* sensor, const float* depth,
                                const float* opacity, const salf_secondary_opts* opts,
                                float* rays_out, void* stream);

/* Check the scene's device status word (synchronises the device).  Returns
 * SALF_ERR_DEVICE if a kernel hit an internal bound since the last check. */
salf_status salf_scene_check(salf_scene* scene);

/*
 * Scene files (checkpoint / resume of a scene; the paper stores trained
 * scenes, Sec. III-A: voxel keys and their records).  salf_scene_save writes
 * the scene's grid (origin, s0, dims, max_level), field mode, storage dtype,
 * the voxel keys (level, ijk) in input order and the current records in input
 * order, in the storage dtype (FP32, or BF16 bits), to `path` (binary,
 * little-endian; layout in csrc/checkpoint.cpp).  It waits for the device
 * (every stream's work on the records ends first).  salf_scene_load reads
 * such a file and builds the scene on ctx's device as salf_build_scene would
 * from the same arrays: the same voxels, records (bit for bit) and outputs.
 * The library keeps each scene's keys for this (13 bytes per voxel of device
 * memory, counted in device_bytes).  Errors: INVALID (null arguments), IO
 * (cannot open, read or write; wrong magic, version or size), and those of
 * salf_build_scene (load) or CUDA (save).
 */
salf_status salf_scene_save(const salf_scene* scene, const char* path);
salf_status salf_scene_load(salf_ctx* ctx, const char* path, salf_scene** out);

/*
 * Serving: a host scheduler thread batches requests from many sensors over
 * one resident scene.  mem_budget_bytes bounds the device memory of in-flight
 * requests (outputs); a request waits until its outputs fit (admission by
 * memory).  Whenever one of the n_streams streams is idle, the oldest waiting
 * request opens a batch, and waiting requests of the same kernel class join
 * it in arrival order (up to 24 per launch): pinhole cameras and explicit
 * rays; fisheye cameras and panoramas; spinning LiDARs (span-parallel rays).
 * Batches of different classes run side by side on different streams, so
 * requests that arrive while others run start without waiting for them to
 * finish.  Each request's outputs are identical to a lone salf_render_rays
 * call (rays are independent; no cross-ray reductions).
 * Statistics: p50 / p99 / max latency (submit -> completion) over the last
 * 65,536 completions; launches, requests launched (their ratio is the mean
 * batch size), the largest batch, and launches that mixed sensor kinds.
 */
typedef struct {
  int64_t submitted, completed, rejected;
  int64_t launches;
  int64_t rays;
  double p50_ms, p99_ms, max_ms;  /* submit -> completion, recent completions */
  int64_t peak_bytes;
  int64_t requests_launched;      /* sum over launches of the requests each carried */
  int64_t max_batch;              /* most requests one launch carried */
  int64_t mixed_launches;         /* launches carrying more than one sensor kind */
  int64_t latency_window;         /* completions the percentiles are taken over */
} salf_serve_stats;

salf_status salf_serve_create(salf_scene* scene, size_t mem_budget_bytes, int32_t n_streams,
                              salf_server** out);
/* Non-blocking.  The sensor descriptor is copied; explicit rays must stay
 * valid (device memory) until the request completes.  Errors: INVALID (bad
 * sensor, or outputs larger than the whole budget), SHUTDOWN. */
salf_status salf_serve_submit(salf_server* srv, const salf_sensor* sensor,
                              const salf_render_opts* opts, uint64_t* ticket);
/* Wait up to timeout_ms (0 = just look, < 0 = forever) for `ticket`.  On
 * completion *done = 1 and `result` receives device pointers into library-
 * owned memory (rgb, depth, opacity, intensity, valid; saved = NULL), valid
 * until salf_serve_release.  Returns TIMEOUT if not done in time (with
 * *done = 0), NOT_FOUND for unknown tickets. */
salf_status salf_serve_poll(salf_server* srv, uint64_t ticket, int32_t timeout_ms,
                            salf_outputs* result, int32_t* done);
salf_status salf_serve_release(salf_server* srv, uint64_t ticket);
salf_status salf_serve_get_stats(salf_server* srv, salf_serve_stats* stats);
/* hold != 0: admit nothing (submitted requests queue); hold = 0: resume.
 * Requests submitted under a hold start together when it is lifted, e.g. all
 * sensors of one time step, so that they share launches. */
salf_status salf_serve_hold(salf_server* srv, int32_t hold);
/* Stops accepting requests, waits for in-flight work, frees everything. */
void salf_serve_destroy(salf_server* srv);

/* Bytes of kernel parameters that one render launch carries from the host:
 * the batch descriptor (scene view and request descriptors, prepared in FP64
 * on the host).  Rays are generated on the device and the scene is resident,
 * so this is all a device-output render sends to the GPU. */
size_t salf_launch_param_bytes(void);

/* Measurement utility, not part of the method: the read bandwidth of this
 * GPU's L2 in GB/s, from `reps` streaming reads of a `bytes`-long device buffer
 * that the call allocates, fills and frees (bytes in [1 MiB, 4 GiB]; a buffer
 * smaller than L2 stays resident after the warm-up reads).  The render kernels
 * take most of their record and structure bytes from L1 and L2, so their L2
 * traffic is reported against this figure.  Synchronous.  Errors: INVALID, CUDA. */
salf_status salf_measure_l2_read(int32_t device, int64_t bytes, int32_t reps, double* gbs);

/* Thread-local message of the last failing call on this thread. */
const char* salf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
