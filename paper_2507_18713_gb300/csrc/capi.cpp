// capi.cpp -- C-ABI entry points of libsalf (declared in include/salf.h):
// context, scene lifetime, request preparation (done in FP64 on the host),
// render / adjoint dispatch, host-memory staging.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <string>

#include "salf_internal.h"

namespace {
thread_local std::string g_err;
}

void salf_set_error(const std::string& msg) { g_err = msg; }

salf_status salf_cuda_fail(cudaError_t e, const char* what) {
  g_err = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? SALF_ERR_OOM : SALF_ERR_CUDA;
}

extern "C" const char* salf_last_error(void) { return g_err.c_str(); }

extern "C" size_t salf_launch_param_bytes(void) { return sizeof(LaunchParams); }

extern "C" salf_status salf_create(int32_t device, salf_ctx** out) {
  if (!out) {
    g_err = "salf_create: null out";
    return SALF_ERR_INVALID;
  }
  *out = nullptr;
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess) return salf_cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= count) {
    g_err = "salf_create: no such device";
    return SALF_ERR_INVALID;
  }
  if ((e = cudaSetDevice(device)) != cudaSuccess) return salf_cuda_fail(e, "cudaSetDevice");
  // the no-alloc entry point's fixed staging array becomes resident here
  const salf_status st = salf_noalloc_setup(device);
  if (st != SALF_OK) return st;
  salf_ctx* c = new salf_ctx();
  c->device = device;
  *out = c;
  return SALF_OK;
}

extern "C" void salf_destroy(salf_ctx* ctx) { delete ctx; }

extern "C" salf_status salf_build_scene(salf_ctx* ctx, const salf_scene_desc* desc,
                                        salf_scene** out) {
  SALF_RANGE("salf_build_scene");
  salf_status st = salf_build_scene_impl(ctx, desc, out);
  if (st != SALF_OK) return st;
  // the keys stay with the scene so that salf_scene_save can write it out
  st = salf_scene_keep_keys(*out, desc);
  if (st != SALF_OK) {
    salf_scene_destroy(*out);
    *out = nullptr;
  }
  return st;
}

extern "C" void salf_scene_destroy(salf_scene* s) {
  if (!s) return;
  cudaSetDevice(s->device);
  cudaDeviceSynchronize();
  for (void* p : s->allocations) cudaFree(p);
  if (s->staging) cudaFree(s->staging);
  if (s->grads) cudaFree(s->grads);
  if (s->raster_vox) cudaFree(s->raster_vox);
  if (s->raster_pairs) cudaFree(s->raster_pairs);
  if (s->raster_count_host) cudaFreeHost(s->raster_count_host);
  if (s->raster_done) cudaEventDestroy(s->raster_done);
  if (s->actor_buf) cudaFree(s->actor_buf);
  if (s->refine_ws) cudaFree(s->refine_ws);
  if (s->refine_host) cudaFreeHost(s->refine_host);
  if (s->actor_done) cudaEventDestroy(s->actor_done);
  if (s->actor_fork) cudaEventDestroy(s->actor_fork);
  if (s->actor_join) cudaEventDestroy(s->actor_join);
  if (s->actor_aux) cudaStreamDestroy(s->actor_aux);
  delete s;
}

extern "C" salf_status salf_scene_get_info(const salf_scene* s, salf_scene_info* info) {
  if (!s || !info) {
    g_err = "salf_scene_get_info: null argument";
    return SALF_ERR_INVALID;
  }
  std::memset(info, 0, sizeof(*info));
  info->n = s->n;
  info->mode = s->mode;
  info->dtype = s->dtype;
  info->max_level = s->K;
  for (int a = 0; a < 3; ++a) info->dims[a] = s->dims[a];
  info->n_level0_cells = s->n_cells0;
  info->n_nodes = s->n_nodes;
  info->device_bytes = s->device_bytes;
  info->dev_params = s->dev.params;
  info->dev_order = s->dev.order;
  return SALF_OK;
}

extern "C" salf_status salf_scene_params(salf_scene* s, void** dev_params, void** dev_grads) {
  if (!s) {
    g_err = "salf_scene_params: null scene";
    return SALF_ERR_INVALID;
  }
  if (dev_params) *dev_params = const_cast<void*>(s->dev.params);
  if (!dev_grads) return SALF_OK;
  std::lock_guard<std::mutex> lk(s->grads_mu);
  if (!s->grads) {
    cudaError_t e;
    if ((e = cudaSetDevice(s->device)) != cudaSuccess) return salf_cuda_fail(e, "cudaSetDevice");
    const size_t bytes = (size_t)(s->n > 0 ? s->n : 1) * SALF_RECORD_SCALARS * sizeof(float);
    float* g = nullptr;
    if ((e = cudaMalloc(&g, bytes)) != cudaSuccess) return salf_cuda_fail(e, "cudaMalloc(grads)");
    if ((e = cudaMemset(g, 0, bytes)) != cudaSuccess) {
      cudaFree(g);
      return salf_cuda_fail(e, "cudaMemset(grads)");
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
      cudaFree(g);
      return salf_cuda_fail(e, "cudaMemset(grads)");
    }
    s->grads = g;
  }
  *dev_grads = s->grads;
  return SALF_OK;
}

extern "C" salf_status salf_scene_check(salf_scene* s) {
  if (!s) {
    g_err = "salf_scene_check: null scene";
    return SALF_ERR_INVALID;
  }
  cudaError_t e;
  if ((e = cudaSetDevice(s->device)) != cudaSuccess) return salf_cuda_fail(e, "cudaSetDevice");
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return salf_cuda_fail(e, "kernel");
  int flag = 0;
  if ((e = cudaMemcpy(&flag, s->dev.status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return salf_cuda_fail(e, "cudaMemcpy(status)");
  if (flag) {
    cudaMemset(s->dev.status, 0, sizeof(int));
    g_err = "device status word " + std::to_string(flag) +
            ((flag & SALF_DEVERR_STEP_CAP) ? " (traversal step bound reached)" : "") +
            ((flag & SALF_DEVERR_SDF_AB) ? " (SDF record with a <= 0 or b <= 0)" : "") +
            ((flag & SALF_DEVERR_ACTOR_CAP) ? " (a ray met more actor boxes than it holds)" : "") +
            ((flag & SALF_DEVERR_BOUNDS) ? " (an adjoint index outside its buffers, skipped)" : "");
    return SALF_ERR_DEVICE;
  }
  return SALF_OK;
}

// Grow the scene's staging buffer (caller holds staging_mu).
static salf_status ensure_staging(salf_scene* s, size_t bytes) {
  if (s->staging_bytes >= bytes) return SALF_OK;
  if (s->staging) {
    cudaDeviceSynchronize();
    cudaFree(s->staging);
    s->staging = nullptr;
    s->staging_bytes = 0;
  }
  cudaError_t e = cudaMalloc(&s->staging, bytes);
  if (e != cudaSuccess) {
    s->staging = nullptr;
    return salf_cuda_fail(e, "cudaMalloc(staging)");
  }
  s->staging_bytes = bytes;
  return SALF_OK;
}

extern "C" salf_status salf_scene_update_params(salf_scene* s, const float* params,
                                                int32_t on_device, void* stream) {
  SALF_RANGE("salf_scene_update_params");
  if (!s || (!params && s->n > 0)) {
    g_err = "salf_scene_update_params: null argument";
    return SALF_ERR_INVALID;
  }
  if (s->n == 0) return SALF_OK;
  if (reinterpret_cast<uintptr_t>(params) & 15u) {
    g_err = "salf_scene_update_params: params must be 16-byte aligned";
    return SALF_ERR_INVALID;
  }
  cudaError_t e;
  if ((e = cudaSetDevice(s->device)) != cudaSuccess) return salf_cuda_fail(e, "cudaSetDevice");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (on_device) {
    e = salf_launch_gather_params(params, s->dev.order, const_cast<void*>(s->dev.params), s->n,
                                  s->dtype, s->mode, s->dev.status, st);
    if (e != cudaSuccess) return salf_cuda_fail(e, "gather params");
    return SALF_OK;
  }
  std::lock_guard<std::mutex> lk(s->staging_mu);
  const size_t bytes = (size_t)s->n * 128;
  salf_status rs = ensure_staging(s, bytes);
  if (rs != SALF_OK) return rs;
  if ((e = cudaMemcpyAsync(s->staging, params, bytes, cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return salf_cuda_fail(e, "cudaMemcpyAsync(params)");
  e = salf_launch_gather_params(static_cast<const float*>(s->staging), s->dev.order,
                                const_cast<void*>(s->dev.params), s->n, s->dtype, s->mode,
                                s->dev.status, st);
  if (e != cudaSuccess) return salf_cuda_fail(e, "gather params");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return salf_cuda_fail(e, "sync");
  return SALF_OK;
}

// ------------------------------------------------------------ requests

static void mat_to_quat(const double* P, double q[4]) {
  // rotation block of a row-major 3x4 [R|t] -> (w, x, y, z), Shoemake's
  // branch on the largest diagonal term
  const double r00 = P[0], r01 = P[1], r02 = P[2], r10 = P[4], r11 = P[5], r12 = P[6],
               r20 = P[8], r21 = P[9], r22 = P[10];
  const double tr = r00 + r11 + r22;
  if (tr > 0) {
    const double s = 2.0 * std::sqrt(tr + 1.0);
    q[0] = 0.25 * s;
    q[1] = (r21 - r12) / s;
    q[2] = (r02 - r20) / s;
    q[3] = (r10 - r01) / s;
  } else if (r00 > r11 && r00 > r22) {
    const double s = 2.0 * std::sqrt(1.0 + r00 - r11 - r22);
    q[0] = (r21 - r12) / s;
    q[1] = 0.25 * s;
    q[2] = (r01 + r10) / s;
    q[3] = (r02 + r20) / s;
  } else if (r11 > r22) {
    const double s = 2.0 * std::sqrt(1.0 + r11 - r00 - r22);
    q[0] = (r02 - r20) / s;
    q[1] = (r01 + r10) / s;
    q[2] = 0.25 * s;
    q[3] = (r12 + r21) / s;
  } else {
    const double s = 2.0 * std::sqrt(1.0 + r22 - r00 - r11);
    q[0] = (r10 - r01) / s;
    q[1] = (r02 + r20) / s;
    q[2] = (r12 + r21) / s;
    q[3] = 0.25 * s;
  }
  const double nn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int k = 0; k < 4; ++k) q[k] /= nn;
}

// Relative rotation R1 R0^T of two 3x4 poses as (world axis, angle), the
// shortest way round: the slerp geodesic from R0 to R1 is
// R(s) = rot(axis, s * angle) R0.
void salf_relative_rotation(const double* pose0, const double* pose1, float axis[3],
                            float* angle) {
  double Rr[12] = {0};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += pose1[4 * i + k] * pose0[4 * j + k];
      Rr[4 * i + j] = acc;
    }
  double q[4];
  mat_to_quat(Rr, q);
  if (q[0] < 0)
    for (int k = 0; k < 4; ++k) q[k] = -q[k];
  const double vn = std::sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  *angle = vn > 0 ? (float)(2.0 * std::atan2(vn, q[0])) : 0.f;
  for (int k = 0; k < 3; ++k) axis[k] = vn > 0 ? (float)(q[k + 1] / vn) : 0.f;
}

// Tile row whose centre-column ray is closest to horizontal in the world
// (launch-order heuristic only: near-horizontal rays are the longest in
// driving scenes; it never changes a result).
static int horizon_tile_row(const salf_sensor* s, int tile_h, int tiles_y) {
  if (s->kind == SALF_RAYS_EXPLICIT || tiles_y <= 1) return 0;
  int best = 0;
  double best_z = 2.0;
  for (int ty = 0; ty < tiles_y; ++ty) {
    const double v = std::min((double)s->height - 0.5, ty * tile_h + 0.5 * tile_h);
    double d[3];
    if (s->kind == SALF_LIDAR_SPIN) {
      const double e = s->elev_max - (s->height > 1 ? (v - 0.5) * ((double)s->elev_max - s->elev_min) /
                                                         (s->height - 1) : 0.0);
      d[0] = std::cos(e);
      d[1] = 0.0;
      d[2] = std::sin(e);
    } else if (s->kind == SALF_PANO_EQUIRECT) {
      const double lat = s->elev_max - (v / s->height) * ((double)s->elev_max - s->elev_min);
      d[0] = 0.0;
      d[1] = -std::sin(lat);
      d[2] = std::cos(lat);
    } else {
      const double my = (v - s->cy) / s->fy;
      if (s->kind == SALF_FISHEYE_EQUIDIST) {
        const double th = std::fabs(my);
        d[0] = 0.0;
        d[1] = (my < 0 ? -1.0 : 1.0) * std::sin(th);
        d[2] = std::cos(th);
      } else {
        d[0] = 0.0;
        d[1] = my;
        d[2] = 1.0;
      }
    }
    const double wz = s->pose0[8] * d[0] + s->pose0[9] * d[1] + s->pose0[10] * d[2];
    const double nn = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const double z = std::fabs(wz / nn);
    if (z < best_z) {
      best_z = z;
      best = ty;
    }
  }
  return best;
}

int64_t salf_request_rays(const salf_sensor* sen) {
  return (int64_t)sen->width * (int64_t)sen->height;
}

salf_status salf_prepare_request(const salf_scene* sc, const salf_sensor* s,
                                 const salf_render_opts* o, ReqDev* r) {
  std::memset(r, 0, sizeof(*r));
  if (s->kind < SALF_PINHOLE || s->kind > SALF_RAYS_EXPLICIT || s->width <= 0 || s->height <= 0 ||
      (int64_t)s->width * s->height > (int64_t)0x7fffffff) {
    g_err = "sensor: bad kind or size";
    return SALF_ERR_INVALID;
  }
  if ((s->kind == SALF_PINHOLE || s->kind == SALF_FISHEYE_EQUIDIST) &&
      !(s->fx > 0 && s->fy > 0 && std::isfinite(s->cx) && std::isfinite(s->cy))) {
    g_err = "sensor: focal lengths must be > 0";
    return SALF_ERR_INVALID;
  }
  if (s->kind == SALF_RAYS_EXPLICIT && (!s->rays || (reinterpret_cast<uintptr_t>(s->rays) & 15u))) {
    g_err = "sensor: explicit rays need a 16-byte aligned array";
    return SALF_ERR_INVALID;
  }
  if (!(s->t_near >= 0) || !(o->t_min_transmittance >= 0) || o->visits_cap < 0) {
    g_err = "sensor/options: t_near and t_min must be >= 0";
    return SALF_ERR_INVALID;
  }
  r->kind = s->kind;
  r->W = s->width;
  r->H = s->height;
  r->inv_fx = s->fx > 0 ? (float)(1.0 / (double)s->fx) : 0.f;
  r->inv_fy = s->fy > 0 ? (float)(1.0 / (double)s->fy) : 0.f;
  r->cx = s->cx;
  r->cy = s->cy;
  r->half_fov = 0.5f * s->fov;
  r->elev_min = s->elev_min;
  r->elev_max = s->elev_max;
  r->elev_step = s->height > 1 ? (float)(((double)s->elev_max - (double)s->elev_min) / (s->height - 1)) : 0.f;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) r->R0[3 * i + j] = (float)s->pose0[4 * i + j];
  {
    double p0[12], p1[12];
    for (int k = 0; k < 12; ++k) {
      p0[k] = s->pose0[k];
      p1[k] = s->pose1[k];
    }
    salf_relative_rotation(p0, p1, r->rel_axis, &r->rel_angle);
  }
  const bool timed = s->t1 > s->t0;
  r->moving = (s->kind == SALF_LIDAR_SPIN && timed) ||
              ((s->kind <= SALF_PANO_EQUIRECT) && s->rolling_shutter && timed && s->height > 1);
  const double inv_sfin = 1.0 / sc->sfin;
  for (int a = 0; a < 3; ++a) {
    const double g0 = (s->pose0[4 * a + 3] - sc->origin[a]) * inv_sfin;
    const double g1 = (s->pose1[4 * a + 3] - sc->origin[a]) * inv_sfin;
    const double f = std::floor(g0);
    if (!std::isfinite(g0) || !std::isfinite(g1) || std::fabs(g0) > 8.0e6 || std::fabs(g1) > 8.0e6) {
      g_err = "sensor: pose translation too far from the scene grid";
      return SALF_ERR_INVALID;
    }
    r->Oi[a] = (int)f;
    r->Of[a] = (float)(g0 - f);
    r->dO[a] = (float)(g1 - g0);
  }
  r->t_near = s->t_near;
  r->t_far = s->t_far > 0 ? s->t_far : std::numeric_limits<float>::infinity();
  r->time0 = (float)s->t0;
  r->time1 = (float)s->t1;
  r->rays = s->rays;
  r->t_min = o->t_min_transmittance;
  for (int k = 0; k < 3; ++k) r->bg[k] = o->background[k];
  r->want_int = o->want_intensity ? 1 : 0;
  r->vcap = o->visits_cap;
  int segs = o->ray_segments;
  if (segs == 0) segs = o->visits_cap > 0 ? 1 : salf_auto_segments(s->kind);
  if (segs != 1 && segs != 2 && segs != 4 && segs != 8) {
    g_err = "options: ray_segments must be 0, 1, 2, 4 or 8";
    return SALF_ERR_INVALID;
  }
  salf_request_tiling(r, s, o->visits_cap > 0 ? 0 : __builtin_ctz((unsigned)segs));
  return SALF_OK;
}

int salf_auto_segments(int kind) {
  switch (kind) {
    case SALF_LIDAR_SPIN: return SALF_SEGMENTS_LIDAR;
    case SALF_FISHEYE_EQUIDIST: return SALF_SEGMENTS_FISHEYE;
    case SALF_PANO_EQUIRECT: return SALF_SEGMENTS_PANORAMA;
    default: return 1;
  }
}

void salf_request_tiling(ReqDev* r, const salf_sensor* s, int seg_shift) {
  if (s->kind == SALF_RAYS_EXPLICIT || s->height == 1) {
    r->tile_w = 32;
    r->tile_h = 1;
  } else if (s->kind == SALF_LIDAR_SPIN) {
    // 4 azimuths x 8 beams per warp: measured faster than 8 x 4 for spinning LiDARs
    r->tile_w = 4;
    r->tile_h = 8;
  } else {
    r->tile_w = SALF_TILE_W;
    r->tile_h = SALF_TILE_H;
  }
  // a warp holds 32 >> seg_shift rays: fewer columns first, then fewer rows
  for (int k = 0; k < seg_shift; ++k) {
    if (r->tile_w > 1)
      r->tile_w >>= 1;
    else
      r->tile_h >>= 1;
  }
  if (s->kind == SALF_LIDAR_SPIN && seg_shift > 0 && s->height > 1) {
    r->tile_w = std::min(SALF_SEG_LIDAR_TILE_W, 32 >> seg_shift);
    r->tile_h = (32 >> seg_shift) / r->tile_w;
  }
  r->seg_shift = seg_shift;
  r->tiles_x = (s->width + r->tile_w - 1) / r->tile_w;
  r->tiles_y = (s->height + r->tile_h - 1) / r->tile_h;
  r->n_tiles = r->tiles_x * r->tiles_y;
  r->first_row = horizon_tile_row(s, r->tile_h, r->tiles_y);
}

static salf_render_opts default_opts() {
  salf_render_opts o;
  std::memset(&o, 0, sizeof(o));
  o.t_min_transmittance = 1e-4f;
  return o;
}

static bool misaligned(const void* p, unsigned a) {
  return p && (reinterpret_cast<uintptr_t>(p) & (a - 1));
}

extern "C" salf_status salf_render_rays(salf_scene* sc, const salf_sensor* sen,
                                        const salf_render_opts* opts, const salf_outputs* out,
                                        void* stream) {
  SALF_RANGE("salf_render_rays");
  if (!sc || !sen || !out) {
    g_err = "salf_render_rays: null argument";
    return SALF_ERR_INVALID;
  }
  const salf_render_opts o = opts ? *opts : default_opts();
  if (!out->rgb && !out->depth && !out->opacity && !out->intensity && !out->saved && !out->valid &&
      !(o.visits_cap > 0 && out->visits) && !out->ray_dump && !out->steps && !out->raydrop) {
    g_err = "salf_render_rays: no output requested";
    return SALF_ERR_INVALID;
  }
  if (o.visits_cap > 0 && (!out->visits || !out->visit_count)) {
    g_err = "salf_render_rays: visits_cap > 0 needs visits and visit_count";
    return SALF_ERR_INVALID;
  }
  if (out->on_host < 0 || out->on_host > 2) {
    g_err = "salf_render_rays: on_host must be 0, 1 or 2";
    return SALF_ERR_INVALID;
  }
  if (out->on_host && (out->ray_dump || out->steps || out->max_alpha)) {
    g_err = "salf_render_rays: ray_dump, steps and max_alpha need device outputs";
    return SALF_ERR_INVALID;
  }
  if (!out->on_host && misaligned(out->saved, 16)) {
    g_err = "salf_render_rays: saved must be 16-byte aligned";
    return SALF_ERR_INVALID;
  }
  cudaError_t e;
  if ((e = cudaSetDevice(sc->device)) != cudaSuccess) return salf_cuda_fail(e, "cudaSetDevice");
  LaunchParams P;
  std::memset(&P, 0, sizeof(P));
  P.S = sc->dev;
  P.n_req = 1;
  ReqDev& r = P.req[0];
  salf_status st = salf_prepare_request(sc, sen, &o, &r);
  if (st != SALF_OK) return st;
  if (out->ray_dump || out->steps || out->max_alpha) salf_request_tiling(&r, sen, 0);
  P.total_tiles = r.n_tiles;
  const size_t R = (size_t)salf_request_rays(sen);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);

  if (!out->on_host) {
    r.rgb = out->rgb;
    r.depth = out->depth;
    r.opacity = out->opacity;
    r.intensity = out->intensity;
    r.saved = out->saved;
    r.valid = out->valid;
    r.vcount = out->visit_count;
    r.visits = out->visits;
    r.ray_dump = out->ray_dump;
    r.steps_out = out->steps;
    r.max_alpha = reinterpret_cast<unsigned*>(out->max_alpha);
    r.raydrop = out->raydrop;
    if ((e = salf_launch_forward(P, cs)) != cudaSuccess) return salf_cuda_fail(e, "forward launch");
    return SALF_OK;
  }

  const size_t vcap = (size_t)std::max(0, o.visits_cap);
  const size_t rays_bytes = sen->kind == SALF_RAYS_EXPLICIT ? R * 32 : 0;
  // Host outputs in page-locked memory the device can address (any
  // cudaHostAlloc / cudaHostRegister buffer under unified addressing): the
  // kernel writes them in place (over NVLink-C2C on Grace systems): no staging
  // buffer and no copy step.  Pageable buffers take the staging path below.
  {
    const void* hp[9] = {out->rgb,   out->depth,
                         out->opacity, out->intensity,
                         out->saved, out->valid,
                         vcap ? out->visit_count : nullptr, vcap ? out->visits : nullptr,
                         out->raydrop};
    void* dp[9] = {};
    bool direct = !misaligned(out->saved, 16);
    for (int i = 0; i < 9 && direct; ++i) {
      if (!hp[i]) continue;
      cudaPointerAttributes at;
      if (cudaPointerGetAttributes(&at, hp[i]) != cudaSuccess) {
        cudaGetLastError();
        direct = false;
      } else if (at.type != cudaMemoryTypeHost || !at.devicePointer) {
        direct = false;
      } else {
        dp[i] = at.devicePointer;
      }
    }
    if (direct && rays_bytes) {
      cudaPointerAttributes at;
      if (cudaPointerGetAttributes(&at, sen->rays) != cudaSuccess) {
        cudaGetLastError();
        direct = false;
      } else if (at.type == cudaMemoryTypeDevice) {
        r.rays = sen->rays;
      } else if (at.type == cudaMemoryTypeHost && at.devicePointer) {
        r.rays = static_cast<const float*>(at.devicePointer);
      } else {
        direct = false;
      }
    }
    if (direct) {
      r.rgb = static_cast<float*>(dp[0]);
      r.depth = static_cast<float*>(dp[1]);
      r.opacity = static_cast<float*>(dp[2]);
      r.intensity = static_cast<float*>(dp[3]);
      r.saved = static_cast<float*>(dp[4]);
      r.valid = static_cast<unsigned char*>(dp[5]);
      r.vcount = static_cast<int*>(dp[6]);
      r.visits = static_cast<int*>(dp[7]);
      r.raydrop = static_cast<float*>(dp[8]);
      if ((e = salf_launch_forward(P, cs)) != cudaSuccess)
        return salf_cuda_fail(e, "forward launch");
      if (out->on_host == 2) return SALF_OK;  // asynchronous: results once the stream drains
      if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) return salf_cuda_fail(e, "render");
      return SALF_OK;
    }
    if (out->on_host == 2) {
      g_err = "salf_render_rays: on_host = 2 needs page-locked host buffers the device can "
              "address (saved 16-byte aligned; explicit rays in device or page-locked memory)";
      return SALF_ERR_INVALID;
    }
    r.rays = sen->rays;
  }

  // Host outputs: render into staging, copy back, wait.
  std::lock_guard<std::mutex> lk(sc->staging_mu);
  size_t off[10], total = 0;
  const size_t sizes[10] = {out->rgb ? R * 12 : 0, out->depth ? R * 4 : 0, out->opacity ? R * 4 : 0,
                            out->intensity ? R * 4 : 0, out->saved ? R * 32 : 0,
                            out->valid ? R : 0, vcap ? R * 4 : 0, vcap ? R * vcap * 4 : 0,
                            rays_bytes, out->raydrop ? R * 4 : 0};
  for (int i = 0; i < 10; ++i) {
    off[i] = total;
    total += (sizes[i] + 255) & ~(size_t)255;
  }
  if ((st = ensure_staging(sc, total)) != SALF_OK) return st;
  char* base = static_cast<char*>(sc->staging);
  r.rgb = out->rgb ? reinterpret_cast<float*>(base + off[0]) : nullptr;
  r.depth = out->depth ? reinterpret_cast<float*>(base + off[1]) : nullptr;
  r.opacity = out->opacity ? reinterpret_cast<float*>(base + off[2]) : nullptr;
  r.intensity = out->intensity ? reinterpret_cast<float*>(base + off[3]) : nullptr;
  r.saved = out->saved ? reinterpret_cast<float*>(base + off[4]) : nullptr;
  r.valid = out->valid ? reinterpret_cast<unsigned char*>(base + off[5]) : nullptr;
  r.vcount = vcap ? reinterpret_cast<int*>(base + off[6]) : nullptr;
  r.visits = vcap ? reinterpret_cast<int*>(base + off[7]) : nullptr;
  r.raydrop = out->raydrop ? reinterpret_cast<float*>(base + off[9]) : nullptr;
  if (rays_bytes) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, sen->rays) == cudaSuccess && at.type == cudaMemoryTypeDevice) {
      r.rays = sen->rays;
    } else {
      cudaGetLastError();
      if ((e = cudaMemcpyAsync(base + off[8], sen->rays, rays_bytes, cudaMemcpyHostToDevice, cs)) !=
          cudaSuccess)
        return salf_cuda_fail(e, "cudaMemcpyAsync(rays)");
      r.rays = reinterpret_cast<const float*>(base + off[8]);
    }
  }
  if ((e = salf_launch_forward(P, cs)) != cudaSuccess) return salf_cuda_fail(e, "forward launch");
  struct Cp {
    void* dst;
    const void* src;
    size_t n;
  } cps[9] = {{out->rgb, r.rgb, sizes[0]},        {out->depth, r.depth, sizes[1]},
              {out->opacity, r.opacity, sizes[2]}, {out->intensity, r.intensity, sizes[3]},
              {out->saved, r.saved, sizes[4]},     {out->valid, r.valid, sizes[5]},
              {out->visit_count, r.vcount, sizes[6]}, {out->visits, r.visits, sizes[7]},
              {out->raydrop, r.raydrop, sizes[9]}};
  for (const Cp& c : cps) {
    if (!c.n || !c.dst) continue;
    if ((e = cudaMemcpyAsync(c.dst, c.src, c.n, cudaMemcpyDeviceToHost, cs)) != cudaSuccess)
      return salf_cuda_fail(e, "cudaMemcpyAsync(outputs)");
  }
  if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) return salf_cuda_fail(e, "render");
  return SALF_OK;
}

extern "C" salf_status salf_render_raster(salf_scene* sc, const salf_sensor* sen,
                                         const salf_render_opts* opts, const salf_outputs* out,
                                         salf_raster_stats* stats, void* stream) {
  SALF_RANGE("salf_render_raster");
  if (!sc || !sen || !out) {
    g_err = "salf_render_raster: null argument";
    return SALF_ERR_INVALID;
  }
  if (sen->kind != SALF_PINHOLE) {
    g_err = "salf_render_raster: pinhole cameras only";
    return SALF_ERR_INVALID;
  }
  if (sen->rolling_shutter && sen->t1 > sen->t0 && sen->height > 1) {
    g_err = "salf_render_raster: one camera pose per frame (no rolling shutter)";
    return SALF_ERR_INVALID;
  }
  if (sen->width > 65535 * 16 || sen->height > 65535 * 16) {
    g_err = "salf_render_raster: image too large";
    return SALF_ERR_INVALID;
  }
  const salf_render_opts o = opts ? *opts : default_opts();
  if (out->on_host || out->ray_dump || out->steps || out->raydrop) {
    g_err = "salf_render_raster: device outputs only (no ray_dump, steps or raydrop)";
    return SALF_ERR_INVALID;
  }
  if (!out->rgb && !out->depth && !out->opacity && !out->intensity && !out->saved && !out->valid &&
      !(o.visits_cap > 0 && out->visits)) {
    g_err = "salf_render_raster: no output requested";
    return SALF_ERR_INVALID;
  }
  if (o.visits_cap > 0 && (!out->visits || !out->visit_count)) {
    g_err = "salf_render_raster: visits_cap > 0 needs visits and visit_count";
    return SALF_ERR_INVALID;
  }
  if (misaligned(out->saved, 16)) {
    g_err = "salf_render_raster: saved must be 16-byte aligned";
    return SALF_ERR_INVALID;
  }
  cudaError_t e;
  if ((e = cudaSetDevice(sc->device)) != cudaSuccess) return salf_cuda_fail(e, "cudaSetDevice");
  ReqDev r;
  salf_status st = salf_prepare_request(sc, sen, &o, &r);
  if (st != SALF_OK) return st;
  salf_request_tiling(&r, sen, 0);  // this path walks whole rays
  r.rgb = out->rgb;
  r.depth = out->depth;
  r.opacity = out->opacity;
  r.intensity = out->intensity;
  r.saved = out->saved;
  r.valid = out->valid;
  r.vcount = out->visit_count;
  r.visits = out->visits;
  return salf_raster_run(sc, r, sen->fx, sen->fy, stats, static_cast<cudaStream_t>(stream));
}

// Oriented box: centre, unit axes (columns of the rotation), half extents.
struct Obb {
  double c[3], ax[3][3], h[3];
};

static Obb actor_obb(const salf_scene* a, const double* pose) {
  Obb b;
  double lo[3], hi[3], cl[3];
  for (int k = 0; k < 3; ++k) {
    lo[k] = a->origin[k] + a->dev.bmin[k] * a->sfin;
    hi[k] = a->origin[k] + a->dev.bmax[k] * a->sfin;
    cl[k] = 0.5 * (lo[k] + hi[k]);
    b.h[k] = 0.5 * (hi[k] - lo[k]);
  }
  for (int i = 0; i < 3; ++i) {
    b.c[i] = pose[4 * i + 3];
    for (int j = 0; j < 3; ++j) {
      b.c[i] += pose[4 * i + j] * cl[j];
      b.ax[j][i] = pose[4 * i + j];  // axis j = column j of the rotation
    }
  }
  return b;
}

// Separating-axis test of two oriented boxes (15 candidate axes); true if
// their interiors overlap by more than `tol` along every axis.
static bool obb_overlap(const Obb& A, const Obb& B, double tol) {
  double d[3];
  for (int k = 0; k < 3; ++k) d[k] = B.c[k] - A.c[k];
  auto dot = [](const double* u, const double* v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; };
  auto separated = [&](const double* L) {
    const double n = std::sqrt(dot(L, L));
    if (n < 1e-12) return false;  // degenerate (parallel edges): covered by the face axes
    double ra = 0, rb = 0;
    for (int k = 0; k < 3; ++k) {
      ra += A.h[k] * std::fabs(dot(A.ax[k], L));
      rb += B.h[k] * std::fabs(dot(B.ax[k], L));
    }
    return std::fabs(dot(d, L)) >= ra + rb - tol * n;
  };
  for (int k = 0; k < 3; ++k)
    if (separated(A.ax[k]) || separated(B.ax[k])) return false;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      const double* u = A.ax[i];
      const double* v = B.ax[j];
      const double L[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2],
                           u[0] * v[1] - u[1] * v[0]};
      if (separated(L)) return false;
    }
  return true;
}

// Checks of an actor list (shared by the forward and the adjoint): every actor
// scene matches the static scene's device, dtype and field mode, poses are
// finite, and the actors' boxes are pairwise disjoint at t0 and at t1.
static salf_status check_actors(const salf_scene* sc, const salf_actor* actors, int32_t n_actors,
                                const char* who) {
  for (int k = 0; k < n_actors; ++k) {
    const salf_scene* a = actors[k].actor;
    if (!a || a->device != sc->device || a->dtype != sc->dtype || a->mode != sc->mode) {
      g_err = std::string(who) + ": actor " + std::to_string(k) +
              " is null or differs from the scene in device, dtype or field mode";
      return SALF_ERR_INVALID;
    }
    for (int q = 0; q < 12; ++q)
      if (!std::isfinite(actors[k].pose0[q]) || !std::isfinite(actors[k].pose1[q])) {
        g_err = std::string(who) + ": non-finite actor pose";
        return SALF_ERR_INVALID;
      }
  }
  // actor boxes pairwise disjoint at t0 and at t1
  for (int i = 0; i < n_actors; ++i) {
    if (actors[i].actor->n == 0) continue;
    for (int j = i + 1; j < n_actors; ++j) {
      if (actors[j].actor->n == 0) continue;
      for (int t = 0; t < 2; ++t) {
        const double* pi = t ? actors[i].pose1 : actors[i].pose0;
        const double* pj = t ? actors[j].pose1 : actors[j].pose0;
        if (obb_overlap(actor_obb(actors[i].actor, pi), actor_obb(actors[j].actor, pj), 1e-9)) {
          g_err = std::string(who) + ": boxes of actors " + std::to_string(i) + " and " +
                  std::to_string(j) + " overlap at t" + std::to_string(t);
          return SALF_ERR_OVERLAP;
        }
      }
    }
  }
  return SALF_OK;
}

// The actor table of one request (FP64 -> FP32 constants), skipping empty
// actors; actor k's adjoint buffer is dparams[k] when dparams is not null.
static std::vector<ActorDev> actor_table(const salf_actor* actors, int32_t n_actors,
                                         const salf_sensor* sen, const ReqDev& r,
                                         float* const* dparams) {
  // per-actor constants (FP64 -> FP32)
  std::vector<ActorDev> ad;
  ad.reserve((size_t)n_actors);
  double os0[3], os1[3];
  for (int a = 0; a < 3; ++a) {
    os0[a] = sen->pose0[4 * a + 3];
    os1[a] = r.moving ? sen->pose1[4 * a + 3] : os0[a];
  }
  for (int k = 0; k < n_actors; ++k) {
    const salf_scene* as = actors[k].actor;
    if (as->n == 0) continue;
    ActorDev A;
    std::memset(&A, 0, sizeof(A));
    A.S = as->dev;
    const double* p0 = actors[k].pose0;
    const double* p1 = actors[k].pose1;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) A.R0[3 * i + j] = (float)p0[4 * i + j];
    salf_relative_rotation(p0, p1, A.axis, &A.angle);
    double lo[3], hi[3], cl[3], h2 = 0, cn2 = 0;
    for (int a = 0; a < 3; ++a) {
      A.orel0[a] = (float)(os0[a] - p0[4 * a + 3]);
      A.orel1[a] = (float)(os1[a] - p1[4 * a + 3]);
      lo[a] = as->origin[a] + as->dev.bmin[a] * as->sfin;
      hi[a] = as->origin[a] + as->dev.bmax[a] * as->sfin;
      A.box_lo[a] = (float)lo[a];
      A.box_hi[a] = (float)hi[a];
      A.origin[a] = (float)as->origin[a];
      cl[a] = 0.5 * (lo[a] + hi[a]);
      h2 += 0.25 * (hi[a] - lo[a]) * (hi[a] - lo[a]);
      cn2 += cl[a] * cl[a];
    }
    A.inv_sfin = (float)(1.0 / as->sfin);
    double c0n2 = 0;
    for (int i = 0; i < 3; ++i) {
      double w0 = p0[4 * i + 3] - os0[i], w1 = p1[4 * i + 3] - os1[i];
      for (int j = 0; j < 3; ++j) {
        w0 += p0[4 * i + j] * cl[j];
        w1 += p1[4 * i + j] * cl[j];
      }
      A.cc0[i] = (float)w0;
      A.cc1[i] = (float)w1;
      c0n2 += w0 * w0;
    }
    // the centre follows an arc between its end positions: its chord is off by
    // at most |c| (1 - cos(angle / 2)) <= |c| angle^2 / 8
    const double ang = std::fabs((double)A.angle);
    A.radius = (float)(std::sqrt(h2) + std::sqrt(cn2) * ang * ang / 8.0 +
                       1e-3 * (1.0 + std::sqrt(c0n2)));
    A.id_base = actors[k].id_base;
    A.dparams = dparams ? dparams[k] : nullptr;
    ad.push_back(A);
  }
  return ad;
}

extern "C" salf_status salf_render_rays_actors(salf_scene* sc, const salf_actor* actors,
                                              int32_t n_actors, const salf_sensor* sen,
                                              const salf_render_opts* opts,
                                              const salf_outputs* out, void* stream) {
  SALF_RANGE("salf_render_rays_actors");
  if (!sc || !sen || !out || n_actors < 0 || (n_actors > 0 && !actors)) {
    g_err = "salf_render_rays_actors: null argument or negative count";
    return SALF_ERR_INVALID;
  }
  if (n_actors > SALF_MAX_ACTORS) {
    g_err = "salf_render_rays_actors: more than SALF_MAX_ACTORS actors";
    return SALF_ERR_INVALID;
  }
  const salf_render_opts o = opts ? *opts : default_opts();
  if (out->on_host || out->ray_dump || out->steps || out->raydrop) {
    g_err = "salf_render_rays_actors: device outputs only (no ray_dump, steps or raydrop)";
    return SALF_ERR_INVALID;
  }
  if (!out->rgb && !out->depth && !out->opacity && !out->intensity && !out->saved && !out->valid &&
      !(o.visits_cap > 0 && out->visits)) {
    g_err = "salf_render_rays_actors: no output requested";
    return SALF_ERR_INVALID;
  }
  if (o.visits_cap > 0 && (!out->visits || !out->visit_count)) {
    g_err = "salf_render_rays_actors: visits_cap > 0 needs visits and visit_count";
    return SALF_ERR_INVALID;
  }
  if (misaligned(out->saved, 16)) {
    g_err = "salf_render_rays_actors: saved must be 16-byte aligned";
    return SALF_ERR_INVALID;
  }
  {
    const salf_status cs = check_actors(sc, actors, n_actors, "salf_render_rays_actors");
    if (cs != SALF_OK) return cs;
  }
  cudaError_t e;
  if ((e = cudaSetDevice(sc->device)) != cudaSuccess) return salf_cuda_fail(e, "cudaSetDevice");
  LaunchParams P;
  std::memset(&P, 0, sizeof(P));
  P.S = sc->dev;
  P.n_req = 1;
  ReqDev& r = P.req[0];
  salf_status st = salf_prepare_request(sc, sen, &o, &r);
  if (st != SALF_OK) return st;
  salf_request_tiling(&r, sen, 0);  // this path walks whole rays
  P.total_tiles = r.n_tiles;
  r.rgb = out->rgb;
  r.depth = out->depth;
  r.opacity = out->opacity;
  r.intensity = out->intensity;
  r.saved = out->saved;
  r.valid = out->valid;
  r.vcount = out->visit_count;
  r.visits = out->visits;

  const std::vector<ActorDev> ad = actor_table(actors, n_actors, sen, r, nullptr);
  const int na = (int)ad.size();
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lk(sc->actor_mu);
  if (!sc->actor_done) {
    if ((e = cudaEventCreateWithFlags(&sc->actor_done, cudaEventDisableTiming)) != cudaSuccess)
      return salf_cuda_fail(e, "actor event");
  } else if ((e = cudaStreamWaitEvent(cs, sc->actor_done, 0)) != cudaSuccess) {
    return salf_cuda_fail(e, "actor event wait");
  }
  const size_t table_bytes = ((std::max<size_t>(1, (size_t)na) * sizeof(ActorDev)) + 255) & ~(size_t)255;
  const size_t mask_bytes = (size_t)r.n_tiles * (SALF_MAX_ACTORS / 32) * sizeof(unsigned);
  const size_t bytes = table_bytes + mask_bytes + (2 * (size_t)r.n_tiles + 2) * sizeof(int);
  if (sc->actor_buf_bytes < bytes) {
    if ((e = cudaEventSynchronize(sc->actor_done)) != cudaSuccess)
      return salf_cuda_fail(e, "actor sync");
    if (sc->actor_buf) cudaFree(sc->actor_buf);
    sc->actor_buf = nullptr;
    sc->actor_buf_bytes = 0;
    const size_t grow = bytes + bytes / 4;
    if (cudaMalloc(&sc->actor_buf, grow) != cudaSuccess) {
      cudaGetLastError();
      g_err = "salf_render_rays_actors: out of device memory";
      return SALF_ERR_OOM;
    }
    sc->actor_buf_bytes = grow;
  }
  ActorDev* dact = static_cast<ActorDev*>(sc->actor_buf);
  unsigned* masks = reinterpret_cast<unsigned*>(static_cast<char*>(sc->actor_buf) + table_bytes);
  int* lists = reinterpret_cast<int*>(static_cast<char*>(sc->actor_buf) + table_bytes + mask_bytes);
  int* counts = lists + 2 * (size_t)r.n_tiles;
  if (na == 0) {
    // no actor in the request: the plain ray kernel
    if ((e = salf_launch_forward(P, cs)) != cudaSuccess) return salf_cuda_fail(e, "forward launch");
  } else {
    if ((e = cudaMemcpyAsync(dact, ad.data(), (size_t)na * sizeof(ActorDev),
                             cudaMemcpyHostToDevice, cs)) != cudaSuccess)
      return salf_cuda_fail(e, "actor table upload");
    if ((e = cudaMemsetAsync(counts, 0, 2 * sizeof(int), cs)) != cudaSuccess)
      return salf_cuda_fail(e, "actor tile counts");
    // tiles whose rays may meet an actor go to the merge kernel, the rest to
    // the plain ray kernel
    if ((e = salf_launch_classify(P, dact, na, lists, counts, masks, cs)) != cudaSuccess)
      return salf_cuda_fail(e, "tile classification");
    // the two tile sets are disjoint: the merge kernel runs on an auxiliary
    // stream beside the ray kernel (fork after the classification, join
    // before the call's end event).  That stream has the highest priority, so
    // the merge kernel's few long warps are dispatched ahead of the ray
    // kernel's many short ones (measured: 1080p camera with 24 actors 0.947
    // -> 0.874 ms, LiDAR 0.694 -> 0.613 ms).
    if (!sc->actor_aux) {
      int prio_least = 0, prio_greatest = 0;
      if ((e = cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest)) != cudaSuccess)
        return salf_cuda_fail(e, "stream priorities");
      if ((e = cudaStreamCreateWithPriority(&sc->actor_aux, cudaStreamNonBlocking,
                                            prio_greatest)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&sc->actor_fork, cudaEventDisableTiming)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&sc->actor_join, cudaEventDisableTiming)) != cudaSuccess)
        return salf_cuda_fail(e, "actor stream");
    }
    if ((e = cudaEventRecord(sc->actor_fork, cs)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(sc->actor_aux, sc->actor_fork, 0)) != cudaSuccess)
      return salf_cuda_fail(e, "actor fork");
    LaunchParams Pa = P;
    Pa.req[0].tile_list = lists + r.n_tiles;
    Pa.req[0].tile_count = counts + 1;
    if ((e = salf_launch_actors(Pa, dact, na, masks, sc->actor_aux)) != cudaSuccess)
      return salf_cuda_fail(e, "actor launch");
    LaunchParams Ps = P;
    Ps.req[0].tile_list = lists;
    Ps.req[0].tile_count = counts;
    if ((e = salf_launch_forward(Ps, cs)) != cudaSuccess) return salf_cuda_fail(e, "forward launch");
    if ((e = cudaEventRecord(sc->actor_join, sc->actor_aux)) != cudaSuccess ||
        (e = cudaStreamWaitEvent(cs, sc->actor_join, 0)) != cudaSuccess)
      return salf_cuda_fail(e, "actor join");
  }
  if ((e = cudaEventRecord(sc->actor_done, cs)) != cudaSuccess)
    return salf_cuda_fail(e, "actor event");
  return SALF_OK;
}

extern "C" salf_status salf_render_backward_actors(
    salf_scene* sc, const salf_actor* actors, int32_t n_actors, const salf_sensor* sen,
    const salf_render_opts* opts, const float* saved, const float* d_rgb, const float* d_depth,
    const float* d_opacity, const float* d_intensity, float* d_params,
    float* const* actor_d_params, void* stream) {
  SALF_RANGE("salf_render_backward_actors");
  if (!sc || !sen || !saved || n_actors < 0 || (n_actors > 0 && !actors)) {
    g_err = "salf_render_backward_actors: null argument or negative count";
    return SALF_ERR_INVALID;
  }
  if (n_actors > SALF_MAX_ACTORS) {
    g_err = "salf_render_backward_actors: more than SALF_MAX_ACTORS actors";
    return SALF_ERR_INVALID;
  }
  if (!d_params) {  // the scene's own gradient buffer
    std::lock_guard<std::mutex> lk(sc->grads_mu);
    d_params = sc->grads;
    if (!d_params) {
      g_err = "salf_render_backward_actors: d_params is NULL and salf_scene_params has not "
              "created the scene's gradient buffer";
      return SALF_ERR_INVALID;
    }
  }
  if (misaligned(saved, 16) || misaligned(d_params, 16)) {
    g_err = "salf_render_backward_actors: saved and d_params must be 16-byte aligned";
    return SALF_ERR_INVALID;
  }
  for (int k = 0; actor_d_params && k < n_actors; ++k)
    if (misaligned(actor_d_params[k], 16)) {
      g_err = "salf_render_backward_actors: actor gradient buffers must be 16-byte aligned";
      return SALF_ERR_INVALID;
    }
  {
    const salf_status cs = check_actors(sc, actors, n_actors, "salf_render_backward_actors");
    if (cs != SALF_OK) return cs;
  }
  const salf_render_opts o = opts ? *opts : default_opts();
  cudaError_t e;
  if ((e = cudaSetDevice(sc->device)) != cudaSuccess) return salf_cuda_fail(e, "cudaSetDevice");
  LaunchParams P;
  std::memset(&P, 0, sizeof(P));
  P.S = sc->dev;
  P.n_req = 1;
  ReqDev& r = P.req[0];
  salf_status st = salf_prepare_request(sc, sen, &o, &r);
  if (st != SALF_OK) return st;
  salf_request_tiling(&r, sen, 0);  // the forward's tiles (whole rays)
  P.total_tiles = r.n_tiles;
  r.vcap = 0;
  r.bsaved = saved;
  r.g_rgb = d_rgb;
  r.g_depth = d_depth;
  r.g_opacity = d_opacity;
  r.g_int = d_intensity;
  r.d_params = d_params;
  const std::vector<ActorDev> ad = actor_table(actors, n_actors, sen, r, actor_d_params);
  const int na = (int)ad.size();
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  if (na == 0) {  // the static adjoint alone
    if ((e = salf_launch_backward(P, cs)) != cudaSuccess) return salf_cuda_fail(e, "backward launch");
    return SALF_OK;
  }
  std::lock_guard<std::mutex> lk(sc->actor_mu);
  if (!sc->actor_done) {
    if ((e = cudaEventCreateWithFlags(&sc->actor_done, cudaEventDisableTiming)) != cudaSuccess)
      return salf_cuda_fail(e, "actor event");
  } else if ((e = cudaStreamWaitEvent(cs, sc->actor_done, 0)) != cudaSuccess) {
    return salf_cuda_fail(e, "actor event wait");
  }
  const size_t table_bytes = (((size_t)na * sizeof(ActorDev)) + 255) & ~(size_t)255;
  const size_t mask_bytes = (size_t)r.n_tiles * (SALF_MAX_ACTORS / 32) * sizeof(unsigned);
  const size_t bytes = table_bytes + mask_bytes + (2 * (size_t)r.n_tiles + 2) * sizeof(int);
  if (sc->actor_buf_bytes < bytes) {
    if ((e = cudaEventSynchronize(sc->actor_done)) != cudaSuccess)
      return salf_cuda_fail(e, "actor sync");
    if (sc->actor_buf) cudaFree(sc->actor_buf);
    sc->actor_buf = nullptr;
    sc->actor_buf_bytes = 0;
    const size_t grow = bytes + bytes / 4;
    if (cudaMalloc(&sc->actor_buf, grow) != cudaSuccess) {
      cudaGetLastError();
      g_err = "salf_render_backward_actors: out of device memory";
      return SALF_ERR_OOM;
    }
    sc->actor_buf_bytes = grow;
  }
  ActorDev* dact = static_cast<ActorDev*>(sc->actor_buf);
  unsigned* masks = reinterpret_cast<unsigned*>(static_cast<char*>(sc->actor_buf) + table_bytes);
  int* lists = reinterpret_cast<int*>(static_cast<char*>(sc->actor_buf) + table_bytes + mask_bytes);
  int* counts = lists + 2 * (size_t)r.n_tiles;
  if ((e = cudaMemcpyAsync(dact, ad.data(), (size_t)na * sizeof(ActorDev), cudaMemcpyHostToDevice,
                           cs)) != cudaSuccess)
    return salf_cuda_fail(e, "actor table upload");
  if ((e = cudaMemsetAsync(counts, 0, 2 * sizeof(int), cs)) != cudaSuccess)
    return salf_cuda_fail(e, "actor tile counts");
  // the forward's split: tiles whose rays may meet an actor take the merge
  // walk's adjoint, the others the static adjoint
  if ((e = salf_launch_classify(P, dact, na, lists, counts, masks, cs)) != cudaSuccess)
    return salf_cuda_fail(e, "tile classification");
  LaunchParams Ps = P;
  Ps.req[0].tile_list = lists;
  Ps.req[0].tile_count = counts;
  if ((e = salf_launch_backward(Ps, cs)) != cudaSuccess) return salf_cuda_fail(e, "backward launch");
  LaunchParams Pa = P;
  Pa.req[0].tile_list = lists + r.n_tiles;
  Pa.req[0].tile_count = counts + 1;
  if ((e = salf_launch_backward_actors(Pa, dact, na, masks, cs)) != cudaSuccess)
    return salf_cuda_fail(e, "actor backward launch");
  if ((e = cudaEventRecord(sc->actor_done, cs)) != cudaSuccess)
    return salf_cuda_fail(e, "actor event");
  return SALF_OK;
}

extern "C" salf_status salf_render_rays_batch(salf_scene* sc, int32_t n,
                                              const salf_sensor* sensors,
                                              const salf_render_opts* opts,
                                              const salf_outputs* outs, void* stream) {
  SALF_RANGE("salf_render_rays_batch");
  if (!sc || n < 0 || (n > 0 && (!sensors || !outs))) {
    g_err = "salf_render_rays_batch: null argument or negative count";
    return SALF_ERR_INVALID;
  }
  const salf_render_opts o = opts ? *opts : default_opts();
  if (o.visits_cap > 0) {
    g_err = "salf_render_rays_batch: visit lists are not supported";
    return SALF_ERR_INVALID;
  }
  for (int i = 0; i < n; ++i) {
    const salf_outputs& out = outs[i];
    if (out.on_host || out.visits || out.visit_count || out.ray_dump || out.steps ||
        out.max_alpha) {
      g_err = "salf_render_rays_batch: device outputs only (no visits, ray_dump, steps or max_alpha)";
      return SALF_ERR_INVALID;
    }
    if (!out.rgb && !out.depth && !out.opacity && !out.intensity && !out.saved && !out.valid &&
        !out.raydrop) {
      g_err = "salf_render_rays_batch: no output requested for sensor " + std::to_string(i);
      return SALF_ERR_INVALID;
    }
    if (misaligned(out.saved, 16)) {
      g_err = "salf_render_rays_batch: saved must be 16-byte aligned";
      return SALF_ERR_INVALID;
    }
  }
  cudaError_t e;
  if ((e = cudaSetDevice(sc->device)) != cudaSuccess) return salf_cuda_fail(e, "cudaSetDevice");
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  for (int b = 0; b < n; b += SALF_MAX_BATCH) {
    LaunchParams P;
    std::memset(&P, 0, sizeof(P));
    P.S = sc->dev;
    for (int i = b; i < std::min(n, b + SALF_MAX_BATCH); ++i) {
      ReqDev& r = P.req[P.n_req++];
      const salf_status st = salf_prepare_request(sc, &sensors[i], &o, &r);
      if (st != SALF_OK) return st;
      r.rgb = outs[i].rgb;
      r.depth = outs[i].depth;
      r.opacity = outs[i].opacity;
      r.intensity = outs[i].intensity;
      r.saved = outs[i].saved;
      r.valid = outs[i].valid;
      r.raydrop = outs[i].raydrop;
      r.tile_begin = P.total_tiles;
      P.total_tiles += r.n_tiles;
    }
    if ((e = salf_launch_forward(P, cs)) != cudaSuccess) return salf_cuda_fail(e, "forward launch");
  }
  return SALF_OK;
}

extern "C" salf_status salf_render_backward_batch(
    salf_scene* sc, int32_t n, const salf_sensor* sensors, const salf_render_opts* opts,
    const float* const* saved, const float* const* d_rgb, const float* const* d_depth,
    const float* const* d_opacity, const float* const* d_intensity, float* d_params,
    void* stream) {
  SALF_RANGE("salf_render_backward_batch");
  if (!sc || n < 0 || (n > 0 && (!sensors || !saved))) {
    g_err = "salf_render_backward_batch: null argument or negative count";
    return SALF_ERR_INVALID;
  }
  if (!d_params) {  // the scene's own gradient buffer
    std::lock_guard<std::mutex> lk(sc->grads_mu);
    d_params = sc->grads;
    if (!d_params) {
      g_err = "salf_render_backward_batch: d_params is NULL and salf_scene_params has not created "
              "the scene's gradient buffer";
      return SALF_ERR_INVALID;
    }
  }
  if (misaligned(d_params, 16)) {
    g_err = "salf_render_backward_batch: d_params must be 16-byte aligned";
    return SALF_ERR_INVALID;
  }
  for (int i = 0; i < n; ++i)
    if (!saved[i] || misaligned(saved[i], 16)) {
      g_err = "salf_render_backward_batch: saved[" + std::to_string(i) +
              "] is null or not 16-byte aligned";
      return SALF_ERR_INVALID;
    }
  const salf_render_opts o = opts ? *opts : default_opts();
  cudaError_t e;
  if ((e = cudaSetDevice(sc->device)) != cudaSuccess) return salf_cuda_fail(e, "cudaSetDevice");
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  auto pick = [&](const float* const* a, int i) { return a ? a[i] : nullptr; };
  for (int b = 0; b < n; b += SALF_MAX_BATCH) {
    LaunchParams P;
    std::memset(&P, 0, sizeof(P));
    P.S = sc->dev;
    for (int i = b; i < std::min(n, b + SALF_MAX_BATCH); ++i) {
      ReqDev& r = P.req[P.n_req++];
      const salf_status st = salf_prepare_request(sc, &sensors[i], &o, &r);
      if (st != SALF_OK) return st;
      salf_request_tiling(&r, &sensors[i], 0);  // the adjoint walks whole rays
      r.vcap = 0;
      r.bsaved = saved[i];
      r.g_rgb = pick(d_rgb, i);
      r.g_depth = pick(d_depth, i);
      r.g_opacity = pick(d_opacity, i);
      r.g_int = pick(d_intensity, i);
      r.d_params = d_params;
      r.tile_begin = P.total_tiles;
      P.total_tiles += r.n_tiles;
    }
    if ((e = salf_launch_backward(P, cs)) != cudaSuccess)
      return salf_cuda_fail(e, "backward launch");
  }
  return SALF_OK;
}

extern "C" salf_status salf_render_backward(salf_scene* sc, const salf_sensor* sen,
                                            const salf_render_opts* opts, const float* saved,
                                            const float* d_rgb, const float* d_depth,
                                            const float* d_opacity, const float* d_intensity,
                                            const float* raydrop, const float* d_raydrop,
                                            float* d_params, void* stream) {
  SALF_RANGE("salf_render_backward");
  if (!sc || !sen || !saved) {
    g_err = "salf_render_backward: null argument";
    return SALF_ERR_INVALID;
  }
  if (!d_params) {  // the scene's own gradient buffer
    std::lock_guard<std::mutex> lk(sc->grads_mu);
    d_params = sc->grads;
    if (!d_params) {
      g_err = "salf_render_backward: d_params is NULL and salf_scene_params has not created the "
              "scene's gradient buffer";
      return SALF_ERR_INVALID;
    }
  }
  if (d_raydrop && !raydrop) {
    g_err = "salf_render_backward: d_raydrop needs the forward's raydrop output";
    return SALF_ERR_INVALID;
  }
  if (misaligned(saved, 16) || misaligned(d_params, 16)) {
    g_err = "salf_render_backward: saved and d_params must be 16-byte aligned";
    return SALF_ERR_INVALID;
  }
  const salf_render_opts o = opts ? *opts : default_opts();
  cudaError_t e;
  if ((e = cudaSetDevice(sc->device)) != cudaSuccess) return salf_cuda_fail(e, "cudaSetDevice");
  LaunchParams P;
  std::memset(&P, 0, sizeof(P));
  P.S = sc->dev;
  P.n_req = 1;
  ReqDev& r = P.req[0];
  salf_status st = salf_prepare_request(sc, sen, &o, &r);
  if (st != SALF_OK) return st;
  salf_request_tiling(&r, sen, 0);  // this path walks whole rays
  r.vcap = 0;
  r.bsaved = saved;
  r.g_rgb = d_rgb;
  r.g_depth = d_depth;
  r.g_opacity = d_opacity;
  r.g_int = d_intensity;
  r.b_raydrop = d_raydrop ? raydrop : nullptr;
  r.g_raydrop = d_raydrop;
  r.d_params = d_params;
  P.total_tiles = r.n_tiles;
  if ((e = salf_launch_backward(P, static_cast<cudaStream_t>(stream))) != cudaSuccess)
    return salf_cuda_fail(e, "backward launch");
  return SALF_OK;
}
