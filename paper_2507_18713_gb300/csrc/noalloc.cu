// noalloc.cu -- salf_render_rays_host_noalloc: the host-output render of
// salf_render_rays without any device allocation.
//
// salf_render_rays with host output buffers renders into a device staging
// buffer that the library grows with cudaMalloc on first use (and frees and
// re-allocates, after a device synchronisation, when a larger frame comes).
// Some callers cannot let a library allocate device memory: real-time loops
// where an allocation's latency and implicit synchronisation are not
// acceptable, host applications whose device memory is reserved up front by
// their own pooling allocator, and plug-ins that their host forbids to
// allocate.  This entry point stages the outputs in a fixed array compiled
// into the library instead (SALF_NOALLOC_STAGING_BYTES).  It calls no
// cudaMalloc, cudaFree or allocating library routine.
//
// The array's device address is looked up with cudaGetSymbolAddress by
// salf_create, once per device, with that device current, and cached.  Under
// lazy module loading (the CUDA default) that lookup is also what loads this
// file's module and so makes the device hold the array: it is resident from
// the first salf_create on a device until the process exits, and a caller
// that reserves device memory in its own pool does so after salf_create.
// Every call on a device shares the array and leaves its contents behind; the
// forward kernel overwrites every output element it stages, so nothing needs
// clearing between calls.  Two calls that overlap on the GPU (for instance
// from two host threads on one device) race on the array: serialise them.
#include <cstring>
#include <mutex>
#include <string>

#include "salf_internal.h"

#define SALF_NOALLOC_STAGING_BYTES (48u << 20)
#define SALF_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_noalloc_staging[SALF_NOALLOC_STAGING_BYTES];

namespace {
std::mutex g_setup_mu;
char* g_staging_ptr[SALF_NOALLOC_MAX_DEVICES] = {};

// Device address of the staging array on `device` (which must be current).
salf_status staging_for_device(int device, char** out) {
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (device < 0 || device >= SALF_NOALLOC_MAX_DEVICES) {
    salf_set_error("no-alloc staging: device index out of range");
    return SALF_ERR_INVALID;
  }
  if (!g_staging_ptr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_staging);
    if (e != cudaSuccess) return salf_cuda_fail(e, "cudaGetSymbolAddress(no-alloc staging)");
    g_staging_ptr[device] = static_cast<char*>(p);
  }
  *out = g_staging_ptr[device];
  return SALF_OK;
}

size_t round256(size_t n) { return (n + 255) & ~(size_t)255; }
}  // namespace

// Called by salf_create with `device` current: resolves (and, under lazy
// module loading, loads) the staging array, so that later no-alloc calls on
// the device find it resident.
salf_status salf_noalloc_setup(int device) {
  char* base = nullptr;
  return staging_for_device(device, &base);
}

extern "C" salf_status salf_render_rays_host_noalloc(salf_scene* sc, const salf_sensor* sen,
                                                     const salf_render_opts* opts,
                                                     const salf_outputs* out, void* stream) {
  SALF_RANGE("salf_render_rays_host_noalloc");
  if (!sc || !sen || !out) {
    salf_set_error("salf_render_rays_host_noalloc: null argument");
    return SALF_ERR_INVALID;
  }
  if (out->visits || out->visit_count || out->ray_dump || out->steps || out->raydrop ||
      out->max_alpha || (opts && opts->visits_cap > 0)) {
    salf_set_error("salf_render_rays_host_noalloc: debug, alpha-maxima and raydrop outputs are "
                   "not supported");
    return SALF_ERR_INVALID;
  }
  if (!out->rgb && !out->depth && !out->opacity && !out->intensity && !out->saved && !out->valid) {
    salf_set_error("salf_render_rays_host_noalloc: no output requested");
    return SALF_ERR_INVALID;
  }
  salf_render_opts o;
  if (opts) {
    o = *opts;
  } else {
    std::memset(&o, 0, sizeof(o));
    o.t_min_transmittance = 1e-4f;
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
  if (sen->kind == SALF_RAYS_EXPLICIT) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, sen->rays) != cudaSuccess ||
        (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      salf_set_error("salf_render_rays_host_noalloc: explicit rays must be device memory");
      return SALF_ERR_INVALID;
    }
  }
  P.total_tiles = r.n_tiles;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  // page-locked, device-addressable host outputs: the kernel writes them in
  // place (no staging, no copy step)
  {
    void* hp[6] = {out->rgb, out->depth, out->opacity, out->intensity, out->saved, out->valid};
    void* dp[6] = {};
    bool direct = (reinterpret_cast<uintptr_t>(out->saved) & 15u) == 0;
    for (int i = 0; i < 6 && direct; ++i) {
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
    if (direct) {
      r.rgb = static_cast<float*>(dp[0]);
      r.depth = static_cast<float*>(dp[1]);
      r.opacity = static_cast<float*>(dp[2]);
      r.intensity = static_cast<float*>(dp[3]);
      r.saved = static_cast<float*>(dp[4]);
      r.valid = static_cast<unsigned char*>(dp[5]);
      if ((e = salf_launch_forward(P, cs)) != cudaSuccess)
        return salf_cuda_fail(e, "forward launch");
      if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) return salf_cuda_fail(e, "render");
      return SALF_OK;
    }
  }
  const size_t R = (size_t)salf_request_rays(sen);
  const size_t sizes[6] = {out->rgb ? R * 12 : 0,       out->depth ? R * 4 : 0,
                           out->opacity ? R * 4 : 0,    out->intensity ? R * 4 : 0,
                           out->saved ? R * 32 : 0,     out->valid ? R : 0};
  size_t off[6], total = 0;
  for (int i = 0; i < 6; ++i) {
    off[i] = total;
    total += round256(sizes[i]);
  }
  if (total > SALF_NOALLOC_STAGING_BYTES) {
    salf_set_error("salf_render_rays_host_noalloc: the requested outputs need " +
                   std::to_string(total) + " bytes of staging, more than the fixed " +
                   std::to_string((size_t)SALF_NOALLOC_STAGING_BYTES) + " bytes");
    return SALF_ERR_INVALID;
  }
  char* base = nullptr;
  if ((st = staging_for_device(sc->device, &base)) != SALF_OK) return st;
  r.rgb = out->rgb ? reinterpret_cast<float*>(base + off[0]) : nullptr;
  r.depth = out->depth ? reinterpret_cast<float*>(base + off[1]) : nullptr;
  r.opacity = out->opacity ? reinterpret_cast<float*>(base + off[2]) : nullptr;
  r.intensity = out->intensity ? reinterpret_cast<float*>(base + off[3]) : nullptr;
  r.saved = out->saved ? reinterpret_cast<float*>(base + off[4]) : nullptr;
  r.valid = out->valid ? reinterpret_cast<unsigned char*>(base + off[5]) : nullptr;
  if ((e = salf_launch_forward(P, cs)) != cudaSuccess) return salf_cuda_fail(e, "forward launch");
  void* dst[6] = {out->rgb, out->depth, out->opacity, out->intensity, out->saved, out->valid};
  for (int i = 0; i < 6; ++i) {
    if (!sizes[i]) continue;
    if ((e = cudaMemcpyAsync(dst[i], base + off[i], sizes[i], cudaMemcpyDeviceToHost, cs)) !=
        cudaSuccess)
      return salf_cuda_fail(e, "cudaMemcpyAsync(outputs)");
  }
  if ((e = cudaStreamSynchronize(cs)) != cudaSuccess) return salf_cuda_fail(e, "render");
  return SALF_OK;
}
