// secondary.cu -- secondary rays (reflection, refraction, shadow) spawned at
// the expected hit point of a primary render (effects named in Sec. V-C and
// Fig. 1; the construction is stated in salf.h).  One thread per primary ray:
// regenerate the ray, locate the voxel holding o + (D/O) d, take the normal
// from its geometry slopes, write one explicit ray.  Elementwise and light:
// 8 B read and 32 B written per ray plus one record chunk and the lookup.
#include <cmath>
#include <cstring>

#include "traverse.cuh"

using namespace salf;

namespace {

bool device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

struct SecondaryParams {
  DevScene S;
  ReqDev Q;              // primary sensor (ray generation only)
  const float* depth;    // R: sum w t_m
  const float* opacity;  // R: sum w
  float* rays;           // R x 8 out
  int kind;
  float eta, min_opacity, offset, t_far;
  float light[3];        // unit, toward the light
  long long R;
};

// Geometry slopes W[0:3] of internal voxel `vox`.
template <int DT>
__device__ __forceinline__ void record_slopes(const DevScene& S, int vox, float g[3]) {
  const float4 c = __ldg(reinterpret_cast<const float4*>(S.params) +
                         (size_t)vox * RecordLayout<DT>::kChunks);
  if (DT == SALF_F32) {
    g[0] = c.x;
    g[1] = c.y;
    g[2] = c.z;
  } else {
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&c);
    const float2 a = __bfloat1622float2(h[0]), b = __bfloat1622float2(h[1]);
    g[0] = a.x;
    g[1] = a.y;
    g[2] = b.x;
  }
}

template <int DT>
__global__ void __launch_bounds__(256) k_secondary(const __grid_constant__ SecondaryParams P) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= P.R) return;
  const DevScene& S = P.S;
  const int u = (int)(i % P.Q.W), v = (int)(i / P.Q.W);
  Ray r;
  gen_ray(P.Q, S, u, v, (int)i, r);
  float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = make_float4(0.f, 0.f, 0.f, 0.f);
  const float O = __ldg(P.opacity + i), D = __ldg(P.depth + i);
  if (r.valid && O >= P.min_opacity && O > 0.f) {
    const float ts = D / O;
    // hit point in finest-cell units: Oi + p
    const double isf = S.inv_sfin;
    double p[3];
    int c[3];
    bool inside = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      p[k] = (double)r.Of[k] + (double)ts * (double)r.d[k] * isf;
      const double f = floor(p[k]);
      c[k] = r.Oi[k] + (int)f;
      inside = inside && c[k] >= 0 && c[k] < S.Gf[k];
    }
    int vox = -1, ls;
    if (inside) vox = find_leaf(S, c[0], c[1], c[2], &ls);
    float g[3] = {0.f, 0.f, 0.f};
    if (vox >= 0) record_slopes<DT>(S, vox, g);
    const float gg = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    if (gg > 0.f) {
      const float inv = -rsqrtf(gg);
      float n[3] = {g[0] * inv, g[1] * inv, g[2] * inv};
      float dn = n[0] * r.d[0] + n[1] * r.d[1] + n[2] * r.d[2];
      if (dn > 0.f) {
        n[0] = -n[0];
        n[1] = -n[1];
        n[2] = -n[2];
        dn = -dn;
      }
      float dir[3], side = 1.f;
      const float cosi = -dn;
      const float k = 1.f - P.eta * P.eta * (1.f - cosi * cosi);
      if (P.kind == SALF_SECONDARY_SHADOW) {
#pragma unroll
        for (int q = 0; q < 3; ++q) dir[q] = P.light[q];
      } else if (P.kind == SALF_SECONDARY_REFRACT && k >= 0.f) {
        const float m = P.eta * cosi - sqrtf(k);
#pragma unroll
        for (int q = 0; q < 3; ++q) dir[q] = P.eta * r.d[q] + m * n[q];
        side = -1.f;
      } else {  // reflection (also total internal reflection)
#pragma unroll
        for (int q = 0; q < 3; ++q) dir[q] = r.d[q] - 2.f * dn * n[q];
      }
      double X[3];
#pragma unroll
      for (int q = 0; q < 3; ++q)
        X[q] = S.origin[q] + ((double)r.Oi[q] + p[q]) / isf + (double)(side * P.offset * n[q]);
      a = make_float4((float)X[0], (float)X[1], (float)X[2], dir[0]);
      b = make_float4(dir[1], dir[2], 0.f, P.t_far > 0.f ? P.t_far : 0.f);
    }
  }
  float4* o = reinterpret_cast<float4*>(P.rays) + 2 * i;
  o[0] = a;
  o[1] = b;
}

extern "C" salf_status salf_secondary_rays(salf_scene* sc, const salf_sensor* sen,
                                           const float* depth, const float* opacity,
                                           const salf_secondary_opts* so, float* rays_out,
                                           void* stream) {
  SALF_RANGE("salf_secondary_rays");
  if (!sc || !sen || !depth || !opacity || !so || !rays_out) {
    salf_set_error("salf_secondary_rays: null argument");
    return SALF_ERR_INVALID;
  }
  if ((reinterpret_cast<uintptr_t>(rays_out) & 15u) != 0) {
    salf_set_error("salf_secondary_rays: rays_out must be 16-byte aligned");
    return SALF_ERR_INVALID;
  }
  if (so->kind < SALF_SECONDARY_REFLECT || so->kind > SALF_SECONDARY_SHADOW) {
    salf_set_error("salf_secondary_rays: bad kind");
    return SALF_ERR_INVALID;
  }
  if (so->kind == SALF_SECONDARY_REFRACT && !(so->eta > 0.f && std::isfinite(so->eta))) {
    salf_set_error("salf_secondary_rays: eta must be > 0");
    return SALF_ERR_INVALID;
  }
  const double ll = (double)so->light_dir[0] * so->light_dir[0] +
                    (double)so->light_dir[1] * so->light_dir[1] +
                    (double)so->light_dir[2] * so->light_dir[2];
  if (so->kind == SALF_SECONDARY_SHADOW && !(ll > 0.0 && std::isfinite(ll))) {
    salf_set_error("salf_secondary_rays: light_dir must be non-zero");
    return SALF_ERR_INVALID;
  }
  if (!(so->min_opacity > 0.f && so->min_opacity <= 1.f) || !(so->offset >= 0.f) ||
      !std::isfinite(so->offset) || !std::isfinite(so->t_far)) {
    salf_set_error("salf_secondary_rays: min_opacity must be in (0, 1], offset >= 0");
    return SALF_ERR_INVALID;
  }
  cudaError_t e;
  if ((e = cudaSetDevice(sc->device)) != cudaSuccess) return salf_cuda_fail(e, "cudaSetDevice");
  if (!device_ptr(depth) || !device_ptr(opacity) || !device_ptr(rays_out) ||
      (sen->kind == SALF_RAYS_EXPLICIT && sen->rays && !device_ptr(sen->rays))) {
    salf_set_error("salf_secondary_rays: depth, opacity, rays_out and explicit rays must be device memory");
    return SALF_ERR_INVALID;
  }
  SecondaryParams P;
  std::memset(&P, 0, sizeof(P));
  P.S = sc->dev;
  salf_render_opts o;
  std::memset(&o, 0, sizeof(o));
  o.t_min_transmittance = 1e-4f;
  o.ray_segments = 1;
  salf_status st = salf_prepare_request(sc, sen, &o, &P.Q);
  if (st != SALF_OK) return st;
  P.depth = depth;
  P.opacity = opacity;
  P.rays = rays_out;
  P.kind = so->kind;
  P.eta = so->eta;
  P.min_opacity = so->min_opacity;
  P.offset = so->offset;
  P.t_far = so->t_far;
  const double il = ll > 0.0 ? 1.0 / std::sqrt(ll) : 0.0;
  for (int k = 0; k < 3; ++k) P.light[k] = (float)(so->light_dir[k] * il);
  P.R = salf_request_rays(sen);
  if (P.R == 0) return SALF_OK;
  const long long blocks = (P.R + 255) / 256;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  if (sc->dev.dtype == SALF_BF16)
    k_secondary<SALF_BF16><<<(unsigned)blocks, 256, 0, cs>>>(P);
  else
    k_secondary<SALF_F32><<<(unsigned)blocks, 256, 0, cs>>>(P);
  if ((e = cudaGetLastError()) != cudaSuccess) return salf_cuda_fail(e, "secondary launch");
  return SALF_OK;
}
