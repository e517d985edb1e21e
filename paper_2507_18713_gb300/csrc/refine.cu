// refine.cu -- densification and pruning of a scene's voxel set (Sec. III-C).
//
// Plan (one thread per voxel): a voxel whose largest composited alpha is
// below the pruning threshold is removed; otherwise a voxel above the finest
// level whose colour-field gradient L1 norm (record slots 4..12) exceeds the
// split threshold becomes its 8 octree children; the rest are kept.  An
// exclusive scan of the output counts (0, 8 or 1) places every voxel's
// output in input order, children in place of their parent.
// Apply (one thread per voxel): writes level, cell and record of each output
// voxel.  A child's record carries its parent's fields exactly: every field
// is affine in the local coordinates and x_parent = (x_child + o) / 2 with
// o in {-1, +1}^3, so the slopes halve and the offsets take W . o / 2 (the
// colour rows have no offset of their own: theirs goes to the SH DC term
// through C0 = 1 / (2 sqrt(pi))).
#include <cstring>
#include <mutex>

#include "scan.cuh"
#include "traverse.cuh"

using namespace salf_scan;

namespace {

constexpr float kSH0 = 0.28209479177387814f;

__global__ void __launch_bounds__(256) k_refine_plan(
    const int4* __restrict__ vox_box, const int* __restrict__ order, int n, int K,
    const float* __restrict__ grads, const float* __restrict__ max_alpha, float split_thr,
    float prune_alpha, unsigned char* __restrict__ action, unsigned* __restrict__ count,
    unsigned long long* __restrict__ stats) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  int act = -1;
  if (p < n) {
    const int v = __ldg(&order[p]);
    const int level = K - __ldg(&vox_box[p]).w;
    const float4* g = reinterpret_cast<const float4*>(grads) + (size_t)v * 8;
    const float4 g1 = __ldg(g + 1), g2 = __ldg(g + 2), g3 = __ldg(g + 3);  // slots 4..15
    const float l1 = fabsf(g1.x) + fabsf(g1.y) + fabsf(g1.z) + fabsf(g1.w) + fabsf(g2.x) +
                     fabsf(g2.y) + fabsf(g2.z) + fabsf(g2.w) + fabsf(g3.x);
    const float a = __ldg(&max_alpha[v]);
    act = a < prune_alpha ? 2 : ((level < K && l1 > split_thr) ? 1 : 0);
    action[v] = (unsigned char)act;
    count[v] = act == 0 ? 1u : (act == 1 ? 8u : 0u);
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const unsigned c = __reduce_add_sync(0xffffffffu, act == k ? 1u : 0u);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&stats[k], (unsigned long long)c);
  }
}

__global__ void __launch_bounds__(256) k_refine_apply(
    const int4* __restrict__ vox_box, const int* __restrict__ order, int n, int K,
    const unsigned char* __restrict__ action, const unsigned long long* __restrict__ offs,
    const float* __restrict__ params, unsigned char* __restrict__ level_out,
    int* __restrict__ ijk_out, float* __restrict__ params_out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int v = __ldg(&order[p]);
  const int act = __ldg(&action[v]);
  if (act == 2) return;
  const int4 b = __ldg(&vox_box[p]);
  const int level = K - b.w;
  const int ijk[3] = {b.x >> b.w, b.y >> b.w, b.z >> b.w};
  float rec[32];
  const float4* src = reinterpret_cast<const float4*>(params) + (size_t)v * 8;
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const float4 q = __ldg(src + k);
    rec[4 * k] = q.x;
    rec[4 * k + 1] = q.y;
    rec[4 * k + 2] = q.z;
    rec[4 * k + 3] = q.w;
  }
  const unsigned long long o = __ldg(&offs[v]);
  if (act == 0) {
    level_out[o] = (unsigned char)level;
#pragma unroll
    for (int a = 0; a < 3; ++a) ijk_out[3 * o + a] = ijk[a];
    float4* dst = reinterpret_cast<float4*>(params_out) + (size_t)o * 8;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      dst[k] = make_float4(rec[4 * k], rec[4 * k + 1], rec[4 * k + 2], rec[4 * k + 3]);
    return;
  }
  for (int c = 0; c < 8; ++c) {
    const float s[3] = {(c & 1) ? 1.f : -1.f, (c & 2) ? 1.f : -1.f, (c & 4) ? 1.f : -1.f};
    float out[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) out[k] = rec[k];
    out[3] = rec[3] + 0.5f * (rec[0] * s[0] + rec[1] * s[1] + rec[2] * s[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) out[a] = 0.5f * rec[a];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const float shift = rec[4 + 3 * r] * s[0] + rec[5 + 3 * r] * s[1] + rec[6 + 3 * r] * s[2];
#pragma unroll
      for (int a = 0; a < 3; ++a) out[4 + 3 * r + a] = 0.5f * rec[4 + 3 * r + a];
      out[13 + 4 * r] = rec[13 + 4 * r] + 0.5f * shift / kSH0;
    }
    out[30] = rec[30] + 0.5f * (rec[27] * s[0] + rec[28] * s[1] + rec[29] * s[2]);
#pragma unroll
    for (int a = 0; a < 3; ++a) out[27 + a] = 0.5f * rec[27 + a];
    const unsigned long long oc = o + (unsigned long long)c;
    level_out[oc] = (unsigned char)(level + 1);
    ijk_out[3 * oc] = 2 * ijk[0] + (c & 1);
    ijk_out[3 * oc + 1] = 2 * ijk[1] + ((c >> 1) & 1);
    ijk_out[3 * oc + 2] = 2 * ijk[2] + ((c >> 2) & 1);
    float4* dst = reinterpret_cast<float4*>(params_out) + (size_t)oc * 8;
#pragma unroll
    for (int k = 0; k < 8; ++k)
      dst[k] = make_float4(out[4 * k], out[4 * k + 1], out[4 * k + 2], out[4 * k + 3]);
  }
}

// Density of the geometry value g (Eq. 1 or Eq. 6) and its derivatives with
// respect to g, a and b.
template <int MODE>
__device__ __forceinline__ float reg_density(float g, float a, float b, float* d_g, float* d_a,
                                             float* d_b) {
  if (MODE == SALF_FIELD_EXP) {
    const float s = __expf(g);
    *d_g = s;
    *d_a = *d_b = 0.f;
    return s;
  }
  const float e = __expf(-fabsf(g) / b);
  const float sg = g > 0.f ? 1.f : (g < 0.f ? -1.f : 0.f);
  const float s = 0.5f * a + 0.5f * a * sg * (1.f - e);
  *d_g = 0.5f * a * e / b;
  *d_a = s / a;
  *d_b = -0.5f * a * g * e / (b * b);
  return s;
}

// Eq. 7's L_reg over the face-adjacent pairs, one thread per voxel: across
// each face, the voxel owning the finest cell just outside its min corner is
// the neighbour when it is at least as large (then it covers the whole face);
// a pair is counted by its smaller voxel, or by the + face of the one on the
// - side when both are equal.  At the centre of the shared face: s = W.[x,1],
// alpha = 1 - exp(-sigma(s) l) (l: the smaller edge, m), n = W[0:3] / |W[0:3]|.
template <int MODE>
__global__ void __launch_bounds__(256) k_reg_loss(const __grid_constant__ DevScene S,
                                                  const float* __restrict__ params, float lam_s,
                                                  float lam_a, float lam_n, float sfin,
                                                  float* __restrict__ loss,
                                                  float* __restrict__ grads) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  float acc = 0.f;
  if (p < S.n) {
    const int4 bi = __ldg(&S.vox_box[p]);
    const int E = 1 << bi.w;
    const int lo[3] = {bi.x, bi.y, bi.z};
    const int vi = __ldg(&S.order[p]);
    const float4 wi = __ldg(reinterpret_cast<const float4*>(params) + (size_t)vi * 8);
    const float4 abi = __ldg(reinterpret_cast<const float4*>(params) + (size_t)vi * 8 + 6);
    const float Wi[4] = {wi.x, wi.y, wi.z, wi.w};
    const float ni = sqrtf(Wi[0] * Wi[0] + Wi[1] * Wi[1] + Wi[2] * Wi[2]);
    for (int f = 0; f < 6; ++f) {
      const int ax = f >> 1;
      const int sgn = (f & 1) ? 1 : -1;
      int c[3] = {lo[0], lo[1], lo[2]};
      c[ax] = sgn > 0 ? lo[ax] + E : lo[ax] - 1;
      if (c[ax] < 0 || c[ax] >= S.Gf[ax]) continue;
      int lsj;
      const int j = salf::find_leaf(S, c[0], c[1], c[2], &lsj);
      if (j < 0 || lsj < bi.w || (lsj == bi.w && sgn < 0)) continue;
      const int4 bj = __ldg(&S.vox_box[j]);
      const int Ej = 1 << bj.w;
      const int vj = __ldg(&S.order[j]);
      const float4 wj = __ldg(reinterpret_cast<const float4*>(params) + (size_t)vj * 8);
      const float4 abj = __ldg(reinterpret_cast<const float4*>(params) + (size_t)vj * 8 + 6);
      const float Wj[4] = {wj.x, wj.y, wj.z, wj.w};
      // local coordinates of the face centre: +-1 on the axis in i; in j from its box
      float xi[3] = {0.f, 0.f, 0.f}, xj[3];
      xi[ax] = (float)sgn;
      const int lj[3] = {bj.x, bj.y, bj.z};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float X = a == ax ? (float)(sgn > 0 ? lo[a] + E : lo[a]) : (float)lo[a] + 0.5f * E;
        xj[a] = (X - ((float)lj[a] + 0.5f * Ej)) / (0.5f * Ej);
      }
      const float si = Wi[0] * xi[0] + Wi[1] * xi[1] + Wi[2] * xi[2] + Wi[3];
      const float sj = Wj[0] * xj[0] + Wj[1] * xj[1] + Wj[2] * xj[2] + Wj[3];
      float gi_g, gi_a, gi_b, gj_g, gj_a, gj_b;
      const float sigi = reg_density<MODE>(si, abi.y, abi.z, &gi_g, &gi_a, &gi_b);
      const float sigj = reg_density<MODE>(sj, abj.y, abj.z, &gj_g, &gj_a, &gj_b);
      const float ell = (float)E * sfin;
      const float ei = __expf(-sigi * ell), ej = __expf(-sigj * ell);
      const float ds = si - sj, da = ej - ei;  // alpha_i - alpha_j = e_j - e_i
      const float nj = sqrtf(Wj[0] * Wj[0] + Wj[1] * Wj[1] + Wj[2] * Wj[2]);
      float ui[3] = {0.f, 0.f, 0.f}, uj[3] = {0.f, 0.f, 0.f};
      if (ni > 0.f)
        for (int a = 0; a < 3; ++a) ui[a] = Wi[a] / ni;
      if (nj > 0.f)
        for (int a = 0; a < 3; ++a) uj[a] = Wj[a] / nj;
      const float dot = ui[0] * uj[0] + ui[1] * uj[1] + ui[2] * uj[2];
      acc += lam_s * fabsf(ds) + lam_a * fabsf(da) + lam_n * (1.f - dot);
      const float cs = lam_s * (ds > 0.f ? 1.f : (ds < 0.f ? -1.f : 0.f));
      const float ca = lam_a * (da > 0.f ? 1.f : (da < 0.f ? -1.f : 0.f));
      // d alpha_k / d sigma_k = exp(-sigma_k l) l
      const float ki = ca * ei * ell, kj = -ca * ej * ell;
      float gi[6], gj[6];  // slots 0..3, a, b
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        gi[a] = cs * xi[a] + ki * gi_g * xi[a];
        gj[a] = -cs * xj[a] + kj * gj_g * xj[a];
        if (ni > 0.f) gi[a] -= lam_n * (uj[a] - ui[a] * dot) / ni;
        if (nj > 0.f) gj[a] -= lam_n * (ui[a] - uj[a] * dot) / nj;
      }
      gi[3] = cs + ki * gi_g;
      gj[3] = -cs + kj * gj_g;
      gi[4] = ki * gi_a;
      gi[5] = ki * gi_b;
      gj[4] = kj * gj_a;
      gj[5] = kj * gj_b;
      float* Gi = grads + (size_t)vi * 32;
      float* Gj = grads + (size_t)vj * 32;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        atomicAdd(Gi + q, gi[q]);
        atomicAdd(Gj + q, gj[q]);
      }
      if (MODE == SALF_FIELD_SDF) {
        atomicAdd(Gi + 25, gi[4]);
        atomicAdd(Gi + 26, gi[5]);
        atomicAdd(Gj + 25, gj[4]);
        atomicAdd(Gj + 26, gj[5]);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0.f) atomicAdd(loss, acc);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

bool misaligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) != 0; }

}  // namespace

extern "C" salf_status salf_scene_refine_plan(salf_scene* sc, const float* grads,
                                             const float* max_alpha, float split_threshold,
                                             float prune_alpha, salf_refine_counts* counts,
                                             void* stream) {
  SALF_RANGE("salf_scene_refine_plan");
  if (!sc || !grads || !max_alpha || !counts) {
    salf_set_error("salf_scene_refine_plan: null argument");
    return SALF_ERR_INVALID;
  }
  if (misaligned16(grads)) {
    salf_set_error("salf_scene_refine_plan: grads must be 16-byte aligned");
    return SALF_ERR_INVALID;
  }
  cudaError_t e;
  if ((e = cudaSetDevice(sc->device)) != cudaSuccess) return salf_cuda_fail(e, "cudaSetDevice");
  std::lock_guard<std::mutex> lk(sc->refine_mu);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long n = sc->n, nn = n > 0 ? n : 1;
  const size_t b_act = align256(nn), b_cnt = align256(nn * 4), b_offs = align256((nn + 1) * 8),
               b_tmp = align256(scan_tmp_elems(nn) * 8), b_stats = 256;
  const size_t need = b_act + b_cnt + b_offs + b_tmp + b_stats;
  if (sc->refine_ws_bytes < need) {
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return salf_cuda_fail(e, "refine sync");
    if (sc->refine_ws) cudaFree(sc->refine_ws);
    sc->refine_ws = nullptr;
    sc->refine_ws_bytes = 0;
    if (cudaMalloc(&sc->refine_ws, need) != cudaSuccess) {
      cudaGetLastError();
      salf_set_error("salf_scene_refine_plan: out of device memory");
      return SALF_ERR_OOM;
    }
    sc->refine_ws_bytes = need;
  }
  if (!sc->refine_host &&
      cudaMallocHost(reinterpret_cast<void**>(&sc->refine_host), 64) != cudaSuccess) {
    cudaGetLastError();
    salf_set_error("salf_scene_refine_plan: cudaMallocHost failed");
    return SALF_ERR_OOM;
  }
  char* w = static_cast<char*>(sc->refine_ws);
  unsigned char* action = reinterpret_cast<unsigned char*>(w);
  unsigned* count = reinterpret_cast<unsigned*>(w + b_act);
  unsigned long long* offs = reinterpret_cast<unsigned long long*>(w + b_act + b_cnt);
  unsigned long long* tmp = reinterpret_cast<unsigned long long*>(w + b_act + b_cnt + b_offs);
  unsigned long long* stats =
      reinterpret_cast<unsigned long long*>(w + b_act + b_cnt + b_offs + b_tmp);
  if ((e = cudaMemsetAsync(stats, 0, 4 * sizeof(unsigned long long), st)) != cudaSuccess)
    return salf_cuda_fail(e, "refine stats");
  if (n > 0) {
    const DevScene& D = sc->dev;
    k_refine_plan<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        D.vox_box, D.order, (int)n, D.K, grads, max_alpha, split_threshold, prune_alpha, action,
        count, stats);
    int launches = 0;
    if ((e = scan_exclusive<unsigned, unsigned long long>(count, n, offs, tmp, st, &launches)) !=
        cudaSuccess)
      return salf_cuda_fail(e, "refine scan");
    k_scan_total<unsigned, unsigned long long><<<1, 1, 0, st>>>(count, n, offs);
    if ((e = cudaMemcpyAsync(stats + 3, offs + n, 8, cudaMemcpyDeviceToDevice, st)) !=
        cudaSuccess)
      return salf_cuda_fail(e, "refine total");
  }
  if ((e = cudaMemcpyAsync(sc->refine_host, stats, 4 * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return salf_cuda_fail(e, "refine counts");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return salf_cuda_fail(e, "refine plan");
  counts->n_kept = (int64_t)sc->refine_host[0];
  counts->n_split = (int64_t)sc->refine_host[1];
  counts->n_pruned = (int64_t)sc->refine_host[2];
  counts->n_new = n > 0 ? (int64_t)sc->refine_host[3] : 0;
  sc->refine_planned = true;
  sc->refine_n_new = counts->n_new;
  return SALF_OK;
}

extern "C" salf_status salf_scene_refine_apply(salf_scene* sc, const float* params,
                                              uint8_t* level_out, int32_t* ijk_out,
                                              float* params_out, void* stream) {
  SALF_RANGE("salf_scene_refine_apply");
  if (!sc || !params) {
    salf_set_error("salf_scene_refine_apply: null argument");
    return SALF_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lk(sc->refine_mu);
  if (!sc->refine_planned) {
    salf_set_error("salf_scene_refine_apply: no plan (call salf_scene_refine_plan first)");
    return SALF_ERR_INVALID;
  }
  if (sc->refine_n_new > 0 && (!level_out || !ijk_out || !params_out)) {
    salf_set_error("salf_scene_refine_apply: null output");
    return SALF_ERR_INVALID;
  }
  if (misaligned16(params) || misaligned16(params_out)) {
    salf_set_error("salf_scene_refine_apply: params and params_out must be 16-byte aligned");
    return SALF_ERR_INVALID;
  }
  cudaError_t e;
  if ((e = cudaSetDevice(sc->device)) != cudaSuccess) return salf_cuda_fail(e, "cudaSetDevice");
  const long long n = sc->n, nn = n > 0 ? n : 1;
  char* w = static_cast<char*>(sc->refine_ws);
  const size_t b_act = align256(nn), b_cnt = align256(nn * 4);
  const unsigned char* action = reinterpret_cast<const unsigned char*>(w);
  const unsigned long long* offs = reinterpret_cast<const unsigned long long*>(w + b_act + b_cnt);
  if (n > 0 && sc->refine_n_new > 0) {
    const DevScene& D = sc->dev;
    k_refine_apply<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        D.vox_box, D.order, (int)n, D.K, action, offs, params, level_out, ijk_out, params_out);
    if ((e = cudaGetLastError()) != cudaSuccess) return salf_cuda_fail(e, "refine apply");
  }
  return SALF_OK;
}

extern "C" salf_status salf_scene_reg_loss(salf_scene* sc, const float* params, float lambda_s,
                                          float lambda_alpha, float lambda_n, float* loss,
                                          float* grads, void* stream) {
  SALF_RANGE("salf_scene_reg_loss");
  if (!sc || !params || !loss || !grads) {
    salf_set_error("salf_scene_reg_loss: null argument");
    return SALF_ERR_INVALID;
  }
  if (misaligned16(params)) {
    salf_set_error("salf_scene_reg_loss: params must be 16-byte aligned");
    return SALF_ERR_INVALID;
  }
  cudaError_t e;
  if ((e = cudaSetDevice(sc->device)) != cudaSuccess) return salf_cuda_fail(e, "cudaSetDevice");
  const DevScene& D = sc->dev;
  if (D.n > 0) {
    const unsigned blocks = (unsigned)((D.n + 255) / 256);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const float sfin = (float)sc->sfin;
    if (D.mode == SALF_FIELD_EXP)
      k_reg_loss<SALF_FIELD_EXP><<<blocks, 256, 0, st>>>(D, params, lambda_s, lambda_alpha,
                                                          lambda_n, sfin, loss, grads);
    else
      k_reg_loss<SALF_FIELD_SDF><<<blocks, 256, 0, st>>>(D, params, lambda_s, lambda_alpha,
                                                          lambda_n, sfin, loss, grads);
    if ((e = cudaGetLastError()) != cudaSuccess) return salf_cuda_fail(e, "reg loss launch");
  }
  return SALF_OK;
}
