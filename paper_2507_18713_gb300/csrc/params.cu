// params.cu -- record upload: input order -> the scene's Morton order, with
// FP32 -> BF16 (round to nearest even) when the scene stores BF16 records, and
// the SDF parameter check (Eq. 6 needs a > 0, b > 0).
#include <cuda_bf16.h>

#include "salf_internal.h"

__global__ void __launch_bounds__(256) k_gather_params(const float* __restrict__ in,
                                                       const int* __restrict__ order,
                                                       void* __restrict__ out, long long n,
                                                       int dtype, int mode, int* status) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float4* src = reinterpret_cast<const float4*>(in) + (size_t)__ldg(&order[p]) * 8;
  float4 q[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) q[k] = __ldg(src + k);
  if (mode == SALF_FIELD_SDF && !(q[6].y > 0.f && q[6].z > 0.f)) atomicOr(status, SALF_DEVERR_SDF_AB);
  if (dtype == SALF_F32) {
    float4* dst = reinterpret_cast<float4*>(out) + (size_t)p * 8;
#pragma unroll
    for (int k = 0; k < 8; ++k) dst[k] = q[k];
  } else {
    uint4* dst = reinterpret_cast<uint4*>(out) + (size_t)p * 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float f[8] = {q[2 * k].x, q[2 * k].y, q[2 * k].z, q[2 * k].w,
                          q[2 * k + 1].x, q[2 * k + 1].y, q[2 * k + 1].z, q[2 * k + 1].w};
      unsigned w4[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const unsigned lo = __bfloat16_as_ushort(__float2bfloat16_rn(f[2 * j]));
        const unsigned hi = __bfloat16_as_ushort(__float2bfloat16_rn(f[2 * j + 1]));
        w4[j] = lo | (hi << 16);
      }
      dst[k] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
    }
  }
}

cudaError_t salf_launch_gather_params(const float* in, const int* order, void* out, int64_t n,
                                      int dtype, int mode, int* status, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  k_gather_params<<<blocks, 256, 0, st>>>(in, order, out, (long long)n, dtype, mode, status);
  return cudaGetLastError();
}
