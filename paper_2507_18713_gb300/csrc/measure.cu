// measure.cu -- L2 read bandwidth of this GPU, measured by a plain streaming
// read of a buffer that fits in L2.  The ray kernels gather most of their
// bytes from L1 and L2, not HBM, so their L2 traffic is reported against this
// figure beside the HBM roofline.  Not part of the rendering method.
#include <cuda_runtime.h>
#include <stdint.h>

#include "salf_internal.h"

namespace {

// Each thread reads 16-byte words in a grid-stride loop (cache-global loads:
// served by L2, not L1) and folds them into one word, stored only if it
// matches a key no buffer holds, so that the loads are not removed.
// The buffer is read `passes` times per launch (a compiler barrier between
// passes keeps each pass's loads), so that the launch overhead is amortised.
__global__ void __launch_bounds__(512) k_l2_read(const uint4* __restrict__ p, int64_t n,
                                                 int passes, unsigned key,
                                                 unsigned* __restrict__ sink) {
  unsigned acc = 0u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
#pragma unroll 1
  for (int pass = 0; pass < passes; ++pass) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
      const uint4 a = __ldcg(p + i), b = __ldcg(p + i + stride), c = __ldcg(p + i + 2 * stride),
                  d = __ldcg(p + i + 3 * stride);
      acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^
             d.z ^ d.w;
    }
    for (; i < n; i += stride) {
      const uint4 a = __ldcg(p + i);
      acc ^= a.x ^ a.y ^ a.z ^ a.w;
    }
    asm volatile("" ::: "memory");
  }
  if (acc == key) sink[0] = acc;
}

}  // namespace

extern "C" salf_status salf_measure_l2_read(int32_t device, int64_t bytes, int32_t reps,
                                            double* gbs) {
  if (!gbs || bytes < (1 << 20) || bytes > ((int64_t)1 << 32) || reps < 1 || reps > 100000) {
    salf_set_error("salf_measure_l2_read: bytes must be in [1 MiB, 4 GiB], reps in [1, 100000]");
    return SALF_ERR_INVALID;
  }
  cudaError_t e;
  if ((e = cudaSetDevice(device)) != cudaSuccess) return salf_cuda_fail(e, "cudaSetDevice");
  int sms = 0;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device)) != cudaSuccess)
    return salf_cuda_fail(e, "device attribute");
  const int64_t n = bytes / 16;
  void* buf = nullptr;
  unsigned* sink = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  salf_status st = SALF_OK;
  float ms = 0.f;
  if ((e = cudaMalloc(&buf, (size_t)n * 16)) != cudaSuccess ||
      (e = cudaMalloc(reinterpret_cast<void**>(&sink), 16)) != cudaSuccess ||
      (e = cudaMemset(buf, 0x5a, (size_t)n * 16)) != cudaSuccess ||
      (e = cudaEventCreate(&a)) != cudaSuccess || (e = cudaEventCreate(&b)) != cudaSuccess) {
    st = salf_cuda_fail(e, "salf_measure_l2_read setup");
  } else {
    const int blocks = sms * 4;  // 4 blocks of 16 warps per SM: 64 warps, all resident
    const uint4* p = static_cast<const uint4*>(buf);
    constexpr int kPasses = 16;
    for (int w = 0; w < 3; ++w) k_l2_read<<<blocks, 512>>>(p, n, 1, 0x1234567u, sink);  // into L2
    cudaEventRecord(a);
    for (int r = 0; r < reps; ++r) k_l2_read<<<blocks, 512>>>(p, n, kPasses, 0x1234567u, sink);
    cudaEventRecord(b);
    if ((e = cudaEventSynchronize(b)) != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaEventElapsedTime(&ms, a, b)) != cudaSuccess) {
      st = salf_cuda_fail(e, "salf_measure_l2_read");
    } else {
      *gbs = (double)n * 16.0 * kPasses * reps / (ms * 1e-3) / 1e9;
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (sink) cudaFree(sink);
  if (buf) cudaFree(buf);
  return st;
}
