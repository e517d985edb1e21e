// scan.cuh -- device-wide exclusive prefix sum (tiles of 4096 elements scanned
// by 1024-thread blocks, block totals scanned recursively, then added back),
// used by the tile rasteriser and by scene refinement.
#pragma once

#include <cuda_runtime.h>

namespace salf_scan {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

template <class T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* total) {
  __shared__ T warp_tot[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    T t = lane < nw ? warp_tot[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) warp_tot[lane] = t;  // inclusive
  }
  __syncthreads();
  const T before = wid > 0 ? warp_tot[wid - 1] : T(0);
  *total = warp_tot[(blockDim.x >> 5) - 1];
  __syncthreads();  // warp_tot is reused by the next call
  return before + x - v;
}

// Exclusive scan of tiles of kScanTile elements; block sums to bsum.
template <class Tin, class Tout>
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const Tin* __restrict__ in, long long n,
                                                             Tout* __restrict__ out,
                                                             Tout* __restrict__ bsum) {
  const long long i0 = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  Tout v[kScanItems];
  Tout s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    v[k] = i0 + k < n ? (Tout)in[i0 + k] : Tout(0);
    s += v[k];
  }
  Tout tot;
  Tout run = block_exclusive_scan<Tout>(s, &tot);
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    if (i0 + k < n) out[i0 + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

template <class T>
__global__ void __launch_bounds__(256) k_scan_add(T* __restrict__ out, long long n,
                                                  const T* __restrict__ boff) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += boff[i / kScanTile];
}

// out[n] = total (the scan's exclusive value past the end).
template <class Tin, class Tout>
__global__ void k_scan_total(const Tin* in, long long n, Tout* out) {
  out[n] = n > 0 ? out[n - 1] + (Tout)in[n - 1] : Tout(0);
}

// Elements of `tmp` scan_exclusive needs for n elements.
inline long long scan_tmp_elems(long long n) {
  long long t = 0;
  while (n > 1) {
    n = (n + kScanTile - 1) / kScanTile;
    t += 2 * n;
  }
  return t + 2;
}

// Device-wide exclusive scan of n elements into out (out may not alias in);
// `launches` counts the kernels enqueued.
template <class Tin, class Tout>
cudaError_t scan_exclusive(const Tin* in, long long n, Tout* out, Tout* tmp, cudaStream_t st,
                           int* launches) {
  if (n <= 0) return cudaSuccess;
  const long long nb = (n + kScanTile - 1) / kScanTile;
  Tout* bsum = tmp;
  Tout* boff = tmp + nb;
  k_scan_tiles<Tin, Tout><<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, out, bsum);
  ++*launches;
  if (nb > 1) {
    cudaError_t e = scan_exclusive<Tout, Tout>(bsum, nb, boff, tmp + 2 * nb, st, launches);
    if (e != cudaSuccess) return e;
    k_scan_add<Tout><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, n, boff);
    ++*launches;
  }
  return cudaGetLastError();
}

}  // namespace salf_scan
