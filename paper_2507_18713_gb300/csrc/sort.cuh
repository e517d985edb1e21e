// sort.cuh -- stable LSD radix sort of (64-bit key, 32-bit value) pairs, 8 bits
// per pass, used by the tile rasteriser and the device scene build.
#pragma once

#include <cuda_runtime.h>

#include "scan.cuh"

namespace salf_sort {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;      // rounds per block
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;

// // LSD radix sort of the pairs, 8 bits per pass.  A block owns kSortTile
// consecutive items, read in rounds of kSortThreads (round r, thread t holds
// item r * kSortThreads + t), so the order of (round, thread) is the input
// order and the scatter below keeps it among equal digits (stable).

// Digit counts of each block's items (hist[digit * nblk + block]).
static __global__ void __launch_bounds__(kSortThreads) k_radix_hist(const unsigned long long* __restrict__ keys,
                                                             long long n, int shift,
                                                             unsigned* __restrict__ hist, int nblk) {
  __shared__ unsigned h[kRadix];
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) h[d] = 0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * kSortTile;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const long long i = base + (long long)r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(unsigned)(keys[i] >> shift) & (kRadix - 1)], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) hist[d * nblk + blockIdx.x] = h[d];
}

// Stable scatter: item goes to scanned_hist[digit][block] + (items of this
// block before it with the same digit).  Per round, lanes with equal digits
// are ranked inside their warp (match), and warps are ranked per digit
// through shared counts.
static __global__ void __launch_bounds__(kSortThreads) k_radix_scatter(
    const unsigned long long* __restrict__ kin, const unsigned* __restrict__ vin,
    unsigned long long* __restrict__ kout, unsigned* __restrict__ vout, long long n, int shift,
    const unsigned* __restrict__ hoff, int nblk) {
  constexpr int kWarps = kSortThreads / 32;
  __shared__ unsigned s_base[kRadix];          // running count per digit (earlier rounds)
  __shared__ unsigned s_warp[kWarps][kRadix];  // this round: count, then exclusive prefix
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads)
    s_base[d] = hoff[d * nblk + blockIdx.x];
  const long long base = (long long)blockIdx.x * kSortTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int r = 0; r < kSortItems; ++r) {
    const long long i = base + (long long)r * kSortThreads + threadIdx.x;
    const bool ok = i < n;
    unsigned long long key = 0;
    unsigned val = 0;
    if (ok) {
      key = kin[i];
      val = vin[i];
    }
    const unsigned d = ok ? (unsigned)(key >> shift) & (kRadix - 1) : (unsigned)kRadix;
    __syncthreads();  // the previous round's prefixes have been read
    for (int k = threadIdx.x; k < kWarps * kRadix; k += kSortThreads) (&s_warp[0][0])[k] = 0;
    __syncthreads();
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned rank = __popc(peers & lt);
    if (ok && rank == 0) s_warp[wid][d] = __popc(peers);
    __syncthreads();
    for (int dd = threadIdx.x; dd < kRadix; dd += kSortThreads) {
      unsigned run = s_base[dd];
#pragma unroll
      for (int w = 0; w < kWarps; ++w) {
        const unsigned c = s_warp[w][dd];
        s_warp[w][dd] = run;
        run += c;
      }
      s_base[dd] = run;
    }
    __syncthreads();
    if (ok) {
      const unsigned pos = s_warp[wid][d] + rank;
      kout[pos] = key;
      vout[pos] = val;
    }
  }
}

// Workspace of radix_sort_pairs for n pairs: the histogram and its scan.
inline long long radix_hist_elems(long long n) {
  const long long nblk = (n + kSortTile - 1) / kSortTile;
  return (long long)kRadix * (nblk > 0 ? nblk : 1);
}

// Sorts (ka, va) by the low `bits` bits of the keys, ping-ponging with (kb,
// vb); returns through *keys / *vals the buffers that hold the result.  hist
// and hoff hold radix_hist_elems(n) elements, htmp scan_tmp_elems of that.
inline cudaError_t radix_sort_pairs(unsigned long long* ka, unsigned* va, unsigned long long* kb,
                                    unsigned* vb, long long n, int bits, unsigned* hist,
                                    unsigned* hoff, unsigned* htmp, cudaStream_t st,
                                    int* launches, unsigned long long** keys, unsigned** vals) {
  const long long nblk = (n + kSortTile - 1) / kSortTile;
  const long long hn = radix_hist_elems(n);
  const int passes = (bits + kRadixBits - 1) / kRadixBits;
  unsigned long long *ki = ka, *ko = kb;
  unsigned *vi = va, *vo = vb;
  for (int pass = 0; pass < passes && n > 0; ++pass) {
    const int shift = kRadixBits * pass;
    k_radix_hist<<<(unsigned)nblk, kSortThreads, 0, st>>>(ki, n, shift, hist, (int)nblk);
    cudaError_t e = salf_scan::scan_exclusive<unsigned, unsigned>(hist, hn, hoff, htmp, st, launches);
    if (e != cudaSuccess) return e;
    k_radix_scatter<<<(unsigned)nblk, kSortThreads, 0, st>>>(ki, vi, ko, vo, n, shift, hoff,
                                                             (int)nblk);
    *launches += 2;
    unsigned long long* tk = ki;
    ki = ko;
    ko = tk;
    unsigned* tv = vi;
    vi = vo;
    vo = tv;
  }
  *keys = ki;
  *vals = vi;
  return cudaGetLastError();
}

}  // namespace salf_sort
