// scene_build_gpu.cu -- salf_build_scene for a voxel set already in device
// memory: the steps of the host build (scene_build.cpp) as kernels, giving
// the same acceleration structure (Sec. III-B stand-in for the octree):
//  1. per voxel its sort key (4x4x4 block of level-0 cells, Morton index of
//     the cell in the block, Morton index of the min corner in the cell) and
//     the range checks; a stable radix sort of (key, voxel) gives the voxel
//     order; neighbours in that order reveal any overlap;
//  2. level-0 occupancy words (atomic OR), each block's first voxel and
//     whether a block holds a split cell; a scan of the words' popcounts gives
//     the cells' ranks;
//  3. the cell table: level-0 voxels directly; one thread per split cell
//     builds its subtree of nodes from the cell's voxels (consecutive in the
//     voxel order) into a slice sized by an upper bound, and turns a cell
//     split once into (first child, child mask);
//  4. upper mask levels and the column pyramid by atomic OR, the tight box by
//     atomic min / max, the voxel boxes, and the records in voxel order.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>

#include "salf_internal.h"
#include "scan.cuh"
#include "sort.cuh"

using namespace salf_scan;
using namespace salf_sort;

namespace {

constexpr int kErrLevel = 1, kErrRange = 2, kErrOverlap = 4;

__device__ __forceinline__ unsigned dmorton6(unsigned x, unsigned y, unsigned z) {
  return (x & 1u) | ((y & 1u) << 1) | ((z & 1u) << 2) | ((x & 2u) << 2) | ((y & 2u) << 3) |
         ((z & 2u) << 4);
}

__device__ __forceinline__ unsigned long long dspread3(unsigned long long x) {
  x &= 0x1fffffULL;
  x = (x | x << 32) & 0x1f00000000ffffULL;
  x = (x | x << 16) & 0x1f0000ff0000ffULL;
  x = (x | x << 8) & 0x100f00f00f00f00fULL;
  x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
  x = (x | x << 2) & 0x1249249249249249ULL;
  return x;
}

struct Grid {
  int K;
  int dims[3];
  int mdim[3];  // level-0 occupancy words per axis
};

__device__ __forceinline__ long long block_of(const Grid& G, long long cx, long long cy,
                                              long long cz) {
  return ((cz >> 2) * G.mdim[1] + (cy >> 2)) * G.mdim[0] + (cx >> 2);
}

// err[0]: error bits; err[1]: smallest offending voxel; err[2]: smallest
// voxel-order position of an overlapping pair
__global__ void k_keys(const uint8_t* __restrict__ level, const int* __restrict__ ijk, long long n,
                       Grid G, unsigned long long* __restrict__ keys, unsigned* __restrict__ vals,
                       int* __restrict__ err) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  int l = level[v];
  bool bad = false;
  if (l > G.K) {
    atomicOr(&err[0], kErrLevel);
    bad = true;
    l = 0;
  }
  unsigned long long f[3];
  for (int a = 0; a < 3; ++a) {
    long long c = ijk[3 * v + a];
    if (c < 0 || c >= ((long long)G.dims[a] << l)) {
      atomicOr(&err[0], kErrRange);
      bad = true;
      c = 0;
    }
    f[a] = (unsigned long long)c << (G.K - l);
  }
  if (bad) atomicMin(&err[1], (int)v);
  const unsigned long long fine = (1ULL << G.K) - 1ULL;
  const long long blk = block_of(G, (long long)(f[0] >> G.K), (long long)(f[1] >> G.K),
                                 (long long)(f[2] >> G.K));
  keys[v] = ((unsigned long long)blk << (6 + 3 * G.K)) |
            ((unsigned long long)dmorton6((unsigned)(f[0] >> G.K) & 3, (unsigned)(f[1] >> G.K) & 3,
                                          (unsigned)(f[2] >> G.K) & 3)
             << (3 * G.K)) |
            (dspread3(f[0] & fine) | (dspread3(f[1] & fine) << 1) | (dspread3(f[2] & fine) << 2));
  vals[v] = (unsigned)v;
}

// A voxel of level l covers the key range [key, key + 8^(K - l)): in key order
// an overlap always shows between neighbours.
__global__ void k_overlap(const unsigned long long* __restrict__ keys,
                          const unsigned* __restrict__ order, const uint8_t* __restrict__ level,
                          long long n, int K, int* __restrict__ err) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x + 1;
  if (p >= n) return;
  const unsigned long long span = 1ULL << (3 * (K - level[order[p - 1]]));
  if (keys[p] < keys[p - 1] + span) {
    atomicOr(&err[0], kErrOverlap);
    atomicMin(&err[2], (int)p);
  }
}

__global__ void k_blocks(const unsigned* __restrict__ order, const uint8_t* __restrict__ level,
                         const int* __restrict__ ijk, long long n, Grid G,
                         unsigned long long* __restrict__ m0, unsigned* __restrict__ split,
                         unsigned* __restrict__ vfirst) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const unsigned v = order[p];
  const int l = level[v];
  const long long cx = ijk[3 * (long long)v] >> l, cy = ijk[3 * (long long)v + 1] >> l,
                  cz = ijk[3 * (long long)v + 2] >> l;
  const long long b = block_of(G, cx, cy, cz);
  atomicOr(&m0[b], 1ULL << dmorton6((unsigned)cx & 3, (unsigned)cy & 3, (unsigned)cz & 3));
  if (l > 0) atomicOr(&split[b], 1u);
  atomicMin(&vfirst[b], (unsigned)p);
}

__global__ void k_popcounts(const unsigned long long* __restrict__ m0, long long nb,
                            unsigned* __restrict__ cnt) {
  const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nb) cnt[b] = (unsigned)__popcll(m0[b]);
}

__global__ void k_mask0(const unsigned long long* __restrict__ m0, const unsigned* __restrict__ rank,
                        const unsigned* __restrict__ split, const unsigned* __restrict__ vfirst,
                        long long nb, uint4* __restrict__ mask0) {
  const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const unsigned long long m = m0[b];
  mask0[b] = make_uint4((unsigned)(m & 0xffffffffULL), (unsigned)(m >> 32), rank[b],
                        (m && !split[b]) ? vfirst[b] : 0xffffffffu);
}

// Cell table, level-0 voxels; for split cells their first voxel and a node
// budget (1 + sum of (level - 1) over the cell's voxels).
__global__ void k_cells(const unsigned* __restrict__ order, const unsigned long long* __restrict__ keys,
                        const uint8_t* __restrict__ level, const int* __restrict__ ijk, long long n,
                        Grid G, const uint4* __restrict__ mask0, int2* __restrict__ cells,
                        int* __restrict__ cell_first, unsigned* __restrict__ node_budget) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const unsigned v = order[p];
  const int l = level[v];
  const long long cx = ijk[3 * (long long)v] >> l, cy = ijk[3 * (long long)v + 1] >> l,
                  cz = ijk[3 * (long long)v + 2] >> l;
  const uint4 w = mask0[block_of(G, cx, cy, cz)];
  const unsigned long long m = ((unsigned long long)w.y << 32) | w.x;
  const unsigned bit = dmorton6((unsigned)cx & 3, (unsigned)cy & 3, (unsigned)cz & 3);
  const unsigned rank = w.z + (unsigned)__popcll(m & ((1ULL << bit) - 1ULL));
  if (l == 0) {
    cells[rank] = make_int2((int)p, 0);
    return;
  }
  const int sh = 3 * G.K;
  const bool first = p == 0 || (keys[p - 1] >> sh) != (keys[p] >> sh);
  if (first) cell_first[rank] = (int)p;
  atomicAdd(&node_budget[rank], (unsigned)(l - 1) + (first ? 1u : 0u));
}

// One thread per split cell: its nodes (the host build's insertion order,
// node ids from the cell's slice), then the once-split form if it applies.
__global__ void k_nodes(const unsigned* __restrict__ order, const unsigned long long* __restrict__ keys,
                        const uint8_t* __restrict__ level, const int* __restrict__ ijk, long long n,
                        int K, const int* __restrict__ cell_first,
                        const unsigned long long* __restrict__ node_off, long long n_cells,
                        int* __restrict__ nodes, int2* __restrict__ cells) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_cells) return;
  const int p0 = cell_first[r];
  if (p0 < 0) return;
  const int base = (int)node_off[r];
  int next = 1;
  const int root = base;
  const int sh = 3 * K;
  const unsigned long long cell = keys[p0] >> sh;
  for (long long p = p0; p < n && (keys[p] >> sh) == cell; ++p) {
    const unsigned v = order[p];
    const int l = level[v];
    const int i = ijk[3 * (long long)v], j = ijk[3 * (long long)v + 1], k = ijk[3 * (long long)v + 2];
    int node = root;
    for (int dl = 1; dl <= l; ++dl) {
      const int s = l - dl;
      const int slot = ((i >> s) & 1) | (((j >> s) & 1) << 1) | (((k >> s) & 1) << 2);
      int* e = &nodes[(size_t)node * 8 + slot];
      if (dl == l) {
        *e = (int)p;
      } else {
        if (*e == -1) *e = -2 - (base + next++);
        node = -2 - *e;
      }
    }
  }
  unsigned cm = 0;
  int first = -1, expect = -1;
  bool flat = true;
  for (int c = 0; c < 8 && flat; ++c) {
    const int e = nodes[(size_t)root * 8 + c];
    if (e == -1) continue;
    if (e < 0 || (expect >= 0 && e != expect)) flat = false;
    if (first < 0) first = e;
    expect = e + 1;
    cm |= 1u << c;
  }
  cells[r] = (flat && cm) ? make_int2(first, (int)cm) : make_int2(-2 - root, 0);
}

__global__ void k_up_from_mask0(const uint4* __restrict__ mask0, Grid G, int up0, int up1,
                                unsigned long long* __restrict__ up) {
  const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nb = (long long)G.mdim[0] * G.mdim[1] * G.mdim[2];
  if (w >= nb) return;
  const uint4 m = mask0[w];
  if (!(m.x | m.y)) return;
  const long long wx = w % G.mdim[0], wy = (w / G.mdim[0]) % G.mdim[1], wz = w / ((long long)G.mdim[0] * G.mdim[1]);
  atomicOr(&up[((wz >> 2) * up1 + (wy >> 2)) * up0 + (wx >> 2)],
           1ULL << dmorton6((unsigned)wx & 3, (unsigned)wy & 3, (unsigned)wz & 3));
}

__global__ void k_up(const unsigned long long* __restrict__ prev, int p0, int p1, int p2, int u0,
                     int u1, unsigned long long* __restrict__ up) {
  const long long w = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= (long long)p0 * p1 * p2) return;
  if (!prev[w]) return;
  const long long wx = w % p0, wy = (w / p0) % p1, wz = w / ((long long)p0 * p1);
  atomicOr(&up[((wz >> 2) * u1 + (wy >> 2)) * u0 + (wx >> 2)],
           1ULL << dmorton6((unsigned)wx & 3, (unsigned)wy & 3, (unsigned)wz & 3));
}

__global__ void k_col0(const uint8_t* __restrict__ level, const int* __restrict__ ijk, long long n,
                       int dims0, int layer_cells, unsigned* __restrict__ col0) {
  const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const int l = level[v];
  const long long cx = ijk[3 * v] >> l, cy = ijk[3 * v + 1] >> l, cz = ijk[3 * v + 2] >> l;
  const int layer = (int)(cz / layer_cells);
  atomicOr(&col0[(size_t)(cy * dims0 + cx) * 4 + (layer >> 5)], 1u << (layer & 31));
}

__global__ void k_colup(const uint4* __restrict__ prev, int p0, int p1, int u0,
                        unsigned* __restrict__ cur) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)p0 * p1) return;
  const uint4 a = prev[e];
  if (!(a.x | a.y | a.z | a.w)) return;
  const long long x = e % p0, y = e / p0;
  unsigned* b = cur + (size_t)((y >> 1) * u0 + (x >> 1)) * 4;
  if (a.x) atomicOr(b, a.x);
  if (a.y) atomicOr(b + 1, a.y);
  if (a.z) atomicOr(b + 2, a.z);
  if (a.w) atomicOr(b + 3, a.w);
}

// Voxel boxes in voxel order and the tight box (box[0..2] min, box[3..5] max).
__global__ void k_boxes(const unsigned* __restrict__ order, const uint8_t* __restrict__ level,
                        const int* __restrict__ ijk, long long n, int K, int4* __restrict__ vox_box,
                        int* __restrict__ box) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const unsigned v = order[p];
  const int l = level[v];
  int lo[3];
  for (int a = 0; a < 3; ++a) lo[a] = ijk[3 * (long long)v + a] << (K - l);
  vox_box[p] = make_int4(lo[0], lo[1], lo[2], K - l);
  for (int a = 0; a < 3; ++a) {
    atomicMin(&box[a], lo[a]);
    atomicMax(&box[3 + a], lo[a] + (1 << (K - l)));
  }
}

int bit_width_ll(unsigned long long x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Temporary device memory freed on scope exit.
struct Temp {
  void* p = nullptr;
  ~Temp() {
    if (p) cudaFree(p);
  }
};

}  // namespace

salf_status salf_build_scene_gpu(salf_ctx* ctx, const salf_scene_desc* d, salf_scene** out) {
  const int K = d->max_level;
  const long long n = d->n;
  cudaError_t ce = cudaSetDevice(ctx->device);
  if (ce != cudaSuccess) return salf_cuda_fail(ce, "cudaSetDevice");
  // grid geometry (host): the same level sizes as the host build
  int mdim[SALF_MAX_MASK_LEVELS][3];
  for (int a = 0; a < 3; ++a) mdim[0][a] = (d->dims[a] + 3) / 4;
  int M = 1;
  while (!(mdim[M - 1][0] == 1 && mdim[M - 1][1] == 1 && mdim[M - 1][2] == 1)) {
    if (M >= SALF_MAX_MASK_LEVELS) {
      salf_set_error("salf_build_scene: grid too large for the pyramid");
      return SALF_ERR_INVALID;
    }
    for (int a = 0; a < 3; ++a) mdim[M][a] = (mdim[M - 1][a] + 3) / 4;
    ++M;
  }
  int layer_cells = 1;
  while ((d->dims[2] + layer_cells - 1) / layer_cells > 128) layer_cells *= 2;
  const int n_layers = (d->dims[2] + layer_cells - 1) / layer_cells;
  int cdim[SALF_MAX_COL_LEVELS][2];
  cdim[0][0] = d->dims[0];
  cdim[0][1] = d->dims[1];
  int CL = 1;
  while ((cdim[CL - 1][0] > 1 || cdim[CL - 1][1] > 1) && CL < SALF_MAX_COL_LEVELS) {
    cdim[CL][0] = (cdim[CL - 1][0] + 1) / 2;
    cdim[CL][1] = (cdim[CL - 1][1] + 1) / 2;
    ++CL;
  }
  const long long nb0 = (long long)mdim[0][0] * mdim[0][1] * mdim[0][2];
  Grid G;
  G.K = K;
  for (int a = 0; a < 3; ++a) {
    G.dims[a] = d->dims[a];
    G.mdim[a] = mdim[0][a];
  }
  const long long nn = std::max(n, 1LL);
  const int key_bits = std::max(1, bit_width_ll((unsigned long long)std::max(nb0 - 1, 1LL)) + 6 + 3 * K);
  if (key_bits > 64) {
    salf_set_error("salf_build_scene: grid too large for 64-bit voxel keys");
    return SALF_ERR_INVALID;
  }

  // temporaries
  const long long hn = radix_hist_elems(nn);
  const size_t b_k = a256(nn * 8), b_v = a256(nn * 4), b_h = a256(hn * 4),
               b_ht = a256(scan_tmp_elems(hn) * 4), b_m0 = a256(nb0 * 8), b_b = a256(nb0 * 4),
               b_rank = a256((nb0 + 1) * 4), b_rt = a256(scan_tmp_elems(nb0) * 4),
               b_cf = a256(nn * 4), b_nb = a256(nn * 4), b_no = a256((nn + 1) * 8),
               b_nt = a256(scan_tmp_elems(nn) * 8), b_err = 256;
  const size_t tbytes = 2 * b_k + 2 * b_v + 2 * b_h + b_ht + b_m0 + 3 * b_b + b_rank + b_rt +
                        b_cf + b_nb + b_no + b_nt + b_err;
  Temp tmp;
  if (cudaMalloc(&tmp.p, tbytes) != cudaSuccess) {
    cudaGetLastError();
    salf_set_error("salf_build_scene: out of device memory (build workspace)");
    return SALF_ERR_OOM;
  }
  char* t = static_cast<char*>(tmp.p);
  size_t o = 0;
  auto take = [&](size_t b) { char* q = t + o; o += b; return q; };
  auto* kA = reinterpret_cast<unsigned long long*>(take(b_k));
  auto* kB = reinterpret_cast<unsigned long long*>(take(b_k));
  auto* vA = reinterpret_cast<unsigned*>(take(b_v));
  auto* vB = reinterpret_cast<unsigned*>(take(b_v));
  auto* hist = reinterpret_cast<unsigned*>(take(b_h));
  auto* hoff = reinterpret_cast<unsigned*>(take(b_h));
  auto* htmp = reinterpret_cast<unsigned*>(take(b_ht));
  auto* m0 = reinterpret_cast<unsigned long long*>(take(b_m0));
  auto* split = reinterpret_cast<unsigned*>(take(b_b));
  auto* vfirst = reinterpret_cast<unsigned*>(take(b_b));
  auto* cnt = reinterpret_cast<unsigned*>(take(b_b));
  auto* rank = reinterpret_cast<unsigned*>(take(b_rank));
  auto* rtmp = reinterpret_cast<unsigned*>(take(b_rt));
  auto* cell_first = reinterpret_cast<int*>(take(b_cf));
  auto* node_budget = reinterpret_cast<unsigned*>(take(b_nb));
  auto* node_off = reinterpret_cast<unsigned long long*>(take(b_no));
  auto* ntmp = reinterpret_cast<unsigned long long*>(take(b_nt));
  auto* err = reinterpret_cast<int*>(take(b_err));  // err[0..2], box[3..8]
  int* box = err + 4;
  cudaStream_t st = 0;
  const auto grid = [](long long m) { return (unsigned)((std::max(m, 1LL) + 255) / 256); };
  int launches = 0;

  int herr[4] = {0, INT_MAX, INT_MAX, 0};
  int hbox[6];
  for (int a = 0; a < 3; ++a) {
    hbox[a] = d->dims[a] << K;
    hbox[3 + a] = 0;
  }
  if ((ce = cudaMemcpy(err, herr, sizeof(herr), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (ce = cudaMemcpy(box, hbox, sizeof(hbox), cudaMemcpyHostToDevice)) != cudaSuccess ||
      (ce = cudaMemsetAsync(m0, 0, nb0 * 8, st)) != cudaSuccess ||
      (ce = cudaMemsetAsync(split, 0, nb0 * 4, st)) != cudaSuccess ||
      (ce = cudaMemsetAsync(vfirst, 0xff, nb0 * 4, st)) != cudaSuccess ||
      (ce = cudaMemsetAsync(cell_first, 0xff, nn * 4, st)) != cudaSuccess ||
      (ce = cudaMemsetAsync(node_budget, 0, nn * 4, st)) != cudaSuccess)
    return salf_cuda_fail(ce, "build workspace init");

  // 1. keys, sort, overlap
  const uint8_t* level = d->level;
  const int* ijk = d->ijk;
  unsigned long long* keys = kA;
  unsigned* order = vA;
  if (n > 0) {
    k_keys<<<grid(n), 256, 0, st>>>(level, ijk, n, G, kA, vA, err);
    if ((ce = radix_sort_pairs(kA, vA, kB, vB, n, key_bits, hist, hoff, htmp, st, &launches, &keys,
                               &order)) != cudaSuccess)
      return salf_cuda_fail(ce, "build sort");
    if (n > 1) k_overlap<<<grid(n - 1), 256, 0, st>>>(keys, order, level, n, K, err);
  }
  if ((ce = cudaMemcpy(herr, err, sizeof(herr), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return salf_cuda_fail(ce, "build checks");
  if (herr[0] & (kErrLevel | kErrRange)) {
    salf_set_error("salf_build_scene: voxel " + std::to_string(herr[1]) +
                   ((herr[0] & kErrLevel) ? " has level > max_level" : " outside the grid"));
    return SALF_ERR_INVALID;
  }
  if (herr[0] & kErrOverlap) {
    unsigned pair[2] = {0, 0};
    cudaMemcpy(pair, order + herr[2] - 1, 8, cudaMemcpyDeviceToHost);
    salf_set_error("salf_build_scene: voxels " + std::to_string(pair[0]) + " and " +
                   std::to_string(pair[1]) + " overlap");
    return SALF_ERR_OVERLAP;
  }

  salf_scene* s = new salf_scene();
  struct Guard {
    salf_scene* s;
    bool keep = false;
    ~Guard() {
      if (!keep) salf_scene_destroy(s);
    }
  } guard{s};
  s->ctx = ctx;
  s->device = ctx->device;
  s->n = n;
  s->mode = d->mode;
  s->dtype = d->dtype;
  s->K = K;
  for (int a = 0; a < 3; ++a) {
    s->dims[a] = d->dims[a];
    s->origin[a] = d->origin[a];
  }
  s->s0 = d->s0;
  s->sfin = d->s0 / (double)(1 << K);
  DevScene& D = s->dev;
  std::memset(&D, 0, sizeof(D));
  salf_status sst;
  auto alloc = [&](size_t bytes, void** p) { return salf_scene_dalloc(s, bytes, p); };

  // 2. level-0 words, ranks
  void* pmask0 = nullptr;
  if ((sst = alloc(nb0 * sizeof(uint4), &pmask0)) != SALF_OK) return sst;
  uint4* mask0 = static_cast<uint4*>(pmask0);
  if (n > 0) k_blocks<<<grid(n), 256, 0, st>>>(order, level, ijk, n, G, m0, split, vfirst);
  k_popcounts<<<grid(nb0), 256, 0, st>>>(m0, nb0, cnt);
  if ((ce = scan_exclusive<unsigned, unsigned>(cnt, nb0, rank, rtmp, st, &launches)) != cudaSuccess)
    return salf_cuda_fail(ce, "build rank scan");
  k_scan_total<unsigned, unsigned><<<1, 1, 0, st>>>(cnt, nb0, rank);
  k_mask0<<<grid(nb0), 256, 0, st>>>(m0, rank, split, vfirst, nb0, mask0);
  unsigned n_cells = 0;
  if ((ce = cudaMemcpy(&n_cells, rank + nb0, 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return salf_cuda_fail(ce, "build cell count");

  // 3. cell table and nodes
  void* pcells = nullptr;
  if ((sst = alloc(std::max<size_t>(n_cells, 1) * sizeof(int2), &pcells)) != SALF_OK) return sst;
  int2* cells = static_cast<int2*>(pcells);
  if ((ce = cudaMemsetAsync(cells, 0xff, std::max<size_t>(n_cells, 1) * sizeof(int2), st)) !=
      cudaSuccess)
    return salf_cuda_fail(ce, "build cells init");
  if (n > 0)
    k_cells<<<grid(n), 256, 0, st>>>(order, keys, level, ijk, n, G, mask0, cells, cell_first,
                                     node_budget);
  unsigned long long n_nodes = 0;
  if (n_cells > 0) {
    if ((ce = scan_exclusive<unsigned, unsigned long long>(node_budget, n_cells, node_off, ntmp, st,
                                                           &launches)) != cudaSuccess)
      return salf_cuda_fail(ce, "build node scan");
    k_scan_total<unsigned, unsigned long long><<<1, 1, 0, st>>>(node_budget, n_cells, node_off);
    if ((ce = cudaMemcpy(&n_nodes, node_off + n_cells, 8, cudaMemcpyDeviceToHost)) != cudaSuccess)
      return salf_cuda_fail(ce, "build node count");
  }
  const size_t nodes_n = std::max<unsigned long long>(n_nodes, 1);
  void* pnodes = nullptr;
  if ((sst = alloc(nodes_n * 8 * sizeof(int), &pnodes)) != SALF_OK) return sst;
  int* nodes = static_cast<int*>(pnodes);
  if ((ce = cudaMemsetAsync(nodes, 0xff, nodes_n * 8 * sizeof(int), st)) != cudaSuccess)
    return salf_cuda_fail(ce, "build nodes init");
  if (n_nodes > 0)
    k_nodes<<<grid(n_cells), 256, 0, st>>>(order, keys, level, ijk, n, K, cell_first, node_off,
                                           n_cells, nodes, cells);

  // 4. upper mask levels
  D.mask0 = mask0;
  for (int m = 1; m < M; ++m) {
    void* pu = nullptr;
    const size_t words = (size_t)mdim[m][0] * mdim[m][1] * mdim[m][2];
    if ((sst = alloc(words * 8, &pu)) != SALF_OK) return sst;
    if ((ce = cudaMemsetAsync(pu, 0, words * 8, st)) != cudaSuccess)
      return salf_cuda_fail(ce, "build mask init");
    auto* up = static_cast<unsigned long long*>(pu);
    if (m == 1)
      k_up_from_mask0<<<grid(nb0), 256, 0, st>>>(mask0, G, mdim[1][0], mdim[1][1], up);
    else
      k_up<<<grid((long long)mdim[m - 1][0] * mdim[m - 1][1] * mdim[m - 1][2]), 256, 0, st>>>(
          D.mask[m - 1], mdim[m - 1][0], mdim[m - 1][1], mdim[m - 1][2], mdim[m][0], mdim[m][1],
          up);
    D.mask[m] = up;
  }
  for (int m = 0; m < M; ++m)
    for (int a = 0; a < 3; ++a) D.mdim[m][a] = mdim[m][a];
  // column pyramid
  for (int c = 0; c < CL; ++c) {
    void* pc = nullptr;
    const size_t e = (size_t)cdim[c][0] * cdim[c][1];
    if ((sst = alloc(e * sizeof(uint4), &pc)) != SALF_OK) return sst;
    if ((ce = cudaMemsetAsync(pc, 0, e * sizeof(uint4), st)) != cudaSuccess)
      return salf_cuda_fail(ce, "build column init");
    if (c == 0) {
      if (n > 0)
        k_col0<<<grid(n), 256, 0, st>>>(level, ijk, n, d->dims[0], layer_cells,
                                        static_cast<unsigned*>(pc));
    } else {
      k_colup<<<grid((long long)cdim[c - 1][0] * cdim[c - 1][1]), 256, 0, st>>>(
          D.col[c - 1], cdim[c - 1][0], cdim[c - 1][1], cdim[c][0], static_cast<unsigned*>(pc));
    }
    D.col[c] = static_cast<uint4*>(pc);
    D.cdim[c][0] = cdim[c][0];
    D.cdim[c][1] = cdim[c][1];
  }
  D.CL = CL;
  {
    int ls = 0;
    while ((1 << ls) < layer_cells) ++ls;
    D.layer_shift = ls + K;
  }
  D.n_layers = n_layers;
  // voxel order, boxes, tight box
  void *pord = nullptr, *pbox = nullptr;
  if ((sst = alloc(nn * sizeof(int), &pord)) != SALF_OK) return sst;
  if ((sst = alloc(nn * sizeof(int4), &pbox)) != SALF_OK) return sst;
  if (n > 0) {
    if ((ce = cudaMemcpyAsync(pord, order, n * sizeof(int), cudaMemcpyDeviceToDevice, st)) !=
        cudaSuccess)
      return salf_cuda_fail(ce, "build order");
    k_boxes<<<grid(n), 256, 0, st>>>(order, level, ijk, n, K, static_cast<int4*>(pbox), box);
  } else if ((ce = cudaMemsetAsync(pord, 0, sizeof(int), st)) != cudaSuccess ||
             (ce = cudaMemsetAsync(pbox, 0, sizeof(int4), st)) != cudaSuccess) {
    return salf_cuda_fail(ce, "build order");
  }
  D.cells = cells;
  D.nodes = nodes;
  D.order = static_cast<int*>(pord);
  D.vox_box = static_cast<int4*>(pbox);
  void* status = nullptr;
  if ((sst = alloc(16, &status)) != SALF_OK) return sst;
  if ((ce = cudaMemsetAsync(status, 0, 16, st)) != cudaSuccess)
    return salf_cuda_fail(ce, "cudaMemset");
  D.status = static_cast<int*>(status);
  void* params = nullptr;
  const size_t rec_bytes = d->dtype == SALF_F32 ? 128 : 64;
  if ((sst = alloc(nn * rec_bytes, &params)) != SALF_OK) return sst;
  D.params = params;
  for (int a = 0; a < 3; ++a) {
    D.origin[a] = d->origin[a];
    D.Gf[a] = d->dims[a] << K;
  }
  D.inv_sfin = 1.0 / s->sfin;
  D.K = K;
  D.M = M;
  D.mode = d->mode;
  D.dtype = d->dtype;
  D.n = (int)n;
  if (n > 0) {
    if ((ce = salf_launch_gather_params(d->params, D.order, params, n, d->dtype, d->mode, D.status,
                                        st)) != cudaSuccess)
      return salf_cuda_fail(ce, "gather params");
  }
  if ((ce = cudaMemcpy(hbox, box, sizeof(hbox), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return salf_cuda_fail(ce, "build box");
  for (int a = 0; a < 3; ++a) {
    D.bmin[a] = n > 0 ? hbox[a] : 0;
    D.bmax[a] = n > 0 ? hbox[3 + a] : 0;
  }
  s->n_cells0 = n_cells;
  s->n_nodes = (int64_t)n_nodes;
  int flag = 0;
  if ((ce = cudaMemcpy(&flag, D.status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return salf_cuda_fail(ce, "build status");
  if (flag & SALF_DEVERR_SDF_AB) {
    salf_set_error("salf_build_scene: SDF records need a > 0 and b > 0 (Eq. 6)");
    return SALF_ERR_INVALID;
  }
  guard.keep = true;
  *out = s;
  return SALF_OK;
}
