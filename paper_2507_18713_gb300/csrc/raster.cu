// raster.cu -- tile rasterisation of a pinhole camera (Sec. III-B,
// "Tile-based Splatting").
//
// Pipeline, all on the device except one read of the pair count:
//  1. k_project: per voxel, the pixel rectangle its projection may cover
//     (near-plane aware, widened by two pixels), the 16 x 16 tiles it touches
//     and its camera-order key;
//  2. exclusive scan of the tile counts -> each voxel's slot range;
//  3. k_emit: one (tile | key, voxel) pair per touched tile;
//  4. stable LSD radix sort of the pairs, 8 bits per pass;
//  5. k_tile_ranges: each tile's slice of the sorted pairs;
//  6. k_raster: one 256-thread block per tile, one thread per pixel; the
//     tile's voxels are staged 64 at a time in shared memory (records raw,
//     boxes as plane offsets) and composited front to back with early
//     termination, with the ray kernel's ray set-up, slab test and field code.
//
// Camera-order key: the L1 distance (in level-0 cells) of the voxel's level-0
// cell from the camera's level-0 cell, then the voxel's octree digits inside
// its level-0 cell, each digit XOR-ed with the camera's side of that node's
// split planes (nearest child first).  Along any ray from the camera every
// axis coordinate moves away from the camera, so the L1 distance of the
// level-0 cells it enters strictly grows, and inside a cell the ray meets
// children in nearest-first octree order: sorting by the key gives every
// pixel's voxels in the order of its ray.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "scan.cuh"
#include "sort.cuh"
#include "traverse.cuh"

using namespace salf;
using namespace salf_scan;
using namespace salf_sort;

namespace {

#ifndef SALF_RASTER_MIN_BLOCKS
#define SALF_RASTER_MIN_BLOCKS 3  // resident tile blocks per SM the register budget allows
#endif

constexpr int kTile = 16;          // tile edge in pixels
constexpr int kRasterThreads = kTile * kTile;
#ifndef SALF_RASTER_CHUNK
#define SALF_RASTER_CHUNK 128
#endif
constexpr int kChunk = SALF_RASTER_CHUNK;  // voxels staged in shared memory at a time

struct ProjParams {
  DevScene S;
  float R0[9];        // camera -> world rotation, row-major
  int Oi[3];          // camera origin, finest cells: Oi + Of
  float Of[3];
  float fx, fy, cx, cy;
  int W, H, tiles_x, tiles_y;
  int ce[3];          // camera's level-0 cell
  int dig_shift;      // 3 K: bits of the octree digits
  unsigned* count;    // tiles per voxel
  uint2* rect;        // tile rectangle (x0 | y0 << 16, x1 | y1 << 16)
  int4* prect;        // pixel rectangle (u0, u1, v0, v1), inclusive
  unsigned long long* key;
  unsigned long long* n_visible;  // voxels listed in at least one tile
};

// ---------------------------------------------------------------- projection

// Tiles, tile rectangle and camera-order key of voxel p; returns the tile count.
__device__ __forceinline__ unsigned project_one(const ProjParams& G, int p) {
  const int4 b = __ldg(&G.S.vox_box[p]);
  const float E = (float)(1 << b.w);
  const int lo[3] = {b.x, b.y, b.z};
  float rl[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) rl[a] = (float)(lo[a] - G.Oi[a]) - G.Of[a];
  // camera coordinates of the min corner and of the three edges
  float base[3], ex[3], ey[3], ez[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    base[j] = G.R0[j] * rl[0] + G.R0[3 + j] * rl[1] + G.R0[6 + j] * rl[2];
    ex[j] = E * G.R0[j];
    ey[j] = E * G.R0[3 + j];
    ez[j] = E * G.R0[6 + j];
  }
  float pc[8][3];
#pragma unroll
  for (int c = 0; c < 8; ++c)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      pc[c][j] = base[j] + ((c & 1) ? ex[j] : 0.f) + ((c & 2) ? ey[j] : 0.f) + ((c & 4) ? ez[j] : 0.f);
  float umin = __int_as_float(0x7f800000), umax = -umin, vmin = umin, vmax = -umin;
  bool front = false;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    if (pc[c][2] > 0.f) {
      front = true;
      const float iz = 1.f / pc[c][2];
      const float u = fmaf(G.fx * pc[c][0], iz, G.cx), v = fmaf(G.fy * pc[c][1], iz, G.cy);
      umin = fminf(umin, u);
      umax = fmaxf(umax, u);
      vmin = fminf(vmin, v);
      vmax = fmaxf(vmax, v);
    }
  }
  unsigned cnt = 0;
  uint2 rc = make_uint2(0, 0);
  int4 pr = make_int4(1, 0, 1, 0);  // empty
  if (front) {
    // box points close to the camera plane project without bound, in the
    // direction of where the box's edges cross that plane
#pragma unroll
    for (int c = 0; c < 8; ++c)
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int c2 = c | (1 << a);
        if (c2 == c) continue;
        const float z1 = pc[c][2], z2 = pc[c2][2];
        if ((z1 > 0.f) == (z2 > 0.f)) continue;
        const float t = z1 / (z1 - z2);
        const float x0 = fmaf(t, pc[c2][0] - pc[c][0], pc[c][0]);
        const float y0 = fmaf(t, pc[c2][1] - pc[c][1], pc[c][1]);
        if (x0 >= 0.f) umax = __int_as_float(0x7f800000);
        if (x0 <= 0.f) umin = -__int_as_float(0x7f800000);
        if (y0 >= 0.f) vmax = __int_as_float(0x7f800000);
        if (y0 <= 0.f) vmin = -__int_as_float(0x7f800000);
      }
    // pixel (u, v) has its ray through (u + 0.5, v + 0.5); two pixels of margin
    const float fu0 = fmaxf(floorf(umin) - 2.f, -1.f), fu1 = fminf(floorf(umax) + 2.f, (float)G.W);
    const float fv0 = fmaxf(floorf(vmin) - 2.f, -1.f), fv1 = fminf(floorf(vmax) + 2.f, (float)G.H);
    const int u0 = max((int)fu0, 0), u1 = min((int)fu1, G.W - 1);
    const int v0 = max((int)fv0, 0), v1 = min((int)fv1, G.H - 1);
    if (u0 <= u1 && v0 <= v1 && fu1 >= 0.f && fv1 >= 0.f && fu0 < (float)G.W && fv0 < (float)G.H) {
      const int tx0 = u0 / kTile, tx1 = u1 / kTile, ty0 = v0 / kTile, ty1 = v1 / kTile;
      cnt = (unsigned)((tx1 - tx0 + 1) * (ty1 - ty0 + 1));
      rc = make_uint2((unsigned)tx0 | ((unsigned)ty0 << 16), (unsigned)tx1 | ((unsigned)ty1 << 16));
      pr = make_int4(u0, u1, v0, v1);
    }
  }
  G.count[p] = cnt;
  G.rect[p] = rc;
  G.prect[p] = pr;
  // camera-order key
  const int K = G.S.K;
  unsigned l1 = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) l1 += (unsigned)abs((lo[a] >> K) - G.ce[a]);
  unsigned long long dig = 0;
  const int lev = K - b.w;  // voxel level: digits 1..lev are defined
  for (int j = 1; j <= lev; ++j) {
    unsigned dj = 0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int node_lo = (lo[a] >> (K - j + 1)) << (K - j + 1);
      const int mid = node_lo + (1 << (K - j));
      const unsigned side = G.Oi[a] >= mid ? 1u : 0u;  // camera at or beyond the split
      dj |= ((((unsigned)lo[a] >> (K - j)) & 1u) ^ side) << a;
    }
    dig |= (unsigned long long)dj << (3 * (K - j));
  }
  G.key[p] = ((unsigned long long)l1 << G.dig_shift) | dig;
  return cnt;
}

__global__ void __launch_bounds__(256) k_project(const __grid_constant__ ProjParams G) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = p < G.S.n;
  unsigned cnt = 0;
  if (live) cnt = project_one(G, p);
  const int nvis = __syncthreads_count(cnt > 0);
  if (threadIdx.x == 0 && nvis) atomicAdd(G.n_visible, (unsigned long long)nvis);
}

__global__ void __launch_bounds__(256) k_emit(const unsigned* __restrict__ count,
                                              const uint2* __restrict__ rect,
                                              const unsigned long long* __restrict__ key,
                                              const unsigned long long* __restrict__ offs, int n,
                                              int tiles_x, int key_bits_low,
                                              unsigned long long* __restrict__ out_key,
                                              unsigned* __restrict__ out_val) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n || count[p] == 0) return;
  const uint2 rc = rect[p];
  const int tx0 = rc.x & 0xffff, ty0 = rc.x >> 16, tx1 = rc.y & 0xffff, ty1 = rc.y >> 16;
  unsigned long long o = offs[p];
  const unsigned long long k = key[p];
  for (int ty = ty0; ty <= ty1; ++ty)
    for (int tx = tx0; tx <= tx1; ++tx, ++o) {
      out_key[o] = ((unsigned long long)(ty * tiles_x + tx) << key_bits_low) | k;
      out_val[o] = (unsigned)p;
    }
}

__global__ void __launch_bounds__(256) k_tile_ranges(const unsigned long long* __restrict__ keys,
                                                     long long n, int low_bits,
                                                     uint2* __restrict__ ranges) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned t = (unsigned)(keys[i] >> low_bits);
  if (i == 0 || (unsigned)(keys[i - 1] >> low_bits) != t) ranges[t].x = (unsigned)i;
  if (i == n - 1 || (unsigned)(keys[i + 1] >> low_bits) != t) ranges[t].y = (unsigned)(i + 1);
}

// ---------------------------------------------------------------- tiles

struct RasterParams {
  DevScene S;
  ReqDev Q;
  const uint2* ranges;
  const unsigned* vox;
  const int4* prect;  // per voxel: pixel rectangle its projection may cover
  int tiles_x;
};

template <int DT, int MODE, bool DUMP>
__global__ void __launch_bounds__(kRasterThreads, SALF_RASTER_MIN_BLOCKS) k_raster(const __grid_constant__ RasterParams RP) {
  constexpr int RQ = RecordLayout<DT>::kChunks;
  constexpr int RS = RQ + 1;  // padded record stride: lanes reading different records hit different banks
  __shared__ float4 s_rec[kChunk * RS];
  __shared__ float s_pl[kChunk][6];  // plane offsets: (lo - Oi) - Of, (hi - Oi) - Of per axis
  __shared__ int4 s_box[kChunk];
  __shared__ int4 s_prect[kChunk];
  __shared__ int s_vox[kChunk];
  const DevScene& S = RP.S;
  const ReqDev& Q = RP.Q;
  const int tile = blockIdx.x;
  const int lane = threadIdx.x & 31;
  const int u = (tile % RP.tiles_x) * kTile + (threadIdx.x % kTile);
  const int v = (tile / RP.tiles_x) * kTile + (threadIdx.x / kTile);
  // this warp's pixels: 16 columns x 2 rows
  const int strip_u0 = (tile % RP.tiles_x) * kTile, strip_u1 = strip_u0 + kTile - 1;
  const int strip_v0 = (tile / RP.tiles_x) * kTile + 2 * (threadIdx.x >> 5), strip_v1 = strip_v0 + 1;
  const bool in_img = u < Q.W && v < Q.H;
  const int ray = v * Q.W + u;

  Ray r;
  Walk w;
  w.alive = false;
  r.valid = false;
  r.d[0] = r.d[1] = r.d[2] = 0.f;
  if (in_img) {
    gen_ray_pinhole(Q, u, v, r);  // the rasteriser serves pinhole cameras with one pose
    walk_init(S, r, w);
  }
  float gam[4];
  sh_basis(r.d, gam);
  const bool want_int = Q.want_int != 0;
  const float tmin = Q.t_min;
  const float t0 = w.t;
  bool pos[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) pos[a] = w.D[a] > 0.f;
  Accum A{1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0};

  const uint2 rg = RP.ranges[tile];
  for (unsigned c0 = rg.x; c0 < rg.y; c0 += kChunk) {
    const int n = (int)min((unsigned)kChunk, rg.y - c0);
    __syncthreads();  // the previous chunk is no longer read
    for (int i = threadIdx.x; i < n * RQ; i += kRasterThreads) {
      const int j = i / RQ, k = i % RQ;
      const unsigned vx = __ldg(&RP.vox[c0 + j]);
      s_rec[j * RS + k] = __ldg(reinterpret_cast<const float4*>(S.params) + (size_t)vx * RQ + k);
    }
    for (int i = threadIdx.x; i < n; i += kRasterThreads) {
      const unsigned vx = __ldg(&RP.vox[c0 + i]);
      const int4 b = __ldg(&S.vox_box[vx]);
      const int E = 1 << b.w;
      const int lo[3] = {b.x, b.y, b.z};
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        s_pl[i][a] = (float)(lo[a] - Q.Oi[a]) - Q.Of[a];
        s_pl[i][3 + a] = (float)(lo[a] + E - Q.Oi[a]) - Q.Of[a];
      }
      s_box[i] = b;
      s_prect[i] = __ldg(&RP.prect[vx]);
      s_vox[i] = (int)vx;
    }
    __syncthreads();
    // voxels whose pixel rectangle meets this warp's 16 x 2 pixel strip
    unsigned sel[kChunk / 32];
#pragma unroll
    for (int q = 0; q < kChunk / 32; ++q) {
      const int j = q * 32 + lane;
      bool meet = false;
      if (j < n) {
        const int4 pr = s_prect[j];
        meet = pr.x <= strip_u1 && pr.y >= strip_u0 && pr.z <= strip_v1 && pr.w >= strip_v0;
      }
      sel[q] = __ballot_sync(0xffffffffu, meet);
    }
    // slab test with the ray kernel's expressions (same plane values)
    auto slab = [&](int j, float* tin_out, float* tout_out) {
      float tx[3], tin = t0;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const float pe = pos[a] ? s_pl[j][3 + a] : s_pl[j][a];
        const float pn = pos[a] ? s_pl[j][a] : s_pl[j][3 + a];
        tx[a] = pe * w.invD[a];
        tin = fmaxf(tin, pn * w.invD[a]);
      }
      // the exit is the nearest exit plane (the ray kernel's tx[ax]: the same value, as the
      // distances are finite), taken as a minimum so the distances stay in registers
      *tin_out = tin;
      *tout_out = fminf(fminf(fminf(tx[0], tx[1]), tx[2]), w.tend);
    };
    // phase 1: which of the strip's voxels this pixel's ray crosses
    unsigned hits[kChunk / 32];
#pragma unroll
    for (int q = 0; q < kChunk / 32; ++q) {
      hits[q] = 0u;
      unsigned m = w.alive ? sel[q] : 0u;
      while (m) {
        const int jj = __ffs(m) - 1;
        m &= m - 1;
        const int j = q * 32 + jj;
        const int4 pr = s_prect[j];  // outside it, the ray misses the box
        if (u < pr.x || u > pr.y || v < pr.z || v > pr.w) continue;
        float tin, tout;
        slab(j, &tin, &tout);
        if (tout > tin) hits[q] |= 1u << jj;
      }
    }
    // phase 2: the lanes composite their next hit together, in list order
#pragma unroll
    for (int q = 0; q < kChunk / 32; ++q) {
      while (__any_sync(0xffffffffu, w.alive && hits[q] != 0u)) {
        if (w.alive && hits[q]) {
          const int jj = __ffs(hits[q]) - 1;
          hits[q] &= hits[q] - 1;
          const int j = q * 32 + jj;
          float tin, tout;
          slab(j, &tin, &tout);
          const int4 b = s_box[j];
          Hit h;
          h.vox = s_vox[j];
          h.ls = b.w;
          h.base[0] = b.x;
          h.base[1] = b.y;
          h.base[2] = b.z;
          h.tin = tin;
          h.tout = tout;
          composite_hit<DT, MODE>(w, h, SharedRec{&s_rec[j * RS]}, want_int, gam, A);
          if (DUMP) {
            if (A.nvis < Q.vcap) Q.visits[(size_t)ray * Q.vcap + A.nvis] = __ldg(&S.order[h.vox]);
          }
          ++A.nvis;
          if (A.T < tmin) w.alive = false;
        }
      }
    }
    if (__syncthreads_count(w.alive) == 0) break;
  }
  if (!in_img) return;
  write_outputs(Q, ray, r.valid, A);
  if (DUMP && Q.vcap > 0) {
    Q.vcount[ray] = A.nvis;
    for (int k = A.nvis; k < Q.vcap; ++k) Q.visits[(size_t)ray * Q.vcap + k] = -1;
  }
}

template <int DT, int MODE>
void launch_raster(const RasterParams& RP, int ntiles, bool dump, cudaStream_t st) {
  if (ntiles <= 0) return;
  if (dump)
    k_raster<DT, MODE, true><<<ntiles, kRasterThreads, 0, st>>>(RP);
  else
    k_raster<DT, MODE, false><<<ntiles, kRasterThreads, 0, st>>>(RP);
}

int bit_width(unsigned long long x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

salf_status salf_raster_run(salf_scene* sc, const ReqDev& r, double fx, double fy,
                            salf_raster_stats* stats, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(sc->raster_mu);
  cudaError_t e;
  // GPU work of this call runs after the previous call's (the workspaces are shared)
  if (!sc->raster_done) {
    if ((e = cudaEventCreateWithFlags(&sc->raster_done, cudaEventDisableTiming)) != cudaSuccess)
      return salf_cuda_fail(e, "raster event");
  } else if ((e = cudaStreamWaitEvent(st, sc->raster_done, 0)) != cudaSuccess) {
    return salf_cuda_fail(e, "raster event wait");
  }
  const DevScene& S = sc->dev;
  const int K = S.K;
  const long long n = S.n;
  const int tiles_x = (r.W + kTile - 1) / kTile, tiles_y = (r.H + kTile - 1) / kTile;
  const int ntiles = tiles_x * tiles_y;
  int ce[3];
  unsigned long long l1max = 0;
  for (int a = 0; a < 3; ++a) {
    ce[a] = floor_div(r.Oi[a], 1 << K);
    const long long d0 = std::llabs((long long)ce[a]);
    const long long d1 = std::llabs((long long)sc->dims[a] - 1 - ce[a]);
    l1max += (unsigned long long)std::max(d0, d1);
  }
  const int low_bits = std::max(bit_width(l1max), 1) + 3 * K;
  const int tile_bits = std::max(bit_width((unsigned long long)(ntiles - 1)), 1);
  if (low_bits + tile_bits > 64) {
    salf_set_error("salf_render_raster: sort key wider than 64 bits for this scene and image");
    return SALF_ERR_INVALID;
  }
  const int key_bits = low_bits + tile_bits;

  // per-voxel workspace
  const long long nn = std::max(n, 1LL);
  const size_t b_count = align256(nn * 4), b_rect = align256(nn * 8), b_key = align256(nn * 8),
               b_offs = align256((nn + 2) * 8), b_tmp = align256(scan_tmp_elems(nn) * 8),
               b_ranges = align256((size_t)ntiles * 8), b_prect = align256(nn * 16);
  const size_t need_vox = b_count + b_rect + b_key + b_offs + b_tmp + b_ranges + b_prect;
  if (sc->raster_vox_bytes < need_vox) {
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return salf_cuda_fail(e, "raster sync");
    if ((e = cudaEventSynchronize(sc->raster_done)) != cudaSuccess)
      return salf_cuda_fail(e, "raster sync");
    if (sc->raster_vox) cudaFree(sc->raster_vox);
    sc->raster_vox = nullptr;
    sc->raster_vox_bytes = 0;
    if (cudaMalloc(&sc->raster_vox, need_vox) != cudaSuccess) {
      cudaGetLastError();
      salf_set_error("salf_render_raster: out of device memory (voxel workspace)");
      return SALF_ERR_OOM;
    }
    sc->raster_vox_bytes = need_vox;
  }
  if (!sc->raster_count_host &&
      cudaMallocHost(reinterpret_cast<void**>(&sc->raster_count_host), 64) != cudaSuccess) {
    cudaGetLastError();
    salf_set_error("salf_render_raster: cudaMallocHost failed");
    return SALF_ERR_OOM;
  }
  char* wv = static_cast<char*>(sc->raster_vox);
  unsigned* count = reinterpret_cast<unsigned*>(wv);
  uint2* rect = reinterpret_cast<uint2*>(wv + b_count);
  unsigned long long* vkey = reinterpret_cast<unsigned long long*>(wv + b_count + b_rect);
  unsigned long long* offs = reinterpret_cast<unsigned long long*>(wv + b_count + b_rect + b_key);
  unsigned long long* stmp =
      reinterpret_cast<unsigned long long*>(wv + b_count + b_rect + b_key + b_offs);
  uint2* ranges = reinterpret_cast<uint2*>(wv + b_count + b_rect + b_key + b_offs + b_tmp);
  int4* prect = reinterpret_cast<int4*>(wv + b_count + b_rect + b_key + b_offs + b_tmp + b_ranges);

  unsigned long long P = 0, visible = 0;
  int launches = 0;
  if (n > 0) {
    ProjParams G;
    std::memset(&G, 0, sizeof(G));
    G.S = S;
    for (int k = 0; k < 9; ++k) G.R0[k] = r.R0[k];
    for (int a = 0; a < 3; ++a) {
      G.Oi[a] = r.Oi[a];
      G.Of[a] = r.Of[a];
      G.ce[a] = ce[a];
    }
    G.fx = (float)fx;
    G.fy = (float)fy;
    G.cx = r.cx;
    G.cy = r.cy;
    G.W = r.W;
    G.H = r.H;
    G.tiles_x = tiles_x;
    G.tiles_y = tiles_y;
    G.dig_shift = 3 * K;
    G.count = count;
    G.rect = rect;
    G.prect = prect;
    G.key = vkey;
    G.n_visible = offs + n + 1;
    if ((e = cudaMemsetAsync(offs + n + 1, 0, 8, st)) != cudaSuccess)
      return salf_cuda_fail(e, "raster counter");
    k_project<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(G);
    if ((e = scan_exclusive<unsigned, unsigned long long>(count, n, offs, stmp, st, &launches)) !=
        cudaSuccess)
      return salf_cuda_fail(e, "raster scan");
    k_scan_total<unsigned, unsigned long long><<<1, 1, 0, st>>>(count, n, offs);
    launches += 2;
    if ((e = cudaMemcpyAsync(sc->raster_count_host, offs + n, 16, cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
      return salf_cuda_fail(e, "raster count copy");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return salf_cuda_fail(e, "raster project");
    P = sc->raster_count_host[0];
    visible = sc->raster_count_host[1];
  }
  if (P > 0xffffffffull - kSortTile) {
    salf_set_error("salf_render_raster: too many (voxel, tile) pairs");
    return SALF_ERR_INVALID;
  }

  // per-pair workspace
  const long long nblk = (long long)((P + kSortTile - 1) / kSortTile);
  const long long hn = (long long)kRadix * std::max(nblk, 1LL);
  const size_t pp = std::max<unsigned long long>(P, 1);
  const size_t b_k = align256(pp * 8), b_v = align256(pp * 4), b_h = align256(hn * 4),
               b_ht = align256(scan_tmp_elems(hn) * 4);
  const size_t need_pairs = 2 * b_k + 2 * b_v + 2 * b_h + b_ht;
  if (sc->raster_pairs_bytes < need_pairs) {
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return salf_cuda_fail(e, "raster sync");
    if ((e = cudaEventSynchronize(sc->raster_done)) != cudaSuccess)
      return salf_cuda_fail(e, "raster sync");
    if (sc->raster_pairs) cudaFree(sc->raster_pairs);
    sc->raster_pairs = nullptr;
    sc->raster_pairs_bytes = 0;
    const size_t grow = need_pairs + need_pairs / 4;
    if (cudaMalloc(&sc->raster_pairs, grow) != cudaSuccess) {
      cudaGetLastError();
      salf_set_error("salf_render_raster: out of device memory (tile lists)");
      return SALF_ERR_OOM;
    }
    sc->raster_pairs_bytes = grow;
  }
  char* wp = static_cast<char*>(sc->raster_pairs);
  unsigned long long* kA = reinterpret_cast<unsigned long long*>(wp);
  unsigned long long* kB = reinterpret_cast<unsigned long long*>(wp + b_k);
  unsigned* vA = reinterpret_cast<unsigned*>(wp + 2 * b_k);
  unsigned* vB = reinterpret_cast<unsigned*>(wp + 2 * b_k + b_v);
  unsigned* hist = reinterpret_cast<unsigned*>(wp + 2 * b_k + 2 * b_v);
  unsigned* hoff = reinterpret_cast<unsigned*>(wp + 2 * b_k + 2 * b_v + b_h);
  unsigned* htmp = reinterpret_cast<unsigned*>(wp + 2 * b_k + 2 * b_v + 2 * b_h);

  if ((e = cudaMemsetAsync(ranges, 0, (size_t)ntiles * 8, st)) != cudaSuccess)
    return salf_cuda_fail(e, "raster ranges");
  unsigned long long* keys = kA;
  unsigned* vals = vA;
  if (P > 0) {
    k_emit<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(count, rect, vkey, offs, (int)n, tiles_x,
                                                          low_bits, kA, vA);
    ++launches;
    if ((e = radix_sort_pairs(kA, vA, kB, vB, (long long)P, key_bits, hist, hoff, htmp, st,
                              &launches, &keys, &vals)) != cudaSuccess)
      return salf_cuda_fail(e, "raster sort");
    k_tile_ranges<<<(unsigned)((P + 255) / 256), 256, 0, st>>>(keys, (long long)P, low_bits,
                                                               ranges);
    ++launches;
  }
  RasterParams RP;
  std::memset(&RP, 0, sizeof(RP));
  RP.S = S;
  RP.Q = r;
  RP.ranges = ranges;
  RP.vox = vals;
  RP.prect = prect;
  RP.tiles_x = tiles_x;
  const bool dump = r.vcap > 0;
  if (S.dtype == SALF_F32 && S.mode == SALF_FIELD_EXP)
    launch_raster<SALF_F32, SALF_FIELD_EXP>(RP, ntiles, dump, st);
  else if (S.dtype == SALF_F32)
    launch_raster<SALF_F32, SALF_FIELD_SDF>(RP, ntiles, dump, st);
  else if (S.mode == SALF_FIELD_EXP)
    launch_raster<SALF_BF16, SALF_FIELD_EXP>(RP, ntiles, dump, st);
  else
    launch_raster<SALF_BF16, SALF_FIELD_SDF>(RP, ntiles, dump, st);
  launches += ntiles > 0 ? 1 : 0;
  if ((e = cudaGetLastError()) != cudaSuccess) return salf_cuda_fail(e, "raster launch");
  if ((e = cudaEventRecord(sc->raster_done, st)) != cudaSuccess)
    return salf_cuda_fail(e, "raster event");
  if (stats) {
    stats->pairs = (int64_t)P;
    stats->tiles = ntiles;
    stats->key_bits = key_bits;
    stats->visible_voxels = (int64_t)visible;
    stats->kernels = launches;
    stats->reserved = 0;
  }
  return SALF_OK;
}
