// scene_build.cpp -- salf_build_scene: validates the voxel set, sorts it in
// block order, builds the occupancy pyramid / level-0 cell table /
// subdivision nodes (the accelerator that stands in for the paper's octree,
// Sec. III-B) and uploads everything to the device.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "salf_internal.h"

namespace {

inline uint64_t spread3(uint64_t x) {
  x &= 0x1fffffULL;
  x = (x | x << 32) & 0x1f00000000ffffULL;
  x = (x | x << 16) & 0x1f0000ff0000ffULL;
  x = (x | x << 8) & 0x100f00f00f00f00fULL;
  x = (x | x << 4) & 0x10c30c30c30c30c3ULL;
  x = (x | x << 2) & 0x1249249249249249ULL;
  return x;
}

inline uint64_t morton3(uint64_t x, uint64_t y, uint64_t z) {
  return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

inline unsigned morton6(unsigned x, unsigned y, unsigned z) {
  return (x & 1u) | ((y & 1u) << 1) | ((z & 1u) << 2) | ((x & 2u) << 2) | ((y & 2u) << 3) |
         ((z & 2u) << 4);
}

struct Scope {  // frees a half-built scene on error
  salf_scene* s;
  bool keep = false;
  ~Scope() {
    if (!keep && s) salf_scene_destroy(s);
  }
};

salf_status dalloc(salf_scene* s, size_t bytes, void** p) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    salf_set_error(std::string("cudaMalloc(") + std::to_string(bytes) + ") failed: " +
                   cudaGetErrorString(e));
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? SALF_ERR_OOM : SALF_ERR_CUDA;
  }
  s->allocations.push_back(*p);
  s->device_bytes += (int64_t)bytes;
  return SALF_OK;
}

template <class T>
salf_status upload(salf_scene* s, const std::vector<T>& v, T** out) {
  void* p = nullptr;
  salf_status st = dalloc(s, v.size() * sizeof(T), &p);
  if (st != SALF_OK) return st;
  if (!v.empty()) {
    cudaError_t e = cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return salf_cuda_fail(e, "cudaMemcpy(scene upload)");
  }
  *out = static_cast<T*>(p);
  return SALF_OK;
}

}  // namespace

salf_status salf_scene_dalloc(salf_scene* s, size_t bytes, void** p) { return dalloc(s, bytes, p); }

salf_status salf_build_scene_impl(salf_ctx* ctx, const salf_scene_desc* d, salf_scene** out) {
  if (!ctx || !d || !out) {
    salf_set_error("salf_build_scene: null argument");
    return SALF_ERR_INVALID;
  }
  *out = nullptr;
  const int K = d->max_level;
  const int64_t n = d->n;
  if (n < 0 || n > (int64_t)0x7ffffff0 || K < 0 || K > 10 || !(d->s0 > 0) ||
      !std::isfinite(d->s0) || (d->mode != SALF_FIELD_EXP && d->mode != SALF_FIELD_SDF) ||
      (d->dtype != SALF_F32 && d->dtype != SALF_BF16)) {
    salf_set_error("salf_build_scene: bad n, max_level, s0, mode or dtype");
    return SALF_ERR_INVALID;
  }
  for (int a = 0; a < 3; ++a) {
    if (d->dims[a] <= 0 || ((int64_t)d->dims[a] << K) > (1 << 21) || !std::isfinite(d->origin[a])) {
      salf_set_error("salf_build_scene: dims must be > 0 with dims << max_level <= 2^21");
      return SALF_ERR_INVALID;
    }
  }
  if (n > 0 && (!d->level || !d->ijk || !d->params)) {
    salf_set_error("salf_build_scene: null level/ijk/params");
    return SALF_ERR_INVALID;
  }
  if (n > 0 && (reinterpret_cast<uintptr_t>(d->params) & 15u)) {
    salf_set_error("salf_build_scene: params must be 16-byte aligned");
    return SALF_ERR_INVALID;
  }
  if (d->keys_on_device) {
    if (!d->params_on_device && n > 0) {
      salf_set_error("salf_build_scene: keys_on_device needs params_on_device");
      return SALF_ERR_INVALID;
    }
    return salf_build_scene_gpu(ctx, d, out);
  }
  cudaError_t ce = cudaSetDevice(ctx->device);
  if (ce != cudaSuccess) return salf_cuda_fail(ce, "cudaSetDevice");

  // ---- sort keys of the min corners (finest units), validation.  Voxels are
  // numbered block by block: the linear index of the 4x4x4 block of level-0
  // cells, then the Morton index of the level-0 cell inside the block, then
  // the Morton index of the min corner inside that cell.  Within a block the
  // level-0 voxels thus follow the occupancy bits, and a block whose occupied
  // cells are all level-0 voxels maps cell -> voxel by a popcount.  Bits: the
  // block index needs 3 (19 - K) at most, the rest 6 + 3 K, so 63 in all.
  int mdim[SALF_MAX_MASK_LEVELS][3];
  for (int a = 0; a < 3; ++a) mdim[0][a] = (d->dims[a] + 3) / 4;
  std::vector<uint64_t> code((size_t)n);
  const uint64_t fine = (1ULL << K) - 1ULL;
  for (int64_t v = 0; v < n; ++v) {
    const int l = d->level[v];
    if (l > K) {
      salf_set_error("salf_build_scene: voxel " + std::to_string(v) + " has level > max_level");
      return SALF_ERR_INVALID;
    }
    uint64_t f[3];
    for (int a = 0; a < 3; ++a) {
      const int64_t c = d->ijk[3 * v + a];
      if (c < 0 || c >= ((int64_t)d->dims[a] << l)) {
        salf_set_error("salf_build_scene: voxel " + std::to_string(v) + " outside the grid");
        return SALF_ERR_INVALID;
      }
      f[a] = (uint64_t)c << (K - l);
    }
    const uint64_t c0[3] = {f[0] >> K, f[1] >> K, f[2] >> K};
    const uint64_t blk =
        ((c0[2] >> 2) * (uint64_t)mdim[0][1] + (c0[1] >> 2)) * (uint64_t)mdim[0][0] + (c0[0] >> 2);
    code[v] = (blk << (6 + 3 * K)) | ((uint64_t)morton6(c0[0] & 3, c0[1] & 3, c0[2] & 3) << (3 * K)) |
              morton3(f[0] & fine, f[1] & fine, f[2] & fine);
  }
  std::vector<int32_t> order((size_t)n);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    if (code[a] != code[b]) return code[a] < code[b];
    return d->level[a] < d->level[b];
  });
  // A voxel of level l lies in one level-0 cell and covers the key range
  // [code, code + 8^(K-l)); in this order an overlap (duplicate, ancestor)
  // always shows up between neighbours.
  for (int64_t p = 1; p < n; ++p) {
    const int32_t a = order[p - 1], b = order[p];
    const uint64_t span = 1ULL << (3 * (K - d->level[a]));
    if (code[b] < code[a] + span) {
      salf_set_error("salf_build_scene: voxels " + std::to_string(a) + " and " +
                     std::to_string(b) + " overlap");
      return SALF_ERR_OVERLAP;
    }
  }

  // ---- occupancy of level-0 cells, rank offsets, cell table, nodes
  const int64_t nb0 = (int64_t)mdim[0][0] * mdim[0][1] * mdim[0][2];
  std::vector<uint64_t> m0((size_t)nb0, 0);
  std::vector<uint32_t> vfirst((size_t)nb0, 0xffffffffu);
  std::vector<uint8_t> split((size_t)nb0, 0);
  auto block_of = [&](int64_t cx, int64_t cy, int64_t cz) {
    return ((cz >> 2) * mdim[0][1] + (cy >> 2)) * mdim[0][0] + (cx >> 2);
  };
  for (int64_t p = 0; p < n; ++p) {
    const int32_t v = order[p];
    const int l = d->level[v];
    const int64_t cx = d->ijk[3 * v] >> l, cy = d->ijk[3 * v + 1] >> l, cz = d->ijk[3 * v + 2] >> l;
    const int64_t b = block_of(cx, cy, cz);
    m0[b] |= 1ULL << morton6(cx & 3, cy & 3, cz & 3);
    if (vfirst[b] == 0xffffffffu) vfirst[b] = (uint32_t)p;
    if (l > 0) split[b] = 1;
  }
  std::vector<uint4> mask0((size_t)nb0);
  int64_t running = 0;
  for (int64_t b = 0; b < nb0; ++b) {
    mask0[b].x = (unsigned)(m0[b] & 0xffffffffULL);
    mask0[b].y = (unsigned)(m0[b] >> 32);
    mask0[b].z = (unsigned)running;
    // voxel of the block's first occupied cell when every occupied cell is
    // one level-0 voxel, else all ones (look the cell up in `cells`)
    mask0[b].w = (m0[b] && !split[b]) ? vfirst[b] : 0xffffffffu;
    running += __builtin_popcountll(m0[b]);
  }
  std::vector<int32_t> entries((size_t)std::max<int64_t>(running, 1), -1);
  std::vector<int32_t> nodes;
  auto new_node = [&]() {
    nodes.insert(nodes.end(), 8, -1);
    return (int32_t)(nodes.size() / 8 - 1);
  };
  for (int64_t p = 0; p < n; ++p) {
    const int32_t v = order[p];
    const int l = d->level[v];
    const int64_t i = d->ijk[3 * v], j = d->ijk[3 * v + 1], k = d->ijk[3 * v + 2];
    const int64_t cx = i >> l, cy = j >> l, cz = k >> l;
    const int64_t b = block_of(cx, cy, cz);
    const unsigned bit = morton6(cx & 3, cy & 3, cz & 3);
    const int64_t rank = mask0[b].z + __builtin_popcountll(m0[b] & ((1ULL << bit) - 1ULL));
    if (l == 0) {
      entries[rank] = (int32_t)p;
      continue;
    }
    if (entries[rank] == -1) entries[rank] = -2 - new_node();
    int32_t node = -2 - entries[rank];
    for (int dl = 1; dl <= l; ++dl) {
      const int sh = l - dl;
      const int slot = (int)(((i >> sh) & 1) | (((j >> sh) & 1) << 1) | (((k >> sh) & 1) << 2));
      if (dl == l) {
        nodes[(size_t)node * 8 + slot] = (int32_t)p;
      } else {
        int32_t e = nodes[(size_t)node * 8 + slot];
        if (e == -1) {
          const int32_t nn = new_node();
          e = -2 - nn;
          nodes[(size_t)node * 8 + slot] = e;
        }
        node = -2 - e;
      }
    }
  }
  if (nodes.empty()) nodes.assign(8, -1);
  // Device cell table: (entry, child mask).  A cell split exactly once, into
  // children that are all voxels or empty, becomes (first child voxel, 8-bit
  // occupancy of its children): the children are consecutive in voxel order,
  // so the traversal finds a child without reading its node.
  std::vector<int2> cells(entries.size());
  for (size_t r = 0; r < entries.size(); ++r) {
    const int32_t e = entries[r];
    cells[r] = make_int2(e, 0);
    if (e > -2) continue;
    const int32_t* ch = &nodes[(size_t)(-2 - e) * 8];
    unsigned cm = 0;
    int32_t first = -1, expect = -1;
    bool flat = true;
    for (int c = 0; c < 8 && flat; ++c) {
      if (ch[c] == -1) continue;
      if (ch[c] < 0 || (expect >= 0 && ch[c] != expect)) flat = false;
      if (first < 0) first = ch[c];
      expect = ch[c] + 1;
      cm |= 1u << c;
    }
    if (flat && cm) cells[r] = make_int2(first, (int)cm);
  }

  // ---- upper pyramid levels
  std::vector<std::vector<uint64_t>> up(1);
  int M = 1;
  {
    std::vector<uint64_t> prev = m0;
    while (!(mdim[M - 1][0] == 1 && mdim[M - 1][1] == 1 && mdim[M - 1][2] == 1)) {
      if (M >= SALF_MAX_MASK_LEVELS) {
        salf_set_error("salf_build_scene: grid too large for the pyramid");
        return SALF_ERR_INVALID;
      }
      for (int a = 0; a < 3; ++a) mdim[M][a] = (mdim[M - 1][a] + 3) / 4;
      std::vector<uint64_t> cur((size_t)mdim[M][0] * mdim[M][1] * mdim[M][2], 0);
      for (int64_t wz = 0; wz < mdim[M - 1][2]; ++wz)
        for (int64_t wy = 0; wy < mdim[M - 1][1]; ++wy)
          for (int64_t wx = 0; wx < mdim[M - 1][0]; ++wx) {
            if (!prev[(wz * mdim[M - 1][1] + wy) * mdim[M - 1][0] + wx]) continue;
            cur[((wz >> 2) * mdim[M][1] + (wy >> 2)) * mdim[M][0] + (wx >> 2)] |=
                1ULL << morton6(wx & 3, wy & 3, wz & 3);
          }
      up.push_back(cur);
      prev.swap(cur);
      ++M;
    }
  }

  // ---- column pyramid: z-layer occupancy per footprint of 2^c x 2^c columns
  int layer_cells = 1;
  while ((d->dims[2] + layer_cells - 1) / layer_cells > 128) layer_cells *= 2;
  const int n_layers = (d->dims[2] + layer_cells - 1) / layer_cells;
  int cdim[SALF_MAX_COL_LEVELS][2];
  cdim[0][0] = d->dims[0];
  cdim[0][1] = d->dims[1];
  std::vector<std::vector<uint4>> cols(1);
  cols[0].assign((size_t)cdim[0][0] * cdim[0][1], make_uint4(0, 0, 0, 0));
  for (int64_t p = 0; p < n; ++p) {
    const int32_t v = order[p];
    const int l = d->level[v];
    const int64_t cx = d->ijk[3 * v] >> l, cy = d->ijk[3 * v + 1] >> l, cz = d->ijk[3 * v + 2] >> l;
    const int layer = (int)(cz / layer_cells);
    uint4& m = cols[0][(size_t)cy * cdim[0][0] + cx];
    unsigned* wds = &m.x;
    wds[layer >> 5] |= 1u << (layer & 31);
  }
  int CL = 1;
  while ((cdim[CL - 1][0] > 1 || cdim[CL - 1][1] > 1) && CL < SALF_MAX_COL_LEVELS) {
    cdim[CL][0] = (cdim[CL - 1][0] + 1) / 2;
    cdim[CL][1] = (cdim[CL - 1][1] + 1) / 2;
    std::vector<uint4> cur((size_t)cdim[CL][0] * cdim[CL][1], make_uint4(0, 0, 0, 0));
    for (int64_t y = 0; y < cdim[CL - 1][1]; ++y)
      for (int64_t x = 0; x < cdim[CL - 1][0]; ++x) {
        const uint4 a = cols[CL - 1][(size_t)y * cdim[CL - 1][0] + x];
        uint4& b = cur[(size_t)(y >> 1) * cdim[CL][0] + (x >> 1)];
        b.x |= a.x;
        b.y |= a.y;
        b.z |= a.z;
        b.w |= a.w;
      }
    cols.push_back(std::move(cur));
    ++CL;
  }

  // ---- device upload
  salf_scene* s = new salf_scene();
  Scope guard{s};
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
  s->n_cells0 = running;
  s->n_nodes = (int64_t)nodes.size() / 8;

  DevScene& D = s->dev;
  std::memset(&D, 0, sizeof(D));
  salf_status st;
  uint4* dmask0 = nullptr;
  if ((st = upload(s, mask0, &dmask0)) != SALF_OK) return st;
  D.mask0 = dmask0;
  for (int m = 1; m < M; ++m) {
    uint64_t* p = nullptr;
    if ((st = upload(s, up[m], &p)) != SALF_OK) return st;
    D.mask[m] = reinterpret_cast<const unsigned long long*>(p);
  }
  for (int m = 0; m < M; ++m)
    for (int a = 0; a < 3; ++a) D.mdim[m][a] = mdim[m][a];
  int2* dcells = nullptr;
  int32_t* dnodes = nullptr;
  int32_t* dorder = nullptr;
  if ((st = upload(s, cells, &dcells)) != SALF_OK) return st;
  if ((st = upload(s, nodes, &dnodes)) != SALF_OK) return st;
  std::vector<int32_t> ord = order;
  if (ord.empty()) ord.push_back(0);
  if ((st = upload(s, ord, &dorder)) != SALF_OK) return st;
  D.cells = dcells;
  D.nodes = dnodes;
  D.order = dorder;
  {
    std::vector<int4> box((size_t)std::max<int64_t>(n, 1), make_int4(0, 0, 0, 0));
    for (int64_t p = 0; p < n; ++p) {
      const int32_t v = order[p];
      const int l = d->level[v];
      box[p] = make_int4((int)(d->ijk[3 * v] << (K - l)), (int)(d->ijk[3 * v + 1] << (K - l)),
                         (int)(d->ijk[3 * v + 2] << (K - l)), K - l);
    }
    int4* dbox = nullptr;
    if ((st = upload(s, box, &dbox)) != SALF_OK) return st;
    D.vox_box = dbox;
  }
  for (int c = 0; c < CL; ++c) {
    uint4* pc = nullptr;
    if ((st = upload(s, cols[c], &pc)) != SALF_OK) return st;
    D.col[c] = pc;
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
  void* status = nullptr;
  if ((st = dalloc(s, 16, &status)) != SALF_OK) return st;
  if ((ce = cudaMemset(status, 0, 16)) != cudaSuccess) return salf_cuda_fail(ce, "cudaMemset");
  D.status = static_cast<int*>(status);
  void* params = nullptr;
  const size_t rec_bytes = d->dtype == SALF_F32 ? 128 : 64;
  if ((st = dalloc(s, (size_t)std::max<int64_t>(n, 1) * rec_bytes, &params)) != SALF_OK) return st;
  D.params = params;
  for (int a = 0; a < 3; ++a) {
    D.origin[a] = d->origin[a];
    D.Gf[a] = d->dims[a] << K;
  }
  D.inv_sfin = 1.0 / s->sfin;
  // tight box of the occupied voxels: rays are clipped to it (no hit outside)
  for (int a = 0; a < 3; ++a) {
    D.bmin[a] = D.Gf[a];
    D.bmax[a] = 0;
  }
  for (int64_t v = 0; v < n; ++v) {
    const int l = d->level[v];
    for (int a = 0; a < 3; ++a) {
      const int lo = d->ijk[3 * v + a] << (K - l);
      D.bmin[a] = std::min(D.bmin[a], lo);
      D.bmax[a] = std::max(D.bmax[a], lo + (1 << (K - l)));
    }
  }
  if (n == 0)
    for (int a = 0; a < 3; ++a) D.bmin[a] = D.bmax[a] = 0;
  D.K = K;
  D.M = M;
  D.mode = d->mode;
  D.dtype = d->dtype;
  D.n = (int)n;

  if (n > 0) {
    const float* src = d->params;
    void* tmp = nullptr;
    if (!d->params_on_device) {
      if ((ce = cudaMalloc(&tmp, (size_t)n * 128)) != cudaSuccess) {
        cudaGetLastError();
        salf_set_error("cudaMalloc(param staging) failed");
        return ce == cudaErrorMemoryAllocation ? SALF_ERR_OOM : SALF_ERR_CUDA;
      }
      ce = cudaMemcpy(tmp, d->params, (size_t)n * 128, cudaMemcpyHostToDevice);
      if (ce != cudaSuccess) {
        cudaFree(tmp);
        return salf_cuda_fail(ce, "cudaMemcpy(params)");
      }
      src = static_cast<const float*>(tmp);
    }
    ce = salf_launch_gather_params(src, dorder, params, n, d->dtype, d->mode, D.status, 0);
    if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
    if (tmp) cudaFree(tmp);
    if (ce != cudaSuccess) return salf_cuda_fail(ce, "gather params");
    int flag = 0;
    if ((ce = cudaMemcpy(&flag, D.status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return salf_cuda_fail(ce, "cudaMemcpy(status)");
    if (flag & SALF_DEVERR_SDF_AB) {
      salf_set_error("salf_build_scene: SDF records need a > 0 and b > 0 (Eq. 6)");
      return SALF_ERR_INVALID;
    }
  }
  guard.keep = true;
  *out = s;
  return SALF_OK;
}
