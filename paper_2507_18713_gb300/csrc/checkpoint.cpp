// checkpoint.cpp -- scene files: salf_scene_save / salf_scene_load.
//
// A scene file holds what salf_build_scene takes (Sec. III-A: the voxel keys
// and their 32-scalar records), so loading it rebuilds the same scene.  The
// keys are kept, in input order, in two device buffers the scene owns (the
// build does not otherwise keep them); the records are read back from the
// scene in its storage dtype and written in input order.
//
// Layout (little-endian, no padding between fields):
//   char[8]  magic "SALFSCN1"
//   int32    version (1), dtype (salf_dtype), mode (salf_field_mode), max_level
//   int64    n
//   float64  origin[3], s0
//   int32    dims[3], reserved (0)
//   uint8    level[n]
//   int32    ijk[3 n]
//   records  n x 32 scalars: FP32, or BF16 (the upper half of the FP32 bits)
#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include "salf_internal.h"

namespace {

constexpr char kMagic[8] = {'S', 'A', 'L', 'F', 'S', 'C', 'N', '1'};
constexpr int32_t kVersion = 1;

struct FileCloser {
  void operator()(std::FILE* f) const {
    if (f) std::fclose(f);
  }
};
using File = std::unique_ptr<std::FILE, FileCloser>;

struct Header {
  int32_t version, dtype, mode, max_level;
  int64_t n;
  double origin[3], s0;
  int32_t dims[3], reserved;
};

bool put(std::FILE* f, const void* p, size_t bytes) {
  return bytes == 0 || std::fwrite(p, 1, bytes, f) == bytes;
}
bool get(std::FILE* f, void* p, size_t bytes) {
  return bytes == 0 || std::fread(p, 1, bytes, f) == bytes;
}

size_t record_bytes(int dtype) { return dtype == SALF_F32 ? 128 : 64; }

}  // namespace

salf_status salf_scene_keep_keys(salf_scene* s, const salf_scene_desc* d) {
  const int64_t n = d->n;
  if (n == 0) return SALF_OK;
  void* lv = nullptr;
  void* ij = nullptr;
  salf_status st = salf_scene_dalloc(s, (size_t)n, &lv);
  if (st != SALF_OK) return st;
  st = salf_scene_dalloc(s, (size_t)n * 3 * sizeof(int32_t), &ij);
  if (st != SALF_OK) return st;
  const cudaMemcpyKind k = d->keys_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  cudaError_t e = cudaMemcpy(lv, d->level, (size_t)n, k);
  if (e == cudaSuccess) e = cudaMemcpy(ij, d->ijk, (size_t)n * 3 * sizeof(int32_t), k);
  if (e != cudaSuccess) return salf_cuda_fail(e, "scene keys copy");
  s->key_level = static_cast<const uint8_t*>(lv);
  s->key_ijk = static_cast<const int32_t*>(ij);
  return SALF_OK;
}

extern "C" salf_status salf_scene_save(const salf_scene* s, const char* path) {
  SALF_RANGE("salf_scene_save");
  if (!s || !path) {
    salf_set_error("salf_scene_save: null argument");
    return SALF_ERR_INVALID;
  }
  const int64_t n = s->n;
  if (n > 0 && (!s->key_level || !s->key_ijk)) {
    salf_set_error("salf_scene_save: the scene keeps no voxel keys");
    return SALF_ERR_INVALID;
  }
  cudaError_t e = cudaSetDevice(s->device);
  if (e != cudaSuccess) return salf_cuda_fail(e, "cudaSetDevice");
  const size_t rb = record_bytes(s->dtype);
  std::vector<uint8_t> level((size_t)n);
  std::vector<int32_t> ijk((size_t)n * 3);
  std::vector<uint8_t> rec((size_t)n * rb), rec_in((size_t)n * rb);
  std::vector<int32_t> order((size_t)n);
  // every stream's work on the records is finished before they are read
  if ((e = cudaDeviceSynchronize()) != cudaSuccess) return salf_cuda_fail(e, "scene sync");
  if (n > 0) {
    e = cudaMemcpy(level.data(), s->key_level, (size_t)n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(ijk.data(), s->key_ijk, ijk.size() * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(rec.data(), s->dev.params, rec.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
      e = cudaMemcpy(order.data(), s->dev.order, order.size() * sizeof(int32_t),
                     cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return salf_cuda_fail(e, "scene read-back");
  }
  // records in input order (order maps internal index -> input index)
  for (int64_t i = 0; i < n; ++i) {
    const int32_t v = order[(size_t)i];
    if (v < 0 || v >= n) {
      salf_set_error("salf_scene_save: corrupt voxel order");
      return SALF_ERR_DEVICE;
    }
    std::memcpy(&rec_in[(size_t)v * rb], &rec[(size_t)i * rb], rb);
  }
  Header h{};
  h.version = kVersion;
  h.dtype = s->dtype;
  h.mode = s->mode;
  h.max_level = s->K;
  h.n = n;
  for (int a = 0; a < 3; ++a) {
    h.origin[a] = s->origin[a];
    h.dims[a] = s->dims[a];
  }
  h.s0 = s->s0;
  File f(std::fopen(path, "wb"));
  if (!f) {
    salf_set_error(std::string("salf_scene_save: cannot open ") + path);
    return SALF_ERR_IO;
  }
  const bool ok = put(f.get(), kMagic, sizeof(kMagic)) && put(f.get(), &h.version, 16) &&
                  put(f.get(), &h.n, 8) && put(f.get(), h.origin, 24) && put(f.get(), &h.s0, 8) &&
                  put(f.get(), h.dims, 12) && put(f.get(), &h.reserved, 4) &&
                  put(f.get(), level.data(), level.size()) &&
                  put(f.get(), ijk.data(), ijk.size() * sizeof(int32_t)) &&
                  put(f.get(), rec_in.data(), rec_in.size());
  if (!ok || std::fflush(f.get()) != 0) {
    salf_set_error(std::string("salf_scene_save: write failed: ") + path);
    return SALF_ERR_IO;
  }
  return SALF_OK;
}

extern "C" salf_status salf_scene_load(salf_ctx* ctx, const char* path, salf_scene** out) {
  SALF_RANGE("salf_scene_load");
  if (!ctx || !path || !out) {
    salf_set_error("salf_scene_load: null argument");
    return SALF_ERR_INVALID;
  }
  *out = nullptr;
  File f(std::fopen(path, "rb"));
  if (!f) {
    salf_set_error(std::string("salf_scene_load: cannot open ") + path);
    return SALF_ERR_IO;
  }
  char magic[8];
  Header h{};
  if (!get(f.get(), magic, 8) || std::memcmp(magic, kMagic, 8) != 0 ||
      !get(f.get(), &h.version, 16) || !get(f.get(), &h.n, 8) || !get(f.get(), h.origin, 24) ||
      !get(f.get(), &h.s0, 8) || !get(f.get(), h.dims, 12) || !get(f.get(), &h.reserved, 4)) {
    salf_set_error(std::string("salf_scene_load: not a scene file: ") + path);
    return SALF_ERR_IO;
  }
  if (h.version != kVersion || (h.dtype != SALF_F32 && h.dtype != SALF_BF16) || h.n < 0 ||
      h.n > (int64_t)0x7ffffff0) {
    salf_set_error("salf_scene_load: unsupported version, dtype or size");
    return SALF_ERR_IO;
  }
  // the file must hold exactly the arrays its header announces
  const int64_t n = h.n;
  const size_t rb = record_bytes(h.dtype);
  const long long want = 8 + 16 + 8 + 24 + 8 + 12 + 4 + n * (1 + 12 + (long long)rb);
  if (std::fseek(f.get(), 0, SEEK_END) != 0 || std::ftell(f.get()) != want ||
      std::fseek(f.get(), 8 + 16 + 8 + 24 + 8 + 12 + 4, SEEK_SET) != 0) {
    salf_set_error("salf_scene_load: file size does not match its header");
    return SALF_ERR_IO;
  }
  std::vector<uint8_t> level((size_t)n);
  std::vector<int32_t> ijk((size_t)n * 3);
  std::vector<uint8_t> rec((size_t)n * rb);
  if (!get(f.get(), level.data(), level.size()) ||
      !get(f.get(), ijk.data(), ijk.size() * sizeof(int32_t)) ||
      !get(f.get(), rec.data(), rec.size())) {
    salf_set_error("salf_scene_load: read failed");
    return SALF_ERR_IO;
  }
  // FP32 records for the build; BF16 widens exactly, so the rebuilt scene
  // stores the same BF16 bits
  std::vector<float> params((size_t)n * SALF_RECORD_SCALARS + 4);
  float* p = params.data();
  while (reinterpret_cast<uintptr_t>(p) & 15u) ++p;  // the build wants 16-byte alignment
  if (h.dtype == SALF_F32) {
    if (n > 0) std::memcpy(p, rec.data(), rec.size());
  } else {
    for (size_t k = 0; k < (size_t)n * SALF_RECORD_SCALARS; ++k) {
      uint16_t b;
      std::memcpy(&b, &rec[2 * k], 2);
      const uint32_t w = (uint32_t)b << 16;
      std::memcpy(&p[k], &w, 4);
    }
  }
  salf_scene_desc d;
  std::memset(&d, 0, sizeof(d));
  d.n = n;
  for (int a = 0; a < 3; ++a) {
    d.origin[a] = h.origin[a];
    d.dims[a] = h.dims[a];
  }
  d.s0 = h.s0;
  d.max_level = h.max_level;
  d.level = level.data();
  d.ijk = ijk.data();
  d.mode = h.mode;
  d.dtype = h.dtype;
  d.params = p;
  return salf_build_scene(ctx, &d, out);
}
