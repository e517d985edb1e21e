// traverse.cuh -- per-ray device code shared by the forward and adjoint
// kernels: sensor ray generation (Fig. 2, Sec. V-C), traversal of the sparse
// voxel structure (Sec. III-B), record loads and the local fields of
// Eq. 1, 2, 5, 6.
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

#include "salf_internal.h"

// Traversal tuning switches (compile-time).
#ifndef SALF_COL_MAX_LS
#define SALF_COL_MAX_LS 0  // > 0: try the column skip only below this pyramid leaf size
#endif
#ifndef SALF_COL_EARLY
#define SALF_COL_EARLY 1  // 1: load the column mask beside the pyramid word; 0: only for empty cells
#endif

namespace salf {

constexpr float kPi = 3.14159265358979323846f;
constexpr float kSH0 = 0.28209479177387814f;  // 1 / (2 sqrt(pi))
constexpr float kSH1 = 0.48860251190291992f;  // sqrt(3) / (2 sqrt(pi))

struct Ray {
  int Oi[3];     // origin, finest-cell units: Oi + Of
  float Of[3];
  float d[3];    // unit direction, world frame
  float tn, tf;  // metres
  float s;       // time fraction (t - t0) / (t1 - t0) of the ray's pose
  bool valid;
};

// Sensor ray of pixel (u, v) / LiDAR (azimuth u, beam v).
__device__ __forceinline__ void gen_ray(const ReqDev& Q, const DevScene& S, int u, int v,
                                        int ray, Ray& r) {
  r.valid = true;
  if (Q.kind == SALF_RAYS_EXPLICIT) {
    const float4* q = reinterpret_cast<const float4*>(Q.rays) + 2 * (size_t)ray;
    float4 a = __ldg(q), b = __ldg(q + 1);
    double o[3] = {(double)a.x, (double)a.y, (double)a.z};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double g = (o[k] - S.origin[k]) * S.inv_sfin;
      double f = floor(g);
      r.Oi[k] = (int)f;
      r.Of[k] = (float)(g - f);
    }
    float dx = a.w, dy = b.x, dz = b.y;
    float nn = dx * dx + dy * dy + dz * dz;
    r.valid = nn > 0.f;
    float inv = nn > 0.f ? rsqrtf(nn) : 0.f;
    r.d[0] = dx * inv;
    r.d[1] = dy * inv;
    r.d[2] = dz * inv;
    r.tn = b.z;
    r.tf = b.w > 0.f ? b.w : __int_as_float(0x7f800000);
    r.s = 0.f;
    return;
  }
  float dc[3];
  float s = 0.f;
  if (Q.kind == SALF_LIDAR_SPIN) {
    float e = Q.elev_max - (float)v * Q.elev_step;
    float se, ce, sp, cp;
    sincosf(e, &se, &ce);
    // azimuth 2 pi u / W as sin/cos(pi x) with x = 2u/W: no rounding of 2 pi
    sincospif(2.f * (float)u / (float)Q.W, &sp, &cp);
    dc[0] = ce * cp;
    dc[1] = ce * sp;
    dc[2] = se;
    if (Q.moving) s = (float)u / (float)Q.W;
  } else {
    float px = (float)u + 0.5f, py = (float)v + 0.5f;
    if (Q.kind == SALF_PINHOLE) {
      dc[0] = (px - Q.cx) * Q.inv_fx;
      dc[1] = (py - Q.cy) * Q.inv_fy;
      dc[2] = 1.f;
    } else if (Q.kind == SALF_FISHEYE_EQUIDIST) {
      float mx = (px - Q.cx) * Q.inv_fx, my = (py - Q.cy) * Q.inv_fy;
      float th = sqrtf(mx * mx + my * my);
      r.valid = th <= Q.half_fov;
      float st, ct;
      sincosf(th, &st, &ct);
      float k = th > 0.f ? st / th : 1.f;
      dc[0] = k * mx;
      dc[1] = k * my;
      dc[2] = ct;
    } else {  // equirectangular panorama
      // longitude 2 pi (px / W - 0.5) as sin/cos(pi x): no rounding of 2 pi
      float lat = Q.elev_max - (py / (float)Q.H) * (Q.elev_max - Q.elev_min);
      float sl, cl, sa, ca;
      sincospif(2.f * px / (float)Q.W - 1.f, &sl, &cl);
      sincosf(lat, &sa, &ca);
      dc[0] = ca * sl;
      dc[1] = -sa;
      dc[2] = ca * cl;
    }
    if (Q.moving) s = (float)v / (float)(Q.H - 1);
  }
  float d0 = Q.R0[0] * dc[0] + Q.R0[1] * dc[1] + Q.R0[2] * dc[2];
  float d1 = Q.R0[3] * dc[0] + Q.R0[4] * dc[1] + Q.R0[5] * dc[2];
  float d2 = Q.R0[6] * dc[0] + Q.R0[7] * dc[1] + Q.R0[8] * dc[2];
  if (s > 0.f && Q.rel_angle != 0.f) {
    // Rodrigues rotation by alpha about k: d + sin(a) (k x d) + (1 - cos(a)) k x (k x d)
    const float a = s * Q.rel_angle;
    float sh, ch;
    sincosf(0.5f * a, &sh, &ch);
    const float sa = 2.f * sh * ch, omc = 2.f * sh * sh;
    const float kx = Q.rel_axis[0], ky = Q.rel_axis[1], kz = Q.rel_axis[2];
    const float cx = ky * d2 - kz * d1, cy = kz * d0 - kx * d2, cz = kx * d1 - ky * d0;
    const float ccx = ky * cz - kz * cy, ccy = kz * cx - kx * cz, ccz = kx * cy - ky * cx;
    d0 = fmaf(omc, ccx, fmaf(sa, cx, d0));
    d1 = fmaf(omc, ccy, fmaf(sa, cy, d1));
    d2 = fmaf(omc, ccz, fmaf(sa, cz, d2));
  }
  float inv = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  r.d[0] = d0 * inv;
  r.d[1] = d1 * inv;
  r.d[2] = d2 * inv;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r.Oi[k] = Q.Oi[k];
    r.Of[k] = fmaf(s, Q.dO[k], Q.Of[k]);
  }
  r.tn = Q.t_near;
  r.tf = Q.t_far;
  r.s = s;
}

// gen_ray for a pinhole camera with one pose for the whole frame (no rolling
// shutter): the same arithmetic as gen_ray's pinhole branch, without the other
// sensor kinds' code, for kernels that serve only such cameras.
__device__ __forceinline__ void gen_ray_pinhole(const ReqDev& Q, int u, int v, Ray& r) {
  r.valid = true;
  const float px = (float)u + 0.5f, py = (float)v + 0.5f;
  const float dc0 = (px - Q.cx) * Q.inv_fx, dc1 = (py - Q.cy) * Q.inv_fy, dc2 = 1.f;
  const float d0 = Q.R0[0] * dc0 + Q.R0[1] * dc1 + Q.R0[2] * dc2;
  const float d1 = Q.R0[3] * dc0 + Q.R0[4] * dc1 + Q.R0[5] * dc2;
  const float d2 = Q.R0[6] * dc0 + Q.R0[7] * dc1 + Q.R0[8] * dc2;
  const float inv = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
  r.d[0] = d0 * inv;
  r.d[1] = d1 * inv;
  r.d[2] = d2 * inv;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    r.Oi[k] = Q.Oi[k];
    r.Of[k] = Q.Of[k];  // fmaf(0, dO, Of) in gen_ray
  }
  r.tn = Q.t_near;
  r.tf = Q.t_far;
  r.s = 0.f;
}

// Debug dump of a generated ray: world origin, unit direction, time, valid.
__device__ __forceinline__ void dump_ray(const ReqDev& Q, const DevScene& S, const Ray& r, int ray) {
  float* p = Q.ray_dump + 8 * (size_t)ray;
  const double sf = 1.0 / S.inv_sfin;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    p[k] = (float)(S.origin[k] + ((double)r.Oi[k] + (double)r.Of[k]) * sf);
    p[3 + k] = r.d[k];
  }
  p[6] = Q.time0 + r.s * (Q.time1 - Q.time0);
  p[7] = r.valid ? 1.f : 0.f;
}

// Traversal state of one ray, all positions relative to the origin cell Oi so
// that plane distances are small integers minus a fraction.
struct Walk {
  int Oi[3];
  float Of[3];
  float D[3];     // direction in finest cells per metre (zero components -> 1e-20)
  float invD[3];  // metres per finest cell
  int c[3];       // current finest cell
  float t;        // entry distance of the current cell
  float tend;     // min(t_far, root-box exit)
  int steps;
  int cl;         // column-pyramid level to try next
  bool alive;
};

// (Re)start a walk at distance t: the cell holding the point there, kept
// inside the tight box of the voxels.
__device__ __forceinline__ void walk_seek(const DevScene& S, Walk& w, float t) {
  w.t = t;
  w.steps = 0;
  w.cl = min(S.CL - 1, 6);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    int q = w.Oi[a] + __float2int_rd(fmaf(t, w.D[a], w.Of[a]));
    w.c[a] = min(max(q, S.bmin[a]), max(S.bmax[a] - 1, S.bmin[a]));
  }
}

__device__ __forceinline__ void walk_init(const DevScene& S, const Ray& r, Walk& w) {
  float isf = (float)S.inv_sfin;
  float t0 = r.tn, t1 = r.tf;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    w.Oi[a] = r.Oi[a];
    w.Of[a] = r.Of[a];
    float D = r.d[a] * isf;
    if (fabsf(D) < 1e-20f) D = 1e-20f;
    w.D[a] = D;
    w.invD[a] = 1.f / D;
    // clip to the tight box of the voxels (no hit can lie outside it)
    float lo = ((float)(S.bmin[a] - r.Oi[a]) - r.Of[a]) * w.invD[a];
    float hi = ((float)(S.bmax[a] - r.Oi[a]) - r.Of[a]) * w.invD[a];
    t0 = fmaxf(t0, fminf(lo, hi));
    t1 = fminf(t1, fmaxf(lo, hi));
  }
  w.alive = r.valid && (t0 < t1);
  w.tend = t1;
  walk_seek(S, w, t0);
}

__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

__device__ __forceinline__ unsigned morton6(unsigned x, unsigned y, unsigned z) {
  return (x & 1u) | ((y & 1u) << 1) | ((z & 1u) << 2) | ((x & 2u) << 2) | ((y & 2u) << 3) |
         ((z & 2u) << 4);
}

// Leaf of the structure containing finest cell (ix, iy, iz): a voxel
// (returns its internal index) or an empty region (returns -1).  *ls = log2 of
// the leaf's edge in finest cells.
__device__ __forceinline__ int find_leaf(const DevScene& S, int ix, int iy, int iz, int* ls) {
  const int K = S.K;
  const unsigned cx = (unsigned)ix >> K, cy = (unsigned)iy >> K, cz = (unsigned)iz >> K;
  const unsigned bx = cx >> 2, by = cy >> 2, bz = cz >> 2;
  const uint4 w = __ldg(&S.mask0[(bz * (unsigned)S.mdim[0][1] + by) * (unsigned)S.mdim[0][0] + bx]);
  const unsigned long long m = ((unsigned long long)w.y << 32) | (unsigned long long)w.x;
  const unsigned bit = morton6(cx & 3, cy & 3, cz & 3);
  if ((m >> bit) & 1ull) {
    const unsigned pre = __popcll(m & ((1ull << bit) - 1ull));
    if (w.w != 0xffffffffu) {  // block of level-0 voxels: no cell-table read
      *ls = K;
      return (int)(w.w + pre);
    }
    const int2 en = __ldg(&S.cells[w.z + pre]);
    int e = en.x;
    int l = K;
    if (en.y) {  // split once: child voxel by rank, no node read
      l = K - 1;
      const unsigned ch = ((ix >> l) & 1) | (((iy >> l) & 1) << 1) | (((iz >> l) & 1) << 2);
      const unsigned cm = (unsigned)en.y;
      e = ((cm >> ch) & 1u) ? e + __popc(cm & ((1u << ch) - 1u)) : -1;
    }
    while (e <= -2) {
      --l;
      const int ch = ((ix >> l) & 1) | (((iy >> l) & 1) << 1) | (((iz >> l) & 1) << 2);
      e = __ldg(&S.nodes[(unsigned)(-2 - e) * 8u + (unsigned)ch]);
    }
    *ls = l;
    return e;
  }
  if ((m >> (bit & 0x38u)) & 0xffull) {
    *ls = K;
    return -1;
  }
  if (m) {
    *ls = K + 1;
    return -1;
  }
  unsigned ux = bx, uy = by, uz = bz;
  for (int lev = 1; lev < S.M; ++lev) {
    const unsigned long long mw =
        __ldg(&S.mask[lev][((uz >> 2) * (unsigned)S.mdim[lev][1] + (uy >> 2)) *
                               (unsigned)S.mdim[lev][0] + (ux >> 2)]);
    const unsigned b = morton6(ux & 3, uy & 3, uz & 3);
    if ((mw >> (b & 0x38u)) & 0xffull) {
      *ls = K + 2 * lev;
      return -1;
    }
    if (mw) {
      *ls = K + 2 * lev + 1;
      return -1;
    }
    ux >>= 2;
    uy >>= 2;
    uz >>= 2;
  }
  *ls = K + 2 * S.M;
  return -1;
}

// Column-pyramid skip at level `cl` from the current (empty) cell: the ray may
// advance through every layer of the 2^cl x 2^cl-column footprint that holds
// no voxel, up to the nearest occupied layer in its direction of travel or the
// footprint's side.  Returns false if the current layer is occupied in the
// footprint (no progress at this level).  Fills the skipped box [lo, hi)
// (finest cells), its exit axis and exit distance.
// Column mask of the footprint (at level cl) that holds the current cell.
__device__ __forceinline__ uint4 col_mask(const DevScene& S, const Walk& w, int cl) {
  const int sh = S.K + cl;
  return __ldg(&S.col[cl][(unsigned)(w.c[1] >> sh) * (unsigned)S.cdim[cl][0] +
                          (unsigned)(w.c[0] >> sh)]);
}

__device__ __forceinline__ bool col_skip(const DevScene& S, const Walk& w, int cl, const uint4 m,
                                         float* t_exit, int lo[3], int hi[3], int* axis) {
  const int sh = S.K + cl;
  const int F = 1 << sh;
  const int fx = w.c[0] >> sh, fy = w.c[1] >> sh;
  const int bx = fx << sh, by = fy << sh;
  const float tx = ((float)((w.D[0] > 0.f ? bx + F : bx) - w.Oi[0]) - w.Of[0]) * w.invD[0];
  const float ty = ((float)((w.D[1] > 0.f ? by + F : by) - w.Oi[1]) - w.Of[1]) * w.invD[1];
  float te = fminf(tx, ty);
  int ax = tx <= ty ? 0 : 1;
  const bool up = w.D[2] > 0.f;
  const int LS = S.layer_shift;
  const int lcur = w.c[2] >> LS;
  // furthest layer the ray reaches inside the footprint (widened toward travel)
  const float zf = (float)w.Oi[2] + fmaf(fminf(te, w.tend), w.D[2], w.Of[2]) + (up ? 1e-3f : -1e-3f);
  int lend = __float2int_rd(zf) >> LS;
  lend = min(max(lend, 0), S.n_layers - 1);
  const unsigned long long lo64 = ((unsigned long long)m.y << 32) | m.x;
  const unsigned long long hi64 = ((unsigned long long)m.w << 32) | m.z;
  int Ls;  // nearest occupied layer at or beyond lcur in the direction of travel
  if (up) {
    const unsigned long long a = lcur < 64 ? (lo64 & (~0ull << lcur)) : 0ull;
    const unsigned long long b = lcur < 64 ? hi64 : (hi64 & (~0ull << (lcur - 64)));
    Ls = a ? (__ffsll((long long)a) - 1) : (b ? (63 + __ffsll((long long)b)) : 1 << 20);
  } else {
    const unsigned long long a = lcur >= 64 ? lo64 : (lo64 & ((2ull << lcur) - 1ull));
    const unsigned long long b = lcur >= 64 ? (hi64 & ((2ull << (lcur - 64)) - 1ull)) : 0ull;
    Ls = b ? (127 - __clzll((long long)b)) : (a ? (63 - __clzll((long long)a)) : -(1 << 20));
  }
  if (Ls == lcur) return false;
  const bool reach = up ? (Ls <= lend) : (Ls >= lend);
  int zlo, zhi;
  if (up) {
    zlo = lcur << LS;
    zhi = (reach ? Ls : lend + 1) << LS;
  } else {
    zlo = (reach ? Ls + 1 : lend) << LS;
    zhi = (lcur + 1) << LS;
  }
  if (reach) {
    const int zb = up ? zlo + (zhi - zlo) : zlo;  // boundary plane of layer Ls facing the ray
    const float tz = ((float)(zb - w.Oi[2]) - w.Of[2]) * w.invD[2];
    if (tz < te) {
      te = tz;
      ax = 2;
    }
  }
  lo[0] = bx;
  hi[0] = bx + F;
  lo[1] = by;
  hi[1] = by + F;
  lo[2] = zlo;
  hi[2] = zhi;
  *axis = ax;
  *t_exit = te;
  return te > w.t;
}

struct Hit {
  int vox;
  int base[3];
  int ls;
  float tin, tout;
};

// Distance at which the ray enters a hit's box, not before t0 (where its walk
// from the start began): the same formula as the entry next_hit reports, but
// independent of where a walk started, so every walk of one ray agrees on it.
__device__ __forceinline__ float hit_entry(const Walk& w, const Hit& h, float t0) {
  const int E = 1 << h.ls;
  float t = t0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const int p = (w.D[a] > 0.f ? h.base[a] : h.base[a] + E) - w.Oi[a];
    t = fmaxf(t, ((float)p - w.Of[a]) * w.invD[a]);
  }
  return t;
}

// Leave the box [lo, hi) through its face on `axis` at distance te: the next
// point to locate is the neighbour cell across that face, the other
// coordinates taken from the exit point, kept inside the box's face and never
// moved backwards (so every hop makes progress).
__device__ __forceinline__ void hop(const DevScene& S, Walk& w, const int lo[3], const int hi[3],
                                    int axis, float te) {
  if (!(te < w.tend) || ++w.steps > S.Gf[0] + S.Gf[1] + S.Gf[2] + 64) {
    if (w.steps > S.Gf[0] + S.Gf[1] + S.Gf[2] + 64) atomicOr(S.status, SALF_DEVERR_STEP_CAP);
    w.alive = false;
    return;
  }
  bool out = false;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (a == axis) {
      const int n = w.D[a] > 0.f ? hi[a] : lo[a] - 1;
      out = n < 0 || n >= S.Gf[a];
      w.c[a] = n;
    } else {
      int q = w.Oi[a] + __float2int_rd(fmaf(te, w.D[a], w.Of[a]));
      q = min(max(q, lo[a]), hi[a] - 1);
      q = min(q, S.Gf[a] - 1);  // boxes start at >= 0, so q >= 0 already
      w.c[a] = w.D[a] > 0.f ? max(q, w.c[a]) : min(q, w.c[a]);
    }
  }
  if (out) w.alive = false;
  w.t = fmaxf(w.t, te);
}

// Advance `w` by one structure step toward the next voxel crossed with
// positive length; true if this step found it (in h).  The caller's warp
// composites the lanes that found one, then calls again: one step per call
// keeps lanes of different rays in step, so a warp costs about its heaviest
// ray, not the sum of per-round maxima (two or three steps per call measured
// slower, and the loop for them cost 1-3% even when it ran once).  Empty space
// is left through the farther of two empty boxes around the current cell: the
// largest empty aligned pyramid cell, and the column-pyramid skip.
// FMIN: take the exit distance as the minimum of the three plane distances
// (the same value as indexing them by the exit axis, as they are finite); the
// indexed form keeps the array in local memory, the minimum does not.  The
// span-parallel kernel measured 1.3% slower with it, so it keeps the indexed
// form.
template <bool FMIN = true>
__device__ __forceinline__ bool next_hit(const DevScene& S, Walk& w, Hit& h) {
  if (w.alive) {
    // the column mask depends only on the cell: issue its load with the pyramid's
    const int cl = w.cl;
#if SALF_COL_EARLY
    const uint4 cmask = col_mask(S, w, cl);
#endif
    int ls;
    const int vox = find_leaf(S, w.c[0], w.c[1], w.c[2], &ls);
    const int E = 1 << ls;
    int lo[3], hi[3];
    float tx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      lo[a] = w.c[a] & ~(E - 1);
      hi[a] = lo[a] + E;
      const int p = (w.D[a] > 0.f ? hi[a] : lo[a]) - w.Oi[a];
      tx[a] = ((float)p - w.Of[a]) * w.invD[a];
    }
    int ax = (tx[0] <= tx[1] && tx[0] <= tx[2]) ? 0 : (tx[1] <= tx[2] ? 1 : 2);
    float te = FMIN ? fminf(fminf(tx[0], tx[1]), tx[2]) : tx[ax];
    bool found = false;
    if (vox >= 0) {
      float tin = w.t;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int p = (w.D[a] > 0.f ? lo[a] : hi[a]) - w.Oi[a];
        tin = fmaxf(tin, ((float)p - w.Of[a]) * w.invD[a]);
      }
      const float tout = fminf(te, w.tend);
      found = tout > tin;
      // start fetching the voxel's record: it is read right after this step
      prefetch_l1(static_cast<const char*>(S.params) +
                  (size_t)vox * (S.dtype == SALF_F32 ? 128u : 64u));
      h.vox = vox;
      h.ls = ls;
      h.base[0] = lo[0];
      h.base[1] = lo[1];
      h.base[2] = lo[2];
      h.tin = tin;
      h.tout = tout;
    } else {
      // empty: the column-pyramid skip replaces the pyramid cell if it goes further
      int clo[3], chi[3], cax;
      float cte;
      bool ok = false;
#if SALF_COL_MAX_LS > 0
      if (ls <= SALF_COL_MAX_LS + S.K)
#endif
      {
#if !SALF_COL_EARLY
        const uint4 cmask = col_mask(S, w, cl);
#endif
        ok = col_skip(S, w, cl, cmask, &cte, clo, chi, &cax);
        w.cl = ok ? min(cl + 1, S.CL - 1) : max(cl - 1, 0);
      }
      if (ok && cte > te) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          lo[a] = clo[a];
          hi[a] = chi[a];
        }
        ax = cax;
        te = cte;
      }
    }
    // one hop for every lane, whichever box it leaves (keeps the warp converged)
    hop(S, w, lo, hi, ax, te);
    return found;
  }
  return false;
}

// ---------------------------------------------------------------- records

template <int DT>
struct Record;  // widened record (BF16 only: FP32 records are read in stages)

// Where a record's 16-byte chunks come from: global memory (read-only path)
// or a copy of the raw record bytes in shared memory.
struct GlobalRec {
  const float4* p;
  __device__ __forceinline__ float4 chunk(int k) const { return __ldg(p + k); }
};
struct SharedRec {
  const float4* p;
  __device__ __forceinline__ float4 chunk(int k) const { return p[k]; }
};

// BF16: 32 bf16 (64 B), widened to FP32 in registers.
template <>
struct Record<SALF_BF16> {
  float v[32];
  template <class Src>
  __device__ __forceinline__ void load(const Src& src) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float4 c = src.chunk(k);
      const uint4 q = make_uint4(__float_as_uint(c.x), __float_as_uint(c.y), __float_as_uint(c.z),
                                 __float_as_uint(c.w));
      unsigned w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        v[8 * k + 2 * j] = __uint_as_float(w4[j] << 16);
        v[8 * k + 2 * j + 1] = __uint_as_float(w4[j] & 0xffff0000u);
      }
    }
  }
};

// Local coordinates of the segment midpoint inside the voxel box
// [base, base + 2^ls) (finest cells): x = (p - centre) / (edge / 2).
__device__ __forceinline__ void local_coords(const Walk& w, const Hit& h, float tm, float x[3]) {
  const float E = (float)(1 << h.ls);
  const float inv_half = __int_as_float((128 - h.ls) << 23);  // 2 / E, exact: E = 2^ls
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float p = fmaf(tm, w.D[a], w.Of[a]);  // relative to the origin cell
    float ctr = (float)(h.base[a] - w.Oi[a]) + 0.5f * E;
    x[a] = (p - ctr) * inv_half;
  }
}

__device__ __forceinline__ float sigmoidf_fast(float z) {
  return __fdividef(1.f, 1.f + __expf(-z));
}

// Eq. 1 (EXP) or Eq. 5-6 (SDF) density at x; `lin` = W . [x, 1].
template <int MODE>
__device__ __forceinline__ float density(const float* rec, const float x[3], float* lin) {
  float s = fmaf(rec[0], x[0], fmaf(rec[1], x[1], fmaf(rec[2], x[2], rec[3])));
  *lin = s;
  if (MODE == SALF_FIELD_EXP) return __expf(s);
  float a = rec[25], b = rec[26];
  float e = __expf(-fabsf(s) / b);
  float sg = (s > 0.f) ? 1.f : ((s < 0.f) ? -1.f : 0.f);
  return 0.5f * a + 0.5f * a * sg * (1.f - e);
}

// Eq. 2 colour: c = sigmoid(W_c x + W_sh gamma(d)).
__device__ __forceinline__ void colour(const float* rec, const float x[3], const float gam[4],
                                       float c[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    float z = rec[4 + 3 * r] * x[0] + rec[5 + 3 * r] * x[1] + rec[6 + 3 * r] * x[2];
    z = fmaf(rec[13 + 4 * r], gam[0], z);
    z = fmaf(rec[14 + 4 * r], gam[1], z);
    z = fmaf(rec[15 + 4 * r], gam[2], z);
    z = fmaf(rec[16 + 4 * r], gam[3], z);
    c[r] = sigmoidf_fast(z);
  }
}

__device__ __forceinline__ float intensity_field(const float* rec, const float x[3]) {
  float z = fmaf(rec[27], x[0], fmaf(rec[28], x[1], fmaf(rec[29], x[2], rec[30])));
  return sigmoidf_fast(z);
}

__device__ __forceinline__ void sh_basis(const float d[3], float gam[4]) {
  gam[0] = kSH0;
  gam[1] = kSH1 * d[1];
  gam[2] = kSH1 * d[2];
  gam[3] = kSH1 * d[0];
}

// Launch-order tile row k -> tile row: first_row, first_row + 1, first_row - 1,
// first_row + 2, ... (rows past one edge continue on the other side).
__device__ __forceinline__ int zigzag_row(int k, int first, int rows) {
  const int below = rows - 1 - first;  // rows after `first`
  const int m = min(first, below);     // pairs that alternate
  if (k <= 2 * m) return (k & 1) ? first + (k + 1) / 2 : first - k / 2;
  const int rest = k - 2 * m;          // only one side left
  return below > first ? first + m + rest : first - m - rest;
}

// Tile of a warp: (pixel column, pixel row) of its first lane.
__device__ __forceinline__ void tile_origin(const ReqDev& Q, int tile, int* u0, int* v0) {
  const int tx = tile % Q.tiles_x, k = tile / Q.tiles_x;
  *u0 = tx * Q.tile_w;
  *v0 = zigzag_row(k, Q.first_row, Q.tiles_y) * Q.tile_h;
}

// Local field of one voxel at local coordinates x (Eq. 1 or 5-6, Eq. 2, and
// the intensity field): density, the affine geometry value, colour,
// intensity, and the SDF parameters a, b.
struct Field {
  float sig, lin, c[3], io, a, b;
  float dr;  // sigmoid of the raydrop logit (record slot 31), when asked for
};

__device__ __forceinline__ float sdf_density(float s, float a, float b) {
  const float e = __expf(-fabsf(s) / b);
  const float sg = (s > 0.f) ? 1.f : ((s < 0.f) ? -1.f : 0.f);
  return 0.5f * a + 0.5f * a * sg * (1.f - e);
}

// FP32 records are read in two stages (a compiler barrier keeps the second
// stage's loads below the first stage's arithmetic), so only half of the
// record is live in registers at a time.  Slots: Wsigma 0-3, W_c 4-12 (rows
// r, g, b), W_sh 13-24 (rows r, g, b), a 25, b 26, W_int 27-30.
template <int DT, int MODE, class Src>
__device__ __forceinline__ void field_eval_src(const Src& p, bool want_int, const float x[3],
                                               const float gam[4], Field& f,
                                               bool want_drop = false) {
  if constexpr (DT == SALF_F32) {
    const float4 q0 = p.chunk(0), q1 = p.chunk(1), q2 = p.chunk(2), q3 = p.chunk(3);
    f.lin = fmaf(q0.x, x[0], fmaf(q0.y, x[1], fmaf(q0.z, x[2], q0.w)));
    float zr = q1.x * x[0] + q1.y * x[1] + q1.z * x[2];
    float zg = q1.w * x[0] + q2.x * x[1] + q2.y * x[2];
    float zb = q2.z * x[0] + q2.w * x[1] + q3.x * x[2];
    zr = fmaf(q3.y, gam[0], zr);
    zr = fmaf(q3.z, gam[1], zr);
    zr = fmaf(q3.w, gam[2], zr);
    asm volatile("" ::: "memory");
    const float4 q4 = p.chunk(4), q5 = p.chunk(5), q6 = p.chunk(6);
    zr = fmaf(q4.x, gam[3], zr);
    zg = fmaf(q4.y, gam[0], zg);
    zg = fmaf(q4.z, gam[1], zg);
    zg = fmaf(q4.w, gam[2], zg);
    zg = fmaf(q5.x, gam[3], zg);
    zb = fmaf(q5.y, gam[0], zb);
    zb = fmaf(q5.z, gam[1], zb);
    zb = fmaf(q5.w, gam[2], zb);
    zb = fmaf(q6.x, gam[3], zb);
    f.a = q6.y;
    f.b = q6.z;
    f.sig = MODE == SALF_FIELD_EXP ? __expf(f.lin) : sdf_density(f.lin, f.a, f.b);
    f.c[0] = sigmoidf_fast(zr);
    f.c[1] = sigmoidf_fast(zg);
    f.c[2] = sigmoidf_fast(zb);
    f.io = 0.f;
    f.dr = 0.f;
    if (want_int || want_drop) {
      const float4 q7 = p.chunk(7);
      if (want_int)
        f.io = sigmoidf_fast(fmaf(q6.w, x[0], fmaf(q7.x, x[1], fmaf(q7.y, x[2], q7.z))));
      if (want_drop) f.dr = sigmoidf_fast(q7.w);
    }
  } else {
    Record<DT> rec;
    rec.load(p);
    f.sig = density<MODE>(rec.v, x, &f.lin);
    colour(rec.v, x, gam, f.c);
    f.io = want_int ? intensity_field(rec.v, x) : 0.f;
    f.dr = want_drop ? sigmoidf_fast(rec.v[31]) : 0.f;
    f.a = rec.v[25];
    f.b = rec.v[26];
  }
}

// Record bytes per voxel and the 16-byte chunks of one record.
template <int DT>
struct RecordLayout {
  static constexpr int kChunks = DT == SALF_F32 ? 8 : 4;
};

template <int DT, int MODE>
__device__ __forceinline__ void field_eval(const DevScene& S, int vox, bool want_int,
                                           const float x[3], const float gam[4], Field& f,
                                           bool want_drop = false) {
  const GlobalRec src{reinterpret_cast<const float4*>(S.params) +
                      (size_t)vox * RecordLayout<DT>::kChunks};
  field_eval_src<DT, MODE>(src, want_int, x, gam, f, want_drop);
}

// Front-to-back accumulators of one ray (Eq. 3-4).
struct Accum {
  float T, C0, C1, C2, Dp, Ip;
  int nvis;
  float Rp;  // sum of T_i alpha_i sigmoid(rho_i) (raydrop, when asked for)
};

// Composite one hit voxel with its field at the segment midpoint: alpha =
// 1 - exp(-sigma delta) (Eq. 4), weight T alpha (Eq. 3).  The ray kernel and
// the tile rasteriser both call this, so their arithmetic is the same.
// Returns 1 - alpha.
template <int DT, int MODE, class Src>
__device__ __forceinline__ float composite_hit(const Walk& w, const Hit& h, const Src& src,
                                              bool want_int, const float gam[4], Accum& A,
                                              bool want_drop = false) {
  const float tm = 0.5f * (h.tin + h.tout);
  const float dl = h.tout - h.tin;
  float x[3];
  local_coords(w, h, tm, x);
  Field f;
  field_eval_src<DT, MODE>(src, want_int, x, gam, f, want_drop);
  const float e = __expf(-f.sig * dl);  // 1 - alpha (Eq. 4)
  const float wgt = A.T * (1.f - e);    // T_i alpha_i (Eq. 3)
  A.C0 = fmaf(wgt, f.c[0], A.C0);
  A.C1 = fmaf(wgt, f.c[1], A.C1);
  A.C2 = fmaf(wgt, f.c[2], A.C2);
  A.Dp = fmaf(wgt, tm, A.Dp);
  if (want_int) A.Ip = fmaf(wgt, f.io, A.Ip);
  if (want_drop) A.Rp = fmaf(wgt, f.dr, A.Rp);
  A.T *= e;
  return e;
}

// Per-ray outputs of a request (colour premultiplied, background added with
// the final transmittance; opacity 1 - T_end, which the weights sum to).
__device__ __forceinline__ void write_outputs(const ReqDev& Q, int ray, bool valid, const Accum& A,
                                              bool want_drop = false) {
  // raydrop: an escaping ray (T_end) returns nothing
  if (want_drop) Q.raydrop[ray] = valid ? A.Rp + A.T : 0.f;
  if (Q.rgb) {
    float* o = Q.rgb + 3 * (size_t)ray;
    o[0] = valid ? fmaf(A.T, Q.bg[0], A.C0) : 0.f;
    o[1] = valid ? fmaf(A.T, Q.bg[1], A.C1) : 0.f;
    o[2] = valid ? fmaf(A.T, Q.bg[2], A.C2) : 0.f;
  }
  const float Op = 1.f - A.T;  // sum of T_i alpha_i telescopes to 1 - T_end (Eq. 3-4)
  if (Q.depth) Q.depth[ray] = A.Dp;
  if (Q.opacity) Q.opacity[ray] = Op;
  if (Q.intensity) Q.intensity[ray] = A.Ip;
  if (Q.saved) {
    float4* s = reinterpret_cast<float4*>(Q.saved) + 2 * (size_t)ray;
    s[0] = make_float4(A.C0, A.C1, A.C2, A.Dp);
    s[1] = make_float4(Op, A.Ip, A.T, (float)A.nvis);
  }
  if (Q.valid) Q.valid[ray] = valid ? 1 : 0;
}

// Products of the transmittances of the spans of a ray (lanes k = 0..K-1 of a
// group of K): *inc = T_0 ... T_k, *ex = T_0 ... T_k-1 (1 for k = 0).  The
// association order is fixed, so the products only fall as the T_k fall.
__device__ __forceinline__ void span_products(float T, int k, int K, float* inc, float* ex) {
  float p = T;
  for (int off = 1; off < K; off <<= 1) {
    const float y = __shfl_up_sync(0xffffffffu, p, off, K);
    if (k >= off) p *= y;
  }
  const float e = __shfl_up_sync(0xffffffffu, p, 1, K);
  *inc = p;
  *ex = k == 0 ? 1.f : e;
}

// Warp tile -> request, pixel.
__device__ __forceinline__ int find_request(const LaunchParams& P, int warp) {
  int r = 0;
  while (r + 1 < P.n_req && warp >= P.req[r + 1].tile_begin) ++r;
  return r;
}

}  // namespace salf
