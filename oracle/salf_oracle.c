/*
 * salf_oracle.c -- FP64 CPU oracle for SaLF ray-cast rendering.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check and the benchmark's CPU
 * baseline).  Plain and slow on purpose: every step is the definition written
 * out, in the order the paper states it.
 *
 * Readings of points the paper leaves open (all shared with the docs):
 *   - gamma(omega), Eq. 2: real spherical harmonics of bands l <= 1, 4 values
 *     [C0, C1*w_y, C1*w_z, C1*w_x], C0 = 1/(2 sqrt(pi)), C1 = sqrt(3)/(2 sqrt(pi)),
 *     no Condon-Shortley sign; omega = the unit ray direction (world frame).
 *   - local coordinates x = (X - voxel centre) / (edge / 2) in [-1, 1]^3,
 *     voxel frames = world frame (rotation q fixed at identity, Sec. III-A).
 *   - Eq. 2 uses x (not the homogeneous x-hat): no colour bias besides SH.
 *   - sampling point (Sec. III-A, after Eq. 4): midpoint of the ray-voxel
 *     segment clipped to [t_near, t_far]; delta = the clipped length.
 *   - a voxel is hit iff that clipped length is > 0; in FP64 "> 0" is read as
 *     "> 1e-9 finest-cell edges", so that rays passing exactly through a
 *     voxel edge or corner (length 0 in exact arithmetic, ~1e-15 after
 *     rounding) count as misses whichever way the rounding goes.
 *   - Eq. 6 with sign(0) = 0.
 *   - depth = sum_i w_i t_mid,i (unnormalised), opacity = sum_i w_i,
 *     intensity = sum_i w_i sigmoid(W_int . x-hat); colour premultiplied,
 *     plus T_end * background.
 *   - early termination: composite voxel i, then stop if T_{i+1} < t_min.
 *   - sensor conventions: see the sensor section below.
 */
#include "salf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define REC 32

typedef struct {
  int32_t l, i, j, k, idx;
} okey;

struct orc_scene {
  int64_t n;
  double origin[3];
  double s0;
  int32_t dims[3];
  int32_t K;
  int32_t mode;
  double min_len; /* hit threshold on the clipped segment length */
  uint8_t* level;
  int32_t* ijk;
  double* params;
  okey* keys; /* sorted by (l, k, j, i) */
};

static int key_cmp(const void* pa, const void* pb) {
  const okey* a = (const okey*)pa;
  const okey* b = (const okey*)pb;
  if (a->l != b->l) return a->l < b->l ? -1 : 1;
  if (a->k != b->k) return a->k < b->k ? -1 : 1;
  if (a->j != b->j) return a->j < b->j ? -1 : 1;
  if (a->i != b->i) return a->i < b->i ? -1 : 1;
  return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int64_t orc_scene_lookup(const orc_scene* s, int32_t level, int32_t i, int32_t j, int32_t k) {
  okey q = {level, i, j, k, -1};
  const okey* f = (const okey*)bsearch(&q, s->keys, (size_t)s->n, sizeof(okey), key_cmp);
  return f ? f->idx : -1;
}

void orc_scene_free(orc_scene* s) {
  if (!s) return;
  free(s->level);
  free(s->ijk);
  free(s->params);
  free(s->keys);
  free(s);
}

/* Sec. III-A: voxels live on the level grids of a root grid; Sec. III-D:
 * voxels are disjoint, so a voxel whose ancestor (or itself) is present
 * again is rejected. */
int orc_scene_create(const orc_scene_desc* d, orc_scene** out) {
  *out = NULL;
  if (d->n < 0 || d->max_level < 0 || d->max_level > 16 || d->s0 <= 0) return 1;
  for (int a = 0; a < 3; ++a)
    if (d->dims[a] <= 0) return 1;
  orc_scene* s = (orc_scene*)calloc(1, sizeof(orc_scene));
  s->n = d->n;
  memcpy(s->origin, d->origin, sizeof(s->origin));
  s->s0 = d->s0;
  memcpy(s->dims, d->dims, sizeof(s->dims));
  s->K = d->max_level;
  s->mode = d->mode;
  s->min_len = 1e-9 * d->s0 / (double)(1 << d->max_level);
  size_t n = (size_t)d->n;
  s->level = (uint8_t*)malloc(n ? n : 1);
  s->ijk = (int32_t*)malloc((n ? n : 1) * 3 * sizeof(int32_t));
  s->params = (double*)malloc((n ? n : 1) * REC * sizeof(double));
  s->keys = (okey*)malloc((n ? n : 1) * sizeof(okey));
  if (n) {
    memcpy(s->level, d->level, n);
    memcpy(s->ijk, d->ijk, n * 3 * sizeof(int32_t));
    memcpy(s->params, d->params, n * REC * sizeof(double));
  }
  for (size_t v = 0; v < n; ++v) {
    int32_t l = s->level[v];
    if (l > s->K) { orc_scene_free(s); return 1; }
    for (int a = 0; a < 3; ++a) {
      int64_t lim = (int64_t)s->dims[a] << l;
      if (s->ijk[3 * v + a] < 0 || s->ijk[3 * v + a] >= lim) { orc_scene_free(s); return 1; }
    }
    if (s->mode == 1 && !(s->params[REC * v + 25] > 0 && s->params[REC * v + 26] > 0)) {
      orc_scene_free(s);
      return 1;
    }
    okey kk = {l, s->ijk[3 * v], s->ijk[3 * v + 1], s->ijk[3 * v + 2], (int32_t)v};
    s->keys[v] = kk;
  }
  qsort(s->keys, n, sizeof(okey), key_cmp);
  for (size_t v = 1; v < n; ++v)
    if (key_cmp(&s->keys[v - 1], &s->keys[v]) == 0) { orc_scene_free(s); return 4; }
  for (size_t v = 0; v < n; ++v) {
    int32_t l = s->level[v];
    for (int32_t la = 0; la < l; ++la) {
      int sh = l - la;
      if (orc_scene_lookup(s, la, s->ijk[3 * v] >> sh, s->ijk[3 * v + 1] >> sh,
                           s->ijk[3 * v + 2] >> sh) >= 0) {
        orc_scene_free(s);
        return 4;
      }
    }
  }
  *out = s;
  return 0;
}

int orc_scene_set_record(orc_scene* s, int64_t v, const double* rec) {
  if (!s || v < 0 || v >= s->n || !rec) return 1;
  if (s->mode == 1 && !(rec[25] > 0 && rec[26] > 0)) return 1;
  memcpy(s->params + (size_t)REC * v, rec, REC * sizeof(double));
  return 0;
}

static void voxel_box(const orc_scene* s, int64_t v, double lo[3], double hi[3], double* edge) {
  int32_t l = s->level[v];
  double e = s->s0 / (double)(1 << l);
  for (int a = 0; a < 3; ++a) {
    lo[a] = s->origin[a] + (double)s->ijk[3 * v + a] * e;
    hi[a] = lo[a] + e;
  }
  *edge = e;
}

/* Ray-box slab test: parameter interval where o + t d is inside [lo, hi). */
static int slab(const double lo[3], const double hi[3], const double o[3], const double d[3],
                double* t0, double* t1) {
  double a = -INFINITY, b = INFINITY;
  for (int ax = 0; ax < 3; ++ax) {
    if (d[ax] != 0.0) {
      double ta = (lo[ax] - o[ax]) / d[ax];
      double tb = (hi[ax] - o[ax]) / d[ax];
      if (ta > tb) { double t = ta; ta = tb; tb = t; }
      if (ta > a) a = ta;
      if (tb < b) b = tb;
    } else if (o[ax] < lo[ax] || o[ax] >= hi[ax]) {
      return 0;
    }
  }
  *t0 = a;
  *t1 = b;
  return 1;
}

static double dmax(double a, double b) { return a > b ? a : b; }
static double dmin(double a, double b) { return a < b ? a : b; }

typedef struct {
  orc_hit* h;
  int64_t n, cap;
} hitvec;

static void hv_push(hitvec* v, int32_t vox, double a, double b) {
  if (v->n == v->cap) {
    v->cap = v->cap ? 2 * v->cap : 64;
    v->h = (orc_hit*)realloc(v->h, (size_t)v->cap * sizeof(orc_hit));
  }
  v->h[v->n].voxel = vox;
  v->h[v->n].t_in = a;
  v->h[v->n].t_out = b;
  v->n++;
}

typedef struct {
  double key;
  orc_hit h;
} skey;

static int skey_cmp(const void* pa, const void* pb) {
  const skey* a = (const skey*)pa;
  const skey* b = (const skey*)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  return a->h.voxel < b->h.voxel ? -1 : (a->h.voxel > b->h.voxel);
}

/* Order hits by their clipped entry distance max(t_in, tn). */
static void sort_hits(hitvec* v, double tn) {
  if (v->n < 2) return;
  skey* k = (skey*)malloc((size_t)v->n * sizeof(skey));
  for (int64_t i = 0; i < v->n; ++i) {
    k[i].key = dmax(v->h[i].t_in, tn);
    k[i].h = v->h[i];
  }
  qsort(k, (size_t)v->n, sizeof(skey), skey_cmp);
  for (int64_t i = 0; i < v->n; ++i) v->h[i] = k[i].h;
  free(k);
}

static int32_t owner_of_fine_cell(const orc_scene* s, const int64_t c[3]) {
  for (int32_t l = 0; l <= s->K; ++l) {
    int sh = s->K - l;
    int64_t v = orc_scene_lookup(s, l, (int32_t)(c[0] >> sh), (int32_t)(c[1] >> sh),
                                 (int32_t)(c[2] >> sh));
    if (v >= 0) return (int32_t)v;
  }
  return -1;
}

static int i32_cmp(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return x < y ? -1 : (x > y);
}

typedef struct {
  int32_t* v;
  int64_t n, cap;
} ivec;

static void iv_push(ivec* v, int32_t x) {
  if (v->n == v->cap) {
    v->cap = v->cap ? 2 * v->cap : 64;
    v->v = (int32_t*)realloc(v->v, (size_t)v->cap * sizeof(int32_t));
  }
  v->v[v->n++] = x;
}

/* Candidate voxels: owners of the finest-level cells the ray passes through
 * (Amanatides-Woo grid walk), optionally with their 26 neighbours.  This only
 * enumerates candidates; which of them are hit is decided by the slab test. */
static void dda_candidates(const orc_scene* s, const double o[3], const double d[3], double tn,
                           double tf, int neighbours, ivec* cand) {
  int64_t Gf[3];
  double sf = s->s0 / (double)(1 << s->K);
  double lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    Gf[a] = (int64_t)s->dims[a] << s->K;
    lo[a] = s->origin[a];
    hi[a] = s->origin[a] + (double)s->dims[a] * s->s0;
  }
  double ra, rb;
  if (!slab(lo, hi, o, d, &ra, &rb)) return;
  double ta = dmax(ra, tn), tb = dmin(rb, tf);
  if (!(ta < tb)) return;
  int64_t c[3], step[3];
  double tmax[3], tdel[3];
  for (int a = 0; a < 3; ++a) {
    double p = o[a] + ta * d[a];
    int64_t ci = (int64_t)floor((p - s->origin[a]) / sf);
    if (ci < 0) ci = 0;
    if (ci >= Gf[a]) ci = Gf[a] - 1;
    c[a] = ci;
    if (d[a] > 0) {
      step[a] = 1;
      tmax[a] = (s->origin[a] + (double)(ci + 1) * sf - o[a]) / d[a];
      tdel[a] = sf / d[a];
    } else if (d[a] < 0) {
      step[a] = -1;
      tmax[a] = (s->origin[a] + (double)ci * sf - o[a]) / d[a];
      tdel[a] = -sf / d[a];
    } else {
      step[a] = 0;
      tmax[a] = INFINITY;
      tdel[a] = INFINITY;
    }
  }
  int32_t last = -2;
  for (;;) {
    if (neighbours) {
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            int64_t q[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
            if (q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] >= Gf[0] || q[1] >= Gf[1] ||
                q[2] >= Gf[2])
              continue;
            int32_t w = owner_of_fine_cell(s, q);
            if (w >= 0) iv_push(cand, w);
          }
    } else {
      int32_t w = owner_of_fine_cell(s, c);
      if (w >= 0 && w != last) iv_push(cand, w);
      last = w;
    }
    int a = 0;
    if (tmax[1] < tmax[a]) a = 1;
    if (tmax[2] < tmax[a]) a = 2;
    if (!(tmax[a] < tb)) break;
    c[a] += step[a];
    tmax[a] += tdel[a];
    if (c[a] < 0 || c[a] >= Gf[a]) break;
  }
}

static void unique_ids(ivec* v) {
  if (v->n < 2) return;
  qsort(v->v, (size_t)v->n, sizeof(int32_t), i32_cmp);
  int64_t w = 1;
  for (int64_t i = 1; i < v->n; ++i)
    if (v->v[i] != v->v[w - 1]) v->v[w++] = v->v[i];
  v->n = w;
}

static void trace_vec(const orc_scene* s, const double o[3], const double d[3], double tn,
                      double tf, int32_t brute, hitvec* out) {
  double lo[3], hi[3], e, a, b;
  out->n = 0;
  if (brute) {
    for (int64_t v = 0; v < s->n; ++v) {
      voxel_box(s, v, lo, hi, &e);
      if (slab(lo, hi, o, d, &a, &b) && dmin(b, tf) - dmax(a, tn) > s->min_len)
        hv_push(out, (int32_t)v, a, b);
    }
  } else {
    ivec cand = {0, 0, 0};
    dda_candidates(s, o, d, tn, tf, 0, &cand);
    unique_ids(&cand);
    for (int64_t i = 0; i < cand.n; ++i) {
      int32_t v = cand.v[i];
      voxel_box(s, v, lo, hi, &e);
      if (slab(lo, hi, o, d, &a, &b) && dmin(b, tf) - dmax(a, tn) > s->min_len)
        hv_push(out, v, a, b);
    }
    free(cand.v);
  }
  sort_hits(out, tn);
}

int64_t orc_trace(const orc_scene* s, const double o[3], const double d[3], double tn, double tf,
                  int32_t brute_force, orc_hit* hits, int64_t cap) {
  hitvec hv = {0, 0, 0};
  trace_vec(s, o, d, tn, tf, brute_force, &hv);
  for (int64_t i = 0; i < hv.n && i < cap; ++i) hits[i] = hv.h[i];
  int64_t n = hv.n;
  free(hv.h);
  return n;
}

int64_t orc_trace_eps(const orc_scene* s, const double o[3], const double d[3], double tn,
                      double tf, double eps_abs, double eps_rel, int32_t sign, int32_t* ids,
                      double* t_in, double* t_out, int64_t cap) {
  ivec cand = {0, 0, 0};
  if (s->n <= 20000) {
    for (int64_t v = 0; v < s->n; ++v) iv_push(&cand, (int32_t)v);
  } else {
    dda_candidates(s, o, d, tn, tf, 1, &cand);
    unique_ids(&cand);
  }
  hitvec hv = {0, 0, 0};
  for (int64_t i = 0; i < cand.n; ++i) {
    int32_t v = cand.v[i];
    double lo[3], hi[3], e, a, b, dist = 0;
    voxel_box(s, v, lo, hi, &e);
    for (int ax = 0; ax < 3; ++ax) {
      double cc = 0.5 * (lo[ax] + hi[ax]) - o[ax];
      dist += cc * cc;
    }
    double eps = eps_abs + eps_rel * sqrt(dist);
    for (int ax = 0; ax < 3; ++ax) {
      lo[ax] -= sign * eps;
      hi[ax] += sign * eps;
    }
    if (slab(lo, hi, o, d, &a, &b) && dmin(b, tf) - dmax(a, tn) > s->min_len)
      hv_push(&hv, v, a, b);
  }
  sort_hits(&hv, tn);
  for (int64_t i = 0; i < hv.n && i < cap; ++i) {
    ids[i] = hv.h[i].voxel;
    if (t_in) t_in[i] = hv.h[i].t_in;
    if (t_out) t_out[i] = hv.h[i].t_out;
  }
  int64_t n = hv.n;
  free(hv.h);
  free(cand.v);
  return n;
}

/* ------------------------------------------------------------------------ */
/* Sensors (Fig. 2, Sec. V-C).  Camera frame: x right, y down, z forward.    */
/* LiDAR frame: x forward, y left, z up.                                     */
/* ------------------------------------------------------------------------ */

static void mat_to_quat(const double* P, double q[4]) {
  /* rotation part of a row-major 3x4 [R|t]; q = (w, x, y, z); Shoemake. */
  double r00 = P[0], r01 = P[1], r02 = P[2];
  double r10 = P[4], r11 = P[5], r12 = P[6];
  double r20 = P[8], r21 = P[9], r22 = P[10];
  double tr = r00 + r11 + r22, S;
  if (tr > 0) {
    S = sqrt(tr + 1.0) * 2.0;
    q[0] = 0.25 * S;
    q[1] = (r21 - r12) / S;
    q[2] = (r02 - r20) / S;
    q[3] = (r10 - r01) / S;
  } else if (r00 > r11 && r00 > r22) {
    S = sqrt(1.0 + r00 - r11 - r22) * 2.0;
    q[0] = (r21 - r12) / S;
    q[1] = 0.25 * S;
    q[2] = (r01 + r10) / S;
    q[3] = (r02 + r20) / S;
  } else if (r11 > r22) {
    S = sqrt(1.0 + r11 - r00 - r22) * 2.0;
    q[0] = (r02 - r20) / S;
    q[1] = (r01 + r10) / S;
    q[2] = 0.25 * S;
    q[3] = (r12 + r21) / S;
  } else {
    S = sqrt(1.0 + r22 - r00 - r11) * 2.0;
    q[0] = (r10 - r01) / S;
    q[1] = (r02 + r20) / S;
    q[2] = (r12 + r21) / S;
    q[3] = 0.25 * S;
  }
}

static void quat_to_mat(const double q[4], double R[9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z);
  R[1] = 2 * (x * y - w * z);
  R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);
  R[4] = 1 - 2 * (x * x + z * z);
  R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);
  R[7] = 2 * (y * z + w * x);
  R[8] = 1 - 2 * (x * x + y * y);
}

/* Pose at fraction s of the way from pose0 to pose1 (3x4 row-major): linear
 * translation, spherical-linear rotation.  At s = 0 the pose is pose0 itself. */
static void interp_pose(const double* pose0, const double* pose1, double s, double R[9],
                        double t[3]) {
  if (s == 0.0) {
    for (int r = 0; r < 3; ++r) {
      for (int c = 0; c < 3; ++c) R[3 * r + c] = pose0[4 * r + c];
      t[r] = pose0[4 * r + 3];
    }
    return;
  }
  double q0[4], q1[4], q[4];
  mat_to_quat(pose0, q0);
  mat_to_quat(pose1, q1);
  double dot = q0[0] * q1[0] + q0[1] * q1[1] + q0[2] * q1[2] + q0[3] * q1[3];
  if (dot < 0) {
    dot = -dot;
    for (int i = 0; i < 4; ++i) q1[i] = -q1[i];
  }
  if (dot > 0.9999999) {
    double nn = 0;
    for (int i = 0; i < 4; ++i) {
      q[i] = (1 - s) * q0[i] + s * q1[i];
      nn += q[i] * q[i];
    }
    nn = sqrt(nn);
    for (int i = 0; i < 4; ++i) q[i] /= nn;
  } else {
    double th = acos(dot), st = sin(th);
    double a = sin((1 - s) * th) / st, b = sin(s * th) / st;
    for (int i = 0; i < 4; ++i) q[i] = a * q0[i] + b * q1[i];
  }
  quat_to_mat(q, R);
  for (int r = 0; r < 3; ++r) t[r] = (1 - s) * pose0[4 * r + 3] + s * pose1[4 * r + 3];
}

static double time_fraction(const orc_sensor* sen, double tau) {
  return sen->t1 > sen->t0 ? (tau - sen->t0) / (sen->t1 - sen->t0) : 0.0;
}

/* Pose at time tau: linear translation, spherical-linear rotation between
 * pose0 (t0) and pose1 (t1).  At the start time the pose is pose0 itself. */
void orc_pose_at(const orc_sensor* sen, double tau, double R[9], double t[3]) {
  interp_pose(sen->pose0, sen->pose1, time_fraction(sen, tau), R, t);
}

static void one_ray(const orc_sensor* sen, int64_t r, double o[3], double d[3], double* tn,
                    double* tf, double* tau, uint8_t* valid) {
  const int64_t W = sen->width, H = sen->height;
  *valid = 1;
  if (sen->kind == 4) {
    double q[8];
    for (int k = 0; k < 8; ++k) q[k] = sen->rays64 ? sen->rays64[8 * r + k] : (double)sen->rays[8 * r + k];
    double nn = 0;
    for (int a = 0; a < 3; ++a) {
      o[a] = q[a];
      d[a] = q[3 + a];
      nn += d[a] * d[a];
    }
    nn = sqrt(nn);
    for (int a = 0; a < 3; ++a) d[a] /= nn;
    *tn = q[6];
    *tf = q[7] > 0 ? q[7] : INFINITY;
    *tau = 0;
    if (!(nn > 0)) *valid = 0;
    return;
  }
  int64_t u = r % W, v = r / W;
  double ds[3];
  if (sen->kind == 3) {
    /* spinning LiDAR: row v = beam (row 0 highest), column u = azimuth */
    double e = sen->elev_max;
    if (H > 1) e = sen->elev_max - (double)v * (sen->elev_max - sen->elev_min) / (double)(H - 1);
    double ph = 2.0 * M_PI * (double)u / (double)W;
    ds[0] = cos(e) * cos(ph);
    ds[1] = cos(e) * sin(ph);
    ds[2] = sin(e);
    *tau = sen->t0 + ((double)u / (double)W) * (sen->t1 - sen->t0);
  } else {
    double px = (double)u + 0.5, py = (double)v + 0.5;
    if (sen->kind == 0) {
      ds[0] = (px - sen->cx) / sen->fx;
      ds[1] = (py - sen->cy) / sen->fy;
      ds[2] = 1.0;
    } else if (sen->kind == 1) {
      /* equidistant: image radius = f * theta */
      double mx = (px - sen->cx) / sen->fx, my = (py - sen->cy) / sen->fy;
      double th = sqrt(mx * mx + my * my);
      if (th > 0.5 * sen->fov) *valid = 0;
      if (th > 0) {
        ds[0] = sin(th) * mx / th;
        ds[1] = sin(th) * my / th;
      } else {
        ds[0] = ds[1] = 0;
      }
      ds[2] = cos(th);
    } else {
      /* equirectangular: longitude across the width (0 at the centre column,
       * increasing to the right), latitude from elev_max (top) to elev_min */
      double lon = 2.0 * M_PI * (px / (double)W - 0.5);
      double lat = sen->elev_max - (py / (double)H) * (sen->elev_max - sen->elev_min);
      ds[0] = cos(lat) * sin(lon);
      ds[1] = -sin(lat);
      ds[2] = cos(lat) * cos(lon);
    }
    *tau = sen->t0;
    if (sen->rolling_shutter && H > 1)
      *tau = sen->t0 + ((double)v / (double)(H - 1)) * (sen->t1 - sen->t0);
  }
  double R[9], t[3];
  orc_pose_at(sen, *tau, R, t);
  double nn = 0;
  for (int a = 0; a < 3; ++a) {
    d[a] = R[3 * a] * ds[0] + R[3 * a + 1] * ds[1] + R[3 * a + 2] * ds[2];
    nn += d[a] * d[a];
    o[a] = t[a];
  }
  nn = sqrt(nn);
  for (int a = 0; a < 3; ++a) d[a] /= nn;
  *tn = sen->t_near;
  *tf = sen->t_far > 0 ? sen->t_far : INFINITY;
}

int orc_gen_rays(const orc_sensor* sen, const int64_t* idx, int64_t m, double* o, double* d,
                 double* tn, double* tf, double* tau, uint8_t* valid) {
  if (sen->width <= 0 || sen->height <= 0) return 1;
  for (int64_t i = 0; i < m; ++i) {
    int64_t r = idx ? idx[i] : i;
    one_ray(sen, r, o + 3 * i, d + 3 * i, tn + i, tf + i, tau + i, valid + i);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Local fields (Eq. 1, 2, 5, 6)                                             */
/* ------------------------------------------------------------------------ */

/* Per ray of a sensor (idx as for orc_render): 1 if the ordered list of
 * voxels crossed with positive length is the same for every box shrunk and
 * grown by eps_abs + eps_rel * (distance of the box centre), else 0 (also 0
 * for invalid rays).  Such a list does not change under position errors
 * below that margin. */
int orc_conditioned(const orc_scene* s, const orc_sensor* sen, const int64_t* idx, int64_t m,
                    double eps_abs, double eps_rel, uint8_t* ok) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < m; ++i) {
    int64_t r = idx ? idx[i] : i;
    double o[3], d[3], tn, tf, tau;
    uint8_t valid;
    one_ray(sen, r, o, d, &tn, &tf, &tau, &valid);
    ok[i] = 0;
    if (!valid) continue;
    ivec cand = {0, 0, 0};
    if (s->n <= 20000) {
      for (int64_t v = 0; v < s->n; ++v) iv_push(&cand, (int32_t)v);
    } else {
      dda_candidates(s, o, d, tn, tf, 1, &cand);
      unique_ids(&cand);
    }
    hitvec hv[2] = {{0, 0, 0}, {0, 0, 0}};
    for (int side = 0; side < 2; ++side) {
      const double sign = side ? 1.0 : -1.0;
      for (int64_t c = 0; c < cand.n; ++c) {
        int32_t v = cand.v[c];
        double lo[3], hi[3], e, a, b, dist = 0;
        voxel_box(s, v, lo, hi, &e);
        for (int ax = 0; ax < 3; ++ax) {
          double cc = 0.5 * (lo[ax] + hi[ax]) - o[ax];
          dist += cc * cc;
        }
        double eps = eps_abs + eps_rel * sqrt(dist);
        for (int ax = 0; ax < 3; ++ax) {
          lo[ax] -= sign * eps;
          hi[ax] += sign * eps;
        }
        if (slab(lo, hi, o, d, &a, &b) && dmin(b, tf) - dmax(a, tn) > s->min_len)
          hv_push(&hv[side], v, a, b);
      }
      sort_hits(&hv[side], tn);
    }
    int same = hv[0].n == hv[1].n;
    for (int64_t k = 0; same && k < hv[0].n; ++k) same = hv[0].h[k].voxel == hv[1].h[k].voxel;
    ok[i] = (uint8_t)same;
    free(hv[0].h);
    free(hv[1].h);
    free(cand.v);
  }
  return 0;
}

void orc_sh_basis(const double dir[3], double g[4]) {
  const double C0 = 0.5 / sqrt(M_PI);
  const double C1 = 0.5 * sqrt(3.0 / M_PI);
  g[0] = C0;
  g[1] = C1 * dir[1];
  g[2] = C1 * dir[2];
  g[3] = C1 * dir[0];
}

static double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

static double sgn(double x) { return (x > 0) - (x < 0); }

void orc_field(const double* rec, int32_t mode, const double x[3], const double dir[3],
               double* sigma, double c[3], double* iota) {
  double xh[4] = {x[0], x[1], x[2], 1.0};
  double g[4];
  orc_sh_basis(dir, g);
  double lin = 0;
  for (int a = 0; a < 4; ++a) lin += rec[a] * xh[a];
  if (mode == 0) {
    *sigma = exp(lin); /* Eq. 1 */
  } else {
    double a = rec[25], b = rec[26]; /* Eq. 5 gives lin = s_pm; Eq. 6 */
    *sigma = 0.5 * a + 0.5 * a * sgn(lin) * (1.0 - exp(-fabs(lin) / b));
  }
  for (int r = 0; r < 3; ++r) { /* Eq. 2 */
    double z = 0;
    for (int a = 0; a < 3; ++a) z += rec[4 + 3 * r + a] * x[a];
    for (int k = 0; k < 4; ++k) z += rec[13 + 4 * r + k] * g[k];
    c[r] = sigmoid(z);
  }
  double zi = 0;
  for (int a = 0; a < 4; ++a) zi += rec[27 + a] * xh[a];
  *iota = sigmoid(zi);
}

/* ------------------------------------------------------------------------ */
/* Rendering (Eq. 3-4)                                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
  int64_t n;            /* composited voxels */
  int32_t* vox;
  double *tm, *dl, *sig, *lin, *c, *io, *dr, *alpha, *T, *w, *x;
  double t_end, gap;
} ray_record;

static void rr_free(ray_record* rr) {
  free(rr->vox);
  free(rr->tm);
  free(rr->dl);
  free(rr->sig);
  free(rr->lin);
  free(rr->c);
  free(rr->io);
  free(rr->dr);
  free(rr->alpha);
  free(rr->T);
  free(rr->w);
  free(rr->x);
}

/* Trace one ray and composite front to back; keeps every per-voxel quantity
 * so that the adjoint can be written as plain sums. */
static void composite_ray(const orc_scene* s, const orc_opts* opt, const double o[3],
                          const double d[3], double tn, double tf, ray_record* rr) {
  hitvec hv = {0, 0, 0};
  trace_vec(s, o, d, tn, tf, opt->brute_force, &hv);
  int64_t m = hv.n;
  size_t M = (size_t)(m ? m : 1);
  rr->vox = (int32_t*)malloc(M * sizeof(int32_t));
  rr->tm = (double*)malloc(M * sizeof(double));
  rr->dl = (double*)malloc(M * sizeof(double));
  rr->sig = (double*)malloc(M * sizeof(double));
  rr->lin = (double*)malloc(M * sizeof(double));
  rr->c = (double*)malloc(3 * M * sizeof(double));
  rr->io = (double*)malloc(M * sizeof(double));
  rr->dr = (double*)malloc(M * sizeof(double));
  rr->alpha = (double*)malloc(M * sizeof(double));
  rr->T = (double*)malloc(M * sizeof(double));
  rr->w = (double*)malloc(M * sizeof(double));
  rr->x = (double*)malloc(3 * M * sizeof(double));
  double T = 1.0, gap = INFINITY;
  int64_t k = 0;
  for (; k < m; ++k) {
    int32_t v = hv.h[k].voxel;
    double lo[3], hi[3], e;
    voxel_box(s, v, lo, hi, &e);
    double a = dmax(hv.h[k].t_in, tn), b = dmin(hv.h[k].t_out, tf);
    double tm = 0.5 * (a + b), dl = b - a;
    double x[3];
    for (int ax = 0; ax < 3; ++ax) {
      double X = o[ax] + tm * d[ax];
      double ctr = 0.5 * (lo[ax] + hi[ax]);
      x[ax] = (X - ctr) / (0.5 * e);
    }
    const double* rec = s->params + (size_t)REC * v;
    double sig, c[3], io;
    orc_field(rec, s->mode, x, d, &sig, c, &io);
    if (!opt->want_intensity) io = 0.0;
    double lin = 0;
    for (int q = 0; q < 3; ++q) lin += rec[q] * x[q];
    lin += rec[3];
    double alpha = 1.0 - exp(-sig * dl); /* Eq. 4 */
    double w = T * alpha;                /* Eq. 3 weight T_i alpha_i */
    rr->vox[k] = v;
    rr->tm[k] = tm;
    rr->dl[k] = dl;
    rr->sig[k] = sig;
    rr->lin[k] = lin;
    for (int q = 0; q < 3; ++q) {
      rr->c[3 * k + q] = c[q];
      rr->x[3 * k + q] = x[q];
    }
    rr->io[k] = io;
    /* raydrop field (paper silent on its form): a per-voxel logit, record
     * slot 31, composited like intensity */
    rr->dr[k] = opt->want_raydrop ? sigmoid(rec[31]) : 0.0;
    rr->alpha[k] = alpha;
    rr->T[k] = T;
    rr->w[k] = w;
    T = T * (1.0 - alpha); /* T_{i+1} = prod_{j<=i} (1 - alpha_j) */
    if (opt->t_min > 0) {
      double g = fabs(log(T) - log(opt->t_min));
      if (g < gap) gap = g;
      if (T < opt->t_min) {
        ++k;
        break;
      }
    }
  }
  rr->n = k;
  rr->t_end = T;
  rr->gap = gap;
  free(hv.h);
}

int orc_render(const orc_scene* s, const orc_sensor* sen, const orc_opts* opt,
               const int64_t* idx, int64_t m, const orc_outputs* out) {
  if (sen->width <= 0 || sen->height <= 0) return 1;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < m; ++i) {
    int64_t r = idx ? idx[i] : i;
    double o[3], d[3], tn, tf, tau;
    uint8_t valid;
    one_ray(sen, r, o, d, &tn, &tf, &tau, &valid);
    double C[3] = {0, 0, 0}, D = 0, O = 0, I = 0, P = 0, Tend = 1.0, gap = INFINITY;
    int64_t nv = 0;
    ray_record rr;
    memset(&rr, 0, sizeof(rr));
    if (valid) {
      composite_ray(s, opt, o, d, tn, tf, &rr);
      if (out->max_alpha) {
#pragma omp critical(salf_max_alpha)
        for (int64_t k = 0; k < rr.n; ++k)
          if (rr.alpha[k] > out->max_alpha[rr.vox[k]]) out->max_alpha[rr.vox[k]] = rr.alpha[k];
      }
      for (int64_t k = 0; k < rr.n; ++k) {
        for (int q = 0; q < 3; ++q) C[q] += rr.w[k] * rr.c[3 * k + q];
        D += rr.w[k] * rr.tm[k];
        O += rr.w[k];
        I += rr.w[k] * rr.io[k];
        P += rr.w[k] * rr.dr[k];
      }
      Tend = rr.t_end;
      gap = rr.gap;
      nv = rr.n;
      for (int q = 0; q < 3; ++q) C[q] += Tend * opt->background[q];
    }
    if (out->rgb)
      for (int q = 0; q < 3; ++q) out->rgb[3 * i + q] = valid ? C[q] : 0.0;
    if (out->depth) out->depth[i] = D;
    if (out->opacity) out->opacity[i] = O;
    if (out->intensity) out->intensity[i] = I;
    if (out->raydrop) out->raydrop[i] = valid ? P + Tend : 0.0;
    if (out->t_end) out->t_end[i] = valid ? Tend : 1.0;
    if (out->term_gap) out->term_gap[i] = gap;
    if (out->n_visits) out->n_visits[i] = (int32_t)nv;
    if (out->valid) out->valid[i] = valid;
    if (out->visits) {
      for (int64_t k = 0; k < out->visits_cap; ++k)
        out->visits[i * out->visits_cap + k] = k < nv ? rr.vox[k] : -1;
    }
    if (valid) rr_free(&rr);
  }
  return 0;
}

#define ADD(p, v)            \
  do {                       \
    double _v = (v);         \
    _Pragma("omp atomic") *(p) += _v; \
  } while (0)

/* Adjoint of Eq. 1-6 for L = sum_r g_r . outputs_r.  With q_k = (c_k, t_mid,k,
 * 1, iota_k, rho_k) (rho_k = sigmoid of the raydrop logit) and w_k = T_k alpha_k,
 * tau_k = sigma_k delta_k:
 *   dL/dtau_k = T_{k+1} (g . q_k) - sum_{j>k} w_j (g . q_j)
 *               - T_end (g_rgb . bg + g_raydrop)
 * (the raydrop output adds T_end like a background of 1), then the chain rule
 * through Eq. 1/6 (density), Eq. 2 (colour) and the sigmoid fields. */
int orc_backward(const orc_scene* s, const orc_sensor* sen, const orc_opts* opt,
                 const int64_t* idx, int64_t m, const double* g_rgb, const double* g_depth,
                 const double* g_opacity, const double* g_intensity, const double* g_raydrop,
                 double* grad) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < m; ++i) {
    int64_t r = idx ? idx[i] : i;
    double o[3], d[3], tn, tf, tau;
    uint8_t valid;
    one_ray(sen, r, o, d, &tn, &tf, &tau, &valid);
    if (!valid) continue;
    double gc[3] = {0, 0, 0}, gd = 0, go = 0, gi = 0;
    if (g_rgb)
      for (int q = 0; q < 3; ++q) gc[q] = g_rgb[3 * i + q];
    if (g_depth) gd = g_depth[i];
    if (g_opacity) go = g_opacity[i];
    if (g_intensity && opt->want_intensity) gi = g_intensity[i];
    double gp = (g_raydrop && opt->want_raydrop) ? g_raydrop[i] : 0.0;
    ray_record rr;
    memset(&rr, 0, sizeof(rr));
    composite_ray(s, opt, o, d, tn, tf, &rr);
    int64_t n = rr.n;
    double* gq = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
    double* suf = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
    for (int64_t k = 0; k < n; ++k)
      gq[k] = gc[0] * rr.c[3 * k] + gc[1] * rr.c[3 * k + 1] + gc[2] * rr.c[3 * k + 2] +
              gd * rr.tm[k] + go + gi * rr.io[k] + gp * rr.dr[k];
    double acc = 0;
    for (int64_t k = n - 1; k >= 0; --k) {
      suf[k] = acc; /* sum_{j>k} w_j gq_j */
      acc += rr.w[k] * gq[k];
    }
    double gbg = gc[0] * opt->background[0] + gc[1] * opt->background[1] +
                 gc[2] * opt->background[2] + gp;
    double gam[4];
    orc_sh_basis(d, gam);
    for (int64_t k = 0; k < n; ++k) {
      int32_t v = rr.vox[k];
      const double* rec = s->params + (size_t)REC * v;
      double* gr = grad + (size_t)REC * v;
      double Tn = rr.T[k] * (1.0 - rr.alpha[k]);
      double dtau = Tn * gq[k] - suf[k] - rr.t_end * gbg;
      double dsig = dtau * rr.dl[k];
      const double* x = rr.x + 3 * k;
      double xh[4] = {x[0], x[1], x[2], 1.0};
      if (s->mode == 0) {
        for (int a = 0; a < 4; ++a) ADD(&gr[a], dsig * rr.sig[k] * xh[a]);
      } else {
        double a = rec[25], b = rec[26], sp = rr.lin[k];
        double ex = exp(-fabs(sp) / b);
        double ds = dsig * (a / (2.0 * b)) * ex;
        for (int q = 0; q < 4; ++q) ADD(&gr[q], ds * xh[q]);
        ADD(&gr[25], dsig * rr.sig[k] / a);
        ADD(&gr[26], dsig * (-a * sp * ex / (2.0 * b * b)));
      }
      for (int q = 0; q < 3; ++q) {
        double cq = rr.c[3 * k + q];
        double dz = rr.w[k] * gc[q] * cq * (1.0 - cq);
        for (int a = 0; a < 3; ++a) ADD(&gr[4 + 3 * q + a], dz * x[a]);
        for (int b = 0; b < 4; ++b) ADD(&gr[13 + 4 * q + b], dz * gam[b]);
      }
      if (opt->want_intensity) {
        double io = rr.io[k];
        double dz = rr.w[k] * gi * io * (1.0 - io);
        for (int a = 0; a < 4; ++a) ADD(&gr[27 + a], dz * xh[a]);
      }
      if (opt->want_raydrop) {
        double dr = rr.dr[k];
        ADD(&gr[31], rr.w[k] * gp * dr * (1.0 - dr));
      }
    }
    free(gq);
    free(suf);
    rr_free(&rr);
  }
  return 0;
}

/* Rounding bound for an FP32 evaluation of orc_backward's sum (not part of
 * the method: a tolerance for comparing an FP32 implementation with this FP64
 * adjoint).  bound (n*32, input order) += per record scalar, over the same
 * rays and hits as orc_backward, the magnitude of each hit's contribution
 * with
 *   - every factor in absolute value and every cancelling sum (the suffix
 *     sums of dL/dtau, g . q) replaced by the sum of its terms' absolute
 *     values;
 *   - the conditioning of the hit's geometry folded in: a position carried
 *     in FP32 relative to the sensor is off by about u t (u the unit
 *     roundoff, t the distance), i.e. by u kappa in local coordinates with
 *     kappa = 1 + 2 t / edge, which moves every field of the voxel by up to
 *     u kappa times its slopes' L1 norm; so a relative factor
 *     Phi = kappa (1 + |slopes|_1) + Lambda, where Lambda = sum over the
 *     ray's hits of (sigma t + tau kappa |W_sigma slopes|_1) bounds the
 *     relative error of any transmittance of the ray in units of u;
 *   - terms proportional to the segment length delta carry its absolute
 *     error u t: a weight w = T (1 - e^{-sigma delta}) becomes
 *     w Phi + T sigma t, and dL/dsigma = dL/dtau delta becomes
 *     |dL/dtau| (delta Phi + t);
 *   - a local-coordinate factor x_a becomes |x_a| + 1 (its absolute error
 *     u kappa is not relative to x_a, which may be exactly 0).
 * An FP32 evaluation in the same order of operations is then expected within
 * a small multiple of u times this bound (plus its own relative rounding). */
int orc_backward_bound(const orc_scene* s, const orc_sensor* sen, const orc_opts* opt,
                       const int64_t* idx, int64_t m, const double* g_rgb, const double* g_depth,
                       const double* g_opacity, const double* g_intensity,
                       const double* g_raydrop, double* bound) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < m; ++i) {
    int64_t r = idx ? idx[i] : i;
    double o[3], d[3], tn, tf, tau;
    uint8_t valid;
    one_ray(sen, r, o, d, &tn, &tf, &tau, &valid);
    if (!valid) continue;
    double gc[3] = {0, 0, 0}, gd = 0, go = 0, gi = 0;
    if (g_rgb)
      for (int q = 0; q < 3; ++q) gc[q] = g_rgb[3 * i + q];
    if (g_depth) gd = g_depth[i];
    if (g_opacity) go = g_opacity[i];
    if (g_intensity && opt->want_intensity) gi = g_intensity[i];
    double gp = (g_raydrop && opt->want_raydrop) ? g_raydrop[i] : 0.0;
    ray_record rr;
    memset(&rr, 0, sizeof(rr));
    composite_ray(s, opt, o, d, tn, tf, &rr);
    int64_t n = rr.n;
    size_t N = (size_t)(n ? n : 1);
    double* gqa = (double*)malloc(N * sizeof(double));
    double* kap = (double*)malloc(N * sizeof(double));
    double* phi = (double*)malloc(N * sizeof(double));
    double* tk = (double*)malloc(N * sizeof(double));
    double* wm = (double*)malloc(N * sizeof(double));
    double lam = 0.0;
    for (int64_t k = 0; k < n; ++k) {
      int32_t v = rr.vox[k];
      const double* rec = s->params + (size_t)REC * v;
      double lo[3], hi[3], e;
      voxel_box(s, v, lo, hi, &e);
      tk[k] = rr.tm[k] + 0.5 * rr.dl[k];
      kap[k] = 1.0 + 2.0 * tk[k] / e;
      double ws = fabs(rec[0]) + fabs(rec[1]) + fabs(rec[2]);
      lam += rr.sig[k] * tk[k] + rr.sig[k] * rr.dl[k] * kap[k] * ws;
      gqa[k] = fabs(gc[0] * rr.c[3 * k]) + fabs(gc[1] * rr.c[3 * k + 1]) +
               fabs(gc[2] * rr.c[3 * k + 2]) + fabs(gd * rr.tm[k]) + fabs(go) +
               fabs(gi * rr.io[k]) + fabs(gp * rr.dr[k]);
    }
    double sabs = 0.0;
    for (int64_t k = 0; k < n; ++k) {
      int32_t v = rr.vox[k];
      const double* rec = s->params + (size_t)REC * v;
      double sl = 0.0;
      for (int q = 0; q < 3; ++q) sl += fabs(rec[q]);
      for (int q = 4; q < 13; ++q) sl += fabs(rec[q]);
      for (int q = 27; q < 30; ++q) sl += fabs(rec[q]);
      phi[k] = kap[k] * (1.0 + sl) + lam;
      wm[k] = rr.w[k] * phi[k] + rr.T[k] * rr.sig[k] * tk[k];
      sabs += wm[k] * gqa[k];
    }
    double gbga = fabs(gc[0] * opt->background[0]) + fabs(gc[1] * opt->background[1]) +
                  fabs(gc[2] * opt->background[2]) + fabs(gp);
    double gam[4];
    orc_sh_basis(d, gam);
    for (int64_t k = 0; k < n; ++k) {
      int32_t v = rr.vox[k];
      const double* rec = s->params + (size_t)REC * v;
      double* bd = bound + (size_t)REC * v;
      double dtm = rr.T[k] * gqa[k] + sabs + rr.t_end * gbga;
      double dsm = dtm * (rr.dl[k] * phi[k] + tk[k]);
      const double* x = rr.x + 3 * k;
      double xa[4] = {fabs(x[0]) + 1.0, fabs(x[1]) + 1.0, fabs(x[2]) + 1.0, 2.0};
      if (s->mode == 0) {
        for (int a = 0; a < 4; ++a) ADD(&bd[a], dsm * rr.sig[k] * xa[a]);
      } else {
        double a = rec[25], b = rec[26], sp = rr.lin[k];
        double ex = exp(-fabs(sp) / b);
        double ds = dsm * (a / (2.0 * b)) * ex * (1.0 + kap[k] / b);
        for (int q = 0; q < 4; ++q) ADD(&bd[q], ds * xa[q]);
        ADD(&bd[25], dsm * rr.sig[k] / a);
        ADD(&bd[26], dsm * a * (fabs(sp) + 1.0) * ex / (2.0 * b * b) * (1.0 + kap[k] / b));
      }
      for (int q = 0; q < 3; ++q) {
        double cq = rr.c[3 * k + q];
        double dz = wm[k] * fabs(gc[q]) * cq * (1.0 - cq);
        for (int a = 0; a < 3; ++a) ADD(&bd[4 + 3 * q + a], dz * xa[a]);
        for (int b = 0; b < 4; ++b) ADD(&bd[13 + 4 * q + b], dz * fabs(gam[b]));
      }
      if (opt->want_intensity) {
        double io = rr.io[k];
        double dz = wm[k] * fabs(gi) * io * (1.0 - io);
        for (int a = 0; a < 4; ++a) ADD(&bd[27 + a], dz * xa[a]);
      }
      if (opt->want_raydrop) {
        double dr = rr.dr[k];
        ADD(&bd[31], wm[k] * fabs(gp) * dr * (1.0 - dr));
      }
    }
    free(gqa);
    free(kap);
    free(phi);
    free(tk);
    free(wm);
    rr_free(&rr);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Dynamic actors (Sec. IV-A)                                                */
/* ------------------------------------------------------------------------ */
/* Each actor is a voxel set in its own canonical frame, placed in the world
 * by its pose at the ray's time (interpolated like the sensor's pose between
 * the sensor's t0 and t1).  A ray is moved into every actor's frame (a rigid
 * map: distances along the ray are unchanged), each frame's voxels are
 * traced, and all hits are composited by Eq. 3-4 in order of entry, each
 * with its field evaluated in its own frame (local coordinates and view
 * direction of the actor's canonical frame). */

typedef struct {
  int32_t frame, voxel;
  double t_in, t_out, key;
} mhit;

static int mhit_cmp(const void* pa, const void* pb) {
  const mhit* a = (const mhit*)pa;
  const mhit* b = (const mhit*)pb;
  if (a->key != b->key) return a->key < b->key ? -1 : 1;
  if (a->frame != b->frame) return a->frame < b->frame ? -1 : 1;
  return a->voxel < b->voxel ? -1 : (a->voxel > b->voxel);
}

int orc_render_actors(const orc_scene* s, const orc_actor* actors, int32_t n_actors,
                      const orc_sensor* sen, const orc_opts* opt, const int64_t* idx, int64_t m,
                      const orc_outputs* out) {
  if (sen->width <= 0 || sen->height <= 0 || n_actors < 0) return 1;
  const int nf = 1 + n_actors;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < m; ++i) {
    int64_t r = idx ? idx[i] : i;
    double o[3], d[3], tn, tf, tau;
    uint8_t valid;
    one_ray(sen, r, o, d, &tn, &tf, &tau, &valid);
    double C[3] = {0, 0, 0}, D = 0, O = 0, I = 0, T = 1.0, gap = INFINITY;
    int64_t nv = 0;
    const double sfr = time_fraction(sen, tau);
    /* the ray in every frame: frame 0 = world (static scene), frame 1 + k = actor k */
    double* fo = (double*)malloc((size_t)nf * 3 * sizeof(double));
    double* fd = (double*)malloc((size_t)nf * 3 * sizeof(double));
    for (int a = 0; a < 3; ++a) {
      fo[a] = o[a];
      fd[a] = d[a];
    }
    for (int k = 0; k < n_actors; ++k) {
      double R[9], t[3], rel[3];
      interp_pose(actors[k].pose0, actors[k].pose1, sfr, R, t);
      for (int a = 0; a < 3; ++a) rel[a] = o[a] - t[a];
      for (int c = 0; c < 3; ++c) { /* R maps canonical -> world; its transpose maps back */
        fo[3 * (1 + k) + c] = R[c] * rel[0] + R[3 + c] * rel[1] + R[6 + c] * rel[2];
        fd[3 * (1 + k) + c] = R[c] * d[0] + R[3 + c] * d[1] + R[6 + c] * d[2];
      }
    }
    mhit* mh = NULL;
    int64_t nh = 0, ch = 0;
    if (valid) {
      for (int f = 0; f < nf; ++f) {
        const orc_scene* sc = f == 0 ? s : actors[f - 1].scene;
        hitvec hv = {0, 0, 0};
        trace_vec(sc, fo + 3 * f, fd + 3 * f, tn, tf, opt->brute_force, &hv);
        for (int64_t q = 0; q < hv.n; ++q) {
          if (nh == ch) {
            ch = ch ? 2 * ch : 64;
            mh = (mhit*)realloc(mh, (size_t)ch * sizeof(mhit));
          }
          mh[nh].frame = f;
          mh[nh].voxel = hv.h[q].voxel;
          mh[nh].t_in = hv.h[q].t_in;
          mh[nh].t_out = hv.h[q].t_out;
          mh[nh].key = dmax(hv.h[q].t_in, tn);
          ++nh;
        }
        free(hv.h);
      }
      if (nh > 1) qsort(mh, (size_t)nh, sizeof(mhit), mhit_cmp);
      for (int64_t k = 0; k < nh; ++k) {
        const int f = mh[k].frame;
        const orc_scene* sc = f == 0 ? s : actors[f - 1].scene;
        const double* of = fo + 3 * f;
        const double* df = fd + 3 * f;
        double lo[3], hi[3], e;
        voxel_box(sc, mh[k].voxel, lo, hi, &e);
        double a = dmax(mh[k].t_in, tn), b = dmin(mh[k].t_out, tf);
        double tm = 0.5 * (a + b), dl = b - a;
        double x[3];
        for (int ax = 0; ax < 3; ++ax)
          x[ax] = (of[ax] + tm * df[ax] - 0.5 * (lo[ax] + hi[ax])) / (0.5 * e);
        double sig, c[3], io;
        orc_field(sc->params + (size_t)REC * mh[k].voxel, sc->mode, x, df, &sig, c, &io);
        if (!opt->want_intensity) io = 0.0;
        double alpha = 1.0 - exp(-sig * dl); /* Eq. 4 */
        double w = T * alpha;                /* Eq. 3 */
        for (int q = 0; q < 3; ++q) C[q] += w * c[q];
        D += w * tm;
        O += w;
        I += w * io;
        if (out->visits && nv < out->visits_cap)
          out->visits[i * out->visits_cap + nv] =
              f == 0 ? mh[k].voxel : actors[f - 1].id_base + mh[k].voxel;
        ++nv;
        T = T * (1.0 - alpha);
        if (opt->t_min > 0) {
          double g = fabs(log(T) - log(opt->t_min));
          if (g < gap) gap = g;
          if (T < opt->t_min) break;
        }
      }
      for (int q = 0; q < 3; ++q) C[q] += T * opt->background[q];
    }
    if (out->rgb)
      for (int q = 0; q < 3; ++q) out->rgb[3 * i + q] = valid ? C[q] : 0.0;
    if (out->depth) out->depth[i] = D;
    if (out->opacity) out->opacity[i] = O;
    if (out->intensity) out->intensity[i] = I;
    if (out->t_end) out->t_end[i] = valid ? T : 1.0;
    if (out->term_gap) out->term_gap[i] = gap;
    if (out->n_visits) out->n_visits[i] = (int32_t)nv;
    if (out->valid) out->valid[i] = valid;
    if (out->visits)
      for (int64_t k = nv; k < out->visits_cap; ++k) out->visits[i * out->visits_cap + k] = -1;
    free(mh);
    free(fo);
    free(fd);
  }
  return 0;
}

/* Adjoint of the actor render (Sec. IV-A: actors are fitted with the scene).
 * The composited hits of one ray, in orc_render_actors' order, with every
 * per-hit quantity the adjoint needs; the field of a hit is evaluated in its
 * own frame (local coordinates and SH direction of that frame). */
typedef struct {
  int64_t n;
  int32_t *frame, *vox;
  double *tm, *dl, *sig, *lin, *c, *io, *alpha, *T, *w, *x, *dir, *edge;
  double t_end;
} actor_record;

static void ar_free(actor_record* a) {
  free(a->frame);
  free(a->vox);
  free(a->tm);
  free(a->dl);
  free(a->sig);
  free(a->lin);
  free(a->c);
  free(a->io);
  free(a->alpha);
  free(a->T);
  free(a->w);
  free(a->x);
  free(a->dir);
  free(a->edge);
}

static void actor_ray(const orc_scene* s, const orc_actor* actors, int32_t n_actors,
                      const orc_opts* opt, const double o[3], const double d[3], double tn,
                      double tf, double sfr, actor_record* ar) {
  const int nf = 1 + n_actors;
  double* fo = (double*)malloc((size_t)nf * 3 * sizeof(double));
  double* fd = (double*)malloc((size_t)nf * 3 * sizeof(double));
  for (int a = 0; a < 3; ++a) {
    fo[a] = o[a];
    fd[a] = d[a];
  }
  for (int k = 0; k < n_actors; ++k) {
    double R[9], t[3], rel[3];
    interp_pose(actors[k].pose0, actors[k].pose1, sfr, R, t);
    for (int a = 0; a < 3; ++a) rel[a] = o[a] - t[a];
    for (int c = 0; c < 3; ++c) {
      fo[3 * (1 + k) + c] = R[c] * rel[0] + R[3 + c] * rel[1] + R[6 + c] * rel[2];
      fd[3 * (1 + k) + c] = R[c] * d[0] + R[3 + c] * d[1] + R[6 + c] * d[2];
    }
  }
  mhit* mh = NULL;
  int64_t nh = 0, ch = 0;
  for (int f = 0; f < nf; ++f) {
    const orc_scene* sc = f == 0 ? s : actors[f - 1].scene;
    hitvec hv = {0, 0, 0};
    trace_vec(sc, fo + 3 * f, fd + 3 * f, tn, tf, opt->brute_force, &hv);
    for (int64_t q = 0; q < hv.n; ++q) {
      if (nh == ch) {
        ch = ch ? 2 * ch : 64;
        mh = (mhit*)realloc(mh, (size_t)ch * sizeof(mhit));
      }
      mh[nh].frame = f;
      mh[nh].voxel = hv.h[q].voxel;
      mh[nh].t_in = hv.h[q].t_in;
      mh[nh].t_out = hv.h[q].t_out;
      mh[nh].key = dmax(hv.h[q].t_in, tn);
      ++nh;
    }
    free(hv.h);
  }
  if (nh > 1) qsort(mh, (size_t)nh, sizeof(mhit), mhit_cmp);
  size_t M = (size_t)(nh ? nh : 1);
  ar->frame = (int32_t*)malloc(M * sizeof(int32_t));
  ar->vox = (int32_t*)malloc(M * sizeof(int32_t));
  ar->tm = (double*)malloc(M * sizeof(double));
  ar->dl = (double*)malloc(M * sizeof(double));
  ar->sig = (double*)malloc(M * sizeof(double));
  ar->lin = (double*)malloc(M * sizeof(double));
  ar->c = (double*)malloc(3 * M * sizeof(double));
  ar->io = (double*)malloc(M * sizeof(double));
  ar->alpha = (double*)malloc(M * sizeof(double));
  ar->T = (double*)malloc(M * sizeof(double));
  ar->w = (double*)malloc(M * sizeof(double));
  ar->x = (double*)malloc(3 * M * sizeof(double));
  ar->dir = (double*)malloc(3 * M * sizeof(double));
  ar->edge = (double*)malloc(M * sizeof(double));
  double T = 1.0;
  int64_t k = 0;
  for (; k < nh; ++k) {
    const int f = mh[k].frame;
    const orc_scene* sc = f == 0 ? s : actors[f - 1].scene;
    const double* of = fo + 3 * f;
    const double* df = fd + 3 * f;
    double lo[3], hi[3], e;
    voxel_box(sc, mh[k].voxel, lo, hi, &e);
    double a = dmax(mh[k].t_in, tn), b = dmin(mh[k].t_out, tf);
    double tm = 0.5 * (a + b), dl = b - a;
    double x[3];
    for (int ax = 0; ax < 3; ++ax)
      x[ax] = (of[ax] + tm * df[ax] - 0.5 * (lo[ax] + hi[ax])) / (0.5 * e);
    const double* rec = sc->params + (size_t)REC * mh[k].voxel;
    double sig, c[3], io;
    orc_field(rec, sc->mode, x, df, &sig, c, &io);
    if (!opt->want_intensity) io = 0.0;
    double lin = rec[3];
    for (int q = 0; q < 3; ++q) lin += rec[q] * x[q];
    double alpha = 1.0 - exp(-sig * dl); /* Eq. 4 */
    ar->frame[k] = f;
    ar->vox[k] = mh[k].voxel;
    ar->tm[k] = tm;
    ar->dl[k] = dl;
    ar->sig[k] = sig;
    ar->lin[k] = lin;
    ar->io[k] = io;
    ar->alpha[k] = alpha;
    ar->T[k] = T;
    ar->w[k] = T * alpha; /* Eq. 3 */
    ar->edge[k] = e;
    for (int q = 0; q < 3; ++q) {
      ar->c[3 * k + q] = c[q];
      ar->x[3 * k + q] = x[q];
      ar->dir[3 * k + q] = df[q];
    }
    T = T * (1.0 - alpha);
    if (opt->t_min > 0 && T < opt->t_min) {
      ++k;
      break;
    }
  }
  ar->n = k;
  ar->t_end = T;
  free(mh);
  free(fo);
  free(fd);
}

/* grad (static, n*32) and actor_grads[k] (actor k's n_k*32, NULL = not
 * wanted) += d/d(record scalars) of sum_r g_r . outputs_r of the actor render,
 * by the same adjoint as orc_backward: with q_k = (c_k, t_mid,k, 1, iota_k),
 *   dL/dtau_k = T_{k+1} (g . q_k) - sum_{j>k} w_j (g . q_j) - T_end (g_rgb . bg),
 * then the chain rule through the hit's field in its own frame. */
int orc_backward_actors(const orc_scene* s, const orc_actor* actors, int32_t n_actors,
                        const orc_sensor* sen, const orc_opts* opt, const int64_t* idx, int64_t m,
                        const double* g_rgb, const double* g_depth, const double* g_opacity,
                        const double* g_intensity, double* grad, double* const* actor_grads) {
  if (sen->width <= 0 || sen->height <= 0 || n_actors < 0) return 1;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < m; ++i) {
    int64_t r = idx ? idx[i] : i;
    double o[3], d[3], tn, tf, tau;
    uint8_t valid;
    one_ray(sen, r, o, d, &tn, &tf, &tau, &valid);
    if (!valid) continue;
    double gc[3] = {0, 0, 0}, gd = 0, go = 0, gi = 0;
    if (g_rgb)
      for (int q = 0; q < 3; ++q) gc[q] = g_rgb[3 * i + q];
    if (g_depth) gd = g_depth[i];
    if (g_opacity) go = g_opacity[i];
    if (g_intensity && opt->want_intensity) gi = g_intensity[i];
    actor_record ar;
    actor_ray(s, actors, n_actors, opt, o, d, tn, tf, time_fraction(sen, tau), &ar);
    int64_t n = ar.n;
    double* gq = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
    double* suf = (double*)malloc((size_t)(n ? n : 1) * sizeof(double));
    for (int64_t k = 0; k < n; ++k)
      gq[k] = gc[0] * ar.c[3 * k] + gc[1] * ar.c[3 * k + 1] + gc[2] * ar.c[3 * k + 2] +
              gd * ar.tm[k] + go + gi * ar.io[k];
    double acc = 0;
    for (int64_t k = n - 1; k >= 0; --k) {
      suf[k] = acc; /* sum_{j>k} w_j gq_j */
      acc += ar.w[k] * gq[k];
    }
    double gbg = gc[0] * opt->background[0] + gc[1] * opt->background[1] +
                 gc[2] * opt->background[2];
    for (int64_t k = 0; k < n; ++k) {
      const int f = ar.frame[k];
      const orc_scene* sc = f == 0 ? s : actors[f - 1].scene;
      double* gbase = f == 0 ? grad : actor_grads[f - 1];
      if (!gbase) continue;
      const double* rec = sc->params + (size_t)REC * ar.vox[k];
      double* gr = gbase + (size_t)REC * ar.vox[k];
      double gam[4];
      orc_sh_basis(ar.dir + 3 * k, gam);
      double Tn = ar.T[k] * (1.0 - ar.alpha[k]);
      double dtau = Tn * gq[k] - suf[k] - ar.t_end * gbg;
      double dsig = dtau * ar.dl[k];
      const double* x = ar.x + 3 * k;
      double xh[4] = {x[0], x[1], x[2], 1.0};
      if (sc->mode == 0) {
        for (int a = 0; a < 4; ++a) ADD(&gr[a], dsig * ar.sig[k] * xh[a]);
      } else {
        double a = rec[25], b = rec[26], sp = ar.lin[k];
        double ex = exp(-fabs(sp) / b);
        double ds = dsig * (a / (2.0 * b)) * ex;
        for (int q = 0; q < 4; ++q) ADD(&gr[q], ds * xh[q]);
        ADD(&gr[25], dsig * ar.sig[k] / a);
        ADD(&gr[26], dsig * (-a * sp * ex / (2.0 * b * b)));
      }
      for (int q = 0; q < 3; ++q) {
        double cq = ar.c[3 * k + q];
        double dz = ar.w[k] * gc[q] * cq * (1.0 - cq);
        for (int a = 0; a < 3; ++a) ADD(&gr[4 + 3 * q + a], dz * x[a]);
        for (int b = 0; b < 4; ++b) ADD(&gr[13 + 4 * q + b], dz * gam[b]);
      }
      if (opt->want_intensity) {
        double io = ar.io[k];
        double dz = ar.w[k] * gi * io * (1.0 - io);
        for (int a = 0; a < 4; ++a) ADD(&gr[27 + a], dz * xh[a]);
      }
    }
    free(gq);
    free(suf);
    ar_free(&ar);
  }
  return 0;
}

/* The rounding bound of orc_backward_bound for orc_backward_actors' sums
 * (same construction; distances and edges are those of each hit's frame). */
int orc_backward_actors_bound(const orc_scene* s, const orc_actor* actors, int32_t n_actors,
                              const orc_sensor* sen, const orc_opts* opt, const int64_t* idx,
                              int64_t m, const double* g_rgb, const double* g_depth,
                              const double* g_opacity, const double* g_intensity, double* bound,
                              double* const* actor_bounds) {
  if (sen->width <= 0 || sen->height <= 0 || n_actors < 0) return 1;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < m; ++i) {
    int64_t r = idx ? idx[i] : i;
    double o[3], d[3], tn, tf, tau;
    uint8_t valid;
    one_ray(sen, r, o, d, &tn, &tf, &tau, &valid);
    if (!valid) continue;
    double gc[3] = {0, 0, 0}, gd = 0, go = 0, gi = 0;
    if (g_rgb)
      for (int q = 0; q < 3; ++q) gc[q] = g_rgb[3 * i + q];
    if (g_depth) gd = g_depth[i];
    if (g_opacity) go = g_opacity[i];
    if (g_intensity && opt->want_intensity) gi = g_intensity[i];
    actor_record ar;
    actor_ray(s, actors, n_actors, opt, o, d, tn, tf, time_fraction(sen, tau), &ar);
    int64_t n = ar.n;
    size_t N = (size_t)(n ? n : 1);
    double* gqa = (double*)malloc(N * sizeof(double));
    double* kap = (double*)malloc(N * sizeof(double));
    double* phi = (double*)malloc(N * sizeof(double));
    double* tk = (double*)malloc(N * sizeof(double));
    double* wm = (double*)malloc(N * sizeof(double));
    double lam = 0.0;
    for (int64_t k = 0; k < n; ++k) {
      const int f = ar.frame[k];
      const orc_scene* sc = f == 0 ? s : actors[f - 1].scene;
      const double* rec = sc->params + (size_t)REC * ar.vox[k];
      tk[k] = ar.tm[k] + 0.5 * ar.dl[k];
      kap[k] = 1.0 + 2.0 * tk[k] / ar.edge[k];
      double ws = fabs(rec[0]) + fabs(rec[1]) + fabs(rec[2]);
      lam += ar.sig[k] * tk[k] + ar.sig[k] * ar.dl[k] * kap[k] * ws;
      gqa[k] = fabs(gc[0] * ar.c[3 * k]) + fabs(gc[1] * ar.c[3 * k + 1]) +
               fabs(gc[2] * ar.c[3 * k + 2]) + fabs(gd * ar.tm[k]) + fabs(go) +
               fabs(gi * ar.io[k]);
    }
    double sabs = 0.0;
    for (int64_t k = 0; k < n; ++k) {
      const int f = ar.frame[k];
      const orc_scene* sc = f == 0 ? s : actors[f - 1].scene;
      const double* rec = sc->params + (size_t)REC * ar.vox[k];
      double sl = 0.0;
      for (int q = 0; q < 3; ++q) sl += fabs(rec[q]);
      for (int q = 4; q < 13; ++q) sl += fabs(rec[q]);
      for (int q = 27; q < 30; ++q) sl += fabs(rec[q]);
      phi[k] = kap[k] * (1.0 + sl) + lam;
      wm[k] = ar.w[k] * phi[k] + ar.T[k] * ar.sig[k] * tk[k];
      sabs += wm[k] * gqa[k];
    }
    double gbga = fabs(gc[0] * opt->background[0]) + fabs(gc[1] * opt->background[1]) +
                  fabs(gc[2] * opt->background[2]);
    for (int64_t k = 0; k < n; ++k) {
      const int f = ar.frame[k];
      const orc_scene* sc = f == 0 ? s : actors[f - 1].scene;
      double* bbase = f == 0 ? bound : actor_bounds[f - 1];
      if (!bbase) continue;
      const double* rec = sc->params + (size_t)REC * ar.vox[k];
      double* bd = bbase + (size_t)REC * ar.vox[k];
      double gam[4];
      orc_sh_basis(ar.dir + 3 * k, gam);
      double dtm = ar.T[k] * gqa[k] + sabs + ar.t_end * gbga;
      double dsm = dtm * (ar.dl[k] * phi[k] + tk[k]);
      const double* x = ar.x + 3 * k;
      double xa[4] = {fabs(x[0]) + 1.0, fabs(x[1]) + 1.0, fabs(x[2]) + 1.0, 2.0};
      if (sc->mode == 0) {
        for (int a = 0; a < 4; ++a) ADD(&bd[a], dsm * ar.sig[k] * xa[a]);
      } else {
        double a = rec[25], b = rec[26], sp = ar.lin[k];
        double ex = exp(-fabs(sp) / b);
        double ds = dsm * (a / (2.0 * b)) * ex * (1.0 + kap[k] / b);
        for (int q = 0; q < 4; ++q) ADD(&bd[q], ds * xa[q]);
        ADD(&bd[25], dsm * ar.sig[k] / a);
        ADD(&bd[26], dsm * a * (fabs(sp) + 1.0) * ex / (2.0 * b * b) * (1.0 + kap[k] / b));
      }
      for (int q = 0; q < 3; ++q) {
        double cq = ar.c[3 * k + q];
        double dz = wm[k] * fabs(gc[q]) * cq * (1.0 - cq);
        for (int a = 0; a < 3; ++a) ADD(&bd[4 + 3 * q + a], dz * xa[a]);
        for (int b = 0; b < 4; ++b) ADD(&bd[13 + 4 * q + b], dz * fabs(gam[b]));
      }
      if (opt->want_intensity) {
        double io = ar.io[k];
        double dz = wm[k] * fabs(gi) * io * (1.0 - io);
        for (int a = 0; a < 4; ++a) ADD(&bd[27 + a], dz * xa[a]);
      }
    }
    free(gqa);
    free(kap);
    free(phi);
    free(tk);
    free(wm);
    ar_free(&ar);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Densification (Sec. III-C)                                                */
/* ------------------------------------------------------------------------ */

void orc_subdivide_record(const double* rec, int32_t child, double* out) {
  const double C0 = 0.28209479177387814; /* 1 / (2 sqrt(pi)) */
  double o[3];
  for (int a = 0; a < 3; ++a) o[a] = ((child >> a) & 1) ? 1.0 : -1.0;
  for (int k = 0; k < REC; ++k) out[k] = rec[k];
  /* geometry W . [x, 1] */
  out[3] = rec[3] + 0.5 * (rec[0] * o[0] + rec[1] * o[1] + rec[2] * o[2]);
  for (int a = 0; a < 3; ++a) out[a] = 0.5 * rec[a];
  /* colour rows: W_c x + W_sh gamma; the constant W_c . o / 2 joins W_sh[r][0] C0 */
  for (int r = 0; r < 3; ++r) {
    double shift = 0.0;
    for (int a = 0; a < 3; ++a) {
      shift += rec[4 + 3 * r + a] * o[a];
      out[4 + 3 * r + a] = 0.5 * rec[4 + 3 * r + a];
    }
    out[13 + 4 * r] = rec[13 + 4 * r] + 0.5 * shift / C0;
  }
  /* intensity W_int . [x, 1] */
  out[30] = rec[30] + 0.5 * (rec[27] * o[0] + rec[28] * o[1] + rec[29] * o[2]);
  for (int a = 0; a < 3; ++a) out[27 + a] = 0.5 * rec[27 + a];
}
