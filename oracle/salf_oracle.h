/*
 * salf_oracle.h -- FP64 CPU oracle for SaLF ray-cast rendering.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link,
 * load or call this code: only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no source with the CUDA library.
 *
 * What it computes (SaLF, arXiv 2507.18713):
 *   - sensor rays: pinhole, equidistant fisheye, equirectangular panorama,
 *     spinning LiDAR, caller-given rays; per-ray time and pose (rolling
 *     shutter / motion, Sec. V-C, Fig. 10);
 *   - the ordered list of voxels a ray crosses with positive length
 *     (Sec. III-B: the octree is only an accelerator, so its result is the
 *     exhaustive ray-box intersection list; voxels are disjoint, Sec. III-D);
 *   - per hit, the local field at the segment midpoint: density by Eq. 1
 *     (EXP) or Eq. 5-6 (SDF), colour by Eq. 2;
 *   - front-to-back compositing by Eq. 3-4;
 *   - the analytic gradient of a linear functional of the outputs with
 *     respect to every record scalar.
 * Everything is double precision.  Status: 0 ok, 1 invalid, 4 overlap.
 */
#ifndef SALF_ORACLE_H
#define SALF_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_scene orc_scene;

typedef struct {
  int64_t n;
  double origin[3];      /* min corner of the root grid (m) */
  double s0;             /* level-0 edge (m) */
  int32_t dims[3];       /* level-0 grid cells */
  int32_t max_level;     /* K */
  int32_t mode;          /* 0: Eq. 1 density; 1: Eq. 5-6 SDF density */
  const uint8_t* level;  /* n */
  const int32_t* ijk;    /* n*3, cell coordinates at the voxel's own level */
  const double* params;  /* n*32 record scalars */
} orc_scene_desc;

typedef struct {
  int32_t kind;          /* 0 pinhole, 1 fisheye, 2 panorama, 3 lidar, 4 explicit */
  int32_t width, height; /* LiDAR: width = azimuth columns, height = beams */
  double fx, fy, cx, cy; /* pixels */
  double fov;            /* fisheye: full field of view (rad) */
  double elev_min, elev_max; /* LiDAR beams / panorama vertical extent (rad) */
  double pose0[12], pose1[12]; /* sensor-to-world 3x4 row-major [R|t] */
  double t0, t1;
  int32_t rolling_shutter;
  double t_near, t_far;  /* t_far <= 0: unbounded */
  const float* rays;     /* explicit: width rows of (o, d, t_near, t_far) */
  const double* rays64;  /* explicit, FP64 rows (used instead of `rays` when set) */
} orc_sensor;

typedef struct {
  double t_min;          /* stop after the voxel that brings T below this; 0 = never */
  double background[3];
  int32_t want_intensity;
  int32_t brute_force;   /* 1: test every voxel; 0: finest-level DDA candidates */
  int32_t want_raydrop;  /* evaluate the raydrop field (record slot 31) */
} orc_opts;

typedef struct {
  double* rgb;           /* m*3 (premultiplied colour + T_end * background) */
  double* depth;         /* m: sum of w * t_mid */
  double* opacity;       /* m: sum of w */
  double* intensity;     /* m: sum of w * iota */
  double* t_end;         /* m: transmittance after the last composited voxel */
  double* term_gap;      /* m: min |ln T_k - ln T_min| over the termination tests */
  int32_t* n_visits;     /* m: composited voxels */
  uint8_t* valid;        /* m */
  int32_t* visits;       /* m*visits_cap input voxel indices in order, -1 padded */
  int32_t visits_cap;
  double* max_alpha;     /* n (input order): largest composited alpha per voxel, max-accumulated */
  double* raydrop;       /* m: sum of w * sigmoid(rho) + T_end (an escaping ray returns nothing) */
} orc_outputs;

typedef struct {
  int32_t voxel;         /* input index */
  double t_in, t_out;    /* unclipped box entry/exit */
} orc_hit;

int orc_scene_create(const orc_scene_desc* desc, orc_scene** out);
void orc_scene_free(orc_scene* s);
int64_t orc_scene_lookup(const orc_scene* s, int32_t level, int32_t i, int32_t j, int32_t k);
/* Replace voxel v's 32 record scalars (input order; for finite differences).
 * Status 1 if v is out of range or an SDF record has a <= 0 or b <= 0. */
int orc_scene_set_record(orc_scene* s, int64_t v, const double* rec);

/* Rays for the given ray indices (idx NULL: all rays 0..m-1). */
int orc_gen_rays(const orc_sensor* sen, const int64_t* idx, int64_t m, double* o, double* d,
                 double* tn, double* tf, double* tau, uint8_t* valid);
void orc_pose_at(const orc_sensor* sen, double tau, double R[9], double t[3]);
void orc_sh_basis(const double dir[3], double g[4]);
void orc_field(const double* rec, int32_t mode, const double x[3], const double dir[3],
               double* sigma, double c[3], double* iota);

/* Hits of one ray in [tn, tf], sorted by entry; returns the hit count (writes
 * at most cap). */
int64_t orc_trace(const orc_scene* s, const double o[3], const double d[3], double tn,
                  double tf, int32_t brute_force, orc_hit* hits, int64_t cap);
/* Same, with every voxel box grown (sign=+1) or shrunk (sign=-1) by
 * eps = eps_abs + eps_rel * |box centre - o|; returns ids sorted by entry and
 * (if t_in / t_out are not NULL) the perturbed boxes' entry / exit. */
int64_t orc_trace_eps(const orc_scene* s, const double o[3], const double d[3], double tn,
                      double tf, double eps_abs, double eps_rel, int32_t sign, int32_t* ids,
                      double* t_in, double* t_out, int64_t cap);

/* Per ray (idx NULL: all rays 0..m-1): 1 if its visit list is the same for
 * every voxel box shrunk and grown by eps_abs + eps_rel * |box centre - o|. */
int orc_conditioned(const orc_scene* s, const orc_sensor* sen, const int64_t* idx, int64_t m,
                    double eps_abs, double eps_rel, uint8_t* ok);

int orc_render(const orc_scene* s, const orc_sensor* sen, const orc_opts* opt,
               const int64_t* idx, int64_t m, const orc_outputs* out);
/* grad (n*32, input order) += d/dparams of
 *   sum_r g_rgb[r].rgb[r] + g_depth[r] depth[r] + g_opacity[r] opacity[r]
 *         + g_intensity[r] intensity[r] + g_raydrop[r] raydrop[r]
 * (any g_* may be NULL). */
int orc_backward(const orc_scene* s, const orc_sensor* sen, const orc_opts* opt,
                 const int64_t* idx, int64_t m, const double* g_rgb, const double* g_depth,
                 const double* g_opacity, const double* g_intensity, const double* g_raydrop,
                 double* grad);
/* A rounding bound for FP32 evaluations of orc_backward's gradient (same
 * arguments): bound (n*32) += per scalar the magnitude of every contribution
 * with absolute factors, absolute-term sums and the hit geometry's FP32
 * conditioning folded in (see the definition).  A tolerance, not part of
 * the method. */
int orc_backward_bound(const orc_scene* s, const orc_sensor* sen, const orc_opts* opt,
                       const int64_t* idx, int64_t m, const double* g_rgb, const double* g_depth,
                       const double* g_opacity, const double* g_intensity,
                       const double* g_raydrop, double* bound);
int orc_num_threads(void);

/* Sec. III-C densification: the record of child `child` (bits x | y << 1 |
 * z << 2 select the upper half per axis) of a voxel split into 8, carrying
 * the parent's fields: every field is affine in the local coordinates and
 * x_parent = (x_child + o) / 2 with o in {-1, +1}^3, so slopes halve and the
 * offsets take W . o / 2 (the colour's, which has no own offset, goes to the
 * SH DC term through C0).  a and b are kept. */
void orc_subdivide_record(const double* rec, int32_t child, double* out);

/* Dynamic actors (Sec. IV-A): an actor is a voxel set in its own canonical
 * frame (an orc_scene built from it), placed in the world by pose0 / pose1
 * (canonical -> world, 3x4 row-major) at the sensor's t0 / t1 and by their
 * interpolation (linear translation, slerp) at a ray's time.  The static
 * scene's hits and every actor's hits (traced in the actor's frame) are
 * composited together in order of entry (ties: static first, then actors in
 * list order, then voxel index); each hit's field uses local coordinates and
 * view direction of its own frame.  Visits report static voxels by input
 * index and actor k's voxels as id_base + input index. */
typedef struct {
  const orc_scene* scene;
  double pose0[12], pose1[12];
  int32_t id_base;
} orc_actor;

int orc_render_actors(const orc_scene* s, const orc_actor* actors, int32_t n_actors,
                      const orc_sensor* sen, const orc_opts* opt, const int64_t* idx, int64_t m,
                      const orc_outputs* out);

/* Adjoint of orc_render_actors (actors are fitted with the scene, Sec. IV-A):
 * grad (static scene, n*32) and actor_grads[k] (actor k's n_k*32; NULL =
 * not wanted) += d/d(record scalars) of sum_r g_r . outputs_r (raydrop is
 * not part of the actor render).  The _bound variant accumulates the FP32
 * rounding bound of orc_backward_bound for the same sums. */
int orc_backward_actors(const orc_scene* s, const orc_actor* actors, int32_t n_actors,
                        const orc_sensor* sen, const orc_opts* opt, const int64_t* idx, int64_t m,
                        const double* g_rgb, const double* g_depth, const double* g_opacity,
                        const double* g_intensity, double* grad, double* const* actor_grads);
int orc_backward_actors_bound(const orc_scene* s, const orc_actor* actors, int32_t n_actors,
                              const orc_sensor* sen, const orc_opts* opt, const int64_t* idx,
                              int64_t m, const double* g_rgb, const double* g_depth,
                              const double* g_opacity, const double* g_intensity, double* bound,
                              double* const* actor_bounds);

#ifdef __cplusplus
}
#endif
#endif
