/* oracle.h -- plain, slow CPU oracle of the 3DGUT-style camera / LiDAR
 * renderer of "SimULi: Real-Time LiDAR and Camera Simulation with Unscented
 * Transforms" (arXiv 2510.12901).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * The same sources are compiled twice: with -DORACLE_F32 every floating-point
 * step runs in float (the precision in which the CUDA kernels take their
 * integer decisions: tile ranges, culls, sort keys, cutoffs), otherwise in
 * double (the reference values for every floating-point output).  Sensor ray
 * tables and the elevation tiling are set-up steps computed in double in both
 * builds.
 *
 * Parity status per function is stated next to each declaration.
 */
#ifndef SIMGUT_ORACLE_H
#define SIMGUT_ORACLE_H
#include <stdint.h>

#ifdef ORACLE_F32
typedef float real;
#else
typedef double real;
#endif

/* Feature kinds: RGB (3 floats, camera), SH (3 (d+1)^2 floats: camera
 * colour, offset 0.5 and clamped at 0 as in 3DGS), LIDAR (3 raw floats:
 * intensity, beta_hit, beta_drop), LIDAR_SH (3 (d+1)^2 floats: the SH^l
 * coefficients of those three channels, Sec. 3.1; zeta = sum_k Y_k(dir)
 * c_k with neither offset nor clamp, dir from the sensor origin of the
 * column pose that sees the mean to the mean). */
enum { OR_FEAT_RGB = 0, OR_FEAT_SH = 1, OR_FEAT_LIDAR = 2, OR_FEAT_LIDAR_SH = 3 };
enum { OR_PINHOLE = 0, OR_FISHEYE = 1 };

/* Gaussian parameters are in the build's own precision (`real`): float in
 * the float build, double in the double build, so that the double build can
 * be differentiated by central differences in double. */
typedef struct {
    int64_t n;
    const real *means;        /* [n,3] */
    const real *log_scales;   /* [n,3] */
    const real *quats;        /* [n,4] (w,x,y,z), normalised here */
    const real *opacity;      /* [n], already in (0,1) */
    const real *features;     /* [n,F] */
    int feature_kind;
    int sh_degree;
    /* Dynamic actors (Sec. 3.1 scene graph; NULL actor_of: all static).
     * Gaussian g with actor_of[g] = a >= 0 has its mean and rotation in
     * actor a's frame; actor_poses[a] (row-major [R | t], actor to world, at
     * the render's timestamp) takes them to world coordinates before
     * projection.  Its SH are evaluated at the view direction expressed in
     * the actor's frame (the appearance turns with the object). */
    const int32_t *actor_of;  /* [n] or NULL */
    int n_actors;
    const float *actor_poses; /* [n_actors,12] */
} or_scene;

typedef struct {
    int model, width, height;
    float fx, fy, cx, cy;
    float k[4];
    float c2w[12];            /* row-major [R | t], OpenCV axes */
    /* Rolling shutter (Sec. 3.2, time-dependent effects): [height,12]
     * camera-to-world pose of every pixel row (the row's exposure time), or
     * NULL for a global shutter (c2w).  A point's pixel comes from the pose
     * of the row it falls in, found as for the LiDAR columns: start from the
     * middle row's pose, then pose_iters times take the pose of the row the
     * point projects to (clamped to the image). */
    const float *row_c2w;
} or_camera;

typedef struct {
    int n_beams, n_cols;
    float az0_deg;
    const float *elev_deg;    /* [n_beams] */
    const float *col_c2w;     /* [n_cols,12] sensor-to-world per column */
    int n_elev_tiles;         /* N_phi */
    int max_rays_per_tile;    /* M */
    int cull_az;              /* dense culling cells over 360 deg */
    int cull_el_per_tile;     /* dense culling cells per elevation tile */
} or_lidar;

typedef struct {
    float alpha_min, alpha_max, t_min, near_dist;
    float ut_alpha, ut_beta, ut_kappa;
    int tile;         /* camera tile edge in pixels */
    int pose_iters;   /* LiDAR column-pose fixed-point iterations */
    int cull;         /* LiDAR ray-based culling on/off */
    int predicate;    /* per-ray extent test (1); 0 only for smooth FD checks */
    int cutoffs;      /* alpha_min / t_min / alpha_max cutoffs (1); 0 for FD */
    /* LiDAR beam divergence delta (radians, 0 = off; Sec. 3.3, Eq. 6): a
     * LiDAR Gaussian's covariance becomes Sigma + (delta |mu - o|)^2
     * (I - d d^T), d = (mu - o)/|mu - o| from the origin o of the column
     * pose that sees the mean, without rescaling the opacity.  The UT then
     * takes its sigma points along the columns of the Cholesky factor of
     * that covariance. */
    float beam_divergence;
    /* SH evaluated per ray (1) instead of once per Gaussian (0, the
     * default).  Eq. 1 writes the colour as SH_i(d) with d the ray
     * direction; 3DGS-style renderers, and this library, evaluate it once
     * per Gaussian at the direction from the sensor origin to the mean.  This
     * option evaluates it at each ray's own direction (in the Gaussian's
     * actor frame), to measure how far the two readings differ.  Forward
     * only: the backward refuses it. */
    int sh_per_ray;
} or_opts;

/* Sensor set-up, computed once per sensor (double in both builds). */
typedef struct {
    int n_tiles_x, n_tiles_y;    /* camera tiles; LiDAR: N_theta, N_phi */
    double theta_max;            /* fisheye validity limit (rad) */
    /* LiDAR */
    float *T;                    /* [N_phi+1] elevation boundaries (deg), float-rounded */
    int n_theta;
    int *sat;                    /* [(A+1)*(E+1)] summed-area table of the ray mask */
    int sat_w, sat_h;            /* A+1, E+1 */
} or_sensor_setup;

/* Per-Gaussian projection record. */
typedef struct {
    int valid;            /* passed validity, opacity and extent tests */
    real mean2d[2];       /* UT mean (px, or az/el degrees) */
    real cov2d[3];        /* UT covariance xx, xy, yy */
    real rect[4];         /* per-ray test box: x_lo, x_hi, y_lo, y_hi */
    int tiles[4];         /* tile range x0, x1 (may exceed N for LiDAR wrap), y0, y1 */
    int count;            /* number of tiles it is binned into */
    real depth;           /* sort key: distance |mu - o| rounded to float */
    int pose_col;         /* LiDAR: column whose pose the centre point used */
    real vmargin;         /* min relative margin of the validity tests (near, theta, opacity) */
    int ut;               /* the unscented transform ran (all sigma points valid) */
    real pmargin;         /* LiDAR: min distance (in columns) of a sigma point's
                             azimuth to a column boundary in the pose choice */
    real cmargin;         /* LiDAR: the same for the centre alone (the sort key's
                             column); 1e30 for cameras */
    real kdelta;          /* LiDAR: largest change of the float32 key if the centre
                             took a neighbouring column's pose; 0 for cameras */
} or_proj;

/* Per-ray outputs and statistics. */
typedef struct {
    real out[3];          /* camera rgb / LiDAR (intensity, beta_hit, beta_drop) sums */
    real alpha;           /* omega = sum alpha_i T_i */
    real depth;           /* Z / omega (camera depth, LiDAR range) or 0 */
    real zsum;            /* Z = sum tau_i alpha_i T_i */
    real t_final;
    int n_visited;        /* list entries visited before termination */
    int n_evaluated;      /* entries that passed the extent test */
    int n_contrib;        /* entries composited */
    real m_rect;          /* min |ray coord - rect edge| over entries that would contribute */
    real m_alpha;         /* min |alpha - alpha_min| / alpha_min over evaluated */
    real m_tmin;          /* min |T' - t_min| / t_min over composited + stopping */
    real m_tau;           /* min |tau| over evaluated */
    real m_order;         /* min relative gap of consecutive sort keys of contributing entries */
    real m_kpose;         /* min cmargin over contributing entries whose key is within
                             their kdelta of another contributing entry's key (a
                             column-pose flip could swap them); 1e30 if none */
} or_ray;

#ifdef __cplusplus
extern "C" {
#endif

or_opts or_default_opts(void);

/* Sec. 3.1: q -> R, log-scale -> scale.  Pinned: R orthonormal, det 1. */
void or_activate(int64_t n, const real *log_scales, const real *quats,
                 real *R_out, real *s_out);

/* Real spherical harmonics up to degree 3 at a unit direction (16 values).
 * Pinned: orthonormality on the sphere, harmonic polynomials. */
void or_sh_basis(const real dir[3], real Y[16]);
void or_sh_basis_grad(const real dir[3], real dY[16][3]);

/* Camera model (Sec. 3.2).  Pinned: k=0 equidistant, round trip. */
double or_fisheye_theta_max(const float k[4]);
int or_camera_project(const or_camera *cam, double theta_max, const or_opts *o,
                      const real xw[3], real uv[2]);
int or_camera_ray(const or_camera *cam, double theta_max, int px, int py,
                  double o[3], double d[3]);

/* Unscented transform of one 3D Gaussian to 2D (Sec. 3.2).
 * Pinned: exact for an affine map; EWA limit; Monte-Carlo moments. */
typedef int (*or_point_map)(void *ctx, const real x[3], int idx, real y[2]);
int or_unscented(const or_opts *o, const real mu[3], const real R[9],
                 const real s[3], or_point_map f, void *ctx, int wrap_first,
                 real mean2d[2], real cov2d[3]);

/* LiDAR sensor set-up: Proc. 1 (ElevationTiling) and the ray-mask summed-area
 * table of App. B.  Pinned: uniform table, M bound, SAT vs brute force. */
void or_elevation_tiling(const float *elev_deg, int n_beams, int n_cols,
                         int n_phi, int M, float *T_out, int *n_theta_out);
int or_elev_tile(const float *T, int n_phi, real el);
int or_elev_cell(const float *T, int n_phi, int per_tile, real el);
int or_az_cell(real az, float az0, int n_cells);
void or_lidar_setup(const or_lidar *L, or_sensor_setup *S);
void or_camera_setup(const or_camera *cam, const or_opts *o, or_sensor_setup *S);
void or_setup_free(or_sensor_setup *S);
int or_sat_count(const or_sensor_setup *S, int x0, int x1, int y0, int y1);
int or_sat_count_wrap(const or_sensor_setup *S, int A, int x0, int x1, int y0, int y1);
void or_lidar_ray(const or_lidar *L, int beam, int col, double o[3], double d[3],
                  double *az_deg, double *el_deg);

/* Projection of every Gaussian (Sec. 3.2 / 3.3, App. B Proc. 2-3). */
void or_project_camera(const or_scene *sc, const or_camera *cam,
                       const or_sensor_setup *S, const or_opts *o,
                       or_proj *out);
void or_project_lidar(const or_scene *sc, const or_lidar *L,
                      const or_sensor_setup *S, const or_opts *o,
                      or_proj *out);

/* Tile lists: every (tile, gaussian) pair sorted by (tile, depth, id).
 * Returns the number of pairs K; ids_out may be NULL to only count.
 * ranges_out [n_tiles*2] start/end.  Pinned: brute-force sort. */
int64_t or_bin_sort(int64_t n, const or_proj *P, int n_tiles_x, int n_tiles_y,
                    int wrap_x, uint32_t *ids_out, uint32_t *tiles_out,
                    int64_t cap, uint32_t *ranges_out);

/* Rendering (Eq. 1, response at tau_max).  `rays` selects rays by linear
 * index (py*W+px or beam*n_cols+col); n_rays<0 renders all.  bruteforce=1
 * walks every projected Gaussian in global (depth,id) order instead of the
 * tile list.  Pinned: closed forms, tiled == brute force, culling and
 * tiling invariance. */
int or_render_camera(const or_scene *sc, const or_camera *cam,
                     const or_opts *o, int bruteforce,
                     const int64_t *rays, int64_t n_rays, or_ray *out);
int or_render_lidar(const or_scene *sc, const or_lidar *L,
                    const or_opts *o, int bruteforce,
                    const int64_t *rays, int64_t n_rays, or_ray *out);

/* Per-ray output decode: LiDAR intensity and ray-drop probability (Sec. 3.2).
 * range = Z / omega, intensity = the first channel of zeta, drop =
 * softmax(zeta_1, zeta_2)[drop] = 1 / (1 + exp(zeta_1 - zeta_2)) with
 * zeta_1 the accumulated beta_hit and zeta_2 the accumulated beta_drop.
 * Pinned: a single Gaussian on a beam (closed form), rays that hit nothing. */
void or_lidar_decode(const or_ray *r, real *range, real *intensity, real *drop);
void or_lidar_decode_n(int64_t n, const or_ray *r, real *range, real *intensity, real *drop);

/* Analytic gradients (Sec. 3.4 differentiable renderer) of
 * L = sum_rays <g_out, outputs> w.r.t. the raw parameters; upstream arrays
 * are indexed by ray id; `rays` (n_rays < 0: all) selects the rays summed.
 * Camera outputs: rgb[3], alpha, depth.  LiDAR outputs: range, intensity,
 * drop, alpha.  grads are [n,3], [n,3], [n,4], [n], [n,F]; accumulated.
 * Pinned: central finite differences of the forward, closed forms.
 * Return -1 (nothing computed) for opts with sh_per_ray set. */
int or_backward_camera(const or_scene *sc, const or_camera *cam,
                       const or_opts *o, const int64_t *rays, int64_t n_rays,
                       const float *g_rgb,
                       const float *g_alpha, const float *g_depth,
                       real *gm, real *gls, real *gq, real *gop, real *gf);
int or_backward_lidar(const or_scene *sc, const or_lidar *L,
                      const or_opts *o, const int64_t *rays, int64_t n_rays,
                      const float *g_range,
                      const float *g_int, const float *g_drop,
                      const float *g_alpha,
                      real *gm, real *gls, real *gq, real *gop, real *gf);

#ifdef __cplusplus
}
#endif
#endif
