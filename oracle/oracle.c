/* oracle.c -- plain CPU oracle of the SimULi / 3DGUT-style renderer.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the CPU
 * baseline of the benchmark; never by the product path.  It shares no code
 * with the CUDA library.  Every step follows the paper's description in the
 * paper's order, with no blocking, fusion or reordering; section, equation and
 * procedure numbers refer to arXiv 2510.12901.
 *
 * Readings of passages the paper leaves open are marked READING below.
 *
 * Built twice: -DORACLE_F32 (float arithmetic) and default (double).
 * Compile with -ffp-contract=off so that no multiply-add is fused.
 */
#include "oracle.h"

#include <float.h>
#include <stdlib.h>
#include <string.h>
#include <tgmath.h>

#define RL(x) ((real)(x))
#define PI_D 3.14159265358979323846
#define DEG_D (180.0 / PI_D)

/* ------------------------------------------------------------------ */
/* Options                                                             */
/* ------------------------------------------------------------------ */

or_opts or_default_opts(void)
{
    or_opts o;
    o.alpha_min = 1.0f / 255.0f;  /* READING: 3DGS cutoff, Sec. 3.2 "as in 3DGS" */
    o.alpha_max = 0.99f;
    o.t_min = 1e-4f;
    o.near_dist = 0.2f;
    o.ut_alpha = 1.0f;            /* READING: scaled UT, alpha=1, beta=2, kappa=0 */
    o.ut_beta = 2.0f;
    o.ut_kappa = 0.0f;
    o.tile = 16;
    o.pose_iters = 2;
    o.cull = 1;
    o.predicate = 1;
    o.cutoffs = 1;
    o.beam_divergence = 0.0f;     /* READING: delta is not stated; off by default */
    o.sh_per_ray = 0;             /* READING: SH once per Gaussian (3DGS practice) */
    return o;
}

/* ------------------------------------------------------------------ */
/* Sec. 3.1: Sigma = R S S^T R^T from a unit quaternion and scales     */
/* ------------------------------------------------------------------ */

static void quat_to_R(const real q[4], real R[9])
{
    real w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = RL(1) - RL(2) * (y * y + z * z);
    R[1] = RL(2) * (x * y - w * z);
    R[2] = RL(2) * (x * z + w * y);
    R[3] = RL(2) * (x * y + w * z);
    R[4] = RL(1) - RL(2) * (x * x + z * z);
    R[5] = RL(2) * (y * z - w * x);
    R[6] = RL(2) * (x * z - w * y);
    R[7] = RL(2) * (y * z + w * x);
    R[8] = RL(1) - RL(2) * (x * x + y * y);
}

static void unit_quat(const real *qin, real q[4], real *norm)
{
    real n = sqrt(RL(qin[0]) * RL(qin[0]) + RL(qin[1]) * RL(qin[1]) +
                  RL(qin[2]) * RL(qin[2]) + RL(qin[3]) * RL(qin[3]));
    for (int i = 0; i < 4; ++i) q[i] = RL(qin[i]) / n;
    if (norm) *norm = n;
}

void or_activate(int64_t n, const real *log_scales, const real *quats,
                 real *R_out, real *s_out)
{
    for (int64_t i = 0; i < n; ++i) {
        real q[4];
        unit_quat(quats + 4 * i, q, NULL);
        quat_to_R(q, R_out + 9 * i);
        for (int k = 0; k < 3; ++k) s_out[3 * i + k] = exp(RL(log_scales[3 * i + k]));
    }
}

/* Inverse covariance A = R diag(1/s^2) R^T, full 3x3 row-major. */
static void inv_cov(const real R[9], const real s[3], real A[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            real acc = 0;
            for (int k = 0; k < 3; ++k)
                acc += R[3 * i + k] * R[3 * j + k] / (s[k] * s[k]);
            A[3 * i + j] = acc;
        }
}

/* ------------------------------------------------------------------ */
/* Real spherical harmonics, degree <= 3 (Sec. 3.1: SH^c in R^48)      */
/* Normalisation K_l^m = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!), times   */
/* sqrt(2) for m != 0; Cartesian forms of the associated Legendre       */
/* polynomials; basis order m = -l..l per degree, with the sign         */
/* convention used by 3DGS-style renderers.                             */
/* ------------------------------------------------------------------ */

/* Actor rotation of Gaussian g (identity for the static background) and,
 * if t is given, its translation. */
static int actor_pose(const or_scene *sc, int64_t g, real Ra[9], real t[3])
{
    int a = sc->actor_of ? sc->actor_of[g] : -1;
    if (a < 0 || a >= sc->n_actors) {
        for (int i = 0; i < 9; ++i) Ra[i] = (i % 4 == 0) ? RL(1) : RL(0);
        if (t) t[0] = t[1] = t[2] = 0;
        return 0;
    }
    const float *P = sc->actor_poses + 12 * a;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) Ra[3 * i + j] = RL(P[4 * i + j]);
        if (t) t[i] = RL(P[4 * i + 3]);
    }
    return 1;
}

/* World mean and rotation of Gaussian g: mu_w = Ra mu + t, R_w = Ra R. */
static void gauss_world(const or_scene *sc, int64_t g, real mu[3], real R[9], real *qn)
{
    real q[4], Rl[9], Ra[9], t[3], ml[3];
    unit_quat(sc->quats + 4 * g, q, qn);
    quat_to_R(q, Rl);
    for (int k = 0; k < 3; ++k) ml[k] = RL(sc->means[3 * g + k]);
    actor_pose(sc, g, Ra, t);
    for (int i = 0; i < 3; ++i) {
        mu[i] = Ra[3 * i] * ml[0] + Ra[3 * i + 1] * ml[1] + Ra[3 * i + 2] * ml[2] + t[i];
        for (int j = 0; j < 3; ++j)
            R[3 * i + j] = Ra[3 * i] * Rl[j] + Ra[3 * i + 1] * Rl[3 + j] + Ra[3 * i + 2] * Rl[6 + j];
    }
}

/* Eq. 6: Sigma_hat = R diag(s^2) R^T + (delta |v|)^2 (I - v v^T / |v|^2)
 *                  = R diag(s^2) R^T + delta^2 (|v|^2 I - v v^T),  v = mu - o. */
static void smoothed_cov(const real R[9], const real s[3], const real v[3], real delta,
                         real C[9])
{
    real vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2], d2 = delta * delta;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            real acc = 0;
            for (int k = 0; k < 3; ++k) acc += R[3 * i + k] * s[k] * s[k] * R[3 * j + k];
            C[3 * i + j] = acc + d2 * ((i == j ? vv : RL(0)) - v[i] * v[j]);
        }
}

/* Lower Cholesky factor L (row-major) of a symmetric positive definite C. */
static void cholesky3(const real C[9], real L[9])
{
    for (int i = 0; i < 9; ++i) L[i] = 0;
    for (int j = 0; j < 3; ++j) {
        real d = C[4 * j];
        for (int k = 0; k < j; ++k) d -= L[3 * j + k] * L[3 * j + k];
        L[4 * j] = sqrt(d);
        for (int i = j + 1; i < 3; ++i) {
            real a = C[3 * i + j];
            for (int k = 0; k < j; ++k) a -= L[3 * i + k] * L[3 * j + k];
            L[3 * i + j] = a / L[4 * j];
        }
    }
}

/* Inverse of a 3x3 matrix by its adjugate. */
static void inverse3(const real C[9], real A[9])
{
    real c00 = C[4] * C[8] - C[5] * C[7], c01 = C[5] * C[6] - C[3] * C[8];
    real c02 = C[3] * C[7] - C[4] * C[6];
    real det = C[0] * c00 + C[1] * c01 + C[2] * c02;
    A[0] = c00 / det;
    A[1] = (C[2] * C[7] - C[1] * C[8]) / det;
    A[2] = (C[1] * C[5] - C[2] * C[4]) / det;
    A[3] = c01 / det;
    A[4] = (C[0] * C[8] - C[2] * C[6]) / det;
    A[5] = (C[2] * C[3] - C[0] * C[5]) / det;
    A[6] = c02 / det;
    A[7] = (C[1] * C[6] - C[0] * C[7]) / det;
    A[8] = (C[0] * C[4] - C[1] * C[3]) / det;
}

static double fact(int k) { double f = 1; for (int i = 2; i <= k; ++i) f *= i; return f; }
static double shK(int l, int m)
{
    int am = m < 0 ? -m : m;
    double k = sqrt((2.0 * l + 1.0) / (4.0 * PI_D) * fact(l - am) / fact(l + am));
    return m == 0 ? k : sqrt(2.0) * k;
}

void or_sh_basis(const real dir[3], real Y[16])
{
    real x = dir[0], y = dir[1], z = dir[2];
    real xx = x * x, yy = y * y, zz = z * z;
    real K00 = RL(shK(0, 0)), K10 = RL(shK(1, 0)), K11 = RL(shK(1, 1));
    real K20 = RL(shK(2, 0)), K21 = RL(shK(2, 1)), K22 = RL(shK(2, 2));
    real K30 = RL(shK(3, 0)), K31 = RL(shK(3, 1)), K32 = RL(shK(3, 2)), K33 = RL(shK(3, 3));
    Y[0] = K00;
    /* l = 1: P_1^1 = -sin(t), P_1^0 = cos(t) */
    Y[1] = -K11 * y;
    Y[2] = K10 * z;
    Y[3] = -K11 * x;
    /* l = 2: P_2^2 = 3 sin^2, P_2^1 = -3 sin cos, P_2^0 = (3 cos^2 - 1)/2;
     * sin^2 sin(2p) = 2xy, sin^2 cos(2p) = x^2 - y^2 */
    Y[4] = RL(3) * K22 * (RL(2) * x * y);
    Y[5] = -RL(3) * K21 * y * z;
    Y[6] = K20 * (RL(2) * zz - xx - yy) / RL(2);
    Y[7] = -RL(3) * K21 * x * z;
    Y[8] = RL(3) * K22 * (xx - yy);
    /* l = 3: P_3^3 = -15 sin^3, P_3^2 = 15 sin^2 cos,
     * P_3^1 = -(3/2) sin (5 cos^2 - 1), P_3^0 = (5 cos^3 - 3 cos)/2 */
    Y[9] = -RL(15) * K33 * y * (RL(3) * xx - yy);
    Y[10] = RL(15) * K32 * (RL(2) * x * y * z);
    Y[11] = -RL(1.5) * K31 * y * (RL(4) * zz - xx - yy);
    Y[12] = K30 * z * (RL(2) * zz - RL(3) * xx - RL(3) * yy) / RL(2);
    Y[13] = -RL(1.5) * K31 * x * (RL(4) * zz - xx - yy);
    Y[14] = RL(15) * K32 * z * (xx - yy);
    Y[15] = -RL(15) * K33 * x * (xx - RL(3) * yy);
}

/* Partial derivatives of the same polynomials w.r.t. (x, y, z). */
void or_sh_basis_grad(const real dir[3], real dY[16][3])
{
    real x = dir[0], y = dir[1], z = dir[2];
    real xx = x * x, yy = y * y, zz = z * z;
    memset(dY, 0, sizeof(real) * 48);
    real K10 = RL(shK(1, 0)), K11 = RL(shK(1, 1));
    real K20 = RL(shK(2, 0)), K21 = RL(shK(2, 1)), K22 = RL(shK(2, 2));
    real K30 = RL(shK(3, 0)), K31 = RL(shK(3, 1)), K32 = RL(shK(3, 2)), K33 = RL(shK(3, 3));
    dY[1][1] = -K11;
    dY[2][2] = K10;
    dY[3][0] = -K11;
    real a = RL(6) * K22;                       /* Y4 = a x y */
    dY[4][0] = a * y; dY[4][1] = a * x;
    real b = RL(3) * K21;                       /* Y5 = -b y z, Y7 = -b x z */
    dY[5][1] = -b * z; dY[5][2] = -b * y;
    dY[7][0] = -b * z; dY[7][2] = -b * x;
    real c = K20 / RL(2);                       /* Y6 = c (2z^2 - x^2 - y^2) */
    dY[6][0] = -RL(2) * c * x; dY[6][1] = -RL(2) * c * y; dY[6][2] = RL(4) * c * z;
    real e = RL(3) * K22;                       /* Y8 = e (x^2 - y^2) */
    dY[8][0] = RL(2) * e * x; dY[8][1] = -RL(2) * e * y;
    real f = RL(15) * K33;                      /* Y9 = -f (3x^2 y - y^3) */
    dY[9][0] = -RL(6) * f * x * y; dY[9][1] = -f * (RL(3) * xx - RL(3) * yy);
    real g = RL(30) * K32;                      /* Y10 = g x y z */
    dY[10][0] = g * y * z; dY[10][1] = g * x * z; dY[10][2] = g * x * y;
    real h = RL(1.5) * K31;                     /* Y11 = -h (4 y z^2 - x^2 y - y^3) */
    dY[11][0] = RL(2) * h * x * y; dY[11][1] = -h * (RL(4) * zz - xx - RL(3) * yy);
    dY[11][2] = -RL(8) * h * y * z;
    real i0 = K30 / RL(2);                      /* Y12 = i (2z^3 - 3x^2 z - 3y^2 z) */
    dY[12][0] = -RL(6) * i0 * x * z; dY[12][1] = -RL(6) * i0 * y * z;
    dY[12][2] = i0 * (RL(6) * zz - RL(3) * xx - RL(3) * yy);
    real j = RL(1.5) * K31;                     /* Y13 = -j (4 x z^2 - x^3 - x y^2) */
    dY[13][0] = -j * (RL(4) * zz - RL(3) * xx - yy); dY[13][1] = RL(2) * j * x * y;
    dY[13][2] = -RL(8) * j * x * z;
    real k = RL(15) * K32;                      /* Y14 = k (x^2 z - y^2 z) */
    dY[14][0] = RL(2) * k * x * z; dY[14][1] = -RL(2) * k * y * z; dY[14][2] = k * (xx - yy);
    real l = RL(15) * K33;                      /* Y15 = -l (x^3 - 3 x y^2) */
    dY[15][0] = -l * (RL(3) * xx - RL(3) * yy); dY[15][1] = RL(6) * l * x * y;
}

/* ------------------------------------------------------------------ */
/* Camera models (Sec. 3.2: "arbitrary" cameras through the UT)        */
/* ------------------------------------------------------------------ */

static double fisheye_poly(const float k[4], double th)
{
    double t2 = th * th;
    return th * (1.0 + t2 * (k[0] + t2 * (k[1] + t2 * (k[2] + t2 * k[3]))));
}
static double fisheye_dpoly(const float k[4], double th)
{
    double t2 = th * th;
    return 1.0 + t2 * (3.0 * k[0] + t2 * (5.0 * k[1] + t2 * (7.0 * k[2] + t2 * 9.0 * k[3])));
}

/* READING: the valid incidence angles are [0, theta_max] with theta_max the
 * first angle where the OpenCV fisheye polynomial stops increasing, capped at
 * pi/2.  Found by a fine scan plus bisection in double. */
double or_fisheye_theta_max(const float k[4])
{
    const double cap = PI_D / 2.0;
    const int steps = 20000;
    double prev = 0.0;
    for (int i = 1; i <= steps; ++i) {
        double th = cap * i / steps;
        if (fisheye_dpoly(k, th) <= 0.0) {
            double lo = prev, hi = th;
            for (int it = 0; it < 200; ++it) {
                double mid = 0.5 * (lo + hi);
                if (fisheye_dpoly(k, mid) > 0.0) lo = mid; else hi = mid;
            }
            return lo;
        }
        prev = th;
    }
    return cap;
}

/* World point -> pixel.  Returns 0 when the point is outside the model's
 * domain (READING: pinhole z > near; fisheye |x| > near and theta <= max). */
/* The camera-to-world pose of pixel row `row` (the global pose without a
 * rolling shutter). */
static const float *row_pose(const or_camera *cam, int row)
{
    return cam->row_c2w ? cam->row_c2w + 12 * row : cam->c2w;
}

static int cam_project_pose(const or_camera *cam, const float *M, double theta_max,
                            const or_opts *o, const real xw[3], real uv[2], real *margin)
{
    real d0 = xw[0] - RL(M[3]), d1 = xw[1] - RL(M[7]), d2 = xw[2] - RL(M[11]);
    /* x_c = R^T (x - t) */
    real x = RL(M[0]) * d0 + RL(M[4]) * d1 + RL(M[8]) * d2;
    real y = RL(M[1]) * d0 + RL(M[5]) * d1 + RL(M[9]) * d2;
    real z = RL(M[2]) * d0 + RL(M[6]) * d1 + RL(M[10]) * d2;
    real nr = RL(o->near_dist);
    if (cam->model == OR_PINHOLE) {
        if (margin) { real m = fabs(z - nr) / nr; if (m < *margin) *margin = m; }
        if (!(z > nr)) return 0;
        uv[0] = RL(cam->fx) * x / z + RL(cam->cx);
        uv[1] = RL(cam->fy) * y / z + RL(cam->cy);
        return 1;
    }
    real r = sqrt(x * x + y * y);
    real dist = sqrt(x * x + y * y + z * z);
    real th = atan2(r, z);
    real tm = RL(theta_max);
    if (margin) {
        real m1 = fabs(dist - nr) / nr, m2 = fabs(th - tm) / tm;
        if (m1 < *margin) *margin = m1;
        if (m2 < *margin) *margin = m2;
    }
    if (!(dist > nr) || !(th <= tm)) return 0;
    real t2 = th * th;
    real thd = th * (RL(1) + t2 * (RL(cam->k[0]) + t2 * (RL(cam->k[1]) +
                     t2 * (RL(cam->k[2]) + t2 * RL(cam->k[3])))));
    if (r > RL(0)) {
        uv[0] = RL(cam->fx) * (thd / r) * x + RL(cam->cx);
        uv[1] = RL(cam->fy) * (thd / r) * y + RL(cam->cy);
    } else {
        uv[0] = RL(cam->cx);
        uv[1] = RL(cam->cy);
    }
    return 1;
}

/* Rolling shutter: the row whose pose sees x (fixed-point iteration from
 * the middle row, see or_camera); *pmargin gets the smallest distance (in
 * rows) of an iterate to a row boundary.  Global shutter: row 0, no
 * iteration. */
static int cam_row_of(const or_camera *cam, double theta_max, const or_opts *o,
                      const real x[3], real *pmargin)
{
    if (!cam->row_c2w) return 0;
    int row = cam->height / 2;
    for (int it = 0; it < o->pose_iters; ++it) {
        real t[2];
        if (!cam_project_pose(cam, row_pose(cam, row), theta_max, o, x, t, NULL)) break;
        real f = t[1], fr = f - floor(f), m = fr < RL(0.5) ? fr : RL(1) - fr;
        if (pmargin && m < *pmargin) *pmargin = m;
        int r = f < RL(0) ? 0 : (f >= RL(cam->height) ? cam->height - 1 : (int)floor(f));
        row = r;
    }
    return row;
}

static int cam_project_margin(const or_camera *cam, double theta_max,
                              const or_opts *o, const real xw[3], real uv[2],
                              real *margin, real *pmargin)
{
    int row = cam_row_of(cam, theta_max, o, xw, pmargin);
    return cam_project_pose(cam, row_pose(cam, row), theta_max, o, xw, uv, margin);
}

int or_camera_project(const or_camera *cam, double theta_max, const or_opts *o,
                      const real xw[3], real uv[2])
{
    return cam_project_margin(cam, theta_max, o, xw, uv, NULL, NULL);
}

/* Pixel centre (px+0.5, py+0.5) -> world ray (double).  Fisheye inverse by
 * bisection on [0, theta_max] (the polynomial is increasing there). */
int or_camera_ray(const or_camera *cam, double theta_max, int px, int py,
                  double o[3], double d[3])
{
    double mx = ((px + 0.5) - (double)cam->cx) / (double)cam->fx;
    double my = ((py + 0.5) - (double)cam->cy) / (double)cam->fy;
    double dc[3];
    if (cam->model == OR_PINHOLE) {
        double n = sqrt(mx * mx + my * my + 1.0);
        dc[0] = mx / n; dc[1] = my / n; dc[2] = 1.0 / n;
    } else {
        double thd = sqrt(mx * mx + my * my);
        if (thd > fisheye_poly(cam->k, theta_max)) return 0;
        double lo = 0.0, hi = theta_max;
        for (int it = 0; it < 200; ++it) {
            double mid = 0.5 * (lo + hi);
            if (fisheye_poly(cam->k, mid) < thd) lo = mid; else hi = mid;
        }
        double th = 0.5 * (lo + hi);
        if (thd > 0.0) {
            dc[0] = sin(th) * mx / thd;
            dc[1] = sin(th) * my / thd;
        } else {
            dc[0] = dc[1] = 0.0;
        }
        dc[2] = cos(th);
    }
    const float *M = row_pose(cam, py);   /* the ray of row py: that row's pose */
    for (int i = 0; i < 3; ++i)
        d[i] = (double)M[4 * i] * dc[0] + (double)M[4 * i + 1] * dc[1] +
               (double)M[4 * i + 2] * dc[2];
    o[0] = M[3]; o[1] = M[7]; o[2] = M[11];
    return 1;
}

/* ------------------------------------------------------------------ */
/* Unscented transform (Sec. 3.2: 7 sigma points -> 2D conic)          */
/* Scaled UT: lambda = a^2 (n + kappa) - n, n = 3; chi_0 = mu,         */
/* chi_{+-i} = mu +- sqrt(n + lambda) s_i R e_i;                       */
/* w0m = lambda/(n+lambda), w0c = w0m + 1 - a^2 + b, wi = 1/(2(n+l)).  */
/* ------------------------------------------------------------------ */

int or_unscented(const or_opts *o, const real mu[3], const real R[9],
                 const real s[3], or_point_map f, void *ctx, int wrap_first,
                 real mean2d[2], real cov2d[3])
{
    const real n = RL(3);
    real a = RL(o->ut_alpha), b = RL(o->ut_beta), kap = RL(o->ut_kappa);
    real lam = a * a * (n + kap) - n;
    real gam = sqrt(n + lam);
    real w0m = lam / (n + lam);
    real w0c = w0m + (RL(1) - a * a + b);
    real wi = RL(1) / (RL(2) * (n + lam));
    real y[7][2];
    int ok = 1;
    for (int p = 0; p < 7; ++p) {
        real x[3] = {mu[0], mu[1], mu[2]};
        if (p > 0) {
            int i = (p - 1) / 2;
            real sg = ((p - 1) % 2 == 0) ? RL(1) : RL(-1);
            for (int r = 0; r < 3; ++r) x[r] += sg * gam * s[i] * R[3 * r + i];
        }
        if (!f(ctx, x, p, y[p])) ok = 0;
    }
    if (!ok) return 0;
    if (wrap_first) {   /* azimuth: unwrap each point to within 180 deg of chi_0 */
        for (int p = 1; p < 7; ++p) {
            real dlt = y[p][0] - y[0][0];
            if (dlt > RL(180)) y[p][0] -= RL(360);
            else if (dlt < RL(-180)) y[p][0] += RL(360);
        }
    }
    real m0 = w0m * y[0][0], m1 = w0m * y[0][1];
    for (int p = 1; p < 7; ++p) { m0 += wi * y[p][0]; m1 += wi * y[p][1]; }
    real c00 = 0, c01 = 0, c11 = 0;
    for (int p = 0; p < 7; ++p) {
        real w = (p == 0) ? w0c : wi;
        real e0 = y[p][0] - m0, e1 = y[p][1] - m1;
        c00 += w * e0 * e0;
        c01 += w * e0 * e1;
        c11 += w * e1 * e1;
    }
    mean2d[0] = m0; mean2d[1] = m1;
    cov2d[0] = c00; cov2d[1] = c01; cov2d[2] = c11;
    return 1;
}

/* ------------------------------------------------------------------ */
/* LiDAR tiling: Proc. 1 ElevationTiling (App. A) and the ray-based     */
/* culling table of App. B (Proc. 2).                                   */
/* ------------------------------------------------------------------ */

/* READING (Proc. 1 is garbled): loop over all r = 400 histogram bins; at
 * each bin append its upper edge while the normalised CDF has reached the
 * next integer (a while loop, so a bin may cross several); the boundaries
 * are mapped back with Phi_min + T/r (Phi_max - Phi_min); the CDF test is
 * done on integer counts (cum * N_phi >= b * total); N_theta is rounded up.
 * Phi holds the elevation of every ray (each beam n_cols times).  The
 * boundaries are rounded to float, and the second histogram (rays per
 * elevation tile) uses the float boundaries, as every later test does. */
void or_elevation_tiling(const float *elev_deg, int n_beams, int n_cols,
                         int n_phi, int M, float *T_out, int *n_theta_out)
{
    const int r = 400;
    double pmin = DBL_MAX, pmax = -DBL_MAX;
    for (int b = 0; b < n_beams; ++b) {
        if (elev_deg[b] < pmin) pmin = elev_deg[b];
        if (elev_deg[b] > pmax) pmax = elev_deg[b];
    }
    int64_t *H = calloc(r, sizeof(int64_t));
    for (int b = 0; b < n_beams; ++b) {
        int bin = (int)floor(((double)elev_deg[b] - pmin) / (pmax - pmin) * r);
        if (bin > r - 1) bin = r - 1;
        if (bin < 0) bin = 0;
        H[bin] += n_cols;
    }
    int64_t total = (int64_t)n_beams * n_cols, cum = 0;
    int nT = 0;
    double Tbin[1024];
    Tbin[nT++] = 0.0;
    int64_t bnext = 1;
    for (int i = 0; i < r; ++i) {
        cum += H[i];
        while (bnext <= n_phi && cum * (int64_t)n_phi >= bnext * total) {
            Tbin[nT++] = (double)(i + 1);
            bnext++;
        }
    }
    for (int j = 0; j <= n_phi; ++j)
        T_out[j] = (float)(pmin + Tbin[j] / r * (pmax - pmin));
    /* re-histogram rays by elevation tile */
    int64_t hmax = 0;
    int64_t *Ht = calloc(n_phi, sizeof(int64_t));
    for (int b = 0; b < n_beams; ++b) Ht[or_elev_tile(T_out, n_phi, RL(elev_deg[b]))] += n_cols;
    for (int j = 0; j < n_phi; ++j) if (Ht[j] > hmax) hmax = Ht[j];
    *n_theta_out = (int)((hmax + M - 1) / M);
    free(H);
    free(Ht);
}

/* Elevation tile: number of interior boundaries T_1..T_{n_phi-1} <= el. */
int or_elev_tile(const float *T, int n_phi, real el)
{
    int e = 0;
    for (int j = 1; j < n_phi; ++j) if (RL(T[j]) <= el) e = j;
    return e;
}

/* Dense culling cell in elevation: `per_tile` uniform cells per tile
 * (READING of r^d = (1600, 8): 8 cells per elevation tile). */
int or_elev_cell(const float *T, int n_phi, int per_tile, real el)
{
    int e = or_elev_tile(T, n_phi, el);
    real lo = RL(T[e]), w = RL(T[e + 1]) - RL(T[e]);
    real f = (el - lo) / w * RL(per_tile);
    int sub;
    if (!(f >= RL(0))) sub = 0;
    else if (f >= RL(per_tile)) sub = per_tile - 1;
    else sub = (int)floor(f);
    if (sub > per_tile - 1) sub = per_tile - 1;
    return e * per_tile + sub;
}

int or_az_cell(real az, float az0, int n_cells)
{
    return (int)floor((az - RL(az0)) * (RL(n_cells) / RL(360)));
}

static int pmod(int a, int n) { int m = a % n; return m < 0 ? m + n : m; }

void or_lidar_ray(const or_lidar *L, int beam, int col, double o[3], double d[3],
                  double *az_deg, double *el_deg)
{
    double az = (double)L->az0_deg + (col + 0.5) * 360.0 / L->n_cols;
    double el = (double)L->elev_deg[beam];
    double u[3] = {cos(el / DEG_D) * cos(az / DEG_D), cos(el / DEG_D) * sin(az / DEG_D),
                   sin(el / DEG_D)};
    const float *P = L->col_c2w + 12 * col;
    for (int i = 0; i < 3; ++i)
        d[i] = (double)P[4 * i] * u[0] + (double)P[4 * i + 1] * u[1] + (double)P[4 * i + 2] * u[2];
    o[0] = P[3]; o[1] = P[7]; o[2] = P[11];
    if (az_deg) *az_deg = az;
    if (el_deg) *el_deg = el;
}

/* ray azimuth as the renderer compares it (rounded to `real`) */
static real lidar_ray_az(const or_lidar *L, int col)
{
    return RL((double)L->az0_deg + (col + 0.5) * 360.0 / L->n_cols);
}

void or_lidar_setup(const or_lidar *L, or_sensor_setup *S)
{
    memset(S, 0, sizeof(*S));
    int nphi = L->n_elev_tiles;
    S->T = malloc(sizeof(float) * (nphi + 1));
    or_elevation_tiling(L->elev_deg, L->n_beams, L->n_cols, nphi,
                        L->max_rays_per_tile, S->T, &S->n_theta);
    S->n_tiles_x = S->n_theta;
    S->n_tiles_y = nphi;
    int A = L->cull_az, E = nphi * L->cull_el_per_tile;
    S->sat_w = A + 1;
    S->sat_h = E + 1;
    /* ray mask: dense cell of every ray (Sec. 3.3 "ray mask") */
    unsigned char *mask = calloc((size_t)A * E, 1);
    for (int b = 0; b < L->n_beams; ++b) {
        int yc = or_elev_cell(S->T, nphi, L->cull_el_per_tile, RL(L->elev_deg[b]));
        for (int c = 0; c < L->n_cols; ++c) {
            int xc = pmod(or_az_cell(lidar_ray_az(L, c), L->az0_deg, A), A);
            mask[(size_t)xc * E + yc] = 1;
        }
    }
    /* summed-area table with a zero first row / column (2D prefix sum) */
    S->sat = calloc((size_t)(A + 1) * (E + 1), sizeof(int));
    for (int x = 1; x <= A; ++x)
        for (int y = 1; y <= E; ++y)
            S->sat[(size_t)x * (E + 1) + y] = mask[(size_t)(x - 1) * E + (y - 1)] +
                                              S->sat[(size_t)(x - 1) * (E + 1) + y] +
                                              S->sat[(size_t)x * (E + 1) + y - 1] -
                                              S->sat[(size_t)(x - 1) * (E + 1) + y - 1];
    free(mask);
}

void or_camera_setup(const or_camera *cam, const or_opts *o, or_sensor_setup *S)
{
    memset(S, 0, sizeof(*S));
    S->n_tiles_x = (cam->width + o->tile - 1) / o->tile;
    S->n_tiles_y = (cam->height + o->tile - 1) / o->tile;
    S->theta_max = cam->model == OR_FISHEYE ? or_fisheye_theta_max(cam->k) : 0.0;
}

void or_setup_free(or_sensor_setup *S)
{
    free(S->T);
    free(S->sat);
    S->T = NULL;
    S->sat = NULL;
}

/* Proc. 2 RayOccupancyCount: rays in dense cells [x0,x1] x [y0,y1]. */
int or_sat_count(const or_sensor_setup *S, int x0, int x1, int y0, int y1)
{
    int H = S->sat_h;
    const int *T = S->sat;
    int A = T[(size_t)(x1 + 1) * H + (y1 + 1)];
    int B = T[(size_t)x0 * H + (y1 + 1)];
    int C = T[(size_t)(x1 + 1) * H + y0];
    int D = T[(size_t)x0 * H + y0];
    return A - B - C + D;
}

/* READING: an azimuth range that crosses the seam is split in two. */
int or_sat_count_wrap(const or_sensor_setup *S, int A, int x0, int x1, int y0, int y1)
{
    if (x1 - x0 + 1 >= A) return or_sat_count(S, 0, A - 1, y0, y1);
    int a = pmod(x0, A), b = pmod(x1, A);
    if (a <= b) return or_sat_count(S, a, b, y0, y1);
    return or_sat_count(S, a, A - 1, y0, y1) + or_sat_count(S, 0, b, y0, y1);
}

/* ------------------------------------------------------------------ */
/* Projection of all Gaussians: UT conic -> extent -> tiles -> counts  */
/* ------------------------------------------------------------------ */

typedef struct {
    const or_camera *cam; double theta_max; const or_opts *o; real margin; real pmargin;
} cam_ctx;

static int cam_point_map(void *vctx, const real x[3], int idx, real y[2])
{
    (void)idx;
    cam_ctx *c = vctx;
    return cam_project_margin(c->cam, c->theta_max, c->o, x, y, &c->margin, &c->pmargin);
}

/* READING of the extent ("culling as in 3DGS", Sec. 3.2): the box of the
 * k-sigma ellipse, k = sqrt(2 ln(sigma / alpha_min)), so that outside it the
 * 2D Gaussian falls below alpha_min. */
static real extent_k(real sigma, real amin) { return sqrt(RL(2) * log(sigma / amin)); }

void or_project_camera(const or_scene *sc, const or_camera *cam,
                       const or_sensor_setup *S, const or_opts *o, or_proj *out)
{
    const int tile = o->tile, ntx = S->n_tiles_x, nty = S->n_tiles_y;
    for (int64_t g = 0; g < sc->n; ++g) {
        or_proj *p = &out[g];
        memset(p, 0, sizeof(*p));
        p->cmargin = RL(1e30);
        real R[9], s[3], mu[3];
        gauss_world(sc, g, mu, R, NULL);
        for (int k = 0; k < 3; ++k) s[k] = exp(RL(sc->log_scales[3 * g + k]));
        real sigma = RL(sc->opacity[g]), amin = RL(o->alpha_min);
        /* the depth key and SH origin: the camera centre, or with a rolling
         * shutter the origin of the row that sees the mean */
        real cm = RL(1e30);
        int row0 = cam_row_of(cam, S->theta_max, o, mu, &cm);
        const float *C0 = row_pose(cam, row0);
        real dx = mu[0] - RL(C0[3]), dy = mu[1] - RL(C0[7]), dz = mu[2] - RL(C0[11]);
        /* sort key: 3DGS-style keys carry float32 depth bits (Sec. 3.2 "as in
         * 3DGS"), so the key is the distance rounded to float */
        p->depth = RL((float)sqrt(dx * dx + dy * dy + dz * dz));
        p->pose_col = row0;
        if (cam->row_c2w) {
            p->cmargin = cm;
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                int rr = row0 + sgn;
                if (rr < 0 || rr >= cam->height) continue;
                const float *Cn = row_pose(cam, rr);
                real ex = mu[0] - RL(Cn[3]), ey = mu[1] - RL(Cn[7]), ez = mu[2] - RL(Cn[11]);
                real kd = fabs(RL((float)sqrt(ex * ex + ey * ey + ez * ez)) - p->depth);
                if (kd > p->kdelta) p->kdelta = kd;
            }
        }
        p->vmargin = fabs(sigma - amin) / amin;
        if (!(sigma >= amin)) continue;
        cam_ctx ctx = {cam, S->theta_max, o, RL(1e30), RL(1e30)};
        int ok = or_unscented(o, mu, R, s, cam_point_map, &ctx, 0, p->mean2d, p->cov2d);
        if (cam->row_c2w) p->pmargin = ctx.pmargin;
        if (ctx.margin < p->vmargin) p->vmargin = ctx.margin;
        if (!ok) continue;
        p->ut = 1;
        real k = extent_k(sigma, amin);
        real hx = k * sqrt(p->cov2d[0]), hy = k * sqrt(p->cov2d[2]);
        p->rect[0] = p->mean2d[0] - hx;
        p->rect[1] = p->mean2d[0] + hx;
        p->rect[2] = p->mean2d[1] - hy;
        p->rect[3] = p->mean2d[1] + hy;
        if (!(p->rect[1] >= RL(0)) || !(p->rect[0] < RL(cam->width)) ||
            !(p->rect[3] >= RL(0)) || !(p->rect[2] < RL(cam->height)))
            continue;
        int x0 = p->rect[0] <= RL(0) ? 0 : (int)floor(p->rect[0] / RL(tile));
        int x1 = p->rect[1] >= RL(cam->width) ? ntx - 1 : (int)floor(p->rect[1] / RL(tile));
        int y0 = p->rect[2] <= RL(0) ? 0 : (int)floor(p->rect[2] / RL(tile));
        int y1 = p->rect[3] >= RL(cam->height) ? nty - 1 : (int)floor(p->rect[3] / RL(tile));
        if (x1 > ntx - 1) x1 = ntx - 1;
        if (y1 > nty - 1) y1 = nty - 1;
        p->tiles[0] = x0; p->tiles[1] = x1; p->tiles[2] = y0; p->tiles[3] = y1;
        p->count = (x1 - x0 + 1) * (y1 - y0 + 1);
        p->valid = 1;
    }
}

/* LiDAR point map (Eq. 3) with the sensor pose of the column that sees the
 * point.  READING (Sec. 3.3 says only "in the same manner as with camera"):
 * start from the mid-sweep pose, then `pose_iters` times take the pose of
 * the column containing the point's azimuth; the final transform gives
 * (azimuth, elevation) in degrees. */
typedef struct {
    const or_lidar *L; const or_opts *o; int col0; real range0; real margin; real pmargin;
} lid_ctx;

static int lidar_col_of(const or_lidar *L, real az, real *pmargin)
{
    real f = (az - RL(L->az0_deg)) * (RL(L->n_cols) / RL(360));
    real fr = f - floor(f);
    real m = fr < RL(0.5) ? fr : RL(1) - fr;
    if (pmargin && m < *pmargin) *pmargin = m;
    int c = (int)floor(f);
    return pmod(c, L->n_cols);
}

static void to_sensor(const float *P, const real x[3], real xs[3])
{
    real d0 = x[0] - RL(P[3]), d1 = x[1] - RL(P[7]), d2 = x[2] - RL(P[11]);
    xs[0] = RL(P[0]) * d0 + RL(P[4]) * d1 + RL(P[8]) * d2;
    xs[1] = RL(P[1]) * d0 + RL(P[5]) * d1 + RL(P[9]) * d2;
    xs[2] = RL(P[2]) * d0 + RL(P[6]) * d1 + RL(P[10]) * d2;
}

static int lidar_point_map(void *vctx, const real x[3], int idx, real y[2])
{
    lid_ctx *c = vctx;
    const or_lidar *L = c->L;
    int col = L->n_cols / 2;
    real xs[3];
    for (int it = 0; it < c->o->pose_iters; ++it) {
        to_sensor(L->col_c2w + 12 * col, x, xs);
        real az = atan2(xs[1], xs[0]) * RL(DEG_D);
        col = lidar_col_of(L, az, &c->pmargin);
    }
    to_sensor(L->col_c2w + 12 * col, x, xs);
    real r = sqrt(xs[0] * xs[0] + xs[1] * xs[1] + xs[2] * xs[2]);
    if (idx == 0) { c->col0 = col; c->range0 = r; }
    {
        real nr = RL(c->o->near_dist), m = fabs(r - nr) / nr;
        if (m < c->margin) c->margin = m;
    }
    if (!(r > RL(c->o->near_dist))) return 0;
    y[0] = atan2(xs[1], xs[0]) * RL(DEG_D);
    y[1] = asin(xs[2] / r) * RL(DEG_D);
    return 1;
}

void or_project_lidar(const or_scene *sc, const or_lidar *L,
                      const or_sensor_setup *S, const or_opts *o, or_proj *out)
{
    const int nphi = L->n_elev_tiles, nth = S->n_theta;
    const int A = L->cull_az, per = L->cull_el_per_tile;
    real T0 = RL(S->T[0]), TN = RL(S->T[nphi]);
    for (int64_t g = 0; g < sc->n; ++g) {
        or_proj *p = &out[g];
        memset(p, 0, sizeof(*p));
        p->cmargin = RL(1e30);
        real R[9], s[3], mu[3];
        gauss_world(sc, g, mu, R, NULL);
        for (int k = 0; k < 3; ++k) s[k] = exp(RL(sc->log_scales[3 * g + k]));
        real sigma = RL(sc->opacity[g]), amin = RL(o->alpha_min);
        lid_ctx ctx = {L, o, 0, 0, RL(1e30), RL(1e30)};
        /* depth key: distance to the sensor origin of the centre's column */
        {
            real y[2];
            lidar_point_map(&ctx, mu, 0, y);
            p->depth = RL((float)ctx.range0);   /* float32 key, as for cameras */
            p->pose_col = ctx.col0;
            /* how close that column choice came to flipping, and what the key
               would be with either neighbouring column's pose */
            p->cmargin = ctx.pmargin;
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                real xs[3];
                to_sensor(L->col_c2w + 12 * pmod(ctx.col0 + sgn, L->n_cols), mu, xs);
                real kd = fabs(RL((float)sqrt(xs[0] * xs[0] + xs[1] * xs[1] + xs[2] * xs[2])) -
                               p->depth);
                if (kd > p->kdelta) p->kdelta = kd;
            }
        }
        p->vmargin = fabs(sigma - amin) / amin;
        if (!(sigma >= amin)) continue;
        ctx.margin = RL(1e30);
        ctx.pmargin = RL(1e30);
        int ok;
        if (o->beam_divergence > 0.0f) {
            /* Eq. 6: the UT of the smoothed covariance, sigma points along the
             * columns of its Cholesky factor (READING) */
            const float *T = L->col_c2w + 12 * ctx.col0;
            real v[3] = {mu[0] - RL(T[3]), mu[1] - RL(T[7]), mu[2] - RL(T[11])}, Cs[9], Lc[9];
            smoothed_cov(R, s, v, RL(o->beam_divergence), Cs);
            cholesky3(Cs, Lc);
            const real one[3] = {1, 1, 1};
            ok = or_unscented(o, mu, Lc, one, lidar_point_map, &ctx, 1, p->mean2d, p->cov2d);
        } else {
            ok = or_unscented(o, mu, R, s, lidar_point_map, &ctx, 1, p->mean2d, p->cov2d);
        }
        p->pmargin = ctx.pmargin;
        if (ctx.margin < p->vmargin) p->vmargin = ctx.margin;
        if (!ok) continue;
        p->ut = 1;
        real k = extent_k(sigma, amin);
        real ha = k * sqrt(p->cov2d[0]), he = k * sqrt(p->cov2d[2]);
        p->rect[0] = p->mean2d[0] - ha;
        p->rect[1] = p->mean2d[0] + ha;
        p->rect[2] = p->mean2d[1] - he;
        p->rect[3] = p->mean2d[1] + he;
        if (!(p->rect[3] >= T0) || !(p->rect[2] <= TN)) continue;
        real elo = p->rect[2] < T0 ? T0 : p->rect[2];
        real ehi = p->rect[3] > TN ? TN : p->rect[3];
        int e0 = or_elev_tile(S->T, nphi, elo), e1 = or_elev_tile(S->T, nphi, ehi);
        int a0, a1, na;
        int full = !(p->rect[1] - p->rect[0] < RL(360));
        if (full) {
            a0 = 0; a1 = nth - 1; na = nth;
        } else {
            a0 = (int)floor((p->rect[0] - RL(L->az0_deg)) * (RL(nth) / RL(360)));
            a1 = (int)floor((p->rect[1] - RL(L->az0_deg)) * (RL(nth) / RL(360)));
            na = a1 - a0 + 1;
            if (na > nth) { na = nth; a1 = a0 + nth - 1; }
        }
        if (o->cull) {   /* App. B Proc. 3: keep only if a ray falls in the dense extent */
            int x0, x1;
            if (full) { x0 = 0; x1 = A - 1; }
            else {
                x0 = or_az_cell(p->rect[0], L->az0_deg, A);
                x1 = or_az_cell(p->rect[1], L->az0_deg, A);
            }
            int y0 = or_elev_cell(S->T, nphi, per, elo), y1 = or_elev_cell(S->T, nphi, per, ehi);
            if (or_sat_count_wrap(S, A, x0, x1, y0, y1) == 0) continue;
        }
        p->tiles[0] = a0; p->tiles[1] = a1; p->tiles[2] = e0; p->tiles[3] = e1;
        p->count = na * (e1 - e0 + 1);
        p->valid = 1;
    }
}

/* ------------------------------------------------------------------ */
/* Binning and the (tile, depth) key sort ("Sort" kernel of Tab. 5)    */
/* READING: total order (tile, depth, gaussian id).                    */
/* ------------------------------------------------------------------ */

typedef struct { uint32_t tile; real depth; uint32_t id; } or_pair;

static int pair_cmp(const void *va, const void *vb)
{
    const or_pair *a = va, *b = vb;
    if (a->tile != b->tile) return a->tile < b->tile ? -1 : 1;
    if (a->depth != b->depth) return a->depth < b->depth ? -1 : 1;
    if (a->id != b->id) return a->id < b->id ? -1 : 1;
    return 0;
}

/* all (tile, gaussian) pairs, optionally only for tiles with mask[t] != 0 */
static or_pair *make_pairs(int64_t n, const or_proj *P, int ntx, int nty,
                           int wrap_x, const unsigned char *mask, int64_t *K_out)
{
    int64_t K = 0;
    for (int64_t g = 0; g < n; ++g) if (P[g].valid) K += P[g].count;
    or_pair *pr = malloc(sizeof(or_pair) * (size_t)(K > 0 ? K : 1));
    int64_t k = 0;
    for (int64_t g = 0; g < n; ++g) {
        const or_proj *p = &P[g];
        if (!p->valid) continue;
        for (int ty = p->tiles[2]; ty <= p->tiles[3]; ++ty)
            for (int tx = p->tiles[0]; tx <= p->tiles[1]; ++tx) {
                int x = wrap_x ? pmod(tx, ntx) : tx;
                uint32_t t = (uint32_t)(ty * ntx + x);
                if (mask && !mask[t]) continue;
                pr[k].tile = t;
                pr[k].depth = p->depth;
                pr[k].id = (uint32_t)g;
                k++;
            }
    }
    (void)nty;
    qsort(pr, (size_t)k, sizeof(or_pair), pair_cmp);
    *K_out = k;
    return pr;
}

int64_t or_bin_sort(int64_t n, const or_proj *P, int ntx, int nty, int wrap_x,
                    uint32_t *ids_out, uint32_t *tiles_out, int64_t cap,
                    uint32_t *ranges_out)
{
    int64_t K;
    or_pair *pr = make_pairs(n, P, ntx, nty, wrap_x, NULL, &K);
    if (ids_out && K <= cap)
        for (int64_t i = 0; i < K; ++i) {
            ids_out[i] = pr[i].id;
            if (tiles_out) tiles_out[i] = pr[i].tile;
        }
    if (ranges_out) {
        int64_t nt = (int64_t)ntx * nty;
        for (int64_t t = 0; t < nt; ++t) { ranges_out[2 * t] = 0; ranges_out[2 * t + 1] = 0; }
        for (int64_t i = 0; i < K; ++i) {
            uint32_t t = pr[i].tile;
            if (i == 0 || pr[i - 1].tile != t) ranges_out[2 * t] = (uint32_t)i;
            ranges_out[2 * t + 1] = (uint32_t)(i + 1);
        }
    }
    free(pr);
    return K;
}

/* ------------------------------------------------------------------ */
/* Per-ray compositing (Eq. 1; response at tau_max, Sec. 3.2)          */
/* ------------------------------------------------------------------ */

typedef struct {
    real A[9];       /* Sigma^{-1} */
    real mu[3];
    real sigma;
    real feat[3];    /* colour, or LiDAR (intensity, beta_hit, beta_drop) */
    int clampc[3];   /* colour channel clamped at 0 (SH) */
    real dir[3];     /* SH direction used */
    real dist;       /* |mu - o_cam| */
    const real *shc; /* SH coefficients [nc][3] (NULL: features are not SH) */
    int nc, lidar_sh;
    real Ra[9];      /* actor rotation (world from the Gaussian's frame) */
} gauss_rt;

static void gauss_prepare(const or_scene *sc, int64_t g, const real ocam[3], real beam,
                          gauss_rt *G)
{
    real R[9], s[3];
    gauss_world(sc, g, G->mu, R, NULL);
    for (int k = 0; k < 3; ++k) s[k] = exp(RL(sc->log_scales[3 * g + k]));
    if (beam > 0) {   /* Eq. 6: the response of the smoothed covariance, opacity unchanged */
        real v[3] = {G->mu[0] - ocam[0], G->mu[1] - ocam[1], G->mu[2] - ocam[2]}, Cs[9];
        smoothed_cov(R, s, v, beam, Cs);
        inverse3(Cs, G->A);
    } else {
        inv_cov(R, s, G->A);
    }
    G->sigma = RL(sc->opacity[g]);
    G->clampc[0] = G->clampc[1] = G->clampc[2] = 0;
    if (sc->feature_kind == OR_FEAT_SH || sc->feature_kind == OR_FEAT_LIDAR_SH) {
        /* READING: SH evaluated once per Gaussian at the direction from the
         * camera centre to its mean (Eq. 1 writes SH_i(d)).  LiDAR (Sec. 3.2
         * writes SH^l_i(d) in zeta): the same, from the sensor origin of the
         * column pose that sees the mean; the channels are intensity and
         * logits, so they get neither the colour offset nor the clamp. */
        const int lidar = sc->feature_kind == OR_FEAT_LIDAR_SH;
        real v[3] = {G->mu[0] - ocam[0], G->mu[1] - ocam[1], G->mu[2] - ocam[2]};
        real nv = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        real Ra[9];
        actor_pose(sc, g, Ra, NULL);
        /* the direction in the Gaussian's own (actor) frame: Ra^T v / |v| */
        for (int k = 0; k < 3; ++k)
            G->dir[k] = (Ra[k] * v[0] + Ra[3 + k] * v[1] + Ra[6 + k] * v[2]) / nv;
        G->dist = nv;
        real Y[16];
        or_sh_basis(G->dir, Y);
        int nc = (sc->sh_degree + 1) * (sc->sh_degree + 1);
        const real *f = sc->features + (size_t)g * nc * 3;
        for (int ch = 0; ch < 3; ++ch) {
            real acc = 0;
            for (int k = 0; k < nc; ++k) acc += Y[k] * RL(f[3 * k + ch]);
            if (!lidar) {
                acc += RL(0.5);
                if (acc < RL(0)) { acc = 0; G->clampc[ch] = 1; }
            }
            G->feat[ch] = acc;
        }
        /* for the per-ray reading (or_opts.sh_per_ray) */
        G->shc = f;
        G->nc = nc;
        G->lidar_sh = lidar;
        for (int k = 0; k < 9; ++k) G->Ra[k] = Ra[k];
    } else {
        for (int ch = 0; ch < 3; ++ch) G->feat[ch] = RL(sc->features[3 * g + ch]);
        G->shc = NULL;
    }
}

/* The features of G seen along ray direction d (or_opts.sh_per_ray): the SH
 * evaluated at d expressed in the Gaussian's actor frame, with the colour
 * offset and clamp for camera SH (as for the per-Gaussian reading). */
static void feat_per_ray(const gauss_rt *G, const real d[3], real feat[3])
{
    real u[3], Y[16];
    for (int k = 0; k < 3; ++k) u[k] = G->Ra[k] * d[0] + G->Ra[3 + k] * d[1] + G->Ra[6 + k] * d[2];
    real nu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    for (int k = 0; k < 3; ++k) u[k] /= nu;
    or_sh_basis(u, Y);
    for (int ch = 0; ch < 3; ++ch) {
        real acc = 0;
        for (int k = 0; k < G->nc; ++k) acc += Y[k] * G->shc[3 * k + ch];
        if (!G->lidar_sh) {
            acc += RL(0.5);
            if (acc < RL(0)) acc = 0;
        }
        feat[ch] = acc;
    }
}

/* tau_max and squared Mahalanobis distance at it: minimum of the quadratic
 * q(tau) = (o + tau d - mu)^T A (o + tau d - mu) = a tau^2 + 2 b tau + c. */
static void response_quadratic(const gauss_rt *G, const real o[3], const real d[3],
                               real *a, real *b, real *c)
{
    real v[3] = {o[0] - G->mu[0], o[1] - G->mu[1], o[2] - G->mu[2]};
    real Ad[3], Av[3];
    for (int i = 0; i < 3; ++i) {
        Ad[i] = G->A[3 * i] * d[0] + G->A[3 * i + 1] * d[1] + G->A[3 * i + 2] * d[2];
        Av[i] = G->A[3 * i] * v[0] + G->A[3 * i + 1] * v[1] + G->A[3 * i + 2] * v[2];
    }
    *a = d[0] * Ad[0] + d[1] * Ad[1] + d[2] * Ad[2];
    *b = d[0] * Av[0] + d[1] * Av[1] + d[2] * Av[2];
    *c = v[0] * Av[0] + v[1] * Av[1] + v[2] * Av[2];
}

static real minr(real a, real b) { return a < b ? a : b; }

/* Is the ray coordinate inside the Gaussian's extent box?  Also tracks the
 * distance to the nearest edge. */
static int inside_rect(const or_proj *p, real rx, real ry, int wrap_az, real *mrect)
{
    real x = rx;
    if (wrap_az) {  /* choose the 360-degree alias of the ray azimuth nearest the box */
        real best = x, bd = RL(1e30);
        for (int k = -2; k <= 2; ++k) {
            real xa = rx + RL(360) * RL(k);
            real dd = fabs(xa - RL(0.5) * (p->rect[0] + p->rect[1]));
            if (dd < bd) { bd = dd; best = xa; }
        }
        x = best;
    }
    real m = minr(minr(fabs(x - p->rect[0]), fabs(x - p->rect[1])),
                  minr(fabs(ry - p->rect[2]), fabs(ry - p->rect[3])));
    if (m < *mrect) *mrect = m;
    return x >= p->rect[0] && x <= p->rect[1] && ry >= p->rect[2] && ry <= p->rect[3];
}

typedef struct {
    int64_t g; real alpha, T, tau, rho, a, b, c; int clamped;
} contrib;

/* Composite one ray over an ordered Gaussian list.  When `rec` is given the
 * composited entries are recorded for the backward pass.
 *
 * Besides the outputs, each ray records how close its discrete decisions
 * came to their thresholds (the m_* margins): the extent test (only for
 * entries that would contribute at the ray), alpha_min, t_min, tau > 0, and
 * the order of consecutive contributing entries' float32 keys. */
static void composite_ray(const or_opts *o, const or_proj *P, const gauss_rt *GR,
                          const uint32_t *list, int64_t nlist,
                          const real org[3], const real dir[3], real rx, real ry,
                          int wrap_az, or_ray *out, contrib *rec, int64_t *nrec)
{
    memset(out, 0, sizeof(*out));
    out->m_rect = out->m_alpha = out->m_tmin = out->m_tau = out->m_order = RL(1e30);
    out->m_kpose = RL(1e30);
    real prev_key = RL(-1);
    /* keys of the entries that reached compositing, for m_kpose */
    real *kk = nlist > 0 ? malloc(sizeof(real) * (size_t)nlist) : NULL;
    uint32_t *kg = nlist > 0 ? malloc(sizeof(uint32_t) * (size_t)nlist) : NULL;
    int64_t nk = 0;
    real T = RL(1), acc[3] = {0, 0, 0}, Z = 0, W = 0;
    real amin = RL(o->alpha_min), amax = RL(o->alpha_max), tmin = RL(o->t_min);
    int64_t nr = 0;
    for (int64_t li = 0; li < nlist; ++li) {
        uint32_t g = list[li];
        out->n_visited++;
        real medge = RL(1e30);
        int inside = !o->predicate || inside_rect(&P[g], rx, ry, wrap_az, &medge);
        const gauss_rt *G = &GR[g];
        real a, b, c;
        response_quadratic(G, org, dir, &a, &b, &c);
        real tau = -b / a;
        /* D2 = q(tau_max), the quadratic evaluated at its minimiser (Sec. 3.2:
         * the response at tau_max).  Evaluated as w^T A w with w = o + tau d - mu
         * rather than as c - b^2/a, which cancels badly when the ray passes
         * far from the Gaussian relative to its size. */
        real e[3], D2 = 0;
        for (int k = 0; k < 3; ++k) e[k] = org[k] + tau * dir[k] - G->mu[k];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) D2 += e[i] * G->A[3 * i + j] * e[j];
        if (D2 < RL(0)) D2 = RL(0);
        real rho = exp(RL(-0.5) * D2);
        real alpha = G->sigma * rho;
        int clamped = 0;
        if (o->cutoffs && alpha > amax) { alpha = amax; clamped = 1; }
        /* an extent-test flip matters only where the entry would contribute */
        if (o->predicate && tau > RL(0) && (!o->cutoffs || alpha >= amin * RL(0.999)))
            if (medge < out->m_rect) out->m_rect = medge;
        if (!inside) continue;
        out->n_evaluated++;
        if (fabs(tau) < out->m_tau) out->m_tau = fabs(tau);
        if (!(tau > RL(0))) continue;   /* READING: nothing behind the origin */
        if (o->cutoffs) {
            real ma = fabs(alpha - amin) / amin;
            if (ma < out->m_alpha) out->m_alpha = ma;
            if (alpha < amin) continue;
        }
        /* order margin between consecutive entries that reach compositing */
        if (prev_key >= RL(0)) {
            real gap = fabs(P[g].depth - prev_key) / P[g].depth;
            if (gap < out->m_order) out->m_order = gap;
        }
        prev_key = P[g].depth;
        /* a key that a column-pose flip could move past another one */
        for (int64_t q = 0; q < nk; ++q) {
            real gap = fabs(P[g].depth - kk[q]);
            if (gap <= P[g].kdelta && P[g].cmargin < out->m_kpose) out->m_kpose = P[g].cmargin;
            if (gap <= P[kg[q]].kdelta && P[kg[q]].cmargin < out->m_kpose)
                out->m_kpose = P[kg[q]].cmargin;
        }
        if (kk) { kk[nk] = P[g].depth; kg[nk] = g; nk++; }
        real Tn = T * (RL(1) - alpha);
        if (o->cutoffs) {
            real mt = fabs(Tn - tmin) / tmin;
            if (mt < out->m_tmin) out->m_tmin = mt;
            if (Tn < tmin) break;   /* READING: 3DGS stops before compositing it */
        }
        real w = alpha * T;
        real fr[3];
        const real *feat = G->feat;
        if (o->sh_per_ray && G->shc) {
            feat_per_ray(G, dir, fr);
            feat = fr;
        }
        for (int ch = 0; ch < 3; ++ch) acc[ch] += w * feat[ch];
        Z += w * tau;
        W += w;
        if (rec) {
            contrib *r = &rec[nr];
            r->g = g; r->alpha = alpha; r->T = T; r->tau = tau; r->rho = rho;
            r->a = a; r->b = b; r->c = c; r->clamped = clamped;
        }
        nr++;
        T = Tn;
        out->n_contrib++;
    }
    for (int ch = 0; ch < 3; ++ch) out->out[ch] = acc[ch];
    out->alpha = W;
    out->zsum = Z;
    out->t_final = T;
    out->depth = W > RL(0) ? Z / W : RL(0);
    if (nrec) *nrec = nr;
    free(kk);
    free(kg);
}

/* ------------------------------------------------------------------ */
/* Full camera / LiDAR renders (tiled or brute force)                  */
/* ------------------------------------------------------------------ */

typedef struct { real depth; uint32_t id; } dkey;
static int dkey_cmp(const void *va, const void *vb)
{
    const dkey *a = va, *b = vb;
    if (a->depth != b->depth) return a->depth < b->depth ? -1 : 1;
    return a->id < b->id ? -1 : (a->id > b->id ? 1 : 0);
}

/* global (depth, id) order of every projected Gaussian (brute force) */
static uint32_t *global_order(int64_t n, const or_proj *P, int64_t *m_out)
{
    dkey *k = malloc(sizeof(dkey) * (size_t)(n > 0 ? n : 1));
    int64_t m = 0;
    for (int64_t g = 0; g < n; ++g)
        if (P[g].valid) { k[m].depth = P[g].depth; k[m].id = (uint32_t)g; m++; }
    qsort(k, (size_t)m, sizeof(dkey), dkey_cmp);
    uint32_t *ids = malloc(sizeof(uint32_t) * (size_t)(m > 0 ? m : 1));
    for (int64_t i = 0; i < m; ++i) ids[i] = k[i].id;
    free(k);
    *m_out = m;
    return ids;
}

/* Shared driver: `ray_fn` gives origin / direction / coordinates / tile of
 * ray r.  Returns 0 on success. */
typedef int (*ray_fn)(const void *ctx, int64_t r, real o[3], real d[3], real *rx,
                      real *ry, uint32_t *tile);

/* ocam: the SH origin, one for all Gaussians, or per Gaussian ([n,3]) when
 * ocam_per_gauss is set. */
static const real *origin_of(const real *ocam, int per_gauss, int64_t g)
{
    return per_gauss ? ocam + 3 * g : ocam;
}

static int render_common(const or_scene *sc, const or_opts *o, const or_proj *P,
                         const real *ocam, int ocam_per_gauss, real beam, int ntx, int nty,
                         int wrap,
                         int bruteforce, const int64_t *rays, int64_t n_rays,
                         int64_t n_total, ray_fn rf, const void *rctx, or_ray *out,
                         /* backward (optional) */
                         void (*bw)(void *, int64_t, const or_ray *, const contrib *,
                                    int64_t, const real *, const real *),
                         void *bwctx)
{
    int64_t nr = n_rays < 0 ? n_total : n_rays;
    gauss_rt *GR = malloc(sizeof(gauss_rt) * (size_t)(sc->n > 0 ? sc->n : 1));
    for (int64_t g = 0; g < sc->n; ++g)
        gauss_prepare(sc, g, origin_of(ocam, ocam_per_gauss, g), beam, &GR[g]);
    int64_t nt = (int64_t)ntx * nty;
    uint32_t *ids = NULL, *ranges = NULL;
    or_pair *pr = NULL;
    int64_t K = 0, m = 0;
    if (bruteforce) {
        ids = global_order(sc->n, P, &m);
    } else {
        unsigned char *mask = calloc((size_t)nt, 1);
        for (int64_t i = 0; i < nr; ++i) {
            real oo[3], dd[3], rx, ry;
            uint32_t t;
            if (rf(rctx, rays ? rays[i] : i, oo, dd, &rx, &ry, &t) == 0) mask[t] = 1;
        }
        pr = make_pairs(sc->n, P, ntx, nty, wrap, mask, &K);
        free(mask);
        ids = malloc(sizeof(uint32_t) * (size_t)(K > 0 ? K : 1));
        ranges = calloc((size_t)nt * 2, sizeof(uint32_t));
        for (int64_t i = 0; i < K; ++i) {
            ids[i] = pr[i].id;
            uint32_t t = pr[i].tile;
            if (i == 0 || pr[i - 1].tile != t) ranges[2 * t] = (uint32_t)i;
            ranges[2 * t + 1] = (uint32_t)(i + 1);
        }
    }
    int64_t maxlist = bruteforce ? m : K;
    contrib *rec = bw ? malloc(sizeof(contrib) * (size_t)(maxlist > 0 ? maxlist : 1)) : NULL;
    for (int64_t i = 0; i < nr; ++i) {
        int64_t r = rays ? rays[i] : i;
        real oo[3], dd[3], rx, ry;
        uint32_t t;
        if (rf(rctx, r, oo, dd, &rx, &ry, &t) != 0) {   /* pixel outside the lens */
            memset(&out[i], 0, sizeof(or_ray));
            out[i].t_final = RL(1);
            out[i].m_rect = out[i].m_alpha = out[i].m_tmin = out[i].m_tau = RL(1e30);
            out[i].m_order = RL(1e30);
            continue;
        }
        const uint32_t *list;
        int64_t nl;
        if (bruteforce) { list = ids; nl = m; }
        else { list = ids + ranges[2 * t]; nl = ranges[2 * t + 1] - ranges[2 * t]; }
        int64_t nrec = 0;
        composite_ray(o, P, GR, list, nl, oo, dd, rx, ry, wrap, &out[i], rec, &nrec);
        if (bw) bw(bwctx, r, &out[i], rec, nrec, oo, dd);
    }
    free(rec);
    free(ids);
    free(ranges);
    free(pr);
    free(GR);
    return 0;
}

typedef struct { const or_camera *cam; double theta_max; int tile, ntx; } cam_rctx;
static int cam_ray_fn(const void *vctx, int64_t r, real o[3], real d[3], real *rx,
                      real *ry, uint32_t *tile)
{
    const cam_rctx *c = vctx;
    int px = (int)(r % c->cam->width), py = (int)(r / c->cam->width);
    double od[3], dd[3];
    *tile = (uint32_t)((py / c->tile) * c->ntx + px / c->tile);
    if (!or_camera_ray(c->cam, c->theta_max, px, py, od, dd)) return 1;
    for (int k = 0; k < 3; ++k) { o[k] = RL(od[k]); d[k] = RL(dd[k]); }
    *rx = RL(px) + RL(0.5);
    *ry = RL(py) + RL(0.5);
    return 0;
}

/* Per-Gaussian SH origins of a camera render: the camera centre, or with a
 * rolling shutter the origin of the row whose pose sees the mean. */
static real *cam_sh_origins(const or_scene *sc, const or_camera *cam, const or_proj *P)
{
    real *o = calloc((size_t)(sc->n > 0 ? sc->n : 1) * 3, sizeof(real));
    for (int64_t g = 0; g < sc->n; ++g) {
        const float *T = row_pose(cam, P[g].pose_col);
        o[3 * g] = RL(T[3]);
        o[3 * g + 1] = RL(T[7]);
        o[3 * g + 2] = RL(T[11]);
    }
    return o;
}

int or_render_camera(const or_scene *sc, const or_camera *cam, const or_opts *o,
                     int bruteforce, const int64_t *rays, int64_t n_rays, or_ray *out)
{
    or_sensor_setup S;
    or_camera_setup(cam, o, &S);
    or_proj *P = malloc(sizeof(or_proj) * (size_t)(sc->n > 0 ? sc->n : 1));
    or_project_camera(sc, cam, &S, o, P);
    real *ocam = cam_sh_origins(sc, cam, P);
    cam_rctx rc = {cam, S.theta_max, o->tile, S.n_tiles_x};
    render_common(sc, o, P, ocam, 1, 0, S.n_tiles_x, S.n_tiles_y, 0, bruteforce, rays,
                  n_rays, (int64_t)cam->width * cam->height, cam_ray_fn, &rc, out,
                  NULL, NULL);
    free(ocam);
    free(P);
    or_setup_free(&S);
    return 0;
}

typedef struct { const or_lidar *L; const or_sensor_setup *S; int *beam_tile; int *col_tile; } lid_rctx;
static int lid_ray_fn(const void *vctx, int64_t r, real o[3], real d[3], real *rx,
                      real *ry, uint32_t *tile)
{
    const lid_rctx *c = vctx;
    int b = (int)(r / c->L->n_cols), col = (int)(r % c->L->n_cols);
    double od[3], dd[3], az, el;
    or_lidar_ray(c->L, b, col, od, dd, &az, &el);
    for (int k = 0; k < 3; ++k) { o[k] = RL(od[k]); d[k] = RL(dd[k]); }
    *rx = lidar_ray_az(c->L, col);
    *ry = RL(c->L->elev_deg[b]);
    *tile = (uint32_t)(c->beam_tile[b] * c->S->n_theta + c->col_tile[col]);
    return 0;
}

static void lidar_ray_tiles(const or_lidar *L, const or_sensor_setup *S, int *bt, int *ct)
{
    for (int b = 0; b < L->n_beams; ++b)
        bt[b] = or_elev_tile(S->T, L->n_elev_tiles, RL(L->elev_deg[b]));
    for (int c = 0; c < L->n_cols; ++c)
        ct[c] = pmod((int)floor((lidar_ray_az(L, c) - RL(L->az0_deg)) *
                                (RL(S->n_theta) / RL(360))), S->n_theta);
}

/* Per-Gaussian SH origins of a LiDAR scene: the sensor origin of the column
 * pose the projection chose for the mean (only LIDAR_SH features use them). */
static real *lidar_sh_origins(const or_scene *sc, const or_lidar *L, const or_proj *P)
{
    real *o = calloc((size_t)(sc->n > 0 ? sc->n : 1) * 3, sizeof(real));
    for (int64_t g = 0; g < sc->n; ++g) {
        const float *T = L->col_c2w + 12 * P[g].pose_col;
        o[3 * g] = RL(T[3]);
        o[3 * g + 1] = RL(T[7]);
        o[3 * g + 2] = RL(T[11]);
    }
    return o;
}

int or_render_lidar(const or_scene *sc, const or_lidar *L, const or_opts *o,
                    int bruteforce, const int64_t *rays, int64_t n_rays, or_ray *out)
{
    or_sensor_setup S;
    or_lidar_setup(L, &S);
    or_proj *P = malloc(sizeof(or_proj) * (size_t)(sc->n > 0 ? sc->n : 1));
    or_project_lidar(sc, L, &S, o, P);
    int *bt = malloc(sizeof(int) * L->n_beams), *ct = malloc(sizeof(int) * L->n_cols);
    lidar_ray_tiles(L, &S, bt, ct);
    lid_rctx rc = {L, &S, bt, ct};
    real *ocam = lidar_sh_origins(sc, L, P);
    render_common(sc, o, P, ocam, 1, RL(o->beam_divergence), S.n_theta, L->n_elev_tiles, 1,
                  bruteforce, rays,
                  n_rays, (int64_t)L->n_beams * L->n_cols, lid_ray_fn, &rc, out, NULL,
                  NULL);
    free(ocam);
    free(bt);
    free(ct);
    free(P);
    or_setup_free(&S);
    return 0;
}

/* Sec. 3.2: intensity = first channel of zeta; ray drop = softmax over the
 * remaining two channels (beta_hit, beta_drop), probability of drop. */
void or_lidar_decode(const or_ray *r, real *range, real *intensity, real *drop)
{
    *range = r->depth;
    *intensity = r->out[0];
    *drop = RL(1) / (RL(1) + exp(r->out[1] - r->out[2]));
}

void or_lidar_decode_n(int64_t n, const or_ray *r, real *range, real *intensity, real *drop)
{
    for (int64_t i = 0; i < n; ++i) or_lidar_decode(&r[i], &range[i], &intensity[i], &drop[i]);
}

/* ------------------------------------------------------------------ */
/* Backward: plain chain rule through the forward above                */
/* ------------------------------------------------------------------ */

typedef struct {
    const or_scene *sc;
    const gauss_rt *GR;   /* filled lazily */
    int lidar;
    const float *g_a, *g_b, *g_c, *g_d, *g_e;  /* per-ray upstream gradients */
    int64_t n_rays_total;
    /* per-Gaussian gradient w.r.t. A (9), mu (3), sigma, feature (3) */
    real *gA, *gmu, *gsig, *gfeat;
} bw_ctx;

/* Gradient of L w.r.t. the accumulated ray quantities Q = (F0, F1, F2, Z, W). */
static void ray_upstream(const bw_ctx *B, int64_t r, const or_ray *ray, real gQ[5])
{
    real W = ray->alpha, Z = ray->zsum;
    if (!B->lidar) {
        gQ[0] = RL(B->g_a[3 * r]); gQ[1] = RL(B->g_a[3 * r + 1]); gQ[2] = RL(B->g_a[3 * r + 2]);
        real gal = RL(B->g_b[r]), gdp = RL(B->g_c[r]);
        gQ[3] = W > RL(0) ? gdp / W : RL(0);
        gQ[4] = gal - (W > RL(0) ? gdp * Z / (W * W) : RL(0));
    } else {
        real grange = RL(B->g_a[r]), gint = RL(B->g_b[r]), gdrop = RL(B->g_c[r]),
             gal = RL(B->g_d[r]);
        real drop = RL(1) / (RL(1) + exp(ray->out[1] - ray->out[2]));
        gQ[0] = gint;
        gQ[1] = -gdrop * drop * (RL(1) - drop);
        gQ[2] = gdrop * drop * (RL(1) - drop);
        gQ[3] = W > RL(0) ? grange / W : RL(0);
        gQ[4] = gal - (W > RL(0) ? grange * Z / (W * W) : RL(0));
    }
}

static void bw_ray(void *vctx, int64_t r, const or_ray *ray, const contrib *rec,
                   int64_t n, const real *org, const real *dir)
{
    bw_ctx *B = vctx;
    real gQ[5];
    ray_upstream(B, r, ray, gQ);
    /* suffix sums S_q(i) = sum_{j>i} q_j alpha_j T_j for q = F0,F1,F2,tau,1 */
    real suf[5] = {0, 0, 0, 0, 0};
    for (int64_t i = n - 1; i >= 0; --i) {
        const contrib *c = &rec[i];
        const gauss_rt *G = &B->GR[c->g];
        real q[5] = {G->feat[0], G->feat[1], G->feat[2], c->tau, RL(1)};
        real wT = c->alpha * c->T;
        real dLdalpha = 0;
        for (int k = 0; k < 5; ++k)
            dLdalpha += gQ[k] * (q[k] * c->T - suf[k] / (RL(1) - c->alpha));
        real dLdtau = gQ[3] * wT;
        for (int ch = 0; ch < 3; ++ch) B->gfeat[3 * c->g + ch] += gQ[ch] * wT;
        for (int k = 0; k < 5; ++k) suf[k] += q[k] * wT;
        /* alpha = sigma * rho (unless clamped at alpha_max) */
        real dLdD2 = 0;
        if (!c->clamped) {
            B->gsig[c->g] += dLdalpha * c->rho;
            dLdD2 = dLdalpha * G->sigma * c->rho * RL(-0.5);
        }
        /* tau = -b/a, D2 = c - b^2/a */
        real a = c->a, b = c->b;
        real dLda = dLdD2 * (b * b / (a * a)) + dLdtau * (b / (a * a));
        real dLdb = dLdD2 * (RL(-2) * b / a) + dLdtau * (RL(-1) / a);
        real dLdc = dLdD2;
        /* a = d^T A d, b = d^T A v, c = v^T A v, v = o - mu */
        real v[3] = {org[0] - G->mu[0], org[1] - G->mu[1], org[2] - G->mu[2]};
        real *gA = B->gA + 9 * c->g;
        for (int i2 = 0; i2 < 3; ++i2)
            for (int j = 0; j < 3; ++j)
                gA[3 * i2 + j] += dLda * dir[i2] * dir[j] + dLdb * dir[i2] * v[j] +
                                  dLdc * v[i2] * v[j];
        real Ad[3], Av[3];
        for (int i2 = 0; i2 < 3; ++i2) {
            Ad[i2] = G->A[3 * i2] * dir[0] + G->A[3 * i2 + 1] * dir[1] + G->A[3 * i2 + 2] * dir[2];
            Av[i2] = G->A[3 * i2] * v[0] + G->A[3 * i2 + 1] * v[1] + G->A[3 * i2 + 2] * v[2];
        }
        /* d b / d v = A d, d c / d v = 2 A v; d v / d mu = -I */
        for (int k = 0; k < 3; ++k)
            B->gmu[3 * c->g + k] -= dLdb * Ad[k] + dLdc * RL(2) * Av[k];
    }
}

/* Map gradients w.r.t. (A, mu, sigma, feature) to the raw parameters. */
static void bw_finish(const or_scene *sc, const gauss_rt *GR, const bw_ctx *B,
                      const real *ocam, int ocam_per_gauss, real beam,
                      real *gm, real *gls, real *gq, real *gop, real *gf)
{
    const int sh = sc->feature_kind == OR_FEAT_SH || sc->feature_kind == OR_FEAT_LIDAR_SH;
    int F = sh ? 3 * (sc->sh_degree + 1) * (sc->sh_degree + 1) : 3;
    for (int64_t g = 0; g < sc->n; ++g) {
        const gauss_rt *G = &GR[g];
        real q[4], qn, R[9], s[3];
        unit_quat(sc->quats + 4 * g, q, &qn);
        quat_to_R(q, R);
        for (int k = 0; k < 3; ++k) s[k] = exp(RL(sc->log_scales[3 * g + k]));
        /* actor: A_w = Ra A Ra^T and mu_w = Ra mu + t, so the gradients in the
         * Gaussian's own frame are Ra^T dL/dA_w Ra and Ra^T dL/dmu_w */
        real Ra[9], GA[9], gmw[3], gmu_w[3];
        actor_pose(sc, g, Ra, NULL);
        const real *GW = B->gA + 9 * g;
        for (int i = 0; i < 3; ++i) gmu_w[i] = B->gmu[3 * g + i];
        real Hw[9];
        if (beam > 0) {
            /* Eq. 6: A = Sigma_hat^-1, so dL/dSigma_hat = -A S A with S the
             * symmetric part of dL/dA; Sigma_hat = Sigma + delta^2 (|v|^2 I -
             * v v^T) adds delta^2 (2 v tr(H) - 2 H v) to dL/dmu (v = mu - o) */
            const real *A = G->A;
            real S[9], T[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) S[3 * i + j] = RL(0.5) * (GW[3 * i + j] + GW[3 * j + i]);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    T[3 * i + j] = S[3 * i] * A[j] + S[3 * i + 1] * A[3 + j] + S[3 * i + 2] * A[6 + j];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    Hw[3 * i + j] = -(A[3 * i] * T[j] + A[3 * i + 1] * T[3 + j] + A[3 * i + 2] * T[6 + j]);
            const real *o = origin_of(ocam, ocam_per_gauss, g);
            real v[3] = {G->mu[0] - o[0], G->mu[1] - o[1], G->mu[2] - o[2]};
            real tr = Hw[0] + Hw[4] + Hw[8], d2 = beam * beam;
            for (int i = 0; i < 3; ++i)
                gmu_w[i] += d2 * (RL(2) * v[i] * tr -
                                  RL(2) * (Hw[3 * i] * v[0] + Hw[3 * i + 1] * v[1] + Hw[3 * i + 2] * v[2]));
        } else {
            for (int i = 0; i < 9; ++i) Hw[i] = GW[i];
        }
        {
            /* Hw (dL/dA_w, or dL/dSigma_w with the filter) in the Gaussian's frame */
            real T[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    T[3 * i + j] = Hw[3 * i] * Ra[j] + Hw[3 * i + 1] * Ra[3 + j] +
                                   Hw[3 * i + 2] * Ra[6 + j];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    GA[3 * i + j] = Ra[i] * T[j] + Ra[3 + i] * T[3 + j] + Ra[6 + i] * T[6 + j];
            const real *m = gmu_w;
            for (int i = 0; i < 3; ++i) gmw[i] = Ra[i] * m[0] + Ra[3 + i] * m[1] + Ra[6 + i] * m[2];
        }
        real gR[9] = {0};
        if (beam > 0) {
            /* Sigma = sum_k s_k^2 r_k r_k^T, GA = dL/dSigma (symmetric) */
            for (int k = 0; k < 3; ++k) {
                real rk[3] = {R[k], R[3 + k], R[6 + k]}, s2 = s[k] * s[k];
                real q2 = 0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) q2 += GA[3 * i + j] * rk[i] * rk[j];
                gls[3 * g + k] += RL(2) * s2 * q2;
                for (int m = 0; m < 3; ++m) {
                    real acc = 0;
                    for (int j = 0; j < 3; ++j) acc += (GA[3 * m + j] + GA[3 * j + m]) * rk[j];
                    gR[3 * m + k] += s2 * acc;
                }
            }
        } else {
            /* A = sum_k u_k r_k r_k^T, u_k = 1/s_k^2 = exp(-2 ls_k), r_k = column k */
            for (int k = 0; k < 3; ++k) {
                real rk[3] = {R[k], R[3 + k], R[6 + k]};
                real u = RL(1) / (s[k] * s[k]);
                real dLdu = 0;
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) dLdu += GA[3 * i + j] * rk[i] * rk[j];
                gls[3 * g + k] += dLdu * RL(-2) * u;
                for (int m = 0; m < 3; ++m) {
                    real acc = 0;
                    for (int j = 0; j < 3; ++j) acc += (GA[3 * m + j] + GA[3 * j + m]) * rk[j];
                    gR[3 * m + k] += u * acc;
                }
            }
        }
        /* R(q_hat): partial derivatives of the rotation matrix entries */
        real w = q[0], x = q[1], y = q[2], z = q[3];
        real dRw[9] = {0, -z, y, z, 0, -x, -y, x, 0};
        real dRx[9] = {0, y, z, y, -2 * x, -w, z, w, -2 * x};
        real dRy[9] = {-2 * y, x, w, x, 0, z, -w, z, -2 * y};
        real dRz[9] = {-2 * z, -w, x, w, -2 * z, y, x, y, 0};
        real gqh[4] = {0, 0, 0, 0};
        for (int i = 0; i < 9; ++i) {
            gqh[0] += RL(2) * dRw[i] * gR[i];
            gqh[1] += RL(2) * dRx[i] * gR[i];
            gqh[2] += RL(2) * dRy[i] * gR[i];
            gqh[3] += RL(2) * dRz[i] * gR[i];
        }
        real dotq = gqh[0] * q[0] + gqh[1] * q[1] + gqh[2] * q[2] + gqh[3] * q[3];
        for (int i = 0; i < 4; ++i) gq[4 * g + i] += (gqh[i] - q[i] * dotq) / qn;
        gop[g] += B->gsig[g];
        for (int k = 0; k < 3; ++k) gm[3 * g + k] += gmw[k];
        const real *gc = B->gfeat + 3 * g;
        if (sh) {
            int nc = (sc->sh_degree + 1) * (sc->sh_degree + 1);
            real Y[16], dY[16][3];
            or_sh_basis(G->dir, Y);
            or_sh_basis_grad(G->dir, dY);
            const real *f = sc->features + (size_t)g * nc * 3;
            real gdir[3] = {0, 0, 0};
            for (int ch = 0; ch < 3; ++ch) {
                if (G->clampc[ch]) continue;
                for (int k = 0; k < nc; ++k) {
                    gf[(size_t)g * F + 3 * k + ch] += Y[k] * gc[ch];
                    for (int t = 0; t < 3; ++t) gdir[t] += gc[ch] * RL(f[3 * k + ch]) * dY[k][t];
                }
            }
            /* dir = Ra^T (mu_w - o)/|mu_w - o|: in the Gaussian's own frame the
             * mean's gradient has the same form as without an actor */
            real dd = gdir[0] * G->dir[0] + gdir[1] * G->dir[1] + gdir[2] * G->dir[2];
            for (int t = 0; t < 3; ++t) gm[3 * g + t] += (gdir[t] - G->dir[t] * dd) / G->dist;
        } else {
            for (int ch = 0; ch < 3; ++ch) gf[(size_t)g * F + ch] += gc[ch];
        }
    }
}

static int backward_common(const or_scene *sc, const or_opts *o, const or_proj *P,
                           const real *ocam, int ocam_per_gauss, real beam, int ntx, int nty,
                           int wrap,
                           int64_t n_total, const int64_t *rays, int64_t n_rays, ray_fn rf,
                           const void *rctx, int lidar,
                           const float *ga, const float *gb, const float *gc,
                           const float *gd, real *gm, real *gls, real *gq,
                           real *gop, real *gf)
{
    if (o->sh_per_ray) return -1;   /* forward-only reading */
    gauss_rt *GR = malloc(sizeof(gauss_rt) * (size_t)(sc->n > 0 ? sc->n : 1));
    for (int64_t g = 0; g < sc->n; ++g)
        gauss_prepare(sc, g, origin_of(ocam, ocam_per_gauss, g), beam, &GR[g]);
    bw_ctx B;
    memset(&B, 0, sizeof(B));
    B.sc = sc; B.GR = GR; B.lidar = lidar;
    B.g_a = ga; B.g_b = gb; B.g_c = gc; B.g_d = gd;
    B.gA = calloc((size_t)sc->n * 9 + 1, sizeof(real));
    B.gmu = calloc((size_t)sc->n * 3 + 1, sizeof(real));
    B.gsig = calloc((size_t)sc->n + 1, sizeof(real));
    B.gfeat = calloc((size_t)sc->n * 3 + 1, sizeof(real));
    int64_t nr = n_rays < 0 ? n_total : n_rays;
    or_ray *out = malloc(sizeof(or_ray) * (size_t)(nr > 0 ? nr : 1));
    render_common(sc, o, P, ocam, ocam_per_gauss, beam, ntx, nty, wrap, 0, rays, n_rays,
                  n_total, rf, rctx, out, bw_ray, &B);
    bw_finish(sc, GR, &B, ocam, ocam_per_gauss, beam, gm, gls, gq, gop, gf);
    free(out);
    free(B.gA); free(B.gmu); free(B.gsig); free(B.gfeat);
    free(GR);
    return 0;
}

int or_backward_camera(const or_scene *sc, const or_camera *cam, const or_opts *o,
                       const int64_t *rays, int64_t n_rays,
                       const float *g_rgb, const float *g_alpha, const float *g_depth,
                       real *gm, real *gls, real *gq, real *gop, real *gf)
{
    if (o->sh_per_ray) return -1;   /* forward-only reading */
    or_sensor_setup S;
    or_camera_setup(cam, o, &S);
    or_proj *P = malloc(sizeof(or_proj) * (size_t)(sc->n > 0 ? sc->n : 1));
    or_project_camera(sc, cam, &S, o, P);
    real *ocam = cam_sh_origins(sc, cam, P);
    cam_rctx rc = {cam, S.theta_max, o->tile, S.n_tiles_x};
    backward_common(sc, o, P, ocam, 1, 0, S.n_tiles_x, S.n_tiles_y, 0,
                    (int64_t)cam->width * cam->height, rays, n_rays, cam_ray_fn, &rc, 0, g_rgb,
                    g_alpha, g_depth, NULL, gm, gls, gq, gop, gf);
    free(ocam);
    free(P);
    or_setup_free(&S);
    return 0;
}

int or_backward_lidar(const or_scene *sc, const or_lidar *L, const or_opts *o,
                      const int64_t *rays, int64_t n_rays,
                      const float *g_range, const float *g_int, const float *g_drop,
                      const float *g_alpha, real *gm, real *gls, real *gq, real *gop,
                      real *gf)
{
    if (o->sh_per_ray) return -1;   /* forward-only reading */
    or_sensor_setup S;
    or_lidar_setup(L, &S);
    or_proj *P = malloc(sizeof(or_proj) * (size_t)(sc->n > 0 ? sc->n : 1));
    or_project_lidar(sc, L, &S, o, P);
    int *bt = malloc(sizeof(int) * L->n_beams), *ct = malloc(sizeof(int) * L->n_cols);
    lidar_ray_tiles(L, &S, bt, ct);
    lid_rctx rc = {L, &S, bt, ct};
    real *ocam = lidar_sh_origins(sc, L, P);
    backward_common(sc, o, P, ocam, 1, RL(o->beam_divergence), S.n_theta, L->n_elev_tiles, 1,
                    (int64_t)L->n_beams * L->n_cols, rays, n_rays, lid_ray_fn, &rc, 1, g_range,
                    g_int,
                    g_drop, g_alpha, gm, gls, gq, gop, gf);
    free(ocam);
    free(bt);
    free(ct);
    free(P);
    or_setup_free(&S);
    return 0;
}
