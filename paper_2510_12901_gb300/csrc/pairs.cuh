// pairs.cuh -- per-(ray, Gaussian) arithmetic shared by the forward and the
// backward kernels, so that both take exactly the same decisions (extent
// test, tau > 0, alpha cutoffs) and see the same values.
//
// Notation (render.cu explains the formulation): M = S^-1 R^T with rows M_k,
// f_k = s_k / (s_i s_j) (rows of cof(M) are f_k M_k), v = mu - o, ray
// direction d = d_T + dd (tile reference + small offset).
//   num = cof(M) (v x d)  = a + P dd          (|num|^2 / |den|^2 = D^2)
//   den = M d             = M d_T + M dd
//   tau_max = (M v) . den / |den|^2
#pragma once

#include "internal.h"

namespace sg {

// moment (mu - o) x d_T with d_T = dh + dl, mu and o floats: accurate to a
// few ulp of the result (TwoSum on mu - o, Kahan's difference of products)
__device__ __forceinline__ void precise_moment(const float mu[3], const float o[3],
                                               const float dh[3], const float dl[3],
                                               float w[3], float vh[3])
{
    float vl[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) sgd::two_diff(mu[k], o[k], vh[k], vl[k]);
    w[0] = sgd::diff_of_products(vh[1], dh[2], vh[2], dh[1]) +
           ((vh[1] * dl[2] - vh[2] * dl[1]) + (vl[1] * dh[2] - vl[2] * dh[1]));
    w[1] = sgd::diff_of_products(vh[2], dh[0], vh[0], dh[2]) +
           ((vh[2] * dl[0] - vh[0] * dl[2]) + (vl[2] * dh[0] - vl[0] * dh[2]));
    w[2] = sgd::diff_of_products(vh[0], dh[1], vh[1], dh[0]) +
           ((vh[0] * dl[1] - vh[1] * dl[0]) + (vl[0] * dh[1] - vl[1] * dh[0]));
}

__device__ __forceinline__ float dot3(const float a[3], const float b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// Camera entry, 9 float4 (one per shared-memory plane):
//   e[0..2] = (P row k, a_k)       e[3..5] = (M row k, M_k . d_T)
//   e[6]    = (M v, sigma)         e[7] = features      e[8] = extent box
// pscale multiplies the P rows and a (planes 0..2), so that |num|^2 comes
// out scaled (the forward folds -1/2 log2(e) of the response into it).
__device__ __forceinline__ void cam_entry(const GRec &r, const float o[3], const float dh[3],
                                          const float dl[3], float4 e[9], float pscale = 1.f)
{
    const float mu[3] = {r.mu_sigma.x, r.mu_sigma.y, r.mu_sigma.z};
    const float M0[3] = {r.m0.x, r.m0.y, r.m0.z}, M1[3] = {r.m1.x, r.m1.y, r.m1.z},
                M2[3] = {r.m2.x, r.m2.y, r.m2.z};
    float w[3], vh[3];
    precise_moment(mu, o, dh, dl, w, vh);
    // P rows: f_k (M_k x v), since M_k . (v x dd) = dd . (M_k x v)
    const float f0 = pscale * r.m0.w, f1 = pscale * r.m1.w, f2 = pscale * r.m2.w;
    e[0] = make_float4(f0 * (M0[1] * vh[2] - M0[2] * vh[1]), f0 * (M0[2] * vh[0] - M0[0] * vh[2]),
                       f0 * (M0[0] * vh[1] - M0[1] * vh[0]), f0 * dot3(M0, w));
    e[1] = make_float4(f1 * (M1[1] * vh[2] - M1[2] * vh[1]), f1 * (M1[2] * vh[0] - M1[0] * vh[2]),
                       f1 * (M1[0] * vh[1] - M1[1] * vh[0]), f1 * dot3(M1, w));
    e[2] = make_float4(f2 * (M2[1] * vh[2] - M2[2] * vh[1]), f2 * (M2[2] * vh[0] - M2[0] * vh[2]),
                       f2 * (M2[0] * vh[1] - M2[1] * vh[0]), f2 * dot3(M2, w));
    e[3] = make_float4(M0[0], M0[1], M0[2], dot3(M0, dh));
    e[4] = make_float4(M1[0], M1[1], M1[2], dot3(M1, dh));
    e[5] = make_float4(M2[0], M2[1], M2[2], dot3(M2, dh));
    e[6] = make_float4(dot3(M0, vh), dot3(M1, vh), dot3(M2, vh), r.mu_sigma.w);
    e[7] = r.feat;
    e[8] = r.rect;
}

struct PairEval {
    float n[3];      // num = cof(M)(v x d)
    float e[3];      // den = M d
    float inv;       // 1 / |den|^2 (fast reciprocal, within 2 ulp)
    float D2, tau, rho, alpha;
    bool clamped;    // alpha hit alpha_max
};

// Evaluate one camera pair, for an entry staged with pscale =
// sqrt(log2(e) / 2) (kResponseScale), whose extent-box test is already
// known (in_box): |num|^2 / |den|^2 is then D^2 log2(e) / 2, and rho =
// 2^-(that) (the hardware exp2, whose error is that of __expf's) without the
// two multiplies of exp(-D^2 / 2).  Returns false when the entry does not
// composite at this ray (outside the box, behind the origin, or below
// alpha_min).  The forward and the backward both decide through this
// function, so they take the same decisions; pe gets the unscaled num and
// D^2 for the gradients.  Branch-free: every value is computed and the tests
// combined at the end, so that evaluations of consecutive entries overlap.
constexpr float kResponseScale = 0.84932180028801904f;   // sqrt(log2(e) / 2)

__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ bool cam_pair_scaled(const float4 q0, const float4 q1, const float4 q2,
                                                const float4 m0, const float4 m1, const float4 m2,
                                                const float4 mv, bool in_box, const float dd[3],
                                                float alpha_min, float alpha_max, PairEval &pe)
{
    const float n0 = q0.w + q0.x * dd[0] + q0.y * dd[1] + q0.z * dd[2];
    const float n1 = q1.w + q1.x * dd[0] + q1.y * dd[1] + q1.z * dd[2];
    const float n2 = q2.w + q2.x * dd[0] + q2.y * dd[1] + q2.z * dd[2];
    pe.e[0] = m0.w + m0.x * dd[0] + m0.y * dd[1] + m0.z * dd[2];
    pe.e[1] = m1.w + m1.x * dd[0] + m1.y * dd[1] + m1.z * dd[2];
    pe.e[2] = m2.w + m2.x * dd[0] + m2.y * dd[1] + m2.z * dd[2];
    pe.inv = __fdividef(1.f, pe.e[0] * pe.e[0] + pe.e[1] * pe.e[1] + pe.e[2] * pe.e[2]);
    pe.tau = (mv.x * pe.e[0] + mv.y * pe.e[1] + mv.z * pe.e[2]) * pe.inv;
    const float d2s = (n0 * n0 + n1 * n1 + n2 * n2) * pe.inv;
    pe.rho = ex2_approx(-d2s);
    const float a = mv.w * pe.rho;
    pe.clamped = a > alpha_max;
    pe.alpha = fminf(a, alpha_max);
    constexpr float kInv = 1.f / kResponseScale;
    pe.n[0] = n0 * kInv;
    pe.n[1] = n1 * kInv;
    pe.n[2] = n2 * kInv;
    pe.D2 = d2s * (kInv * kInv);
    return in_box && pe.tau > 0.f && pe.alpha >= alpha_min;
}

// The lanes of 8x4 sub-block `sub` whose pixel centres lie in an entry's
// box, from the entry's word of tile columns and rows in the box (bits 0-15:
// the tile's columns, 16-31: its rows; written with the tile ranges by the
// same float comparisons as the per-ray test): the sub-block's 8 column bits
// in every byte, a byte kept where the sub-block's row is in the box (the
// multiply by 0x00204081 moves bit r of the 4 row bits to bit 8 r).
__device__ __forceinline__ uint32_t word_lanes(uint32_t cr, int sub)
{
    const uint32_t cols = (cr >> (8 * (sub & 1))) & 0xffu;
    const uint32_t rows = (cr >> (16 + 4 * (sub >> 1))) & 0xfu;
    return (cols * 0x01010101u) & ((((rows * 0x00204081u) & 0x01010101u)) * 0xffu);
}

// LiDAR entries keep per-column quantities (each column has its own sensor
// origin o_c), in a warp's shared block s[kLidPlanes][32] of float4:
//   planes 0..2, entry j at s[k][j]: (M row 0, sigma), (M row 1, f0),
//     (M row 2, f1)   (f: features);
//   then per entry j, quantity k and column slot sl (lid_col): k = 0..2
//   (P row k, a_k) and k = 3 (u = M v, f2), with v = mu - o_c, a = diag(f')
//   M (v x d_T) and P rows f'_k (M_k x v) as for cameras (f'_k = s_k /
//   (s_i s_j)).  The column slots of one (entry, quantity) are adjacent, so
//   the lanes of a warp, whose rays lie in different columns, read one
//   entry's quantity without bank conflicts; entries are 17 float4 apart (16
//   used), so that the lanes staging 32 entries at once write to distinct
//   banks.
constexpr int kLidEntryStride = 4 * kLidarColsMax + 1;
constexpr int kLidPlanes = (3 * 32 + 32 * kLidEntryStride + 31) / 32;   // float4 rows of 32

__device__ __forceinline__ float4 &lid_col(float4 (*s)[32], int j, int k, int sl)
{
    return (&s[0][0])[3 * 32 + j * kLidEntryStride + k * kLidarColsMax + sl];
}
// the (u, f2) quantity of entry j for the column slot of plane base sb = 3 + 4 sl
__device__ __forceinline__ float4 lid_u(float4 (*s)[32], int j, int sb)
{
    return lid_col(s, j, 3, (sb - 3) >> 2);
}

__device__ __forceinline__ void lidar_entry(const GRec &r, const float *poses, int col0,
                                            int ncols, const float dh[3], const float dl[3],
                                            float4 (*s)[32], int pos)
{
    const float mu[3] = {r.mu_sigma.x, r.mu_sigma.y, r.mu_sigma.z};
    const float M0[3] = {r.m0.x, r.m0.y, r.m0.z}, M1[3] = {r.m1.x, r.m1.y, r.m1.z},
                M2[3] = {r.m2.x, r.m2.y, r.m2.z};
    const float f0 = r.m0.w, f1 = r.m1.w, f2 = r.m2.w;
    s[0][pos] = make_float4(M0[0], M0[1], M0[2], r.mu_sigma.w);
    s[1][pos] = make_float4(M1[0], M1[1], M1[2], r.feat.x);
    s[2][pos] = make_float4(M2[0], M2[1], M2[2], r.feat.y);
    for (int sl = 0; sl < ncols; ++sl) {
        const float *Po = poses + 12 * (col0 + sl);
        const float o[3] = {Po[3], Po[7], Po[11]};
        float w[3], vh[3];
        precise_moment(mu, o, dh, dl, w, vh);
        lid_col(s, pos, 0, sl) = make_float4(f0 * (M0[1] * vh[2] - M0[2] * vh[1]),
                                             f0 * (M0[2] * vh[0] - M0[0] * vh[2]),
                                             f0 * (M0[0] * vh[1] - M0[1] * vh[0]), f0 * dot3(M0, w));
        lid_col(s, pos, 1, sl) = make_float4(f1 * (M1[1] * vh[2] - M1[2] * vh[1]),
                                             f1 * (M1[2] * vh[0] - M1[0] * vh[2]),
                                             f1 * (M1[0] * vh[1] - M1[1] * vh[0]), f1 * dot3(M1, w));
        lid_col(s, pos, 2, sl) = make_float4(f2 * (M2[1] * vh[2] - M2[2] * vh[1]),
                                             f2 * (M2[2] * vh[0] - M2[0] * vh[2]),
                                             f2 * (M2[0] * vh[1] - M2[1] * vh[0]), f2 * dot3(M2, w));
        lid_col(s, pos, 3, sl) = make_float4(dot3(M0, vh), dot3(M1, vh), dot3(M2, vh), r.feat.z);
    }
}

// Evaluate one LiDAR pair (entry j of the warp's block, planes of its
// column slot from sb = 3 + 4 sl) whose box test is already known (in_box).
__device__ __forceinline__ bool lidar_pair_in(float4 (*s)[32], int j, int sb, bool in_box,
                                              const float dd[3], const float d[3],
                                              float alpha_min, float alpha_max, PairEval &pe)
{
    // every operation spelled out (fused multiply-adds in a fixed order), so
    // that each call site computes the same bits: the forward evaluates a
    // pair in whichever lane its compaction gives it, the backward in the
    // ray's own lane
    const float4 m0 = s[0][j], m1 = s[1][j], m2 = s[2][j];
    const int sl = (sb - 3) >> 2;
    const float4 q0 = lid_col(s, j, 0, sl), q1 = lid_col(s, j, 1, sl), q2 = lid_col(s, j, 2, sl),
                 u = lid_col(s, j, 3, sl);
    pe.n[0] = __fmaf_rn(q0.z, dd[2], __fmaf_rn(q0.y, dd[1], __fmaf_rn(q0.x, dd[0], q0.w)));
    pe.n[1] = __fmaf_rn(q1.z, dd[2], __fmaf_rn(q1.y, dd[1], __fmaf_rn(q1.x, dd[0], q1.w)));
    pe.n[2] = __fmaf_rn(q2.z, dd[2], __fmaf_rn(q2.y, dd[1], __fmaf_rn(q2.x, dd[0], q2.w)));
    pe.e[0] = __fmaf_rn(m0.z, d[2], __fmaf_rn(m0.y, d[1], __fmul_rn(m0.x, d[0])));
    pe.e[1] = __fmaf_rn(m1.z, d[2], __fmaf_rn(m1.y, d[1], __fmul_rn(m1.x, d[0])));
    pe.e[2] = __fmaf_rn(m2.z, d[2], __fmaf_rn(m2.y, d[1], __fmul_rn(m2.x, d[0])));
    const float ee = __fmaf_rn(pe.e[2], pe.e[2],
                               __fmaf_rn(pe.e[1], pe.e[1], __fmul_rn(pe.e[0], pe.e[0])));
    pe.inv = __fdividef(1.f, ee);
    const float nn = __fmaf_rn(pe.n[2], pe.n[2],
                               __fmaf_rn(pe.n[1], pe.n[1], __fmul_rn(pe.n[0], pe.n[0])));
    pe.D2 = __fmul_rn(nn, pe.inv);
    const float ue = __fmaf_rn(u.z, pe.e[2], __fmaf_rn(u.y, pe.e[1], __fmul_rn(u.x, pe.e[0])));
    pe.tau = __fmul_rn(ue, pe.inv);
    pe.rho = __expf(__fmul_rn(-0.5f, pe.D2));
    const float a = __fmul_rn(m0.w, pe.rho);
    pe.clamped = a > alpha_max;
    pe.alpha = fminf(a, alpha_max);
    return in_box && pe.tau > 0.f && pe.alpha >= alpha_min;
}

// Ray set-up of a sensor whose rays have their own poses (LiDAR columns,
// rolling-shutter camera rows), shared by forward and backward: the
// reference direction of the work item (sensor-frame u under the reference
// pose Pr, double, split into two floats), the ray's offset from it under
// its own pose Pc (e: its sensor-frame offset from u) and its full
// direction.
__device__ __forceinline__ void sensor_ray(const float *Pr, double u0, double u1, double u2,
                                           const float *Pc, const float4 e, float dh[3],
                                           float dl[3], float dd[3], float d[3])
{
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        double dv = (double)Pr[4 * i] * u0 + (double)Pr[4 * i + 1] * u1 + (double)Pr[4 * i + 2] * u2;
        dh[i] = (float)dv;
        dl[i] = (float)(dv - (double)dh[i]);
    }
    const float uf[3] = {(float)u0, (float)u1, (float)u2};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        // R_c (u - u_T) + (R_c - R_ref) u_T
        dd[i] = (Pc[4 * i] * e.x + Pc[4 * i + 1] * e.y + Pc[4 * i + 2] * e.z) +
                ((Pc[4 * i] - Pr[4 * i]) * uf[0] + (Pc[4 * i + 1] - Pr[4 * i + 1]) * uf[1] +
                 (Pc[4 * i + 2] - Pr[4 * i + 2]) * uf[2]);
        d[i] = dh[i] + dd[i];
    }
}

// LiDAR ray set-up: the work item's reference column and direction.
__device__ __forceinline__ void lidar_ray(const LidarItem &it, const double *item_u, int item_id,
                                          const float *poses, const float4 e, int c, float dh[3],
                                          float dl[3], float dd[3], float d[3])
{
    sensor_ray(poses + 12 * it.ref_col, item_u[3 * item_id], item_u[3 * item_id + 1],
               item_u[3 * item_id + 2], poses + 12 * c, e, dh, dl, dd, d);
}

}  // namespace sg
