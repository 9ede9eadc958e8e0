// project.cu -- per-Gaussian projection (Sec. 3.2 camera, Sec. 3.3 LiDAR):
// activation (Sec. 3.1), the unscented transform of 7 sigma points through
// the sensor model, the extent box, the tile range, ray-based culling
// (App. B, Proc. 2-3), the depth key and the render record.
//
// One thread per Gaussian; every input plane is read once with coalesced
// 4-byte loads and every output is written once.  The kernel is bound by HBM
// traffic (about 100 bytes read and 150 written per Gaussian).
#include <math.h>

#include "internal.h"
#include "tma.cuh"

namespace sg {

struct CamParams {
    int model, W, H, ntx, nty, pose_iters;
    float fx, fy, cx, cy, k0, k1, k2, k3, theta_max;
};

struct UTParams {
    float lam_gamma, w0m, w0c, wi;   // spread sqrt(n+lambda) and the weights
    float alpha_min, near_dist;
    float beam;                      // LiDAR beam divergence (radians), 0 = off
};

static UTParams ut_params(const sg_render_opts &o)
{
    UTParams u;
    const float n = 3.0f;
    float a = o.ut_alpha, k = o.ut_kappa, b = o.ut_beta;
    float lam = a * a * (n + k) - n;
    u.lam_gamma = sqrtf(n + lam);
    u.w0m = lam / (n + lam);
    u.w0c = u.w0m + (1.0f - a * a + b);
    u.wi = 1.0f / (2.0f * (n + lam));
    u.alpha_min = o.alpha_min;
    u.near_dist = o.near_dist;
    u.beam = o.beam_divergence;
    return u;
}

struct Activated {
    float mu[3], R[9], s[3], sigma;
};

__device__ __forceinline__ Activated activate(const float *__restrict__ planes, int64_t pitch,
                                              int64_t g)
{
    Activated a;
    for (int k = 0; k < 3; ++k) {
        a.mu[k] = planes[(Scene::kMean + k) * pitch + g];
        a.s[k] = expf(planes[(Scene::kLogScale + k) * pitch + g]);
    }
    float qw = planes[(Scene::kQuat + 0) * pitch + g], qx = planes[(Scene::kQuat + 1) * pitch + g];
    float qy = planes[(Scene::kQuat + 2) * pitch + g], qz = planes[(Scene::kQuat + 3) * pitch + g];
    float qn = sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw /= qn; qx /= qn; qy /= qn; qz /= qn;
    a.R[0] = 1.f - 2.f * (qy * qy + qz * qz);
    a.R[1] = 2.f * (qx * qy - qw * qz);
    a.R[2] = 2.f * (qx * qz + qw * qy);
    a.R[3] = 2.f * (qx * qy + qw * qz);
    a.R[4] = 1.f - 2.f * (qx * qx + qz * qz);
    a.R[5] = 2.f * (qy * qz - qw * qx);
    a.R[6] = 2.f * (qx * qz - qw * qy);
    a.R[7] = 2.f * (qy * qz + qw * qx);
    a.R[8] = 1.f - 2.f * (qx * qx + qy * qy);
    a.sigma = planes[Scene::kOpacity * pitch + g];
    return a;
}

// Dynamic actors (Sec. 3.1 scene graph): the pose of Gaussian g's actor,
// rows of [R | t] (actor to world); false for the static background.
__device__ __forceinline__ bool actor_of(const ActorParams &A, int64_t g, float4 P[3])
{
    const int k = A.of ? A.of[g] : -1;
    if (k < 0 || k >= A.n) return false;
    const float4 *p = reinterpret_cast<const float4 *>(A.poses) + 3 * k;
    P[0] = __ldg(p);
    P[1] = __ldg(p + 1);
    P[2] = __ldg(p + 2);
    return true;
}

// Mean and rotation of an actor's Gaussian to the world: mu_w = Ra mu + t,
// R_w = Ra R.
__device__ __forceinline__ void to_world(const ActorParams &A, int64_t g, Activated &a)
{
    float4 P[3];
    if (!actor_of(A, g, P)) return;
    const float Ra[9] = {P[0].x, P[0].y, P[0].z, P[1].x, P[1].y, P[1].z, P[2].x, P[2].y, P[2].z};
    const float m[3] = {a.mu[0], a.mu[1], a.mu[2]};
    const float t[3] = {P[0].w, P[1].w, P[2].w};
    float R[9];
    for (int i = 0; i < 3; ++i) {
        a.mu[i] = Ra[3 * i] * m[0] + Ra[3 * i + 1] * m[1] + Ra[3 * i + 2] * m[2] + t[i];
        for (int j = 0; j < 3; ++j)
            R[3 * i + j] = Ra[3 * i] * a.R[j] + Ra[3 * i + 1] * a.R[3 + j] + Ra[3 * i + 2] * a.R[6 + j];
    }
    for (int i = 0; i < 9; ++i) a.R[i] = R[i];
}

// A world direction in the frame of Gaussian g's actor (Ra^T d), where its
// SH are defined; unchanged for the static background.
__device__ __forceinline__ void dir_to_actor(const ActorParams &A, int64_t g, float d[3])
{
    float4 P[3];
    if (!actor_of(A, g, P)) return;
    const float x = d[0], y = d[1], z = d[2];
    d[0] = P[0].x * x + P[1].x * y + P[2].x * z;
    d[1] = P[0].y * x + P[1].y * y + P[2].y * z;
    d[2] = P[0].z * x + P[1].z * y + P[2].z * z;
}

// Render record: M = S^-1 R^T (row i = column i of R over s_i) and the
// cofactor weights f_i = s_i / (s_j s_k) (row i of cof(M) = f_i M_i).
__device__ __forceinline__ void write_record(GRec *rec, int64_t g, const Activated &a,
                                             float f0, float f1, float f2, float4 rect,
                                             float fw = 0.f)
{
    GRec r;
    r.mu_sigma = make_float4(a.mu[0], a.mu[1], a.mu[2], a.sigma);
    float i0 = 1.f / a.s[0], i1 = 1.f / a.s[1], i2 = 1.f / a.s[2];
    r.m0 = make_float4(a.R[0] * i0, a.R[3] * i0, a.R[6] * i0, a.s[0] / (a.s[1] * a.s[2]));
    r.m1 = make_float4(a.R[1] * i1, a.R[4] * i1, a.R[7] * i1, a.s[1] / (a.s[0] * a.s[2]));
    r.m2 = make_float4(a.R[2] * i2, a.R[5] * i2, a.R[8] * i2, a.s[2] / (a.s[0] * a.s[1]));
    r.feat = make_float4(f0, f1, f2, fw);
    r.rect = rect;
    rec[g] = r;
}

// Real spherical harmonics of degree <= 3 (normalised, Condon-Shortley
// phase, m = -l..l order).  Constants: sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!),
// times sqrt(2) for m != 0, times the leading factor of P_l^|m|.
// base[(3 k + ch) stride]: coefficient k of channel ch (the Gaussian's entry
// of the SH planes, in global memory or staged in shared memory).
__device__ __forceinline__ void sh_eval(const float *__restrict__ base, int64_t stride, int deg,
                                        float x, float y, float z, float c[3])
{
    float Y[16];
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = 0.28209479177387814f;
    if (deg >= 1) {
        Y[1] = -0.48860251190291992f * y;
        Y[2] = 0.48860251190291992f * z;
        Y[3] = -0.48860251190291992f * x;
    }
    if (deg >= 2) {
        Y[4] = 1.0925484305920792f * x * y;
        Y[5] = -1.0925484305920792f * y * z;
        Y[6] = 0.31539156525252005f * (2.f * zz - xx - yy);
        Y[7] = -1.0925484305920792f * x * z;
        Y[8] = 0.54627421529603959f * (xx - yy);
    }
    if (deg >= 3) {
        Y[9] = -0.59004358992664352f * y * (3.f * xx - yy);
        Y[10] = 2.8906114426405538f * x * y * z;
        Y[11] = -0.45704579946446572f * y * (4.f * zz - xx - yy);
        Y[12] = 0.37317633259011540f * z * (2.f * zz - 3.f * xx - 3.f * yy);
        Y[13] = -0.45704579946446572f * x * (4.f * zz - xx - yy);
        Y[14] = 1.4453057213202769f * z * (xx - yy);
        Y[15] = -0.59004358992664352f * x * (xx - 3.f * yy);
    }
    // unrolled over the 16 coefficients (predicated by the degree), so that a
    // channel's loads are all in flight at once rather than one per FMA
    const int nc = (deg + 1) * (deg + 1);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float f[16];
#pragma unroll
        for (int k = 0; k < 16; ++k)
            f[k] = k < nc ? base[(3 * k + ch) * stride] : 0.f;
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 16; ++k) acc += k < nc ? Y[k] * f[k] : 0.f;
        c[ch] = acc;
    }
}

// Pixel of a world point; returns false outside the model's domain
// (pinhole: z > near; fisheye: |x| > near and theta <= theta_max).
// c2w: row-major [R | t] camera-to-world pose (shared memory).
__device__ __forceinline__ bool cam_point(const CamParams &C, const float *c2w, float near_dist,
                                          const float x[3], float &u, float &v)
{
    float d0 = x[0] - c2w[3], d1 = x[1] - c2w[7], d2 = x[2] - c2w[11];
    float xc = c2w[0] * d0 + c2w[4] * d1 + c2w[8] * d2;
    float yc = c2w[1] * d0 + c2w[5] * d1 + c2w[9] * d2;
    float zc = c2w[2] * d0 + c2w[6] * d1 + c2w[10] * d2;
    if (C.model == SG_CAMERA_PINHOLE) {
        if (!(zc > near_dist)) return false;
        u = C.fx * xc / zc + C.cx;
        v = C.fy * yc / zc + C.cy;
        return true;
    }
    float r = sqrtf(xc * xc + yc * yc);
    float dist = sqrtf(xc * xc + yc * yc + zc * zc);
    float th = atan2f(r, zc);
    if (!(dist > near_dist) || !(th <= C.theta_max)) return false;
    float t2 = th * th;
    float thd = th * (1.f + t2 * (C.k0 + t2 * (C.k1 + t2 * (C.k2 + t2 * C.k3))));
    if (r > 0.f) {
        u = C.fx * (thd / r) * xc + C.cx;
        v = C.fy * (thd / r) * yc + C.cy;
    } else {
        u = C.cx;
        v = C.cy;
    }
    return true;
}

// Testing hook (sg_debug_bulk_wait): non-zero makes the projection's first
// wait for its bulk copies give up at once, so that the status path runs;
// the wait that follows (before any staged value is read and before the
// block exits) keeps its full bound.  In device memory, so that replays of
// captured launch sequences see it.
__device__ uint32_t g_bulk_give_up = 0u;

// The block's bulk copies: false if the first wait gave up (the status word
// is then set and a second bounded wait follows).
__device__ __forceinline__ void bulk_wait(uint64_t *bar, uint32_t *status)
{
    const bool forced = *(volatile uint32_t *)&g_bulk_give_up != 0u;
    if (forced || !mbar_wait(bar, 0)) {
        atomicOr(status, kStatusBulkCopy);
        mbar_wait(bar, 0);
    }
}

#ifndef SG_PROJ_MINB
#define SG_PROJ_MINB 4
#endif
// Rolling shutter: the pose of the pixel row that sees x, found from the
// middle row by taking the row x projects to, pose_iters times (clamped to
// the image; an iterate outside the model's domain stops the iteration).
__device__ __forceinline__ int cam_row(const CamParams &C, const float *poses, float near_dist,
                                       const float x[3])
{
    int row = C.H / 2;
    for (int it = 0; it < C.pose_iters; ++it) {
        float u, v;
        if (!cam_point(C, poses + 12 * row, near_dist, x, u, v)) break;
        row = v < 0.f ? 0 : (v >= (float)C.H ? C.H - 1 : (int)floorf(v));
    }
    return row;
}

// kRS: rolling shutter, the RenderDesc's poses are per pixel row; each point
// (the mean and every sigma point) takes the pose of its row, and the row of
// the mean goes into the record (the backward's SH origin).
template <bool kRS>
__global__ void __launch_bounds__(256, SG_PROJ_MINB)
k_project_camera(const float *__restrict__ planes, int64_t pitch, int64_t n, int feature_kind,
                 int sh_degree, ActorParams A, CamParams C, const RenderDesc *__restrict__ D,
                 UTParams U,
                 GRec *__restrict__ rec,
                 float4 *__restrict__ rect_out, int4 *__restrict__ tiles_out,
                 float *__restrict__ depth_out, uint32_t *__restrict__ count_out,
                 float2 *__restrict__ mean_out, float4 *__restrict__ cov_out,
                 uint32_t *__restrict__ status)
{
    __shared__ float s_c2w[12];   // the pose, from the render's descriptor
    // SH features: the block's run of every coefficient plane, [plane][thread],
    // brought in by bulk copies (TMA) while the sigma points are projected
    extern __shared__ float s_feat[];
    __shared__ uint64_t s_bar;
    const int n_stage =
        feature_kind == SG_FEATURES_SH ? 3 * (sh_degree + 1) * (sh_degree + 1) : 0;
    if (threadIdx.x < 12) s_c2w[threadIdx.x] = D->c2w[threadIdx.x];
    if (threadIdx.x == 0 && n_stage) mbar_init(&s_bar);
    __syncthreads();
    const int64_t g0 = (int64_t)blockIdx.x * blockDim.x;
    if (threadIdx.x == 0 && n_stage) {
        // planes are 128-byte aligned and pitch floats long (a multiple of
        // 32), so each run starts 16-byte aligned and ends inside its plane
        const int64_t run = pitch - g0 < (int64_t)blockDim.x ? pitch - g0 : (int64_t)blockDim.x;
        const uint32_t bytes = 4u * (uint32_t)run;
        mbar_arrive_expect(&s_bar, bytes * (uint32_t)n_stage);
        for (int p = 0; p < n_stage; ++p)
            bulk_copy_g2s(s_feat + p * blockDim.x, planes + (Scene::kFeat + p) * pitch + g0, bytes,
                          &s_bar);
    }
    int64_t g = g0 + threadIdx.x;
    if (g == 0) *status = 0u;     // a new render: no device wait has given up
    if (g >= n) return;           // (thread 0 of a block always has a Gaussian)
    const float *poses = kRS ? D->poses : nullptr;
    Activated a = activate(planes, pitch, g);
    to_world(A, g, a);
    // the mean's pose: the camera's, or that of the row that sees the mean
    int row0 = 0;
    const float *P0 = s_c2w;
    if constexpr (kRS) {
        row0 = cam_row(C, poses, U.near_dist, a.mu);
        P0 = poses + 12 * row0;
    }
    float dx = a.mu[0] - P0[3], dy = a.mu[1] - P0[7], dz = a.mu[2] - P0[11];
    float dist = sqrtf(dx * dx + dy * dy + dz * dz);
    depth_out[g] = dist;
    uint32_t count = 0;
    float4 rect = make_float4(0.f, 0.f, 0.f, 0.f);
    int4 tl = make_int4(0, -1, 0, -1);
    float2 m2 = make_float2(0.f, 0.f);
    float4 cv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (a.sigma >= U.alpha_min) {
        // sigma points chi_0 = mu, chi_{+-i} = mu +- sqrt(n+lambda) s_i R e_i
        float uu[7], vv[7];
        bool ok = cam_point(C, P0, U.near_dist, a.mu, uu[0], vv[0]);
#pragma unroll
        for (int p = 1; p < 7; ++p) {
            int i = (p - 1) >> 1;
            float sg = ((p - 1) & 1) ? -1.f : 1.f;
            float x[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) x[r] = a.mu[r] + sg * U.lam_gamma * a.s[i] * a.R[3 * r + i];
            const float *Pp = s_c2w;
            if constexpr (kRS) Pp = poses + 12 * cam_row(C, poses, U.near_dist, x);
            ok = cam_point(C, Pp, U.near_dist, x, uu[p], vv[p]) && ok;
        }
        if (ok) {
            float mu_u = U.w0m * uu[0], mu_v = U.w0m * vv[0];
#pragma unroll
            for (int p = 1; p < 7; ++p) { mu_u += U.wi * uu[p]; mu_v += U.wi * vv[p]; }
            float cxx = 0.f, cxy = 0.f, cyy = 0.f;
#pragma unroll
            for (int p = 0; p < 7; ++p) {
                float w = p == 0 ? U.w0c : U.wi;
                float eu = uu[p] - mu_u, ev = vv[p] - mu_v;
                cxx += w * eu * eu;
                cxy += w * eu * ev;
                cyy += w * ev * ev;
            }
            // extent: the k-sigma box, k = sqrt(2 ln(sigma / alpha_min))
            float k = sqrtf(2.f * logf(a.sigma / U.alpha_min));
            float hx = k * sqrtf(cxx), hy = k * sqrtf(cyy);
            rect = make_float4(mu_u - hx, mu_u + hx, mu_v - hy, mu_v + hy);
            m2 = make_float2(mu_u, mu_v);
            cv = make_float4(cxx, cxy, cyy, 0.f);
            if (rect.y >= 0.f && rect.x < (float)C.W && rect.w >= 0.f && rect.z < (float)C.H) {
                int x0 = rect.x <= 0.f ? 0 : (int)floorf(rect.x / (float)kTile);
                int x1 = rect.y >= (float)C.W ? C.ntx - 1 : (int)floorf(rect.y / (float)kTile);
                int y0 = rect.z <= 0.f ? 0 : (int)floorf(rect.z / (float)kTile);
                int y1 = rect.w >= (float)C.H ? C.nty - 1 : (int)floorf(rect.w / (float)kTile);
                x1 = min(x1, C.ntx - 1);
                y1 = min(y1, C.nty - 1);
                tl = make_int4(x0, x1, y0, y1);
                count = (uint32_t)((x1 - x0 + 1) * (y1 - y0 + 1));
            }
        }
    }
    count_out[g] = count;
    rect_out[g] = rect;
    tiles_out[g] = tl;
    mean_out[g] = m2;
    cov_out[g] = cv;
    if (count == 0) {
        // the block's copies land before its last thread leaves
        if (threadIdx.x == 0 && n_stage) bulk_wait(&s_bar, status);
        return;
    }
    float c[3];
    if (feature_kind == SG_FEATURES_SH) {
        bulk_wait(&s_bar, status);
        float inv = 1.f / dist;
        float d[3] = {dx * inv, dy * inv, dz * inv};
        dir_to_actor(A, g, d);
        sh_eval(s_feat + threadIdx.x, blockDim.x, sh_degree, d[0], d[1], d[2], c);
        for (int ch = 0; ch < 3; ++ch) c[ch] = fmaxf(c[ch] + 0.5f, 0.f);   // colour offset, clamp
    } else {
        for (int ch = 0; ch < 3; ++ch) c[ch] = planes[(Scene::kFeat + ch) * pitch + g];
    }
    write_record(rec, g, a, c[0], c[1], c[2], rect, __uint_as_float((uint32_t)row0));
}

sg_status project_camera(const Scene &sc, const Camera &cam, const sg_render_opts &o, Frame &fr,
                         cudaStream_t st, bool rolling)
{
    CamParams C;
    C.model = cam.model;
    C.W = cam.width;
    C.H = cam.height;
    C.ntx = cam.ntx;
    C.nty = cam.nty;
    C.fx = cam.fx; C.fy = cam.fy; C.cx = cam.cx; C.cy = cam.cy;
    C.k0 = cam.k[0]; C.k1 = cam.k[1]; C.k2 = cam.k[2]; C.k3 = cam.k[3];
    C.theta_max = (float)cam.theta_max;
    C.pose_iters = o.pose_iters;
    UTParams U = ut_params(o);
    if (sc.n == 0) return SG_OK;
    unsigned grid = (unsigned)((sc.n + 255) / 256);
    auto kern = rolling ? k_project_camera<true> : k_project_camera<false>;
    // shared memory for the SH planes the kernel stages (48 KB at degree 3)
    const int n_stage =
        sc.feature_kind == SG_FEATURES_SH ? 3 * (sc.sh_degree + 1) * (sc.sh_degree + 1) : 0;
    const size_t smem = sizeof(float) * 256 * (size_t)n_stage;
    static bool attr_set[2] = {false, false};
    if (!attr_set[rolling ? 1 : 0]) {
        SG_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(sizeof(float) * 256 * 48)));
        attr_set[rolling ? 1 : 0] = true;
    }
    kern<<<grid, 256, smem, st>>>(
        sc.d_planes, sc.pitch, sc.n, sc.feature_kind, sc.sh_degree, actor_params(sc), C,
        (const RenderDesc *)fr.desc.p, U, (GRec *)fr.rec.p,
        (float4 *)fr.rect.p, (int4 *)fr.tiles.p, (float *)fr.depth.p, (uint32_t *)fr.count.p,
        (float2 *)fr.mean2d.p, (float4 *)fr.cov2d.p, (uint32_t *)fr.scalars.p + kScalStatus);
    SG_LAUNCHED();
    return SG_OK;
}

// ------------------------------------------------------------------ LiDAR

struct LidParams {
    int n_cols, nphi, n_theta, A, per, pose_iters;
    float az0, T0, TN;
    const float *T;
    const int *sat;
    const float *poses;   // [n_cols*12], set in the kernel from the render's descriptor
};

__device__ __forceinline__ int pmod(int a, int n)
{
    int m = a % n;
    return m < 0 ? m + n : m;
}

// sensor-frame coordinates of x under the column pose P (row-major 3x4
// c2w, 16-byte aligned: three float4 loads)
__device__ __forceinline__ void to_sensor(const float *__restrict__ P, const float x[3],
                                          float xs[3])
{
    const float4 r0 = __ldg(reinterpret_cast<const float4 *>(P));
    const float4 r1 = __ldg(reinterpret_cast<const float4 *>(P) + 1);
    const float4 r2 = __ldg(reinterpret_cast<const float4 *>(P) + 2);
    float d0 = x[0] - r0.w, d1 = x[1] - r1.w, d2 = x[2] - r2.w;
    xs[0] = r0.x * d0 + r1.x * d1 + r2.x * d2;
    xs[1] = r0.y * d0 + r1.y * d1 + r2.y * d2;
    xs[2] = r0.z * d0 + r1.z * d1 + r2.z * d2;
}

__device__ __forceinline__ int col_of_az(const LidParams &L, float az)
{
    return pmod((int)floorf((az - L.az0) * ((float)L.n_cols / 360.0f)), L.n_cols);
}

// Column whose pose sees the point: start at mid-sweep, then take the
// column of the point's azimuth `pose_iters` times; xs = the point in that
// column's sensor frame and *az_deg its azimuth there.  The point is
// transformed again only when the column changes, and the last azimuth is
// reused when the last step kept the column (the same values as
// transforming and measuring anew).
__device__ __forceinline__ int lidar_col(const LidParams &L, const float x[3], float xs[3],
                                         float *az_deg)
{
    int col = L.n_cols / 2;
    to_sensor(L.poses + 12 * col, x, xs);
    bool fresh = false;          // *az_deg belongs to the current xs
    for (int it = 0; it < L.pose_iters; ++it) {
        *az_deg = atan2f(xs[1], xs[0]) * 57.295779513082321f;
        const int c2 = col_of_az(L, *az_deg);
        fresh = c2 == col;
        if (!fresh) {
            col = c2;
            to_sensor(L.poses + 12 * col, x, xs);
        }
    }
    if (!fresh) *az_deg = atan2f(xs[1], xs[0]) * 57.295779513082321f;
    return col;
}

__device__ __forceinline__ int elev_tile(const LidParams &L, float el)
{
    int lo = 1, hi = L.nphi - 1, e = 0;
    while (lo <= hi) {
        int m = (lo + hi) >> 1;
        if (L.T[m] <= el) { e = m; lo = m + 1; } else hi = m - 1;
    }
    return e;
}

__device__ __forceinline__ int elev_cell(const LidParams &L, float el)
{
    int e = elev_tile(L, el);
    float f = (el - L.T[e]) / (L.T[e + 1] - L.T[e]) * (float)L.per;
    int sub = !(f >= 0.f) ? 0 : (f >= (float)L.per ? L.per - 1 : (int)floorf(f));
    return e * L.per + min(sub, L.per - 1);
}

__device__ __forceinline__ int sat_count(const LidParams &L, int x0, int x1, int y0, int y1)
{
    const int H = L.nphi * L.per + 1;
    return L.sat[(x1 + 1) * H + (y1 + 1)] - L.sat[x0 * H + (y1 + 1)] -
           L.sat[(x1 + 1) * H + y0] + L.sat[x0 * H + y0];
}

// Proc. 2 RayOccupancyCount with an azimuth range split at the seam.
__device__ __forceinline__ int sat_count_wrap(const LidParams &L, int x0, int x1, int y0, int y1)
{
    if (x1 - x0 + 1 >= L.A) return sat_count(L, 0, L.A - 1, y0, y1);
    int a = pmod(x0, L.A), b = pmod(x1, L.A);
    if (a <= b) return sat_count(L, a, b, y0, y1);
    return sat_count(L, a, L.A - 1, y0, y1) + sat_count(L, 0, b, y0, y1);
}

// Beam divergence (Sec. 3.3, Eq. 6): the smoothed covariance
// Sigma + delta^2 (|v|^2 I - v v^T) of a LiDAR Gaussian with world rotation
// R and scales s, v = mu - o (o the origin of mu's column pose).
__device__ __forceinline__ void smoothed_cov(const float R[9], const float s[3],
                                             const float v[3], float delta, float C[9])
{
    const float vv = v[0] * v[0] + v[1] * v[1] + v[2] * v[2], d2 = delta * delta;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < 3; ++k) acc += R[3 * i + k] * (s[k] * s[k]) * R[3 * j + k];
            C[3 * i + j] = acc + d2 * ((i == j ? vv : 0.f) - v[i] * v[j]);
        }
}

// Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations
// (each zeroes one off-diagonal entry; Golub & Van Loan, Sec. 8.5): C is
// overwritten, Q gets the eigenvectors as columns, lam the eigenvalues.
__device__ __forceinline__ void jacobi_eigen3(float C[9], float Q[9], float lam[3])
{
#pragma unroll
    for (int i = 0; i < 9; ++i) Q[i] = (i % 4 == 0) ? 1.f : 0.f;
    for (int sweep = 0; sweep < 6; ++sweep) {
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int p = r == 2 ? 1 : 0, q = r == 0 ? 1 : 2;
            const float apq = C[3 * p + q];
            if (fabsf(apq) <= 1e-30f) continue;
            const float theta = (C[3 * q + q] - C[3 * p + p]) / (2.f * apq);
            const float t = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
            const float c = 1.f / sqrtf(t * t + 1.f), sn = t * c;
            // C <- J^T C J, J the rotation in the (p, q) plane
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float ckp = C[3 * k + p], ckq = C[3 * k + q];
                C[3 * k + p] = c * ckp - sn * ckq;
                C[3 * k + q] = sn * ckp + c * ckq;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float cpk = C[3 * p + k], cqk = C[3 * q + k];
                C[3 * p + k] = c * cpk - sn * cqk;
                C[3 * q + k] = sn * cpk + c * cqk;
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float qkp = Q[3 * k + p], qkq = Q[3 * k + q];
                Q[3 * k + p] = c * qkp - sn * qkq;
                Q[3 * k + q] = sn * qkp + c * qkq;
            }
        }
    }
    lam[0] = fmaxf(C[0], 1e-30f);
    lam[1] = fmaxf(C[4], 1e-30f);
    lam[2] = fmaxf(C[8], 1e-30f);
}

// Lower Cholesky factor (row-major) of a symmetric positive definite 3x3.
__device__ __forceinline__ void cholesky3(const float C[9], float Lc[9])
{
    const float l00 = sqrtf(fmaxf(C[0], 1e-30f));
    const float l10 = C[3] / l00, l20 = C[6] / l00;
    const float l11 = sqrtf(fmaxf(C[4] - l10 * l10, 1e-30f));
    const float l21 = (C[7] - l20 * l10) / l11;
    const float l22 = sqrtf(fmaxf(C[8] - l20 * l20 - l21 * l21, 1e-30f));
    Lc[0] = l00; Lc[1] = 0.f; Lc[2] = 0.f;
    Lc[3] = l10; Lc[4] = l11; Lc[5] = 0.f;
    Lc[6] = l20; Lc[7] = l21; Lc[8] = l22;
}

// kSH: the scene carries SH^l features; kBeam: beam divergence on (the UT
// runs over the smoothed covariance's Cholesky columns, and the record
// holds its eigen-frame: M = diag(lam)^-1/2 Q^T, the form the compositing
// takes).  Templates, so that the plain path keeps its registers.  Four
// blocks per SM (64 registers, a few bytes spilled): the kernel waits on
// dependent pose loads and atan2f / asinf chains, and 32 warps per SM hide
// more of that than 24 at 76 registers (street sweep, 2M Gaussians: 0.266 ->
// 0.253 ms; with SH^l features 0.400 -> 0.337 ms; beam divergence 0.435 ->
// 0.407 ms).
template <bool kSH, bool kBeam>
__global__ void __launch_bounds__(256, 4)
k_project_lidar(const float *__restrict__ planes, int64_t pitch, int64_t n, int sh_degree,
                ActorParams A, LidParams Lp, const RenderDesc *__restrict__ D, UTParams U,
                int cull, GRec *__restrict__ rec, float4 *__restrict__ rect_out,
                int4 *__restrict__ tiles_out, float *__restrict__ depth_out,
                uint32_t *__restrict__ count_out, float2 *__restrict__ mean_out,
                float4 *__restrict__ cov_out, uint32_t *__restrict__ status)
{
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g == 0) *status = 0u;     // a new render: no look-back wait has given up
    if (g >= n) return;
    LidParams L = Lp;
    L.poses = D->poses;
    Activated a = activate(planes, pitch, g);
    to_world(A, g, a);
    float xs0[3], az0;               // chi_0 = mu, also the depth key
    const int col0 = lidar_col(L, a.mu, xs0, &az0);
    const float r0 = sqrtf(xs0[0] * xs0[0] + xs0[1] * xs0[1] + xs0[2] * xs0[2]);
    depth_out[g] = r0;
    uint32_t count = 0;
    float4 rect = make_float4(0.f, 0.f, 0.f, 0.f);
    int4 tl = make_int4(0, -1, 0, -1);
    float2 m2 = make_float2(0.f, 0.f);
    float4 cv = make_float4(0.f, 0.f, 0.f, 0.f);
    // sigma-point directions: the columns of R diag(s), or of the Cholesky
    // factor of the smoothed covariance
    float Dm[9];
    if constexpr (kBeam) {
        const float *P = L.poses + 12 * col0;
        const float v[3] = {a.mu[0] - P[3], a.mu[1] - P[7], a.mu[2] - P[11]};
        float Cs[9], lam[3];
        smoothed_cov(a.R, a.s, v, U.beam, Cs);
        cholesky3(Cs, Dm);
        jacobi_eigen3(Cs, a.R, lam);
#pragma unroll
        for (int k = 0; k < 3; ++k) a.s[k] = sqrtf(lam[k]);
    } else {
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int i = 0; i < 3; ++i) Dm[3 * r + i] = a.s[i] * a.R[3 * r + i];
    }
    if (a.sigma >= U.alpha_min) {
        float az[7], el[7];
        bool ok = true;
        ok = r0 > U.near_dist;
        az[0] = az0;
        el[0] = asinf(xs0[2] / r0) * 57.295779513082321f;
#pragma unroll
        for (int p = 1; p < 7; ++p) {
            const int i = (p - 1) >> 1;
            const float sg = ((p - 1) & 1) ? -1.f : 1.f;
            float x[3], xs[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) x[r] = a.mu[r] + sg * U.lam_gamma * Dm[3 * r + i];
            lidar_col(L, x, xs, &az[p]);
            const float r = sqrtf(xs[0] * xs[0] + xs[1] * xs[1] + xs[2] * xs[2]);
            ok = ok && (r > U.near_dist);
            el[p] = asinf(xs[2] / r) * 57.295779513082321f;
        }
        if (ok) {
#pragma unroll
            for (int p = 1; p < 7; ++p) {   // unwrap to within 180 deg of chi_0
                float d = az[p] - az[0];
                if (d > 180.f) az[p] -= 360.f;
                else if (d < -180.f) az[p] += 360.f;
            }
            float ma = U.w0m * az[0], me = U.w0m * el[0];
#pragma unroll
            for (int p = 1; p < 7; ++p) { ma += U.wi * az[p]; me += U.wi * el[p]; }
            float caa = 0.f, cae = 0.f, cee = 0.f;
#pragma unroll
            for (int p = 0; p < 7; ++p) {
                float w = p == 0 ? U.w0c : U.wi;
                float ea = az[p] - ma, ee = el[p] - me;
                caa += w * ea * ea;
                cae += w * ea * ee;
                cee += w * ee * ee;
            }
            float k = sqrtf(2.f * logf(a.sigma / U.alpha_min));
            float ha = k * sqrtf(caa), he = k * sqrtf(cee);
            rect = make_float4(ma - ha, ma + ha, me - he, me + he);
            m2 = make_float2(ma, me);
            cv = make_float4(caa, cae, cee, 0.f);
            if (rect.w >= L.T0 && rect.z <= L.TN) {
                float elo = rect.z < L.T0 ? L.T0 : rect.z;
                float ehi = rect.w > L.TN ? L.TN : rect.w;
                int e0 = elev_tile(L, elo), e1 = elev_tile(L, ehi);
                bool full = !(rect.y - rect.x < 360.f);
                int a0, a1, na;
                if (full) {
                    a0 = 0; a1 = L.n_theta - 1; na = L.n_theta;
                } else {
                    float sc = (float)L.n_theta / 360.0f;
                    a0 = (int)floorf((rect.x - L.az0) * sc);
                    a1 = (int)floorf((rect.y - L.az0) * sc);
                    na = a1 - a0 + 1;
                    if (na > L.n_theta) { na = L.n_theta; a1 = a0 + L.n_theta - 1; }
                }
                bool keep = true;
                if (cull) {   // App. B Proc. 3: keep only if the dense extent holds a ray
                    int x0, x1;
                    if (full) { x0 = 0; x1 = L.A - 1; }
                    else {
                        float sc = (float)L.A / 360.0f;
                        x0 = (int)floorf((rect.x - L.az0) * sc);
                        x1 = (int)floorf((rect.y - L.az0) * sc);
                    }
                    keep = sat_count_wrap(L, x0, x1, elev_cell(L, elo), elev_cell(L, ehi)) > 0;
                }
                if (keep) {
                    tl = make_int4(a0, a1, e0, e1);
                    count = (uint32_t)(na * (e1 - e0 + 1));
                }
            }
        }
    }
    count_out[g] = count;
    rect_out[g] = rect;
    tiles_out[g] = tl;
    mean_out[g] = m2;
    cov_out[g] = cv;
    if (count == 0) return;
    if constexpr (kSH) {
        // SH^l at the direction from the origin of mu's column pose to mu;
        // the column goes into the record for the backward
        const float *P = L.poses + 12 * col0;
        const float vx = a.mu[0] - P[3], vy = a.mu[1] - P[7], vz = a.mu[2] - P[11];
        const float inv = 1.f / sqrtf(vx * vx + vy * vy + vz * vz);
        float d[3] = {vx * inv, vy * inv, vz * inv}, c[3];
        dir_to_actor(A, g, d);
        sh_eval(planes + Scene::kFeat * pitch + g, pitch, sh_degree, d[0], d[1], d[2], c);
        write_record(rec, g, a, c[0], c[1], c[2], rect, __uint_as_float((uint32_t)col0));
        return;
    }
    // the column of mu's pose goes into the record (the backward's origin)
    write_record(rec, g, a, planes[(Scene::kFeat + 0) * pitch + g],
                 planes[(Scene::kFeat + 1) * pitch + g], planes[(Scene::kFeat + 2) * pitch + g],
                 rect, __uint_as_float((uint32_t)col0));
}

sg_status project_lidar(const Scene &sc, const Lidar &Ld, const sg_render_opts &o, Frame &fr,
                        cudaStream_t st)
{
    LidParams L;
    L.n_cols = Ld.n_cols;
    L.nphi = Ld.nphi;
    L.n_theta = Ld.n_theta;
    L.A = Ld.cull_az;
    L.per = Ld.cull_el;
    L.pose_iters = o.pose_iters;
    L.az0 = Ld.az0;
    L.T0 = Ld.T[0];
    L.TN = Ld.T[Ld.nphi];
    L.T = Ld.d_T;
    L.sat = Ld.d_sat;
    L.poses = nullptr;
    UTParams U = ut_params(o);
    if (sc.n == 0) return SG_OK;
    unsigned grid = (unsigned)((sc.n + 255) / 256);
    const bool sh = sc.feature_kind == SG_FEATURES_LIDAR_SH, beam = o.beam_divergence > 0.f;
    auto kern = sh ? (beam ? k_project_lidar<true, true> : k_project_lidar<true, false>)
                   : (beam ? k_project_lidar<false, true> : k_project_lidar<false, false>);
    kern<<<grid, 256, 0, st>>>(
        sc.d_planes, sc.pitch, sc.n, sc.sh_degree, actor_params(sc), L,
        (const RenderDesc *)fr.desc.p, U, o.cull,
        (GRec *)fr.rec.p, (float4 *)fr.rect.p,
        (int4 *)fr.tiles.p, (float *)fr.depth.p, (uint32_t *)fr.count.p, (float2 *)fr.mean2d.p,
        (float4 *)fr.cov2d.p, (uint32_t *)fr.scalars.p + kScalStatus);
    SG_LAUNCHED();
    return SG_OK;
}

}  // namespace sg

extern "C" sg_status sg_debug_bulk_wait(int give_up)
{
    const uint32_t v = give_up ? 1u : 0u;
    SG_CUDA(cudaDeviceSynchronize());   // no kernel reads it meanwhile
    SG_CUDA(cudaMemcpyToSymbol(sg::g_bulk_give_up, &v, sizeof(v)));
    return SG_OK;
}
