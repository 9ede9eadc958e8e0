// backward.cu -- gradients of the compositing (the differentiable renderer
// of Sec. 3.2 / 3.4) w.r.t. means, log-scales, quaternions, opacities and
// features.  The unscented transform only selects tiles (a piecewise-constant
// choice) and is not differentiated.
//
// Per ray, the list is walked back to front from the last composited entry,
// recomputing every pair with the forward's own arithmetic (pairs.cuh) so
// that the same entries contribute; transmittance is recovered as
// T_i = T_{i+1} / (1 - alpha_i) from the saved final value.  With
// Q = (F0, F1, F2, Z, W) = sum_i (c_i, tau_i, 1) alpha_i T_i,
//   dQ/dalpha_i = q_i T_i - (sum_{j>i} q_j alpha_j T_j) / (1 - alpha_i).
// The closest approach gives the geometric gradients in a stable form: with
// q* = M (o + tau d - mu) = (num x den) / |den|^2 (the closest point in the
// Gaussian's frame, no cancellation) and p = M^-1 q* = M^T diag(s^2) q*,
//   dD^2/dM = 2 q* p^T,          dD^2/dmu = -2 M^T q*,
//   dtau/dM = -(den p^T + q* d^T) / |den|^2,   dtau/dmu = M^T den / |den|^2
// (envelope theorem at tau_max).  Per (tile, Gaussian) the 16 partial sums
// dL/dM (9), dL/dmu (3), dL/dsigma, dL/dfeature (3) are reduced over the
// warp, then the block, before one float atomic each.  A last per-Gaussian
// kernel maps them to the raw parameters (M = S^-1 R^T, R of the normalised
// quaternion, SH colour at the direction from the camera to the mean).
#include <math.h>

#include "pairs.cuh"
#include "render.cuh"

namespace sg {

constexpr int kG = 16;          // accumulated partials per Gaussian
constexpr int kBwBatch = 64;    // camera list entries per shared-memory batch

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Gradient partials of one composited pair.
//   Mr: rows of M; d: ray direction; dLdD2, dLdtau: upstream.
__device__ __forceinline__ void pair_geometry_grads(const float Mr[9], const PairEval &pe,
                                                    const float d[3], float dLdD2, float dLdtau,
                                                    float g[kG])
{
    // q* = (num x den) * inv
    const float *n = pe.n, *e = pe.e;
    const float qs[3] = {(n[1] * e[2] - n[2] * e[1]) * pe.inv, (n[2] * e[0] - n[0] * e[2]) * pe.inv,
                         (n[0] * e[1] - n[1] * e[0]) * pe.inv};
    // p = M^-1 q* = sum_k s_k^2 q*_k M_k,  s_k^2 = 1 / |M_k|^2
    float p[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float *Mk = Mr + 3 * k;
        const float s2 = 1.f / (Mk[0] * Mk[0] + Mk[1] * Mk[1] + Mk[2] * Mk[2]);
        const float c = s2 * qs[k];
        p[0] += c * Mk[0];
        p[1] += c * Mk[1];
        p[2] += c * Mk[2];
    }
    const float a2 = 2.f * dLdD2, ti = dLdtau * pe.inv;
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            g[3 * k + j] = a2 * qs[k] * p[j] - ti * (e[k] * p[j] + qs[k] * d[j]);
#pragma unroll
    for (int j = 0; j < 3; ++j)
        g[9 + j] = -a2 * (Mr[j] * qs[0] + Mr[3 + j] * qs[1] + Mr[6 + j] * qs[2]) +
                   ti * (Mr[j] * e[0] + Mr[3 + j] * e[1] + Mr[6 + j] * e[2]);
}

// Back-to-front step for one composited entry: returns the partials.
//   q = (f0, f1, f2): features; gQ upstream of (F0, F1, F2, Z, W);
//   T: transmittance after this entry (updated to before it); S: suffix sums.
__device__ __forceinline__ void composite_grads(const PairEval &pe, float sigma, const float q[3],
                                                const float gQ[5], float &T, float S[5],
                                                const float Mr[9], const float d[3], float g[kG])
{
    const float one_m = 1.f - pe.alpha;
    const float Tb = T / one_m;
    const float w = pe.alpha * Tb;
    const float qq[5] = {q[0], q[1], q[2], pe.tau, 1.f};
    float dLda = 0.f;
#pragma unroll
    for (int k = 0; k < 5; ++k) dLda += gQ[k] * (qq[k] * Tb - S[k] / one_m);
#pragma unroll
    for (int k = 0; k < 5; ++k) S[k] += qq[k] * w;
    T = Tb;
    const float dLdtau = gQ[3] * w;
    float dLdD2 = 0.f;
    g[12] = 0.f;
    if (!pe.clamped) {
        g[12] = dLda * pe.rho;                       // d alpha / d sigma = rho
        dLdD2 = dLda * sigma * pe.rho * -0.5f;       // d alpha / d D^2
    }
    g[13] = gQ[0] * w;
    g[14] = gQ[1] * w;
    g[15] = gQ[2] * w;
    pair_geometry_grads(Mr, pe, d, dLdD2, dLdtau, g);
}

// ------------------------------------------------------------------ camera
__global__ void __launch_bounds__(kCamThreads)
k_backward_camera(CamRender P, const GRec *__restrict__ rec, const uint32_t *__restrict__ ids,
                  const uint2 *__restrict__ ranges, const uint32_t *__restrict__ order,
                  const float4 *__restrict__ pix,
                  const double *__restrict__ tile_dir, const RenderDesc *__restrict__ D,
                  const float4 *__restrict__ ray_state,
                  const uint32_t *__restrict__ n_contrib, const float *__restrict__ g_rgb,
                  const float *__restrict__ g_alpha, const float *__restrict__ g_depth,
                  float *__restrict__ gacc)
{
    __shared__ float4 s_e[9][kBwBatch];
    __shared__ uint32_t s_id[kBwBatch];
    __shared__ float s_red[kBwBatch][kCamThreads / 32][kG];
    __shared__ float s_ref[6];
    __shared__ uint32_t s_max;
    __shared__ CamPose s_pose;
    load_cam_pose(D, s_pose);
    __syncthreads();
    const int tile = (int)order[blockIdx.x], tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = tile % P.ntx, ty = tile / P.ntx;
    const int px = tx * kTile + (tid % kTile), py = ty * kTile + (tid / kTile);
    if (tid == 0) {
        cam_tile_ref(s_pose, tile_dir, tile, s_ref);
        s_max = 0;
    }
    __syncthreads();
    const float dh[3] = {s_ref[0], s_ref[1], s_ref[2]};
    const float dl[3] = {s_ref[3], s_ref[4], s_ref[5]};
    const bool inside = px < P.W && py < P.H;
    const int64_t pidx = (int64_t)py * P.W + px;
    const float4 e = inside ? pix[pidx] : make_float4(0.f, 0.f, 0.f, 0.f);
    const bool ray_ok = inside && e.w > 0.f;
    float dd[3], d[3];
    cam_ray_offset(s_pose, e, dd);
#pragma unroll
    for (int i = 0; i < 3; ++i) d[i] = dh[i] + dd[i];
    const float rx = (float)px + 0.5f, ry = (float)py + 0.5f;
    uint32_t last = 0;
    float T = 1.f, gQ[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, S[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (ray_ok) {
        const float4 st = ray_state[pidx];
        last = n_contrib[pidx];
        T = st.x;
        const float W = st.y, Z = st.z;
        if (g_rgb) {
            gQ[0] = g_rgb[3 * pidx];
            gQ[1] = g_rgb[3 * pidx + 1];
            gQ[2] = g_rgb[3 * pidx + 2];
        }
        const float gd = g_depth ? g_depth[pidx] : 0.f;
        const float ga = g_alpha ? g_alpha[pidx] : 0.f;
        gQ[3] = W > 0.f ? gd / W : 0.f;
        gQ[4] = ga - (W > 0.f ? gd * Z / (W * W) : 0.f);
        if (last) atomicMax(&s_max, last);
    }
    __syncthreads();
    const uint2 rg = ranges[tile];
    const uint32_t nmax = s_max;
    for (int32_t bend = (int32_t)nmax; bend > 0; bend -= kBwBatch) {
        const int32_t bstart = max(0, bend - kBwBatch);
        const int cnt = bend - bstart;
        if (tid < cnt) {
            const uint32_t g = ids[rg.x + bstart + tid];
            float4 ent[9];
            cam_entry(rec[g], s_pose.t, dh, dl, ent);
#pragma unroll
            for (int k = 0; k < 9; ++k) s_e[k][tid] = ent[k];
            s_id[tid] = g;
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            float gl[kG];
#pragma unroll
            for (int k = 0; k < kG; ++k) gl[k] = 0.f;
            PairEval pe;
            if ((uint32_t)(bstart + j) < last &&
                cam_pair(s_e[0][j], s_e[1][j], s_e[2][j], s_e[3][j], s_e[4][j], s_e[5][j],
                         s_e[6][j], s_e[8][j], dd, rx, ry, P.alpha_min, P.alpha_max, pe)) {
                const float4 m0 = s_e[3][j], m1 = s_e[4][j], m2 = s_e[5][j];
                const float Mr[9] = {m0.x, m0.y, m0.z, m1.x, m1.y, m1.z, m2.x, m2.y, m2.z};
                const float4 col = s_e[7][j];
                const float q[3] = {col.x, col.y, col.z};
                composite_grads(pe, s_e[6][j].w, q, gQ, T, S, Mr, d, gl);
            }
#pragma unroll
            for (int k = 0; k < kG; ++k) {
                const float v = warp_sum(gl[k]);
                if (lane == 0) s_red[j][warp][k] = v;
            }
        }
        __syncthreads();
        for (int i = tid; i < cnt * kG; i += kCamThreads) {
            const int j = i / kG, k = i % kG;
            float v = 0.f;
#pragma unroll
            for (int w = 0; w < kCamThreads / 32; ++w) v += s_red[j][w][k];
            if (v != 0.f) atomicAdd(&gacc[(int64_t)s_id[j] * kG + k], v);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ LiDAR
__global__ void __launch_bounds__(32 * kLidarWarps)
k_backward_lidar(LidRender P, const LidarItem *__restrict__ items,
                 const uint32_t *__restrict__ item_rays, const float4 *__restrict__ ray_e,
                 const double *__restrict__ item_u, const float *__restrict__ poses,
                 const float *__restrict__ az_col, const float *__restrict__ elev,
                 const GRec *__restrict__ rec, const uint32_t *__restrict__ ids,
                 const uint2 *__restrict__ ranges, const float4 *__restrict__ ray_state,
                 const uint32_t *__restrict__ n_contrib, const float *__restrict__ g_range,
                 const float *__restrict__ g_int, const float *__restrict__ g_drop,
                 const float *__restrict__ g_alpha, float *__restrict__ gacc)
{
    __shared__ float s_all[kLidarWarps][kLidEntry][32];
    __shared__ uint32_t s_ids[kLidarWarps][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int item_id = blockIdx.x * kLidarWarps + wib;
    if (item_id >= P.n_items) return;
    float(*s)[32] = s_all[wib];
    const LidarItem it = items[item_id];
    const uint32_t ray = item_rays[it.ray_off + lane];
    const bool valid = ray != 0xffffffffu;
    const int c = valid ? (int)(ray % (uint32_t)P.n_cols) : it.col0;
    const int b = valid ? (int)(ray / (uint32_t)P.n_cols) : 0;
    const int sb = kLidCommon + kLidPerCol * (c - it.col0);
    float dh[3], dl[3], dd[3], d[3];
    lidar_ray(it, item_u, item_id, poses, ray_e[it.ray_off + lane], c, dh, dl, dd, d);
    const float raz = az_col[c], rel = elev[b];
    uint32_t last = 0;
    float T = 1.f, gQ[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, S[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    if (valid) {
        const float4 st = ray_state[ray];
        last = n_contrib[ray];
        T = st.x;
        const float W = st.y, Z = st.z, drop = st.w;
        const float gr = g_range ? g_range[ray] : 0.f;
        const float gi = g_int ? g_int[ray] : 0.f;
        const float gp = g_drop ? g_drop[ray] : 0.f;
        const float ga = g_alpha ? g_alpha[ray] : 0.f;
        // drop = softmax(F1, F2)[drop] = 1 / (1 + exp(F1 - F2))
        const float dd_ = drop * (1.f - drop);
        gQ[0] = gi;
        gQ[1] = -gp * dd_;
        gQ[2] = gp * dd_;
        gQ[3] = W > 0.f ? gr / W : 0.f;
        gQ[4] = ga - (W > 0.f ? gr * Z / (W * W) : 0.f);
    }
    uint32_t nmax = last;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nmax = max(nmax, __shfl_xor_sync(0xffffffffu, nmax, o));
    const uint2 rg = ranges[it.tile];
    for (int32_t bend = (int32_t)nmax; bend > 0; bend -= 32) {
        const int32_t bstart = max(0, bend - 32);
        const int cnt = bend - bstart;
        __syncwarp();
        if (lane < cnt) {
            const uint32_t g = ids[rg.x + bstart + lane];
            lidar_entry(rec[g], poses, it.col0, it.ncols, dh, dl, s, lane);
            s_ids[wib][lane] = g;
        }
        __syncwarp();
        for (int j = cnt - 1; j >= 0; --j) {
            float gl[kG];
#pragma unroll
            for (int k = 0; k < kG; ++k) gl[k] = 0.f;
            PairEval pe;
            if ((uint32_t)(bstart + j) < last &&
                lidar_pair(s, j, sb, raz, rel, dd, d, P.alpha_min, P.alpha_max, pe)) {
                float Mr[9];
#pragma unroll
                for (int k = 0; k < 9; ++k) Mr[k] = s[k][j];
                const float q[3] = {s[13][j], s[14][j], s[15][j]};
                composite_grads(pe, s[12][j], q, gQ, T, S, Mr, d, gl);
            }
            const uint32_t g = s_ids[wib][j];
#pragma unroll
            for (int k = 0; k < kG; ++k) {
                const float v = warp_sum(gl[k]);
                if (lane == k && v != 0.f) atomicAdd(&gacc[(int64_t)g * kG + k], v);
            }
        }
    }
}

// ------------------------------------------------------------------ parameters
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, float Y[16],
                                              float dY[16][3])
{
    const float xx = x * x, yy = y * y, zz = z * z;
    for (int k = 0; k < 16; ++k) { Y[k] = 0.f; dY[k][0] = dY[k][1] = dY[k][2] = 0.f; }
    Y[0] = 0.28209479177387814f;
    if (deg >= 1) {
        const float c = 0.48860251190291992f;
        Y[1] = -c * y; dY[1][1] = -c;
        Y[2] = c * z;  dY[2][2] = c;
        Y[3] = -c * x; dY[3][0] = -c;
    }
    if (deg >= 2) {
        const float a = 1.0925484305920792f, b = 0.31539156525252005f, h = 0.54627421529603959f;
        Y[4] = a * x * y;  dY[4][0] = a * y; dY[4][1] = a * x;
        Y[5] = -a * y * z; dY[5][1] = -a * z; dY[5][2] = -a * y;
        Y[6] = b * (2.f * zz - xx - yy);
        dY[6][0] = -2.f * b * x; dY[6][1] = -2.f * b * y; dY[6][2] = 4.f * b * z;
        Y[7] = -a * x * z; dY[7][0] = -a * z; dY[7][2] = -a * x;
        Y[8] = h * (xx - yy); dY[8][0] = 2.f * h * x; dY[8][1] = -2.f * h * y;
    }
    if (deg >= 3) {
        const float c0 = 0.59004358992664352f, c1 = 2.8906114426405538f;
        const float c2 = 0.45704579946446572f, c3 = 0.37317633259011540f;
        const float c5 = 1.4453057213202769f;
        Y[9] = -c0 * y * (3.f * xx - yy);
        dY[9][0] = -6.f * c0 * x * y; dY[9][1] = -c0 * (3.f * xx - 3.f * yy);
        Y[10] = c1 * x * y * z;
        dY[10][0] = c1 * y * z; dY[10][1] = c1 * x * z; dY[10][2] = c1 * x * y;
        Y[11] = -c2 * y * (4.f * zz - xx - yy);
        dY[11][0] = 2.f * c2 * x * y; dY[11][1] = -c2 * (4.f * zz - xx - 3.f * yy);
        dY[11][2] = -8.f * c2 * y * z;
        Y[12] = c3 * z * (2.f * zz - 3.f * xx - 3.f * yy);
        dY[12][0] = -6.f * c3 * x * z; dY[12][1] = -6.f * c3 * y * z;
        dY[12][2] = c3 * (6.f * zz - 3.f * xx - 3.f * yy);
        Y[13] = -c2 * x * (4.f * zz - xx - yy);
        dY[13][0] = -c2 * (4.f * zz - 3.f * xx - yy); dY[13][1] = 2.f * c2 * x * y;
        dY[13][2] = -8.f * c2 * x * z;
        Y[14] = c5 * z * (xx - yy);
        dY[14][0] = 2.f * c5 * x * z; dY[14][1] = -2.f * c5 * y * z; dY[14][2] = c5 * (xx - yy);
        Y[15] = -c0 * x * (xx - 3.f * yy);
        dY[15][0] = -c0 * (3.f * xx - 3.f * yy); dY[15][1] = 6.f * c0 * x * y;
    }
}

__global__ void k_param_grads(const float *__restrict__ planes, int64_t pitch, int64_t n,
                              int feature_kind, int sh_degree, int F, float ox, float oy,
                              float oz, const float *__restrict__ gacc, float *__restrict__ gm,
                              float *__restrict__ gls, float *__restrict__ gq,
                              float *__restrict__ gop, float *__restrict__ gf)
{
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n) return;
    float G[kG];
    bool any = false;
#pragma unroll
    for (int k = 0; k < kG; ++k) {
        G[k] = gacc[g * kG + k];
        any = any || G[k] != 0.f;
    }
    if (!any) return;
    float q[4];
    for (int k = 0; k < 4; ++k) q[k] = planes[(Scene::kQuat + k) * pitch + g];
    const float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
    const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                        2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                        2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    // M_k = r_k / s_k (r_k = column k of R): dL/dls_k = -G_k . M_k,
    // dL/dr_k = G_k / s_k
    float gR[9];
    for (int k = 0; k < 3; ++k) {
        const float s = expf(planes[(Scene::kLogScale + k) * pitch + g]);
        const float rk[3] = {R[k], R[3 + k], R[6 + k]};
        const float Gk[3] = {G[3 * k], G[3 * k + 1], G[3 * k + 2]};
        if (gls) gls[3 * g + k] += -(Gk[0] * rk[0] + Gk[1] * rk[1] + Gk[2] * rk[2]) / s;
        for (int i = 0; i < 3; ++i) gR[3 * i + k] = Gk[i] / s;
    }
    if (gq) {
        // partial derivatives of R(w,x,y,z) (entries row-major), times 2
        const float dRw[9] = {0, -z, y, z, 0, -x, -y, x, 0};
        const float dRx[9] = {0, y, z, y, -2 * x, -w, z, w, -2 * x};
        const float dRy[9] = {-2 * y, x, w, x, 0, z, -w, z, -2 * y};
        const float dRz[9] = {-2 * z, -w, x, w, -2 * z, y, x, y, 0};
        float gqh[4] = {0, 0, 0, 0};
        for (int i = 0; i < 9; ++i) {
            gqh[0] += 2.f * dRw[i] * gR[i];
            gqh[1] += 2.f * dRx[i] * gR[i];
            gqh[2] += 2.f * dRy[i] * gR[i];
            gqh[3] += 2.f * dRz[i] * gR[i];
        }
        const float dot = gqh[0] * w + gqh[1] * x + gqh[2] * y + gqh[3] * z;
        const float qh[4] = {w, x, y, z};
        for (int i = 0; i < 4; ++i) gq[4 * g + i] += (gqh[i] - qh[i] * dot) / qn;
    }
    if (gop) gop[g] += G[12];
    float gmu[3] = {G[9], G[10], G[11]};
    const float gc[3] = {G[13], G[14], G[15]};
    if (feature_kind == SG_FEATURES_SH) {
        const float mx = planes[(Scene::kMean + 0) * pitch + g] - ox;
        const float my = planes[(Scene::kMean + 1) * pitch + g] - oy;
        const float mz = planes[(Scene::kMean + 2) * pitch + g] - oz;
        const float dist = sqrtf(mx * mx + my * my + mz * mz);
        const float inv = 1.f / dist;
        const float dx = mx * inv, dy = my * inv, dz = mz * inv;
        float Y[16], dY[16][3];
        sh_basis_grad(sh_degree, dx, dy, dz, Y, dY);
        const int nc = (sh_degree + 1) * (sh_degree + 1);
        float gdir[3] = {0.f, 0.f, 0.f};
        for (int ch = 0; ch < 3; ++ch) {
            float acc = 0.f;
            for (int k = 0; k < nc; ++k) acc += Y[k] * planes[(Scene::kFeat + 3 * k + ch) * pitch + g];
            if (acc + 0.5f < 0.f) continue;   // clamped colour channel
            for (int k = 0; k < nc; ++k) {
                if (gf) gf[g * F + 3 * k + ch] += Y[k] * gc[ch];
                const float f = planes[(Scene::kFeat + 3 * k + ch) * pitch + g];
                gdir[0] += gc[ch] * f * dY[k][0];
                gdir[1] += gc[ch] * f * dY[k][1];
                gdir[2] += gc[ch] * f * dY[k][2];
            }
        }
        const float dd = gdir[0] * dx + gdir[1] * dy + gdir[2] * dz;
        gmu[0] += (gdir[0] - dx * dd) * inv;
        gmu[1] += (gdir[1] - dy * dd) * inv;
        gmu[2] += (gdir[2] - dz * dd) * inv;
    } else if (gf) {
        for (int ch = 0; ch < 3; ++ch) gf[g * F + ch] += gc[ch];
    }
    if (gm)
        for (int k = 0; k < 3; ++k) gm[3 * g + k] += gmu[k];
}

static sg_status finish(const Scene &sc, Frame &fr, const float o[3], const sg_grads &g,
                        cudaStream_t st)
{
    if (sc.n == 0) return SG_OK;
    k_param_grads<<<(unsigned)((sc.n + 127) / 128), 128, 0, st>>>(
        sc.d_planes, sc.pitch, sc.n, sc.feature_kind, sc.sh_degree, sc.F, o[0], o[1], o[2],
        (const float *)fr.gacc.p, g.d_g_means, g.d_g_log_scales, g.d_g_quats, g.d_g_opacity,
        g.d_g_features);
    SG_LAUNCHED();
    return SG_OK;
}

sg_status backward_camera(const Scene &sc, const Camera &cam, Frame &fr, const float *g_rgb,
                          const float *g_alpha, const float *g_depth, const sg_grads &g,
                          cudaStream_t st)
{
    sg_status s = ensure(fr.gacc, sizeof(float) * kG * (sc.n > 0 ? sc.n : 1));
    if (s != SG_OK) return s;
    SG_CUDA(cudaMemsetAsync(fr.gacc.p, 0, sizeof(float) * kG * sc.n, st));
    const CamRender P = cam_render_params(cam, fr.opts);
    k_backward_camera<<<(unsigned)(cam.ntx * cam.nty), kCamThreads, 0, st>>>(
        P, (const GRec *)fr.rec.p, (const uint32_t *)fr.pvals[fr.pair_buf].p,
        (const uint2 *)fr.ranges.p, (const uint32_t *)fr.order.p, cam.d_pix, cam.d_tile_dir,
        (const RenderDesc *)fr.desc.p, (const float4 *)fr.ray_state.p,
        (const uint32_t *)fr.n_contrib.p, g_rgb, g_alpha, g_depth, (float *)fr.gacc.p);
    SG_LAUNCHED();
    const float o[3] = {fr.c2w[3], fr.c2w[7], fr.c2w[11]};
    return finish(sc, fr, o, g, st);
}

sg_status backward_lidar(const Scene &sc, const Lidar &L, Frame &fr, const float *g_range,
                         const float *g_int, const float *g_drop, const float *g_alpha,
                         const sg_grads &g, cudaStream_t st)
{
    sg_status s = ensure(fr.gacc, sizeof(float) * kG * (sc.n > 0 ? sc.n : 1));
    if (s != SG_OK) return s;
    SG_CUDA(cudaMemsetAsync(fr.gacc.p, 0, sizeof(float) * kG * sc.n, st));
    const LidRender P = lidar_render_params(L, fr.opts);
    if (L.n_items > 0) {
        unsigned grid = (unsigned)((L.n_items + kLidarWarps - 1) / kLidarWarps);
        k_backward_lidar<<<grid, 32 * kLidarWarps, 0, st>>>(
            P, L.d_items, L.d_item_rays, L.d_ray_e, L.d_tile_u, fr.d_lidar_poses, L.d_az,
            L.d_elev, (const GRec *)fr.rec.p, (const uint32_t *)fr.pvals[fr.pair_buf].p,
            (const uint2 *)fr.ranges.p, (const float4 *)fr.ray_state.p,
            (const uint32_t *)fr.n_contrib.p, g_range, g_int, g_drop, g_alpha,
            (float *)fr.gacc.p);
        SG_LAUNCHED();
    }
    const float o[3] = {0.f, 0.f, 0.f};
    return finish(sc, fr, o, g, st);
}

}  // namespace sg
