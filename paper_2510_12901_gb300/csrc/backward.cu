// backward.cu -- gradients of the compositing (the differentiable renderer
// of Sec. 3.2 / 3.4) w.r.t. means, log-scales, quaternions, opacities and
// features.  The unscented transform only selects tiles (a piecewise-constant
// choice) and is not differentiated.
//
// The backward runs over the forward's own work items (segments of a tile
// list x sub-blocks for the camera, segments x LiDAR work items), with the
// forward's staging and pair arithmetic (pairs.cuh), so that the same
// entries contribute.  Each segment is walked front to back from the state
// the forward's merge left for it (transmittance T and the sums (F, Z, W)
// before the segment).  With Q = (F0, F1, F2, Z, W) = sum_i (c_i, tau_i, 1)
// alpha_i T_i and U = gQ . Q (gQ = dL/dQ), the gradient of a composited
// entry's alpha is
//   dL/dalpha_i = (gQ . q_i) T_i - (U - U_{<=i}) / (1 - alpha_i),
// where U comes from the ray's saved final (F, Z, W) and U_{<=i} is the
// prefix sum up to and including entry i; T_{i+1} = T_i (1 - alpha_i) is
// the forward's own product.  The closest approach gives the geometric
// gradients in a stable form: with q* = M (o + tau d - mu) = (num x den) /
// |den|^2 (the closest point in the Gaussian's frame, no cancellation) and
// p = M^-1 q* = M^T diag(s^2) q*,
//   dD^2/dM = 2 q* p^T,          dD^2/dmu = -2 M^T q*,
//   dtau/dM = -(den p^T + q* d^T) / |den|^2,   dtau/dmu = M^T den / |den|^2
// (envelope theorem at tau_max).  Per staged entry the 16 partials dL/dM
// (9), dL/dmu (3), dL/dsigma, dL/dfeature (3) are summed over the warp by a
// transposing butterfly (16 shuffles) and added with 16 float atomics.  A
// last per-Gaussian kernel maps them to the raw parameters (M = S^-1 R^T, R
// of the normalised quaternion, SH colour at the direction from the camera
// to the mean).
#include <math.h>

#include "pairs.cuh"
#include "render.cuh"

namespace sg {

constexpr int kG = 16;          // accumulated partials per Gaussian
constexpr int kBwWarps = 4;     // warps per block of the persistent backward grids

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

// Front-to-back step for one composited entry: returns the partials.
//   q = (f0, f1, f2): features; gQ: upstream of (F0, F1, F2, Z, W);
//   T: transmittance before the entry (updated to after it); U: gQ . Q
//   before the entry (updated); Ut: gQ . Q of the whole ray.
__device__ __forceinline__ void composite_grads(const PairEval &pe, float sigma, const float q[3],
                                                const float gQ[5], float &T, float &U, float Ut,
                                                const float Mr[9], const float d[3], float g[kG])
{
    const float w = pe.alpha * T;
    const float gq = gQ[0] * q[0] + gQ[1] * q[1] + gQ[2] * q[2] + gQ[3] * pe.tau + gQ[4];
    const float Ua = U + gq * w;
    const float dLda = gq * T - (Ut - Ua) / (1.f - pe.alpha);
    U = Ua;
    T = T * (1.f - pe.alpha);
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

// Sum g[16] over the warp and add it to acc[0..15]: a butterfly that halves
// the vector at each of the first four levels (8 + 4 + 2 + 1 shuffles) and
// leaves lane L with component 8 b4 + 4 b3 + 2 b2 + b1 (b = bits of L)
// summed over 16 lanes; the last shuffle adds the other half.
__device__ __forceinline__ void warp_reduce_add16(const float g[kG], float *acc)
{
    const int lane = threadIdx.x & 31;
    const bool h1 = lane & 16, h2 = lane & 8, h3 = lane & 4, h4 = lane & 2;
    float a8[8], a4[4], a2[2];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const float mine = h1 ? g[8 + k] : g[k], other = h1 ? g[k] : g[8 + k];
        a8[k] = mine + __shfl_xor_sync(0xffffffffu, other, 16);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float mine = h2 ? a8[4 + k] : a8[k], other = h2 ? a8[k] : a8[4 + k];
        a4[k] = mine + __shfl_xor_sync(0xffffffffu, other, 8);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float mine = h3 ? a4[2 + k] : a4[k], other = h3 ? a4[k] : a4[2 + k];
        a2[k] = mine + __shfl_xor_sync(0xffffffffu, other, 4);
    }
    float a1 = (h4 ? a2[1] : a2[0]) + __shfl_xor_sync(0xffffffffu, h4 ? a2[0] : a2[1], 2);
    a1 += __shfl_xor_sync(0xffffffffu, a1, 1);
    const int comp = (h1 ? 8 : 0) + (h2 ? 4 : 0) + (h3 ? 2 : 0) + (h4 ? 1 : 0);
    if (!(lane & 1) && a1 != 0.f) atomicAdd(acc + comp, a1);
}

// Upstream of (F0, F1, F2, Z, W) for a camera ray from dL/d(rgb, alpha,
// depth), depth = Z / W.
__device__ __forceinline__ void camera_gQ(const float *g_rgb, const float *g_alpha,
                                          const float *g_depth, int64_t r, float W, float Z,
                                          float gQ[5])
{
    gQ[0] = g_rgb ? g_rgb[3 * r] : 0.f;
    gQ[1] = g_rgb ? g_rgb[3 * r + 1] : 0.f;
    gQ[2] = g_rgb ? g_rgb[3 * r + 2] : 0.f;
    const float gd = g_depth ? g_depth[r] : 0.f, ga = g_alpha ? g_alpha[r] : 0.f;
    gQ[3] = W > 0.f ? gd / W : 0.f;
    gQ[4] = ga - (W > 0.f ? gd * Z / (W * W) : 0.f);
}

// ------------------------------------------------------------------ camera
// Six blocks per SM (80 registers, 20 bytes spilled): the differentiable
// street step 4.64 -> 4.60 ms against five at 96 registers.
__global__ void __launch_bounds__(32 * kBwWarps, 6)
k_backward_camera(CamRender P, const GRec *__restrict__ rec, const uint32_t *__restrict__ ids,
                  const uint2 *__restrict__ ranges, const uint2 *__restrict__ items,
                  const uint2 *__restrict__ tile_info, const uint32_t *__restrict__ counts,
                  const uint32_t *__restrict__ crw, uint32_t *__restrict__ counter,
                  const float4 *__restrict__ partials, const float4 *__restrict__ pix,
                  const double *__restrict__ tile_dir, const RenderDesc *__restrict__ D,
                  const float4 *__restrict__ ray_state, const float4 *__restrict__ ray_feat,
                  const uint32_t *__restrict__ n_contrib, const float *__restrict__ g_rgb,
                  const float *__restrict__ g_alpha, const float *__restrict__ g_depth,
                  float *__restrict__ gacc)
{
    __shared__ float4 s_all[kBwWarps][8][32];
    __shared__ uint32_t s_pos[kBwWarps][32], s_lanes[kBwWarps][32], s_gid[kBwWarps][32];
    __shared__ float s_refs[kBwWarps][6];
    __shared__ CamPose s_pose;
    load_cam_pose(D, s_pose);
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float4(*s_e)[32] = s_all[wib];
    float *s_ref = s_refs[wib];
    const uint32_t n_items = counts[0];
    while (true) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(counter, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        const uint2 it = items[item];
        const int tile = (int)it.x, seg = (int)(it.y >> 3), sub = (int)(it.y & 7);
        const uint2 ti = tile_info[tile];
        const int tx = tile % P.ntx, ty = tile / P.ntx;
        const int sbx = tx * kTile + 8 * (sub & 1), sby = ty * kTile + 4 * (sub >> 1);
        const int px = sbx + (lane & 7), py = sby + (lane >> 3);
        const bool inside = px < P.W && py < P.H;
        const int64_t pidx = (int64_t)py * P.W + px;
        const float4 e = inside ? pix[pidx] : make_float4(0.f, 0.f, 0.f, 0.f);
        const bool ray_ok = inside && e.w > 0.f;
        const uint32_t last = ray_ok ? n_contrib[pidx] : 0u;
        const uint2 rg = ranges[tile];
        const uint32_t lo = rg.x + (uint32_t)seg * kSegLen;
        uint32_t hi = min(rg.y, lo + kSegLen);
        uint32_t lim = rg.x + last;                    // entries idx < lim may contribute
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lim = max(lim, __shfl_xor_sync(0xffffffffu, lim, o));
        hi = min(hi, lim);
        if (hi <= lo) continue;                        // nothing of this segment composited
        if (lane == 0) cam_tile_ref(s_pose, tile_dir, tile, s_ref);
        __syncwarp();
        const float dh[3] = {s_ref[0], s_ref[1], s_ref[2]};
        const float dl[3] = {s_ref[3], s_ref[4], s_ref[5]};
        float dd[3], d[3];
        cam_ray_offset(s_pose, e, dd);
#pragma unroll
        for (int i = 0; i < 3; ++i) d[i] = dh[i] + dd[i];
        // state before the segment, upstream, totals
        float T = 1.f, Qp[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (seg > 0) {
            const float4 *pq = partials + ((size_t)(ti.y + seg) * 256 + sub * 32 + lane) * 2;
            const float4 u = pq[0], v = pq[1];
            Qp[0] = u.x; Qp[1] = u.y; Qp[2] = u.z; Qp[3] = v.x; Qp[4] = u.w;
            T = v.y;
        }
        float gQ[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, Ut = 0.f, U = 0.f;
        if (ray_ok) {
            const float4 st = ray_state[pidx], F = ray_feat[pidx];
            camera_gQ(g_rgb, g_alpha, g_depth, pidx, st.y, st.z, gQ);
            Ut = gQ[0] * F.x + gQ[1] * F.y + gQ[2] * F.z + gQ[3] * st.z + gQ[4] * st.y;
            U = gQ[0] * Qp[0] + gQ[1] * Qp[1] + gQ[2] * Qp[2] + gQ[3] * Qp[3] + gQ[4] * Qp[4];
        }
        // the next batch's column/row word and id, loaded one batch ahead
        uint32_t ncr = 0u, nid = 0u;
        if (lo + lane < hi) {
            ncr = crw[lo + lane];
            nid = ids[lo + lane];
        }
        for (uint32_t base = lo; base < hi; base += 32) {
            // lanes whose composited entries reach this batch: an entry that
            // reaches none of them contributes to no ray and is not staged
            const uint32_t act = __ballot_sync(0xffffffffu, rg.x + last > base);
            const uint32_t idx = base + lane;
            const uint32_t g = nid;
            const uint32_t lm = word_lanes(ncr, sub) & act;
            const bool ov = lm != 0u;
            if (idx + 32 < hi) {
                ncr = crw[idx + 32];
                nid = ids[idx + 32];
            } else {
                ncr = 0u;
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, ov);
            if (bal == 0u) continue;
            __syncwarp();
            if (ov) {
                const int pos = __popc(bal & ((1u << lane) - 1u));
                float4 ent[9];
                cam_entry(rec[g], s_pose.t, dh, dl, ent, kResponseScale);
#pragma unroll
                for (int k = 0; k < 8; ++k) s_e[k][pos] = ent[k];
                s_lanes[wib][pos] = lm;
                s_pos[wib][pos] = idx + 1 - rg.x;
                s_gid[wib][pos] = g;
            }
            __syncwarp();
            const int n = __popc(bal);
            for (int j = 0; j < n; ++j) {
                PairEval pe;
                bool ok = cam_pair_scaled(s_e[0][j], s_e[1][j], s_e[2][j], s_e[3][j], s_e[4][j],
                                          s_e[5][j], s_e[6][j], (s_lanes[wib][j] >> lane) & 1u, dd,
                                          P.alpha_min, P.alpha_max, pe);
                ok = ok && s_pos[wib][j] <= last;
                if (!__any_sync(0xffffffffu, ok)) continue;
                float g[kG];
#pragma unroll
                for (int k = 0; k < kG; ++k) g[k] = 0.f;
                if (ok) {
                    const float4 m0 = s_e[3][j], m1 = s_e[4][j], m2 = s_e[5][j];
                    const float Mr[9] = {m0.x, m0.y, m0.z, m1.x, m1.y, m1.z, m2.x, m2.y, m2.z};
                    const float4 col = s_e[7][j];
                    const float q[3] = {col.x, col.y, col.z};
                    composite_grads(pe, s_e[6][j].w, q, gQ, T, U, Ut, Mr, d, g);
                }
                warp_reduce_add16(g, gacc + (int64_t)s_gid[wib][j] * kG);
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ rolling shutter
// The camera backward with a pose per pixel row: the rolling-shutter
// forward's staging (row slots as LiDAR columns) and ray set-up.
__global__ void __launch_bounds__(32 * kBwWarps, 4)
k_backward_camera_rs(CamRender P, const GRec *__restrict__ rec, const uint32_t *__restrict__ ids,
                     const uint2 *__restrict__ ranges, const uint2 *__restrict__ items,
                     const uint2 *__restrict__ tile_info, const uint32_t *__restrict__ counts,
                     const uint32_t *__restrict__ crw, uint32_t *__restrict__ counter,
                     const float4 *__restrict__ partials, const float4 *__restrict__ pix,
                     const double *__restrict__ tile_dir, const float *__restrict__ poses,
                     const float4 *__restrict__ ray_state, const float4 *__restrict__ ray_feat,
                     const uint32_t *__restrict__ n_contrib, const float *__restrict__ g_rgb,
                     const float *__restrict__ g_alpha, const float *__restrict__ g_depth,
                     float *__restrict__ gacc)
{
    __shared__ float4 s_all[kBwWarps][kLidPlanes][32];
    __shared__ uint32_t s_pos[kBwWarps][32], s_lanes[kBwWarps][32], s_gid[kBwWarps][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float4(*s)[32] = s_all[wib];
    const uint32_t n_items = counts[0];
    while (true) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(counter, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        const uint2 it = items[item];
        const int tile = (int)it.x, seg = (int)(it.y >> 3), sub = (int)(it.y & 7);
        const uint2 ti = tile_info[tile];
        const int tx = tile % P.ntx, ty = tile / P.ntx;
        const int sbx = tx * kTile + 8 * (sub & 1), sby = ty * kTile + 4 * (sub >> 1);
        const int px = sbx + (lane & 7), py = sby + (lane >> 3);
        const bool inside = px < P.W && py < P.H;
        const int64_t pidx = (int64_t)py * P.W + px;
        const float4 e = inside ? pix[pidx] : make_float4(0.f, 0.f, 0.f, 0.f);
        const bool ray_ok = inside && e.w > 0.f;
        const uint32_t last = ray_ok ? n_contrib[pidx] : 0u;
        const uint2 rg = ranges[tile];
        const uint32_t lo = rg.x + (uint32_t)seg * kSegLen;
        uint32_t hi = min(rg.y, lo + kSegLen);
        uint32_t lim = rg.x + last;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lim = max(lim, __shfl_xor_sync(0xffffffffu, lim, o));
        hi = min(hi, lim);
        if (hi <= lo) continue;
        const int nrows = min(4, P.H - sby);
        const int row = py < P.H ? py : sby;
        const int sb = 3 + 4 * (row - sby);
        float dh[3], dl[3], dd[3], d[3];
        {
            const double *u = tile_dir + 3 * tile;
            sensor_ray(poses + 12 * sby, u[0], u[1], u[2], poses + 12 * row, e, dh, dl, dd, d);
        }
        float T = 1.f, Qp[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (seg > 0) {
            const float4 *pq = partials + ((size_t)(ti.y + seg) * 256 + sub * 32 + lane) * 2;
            const float4 u = pq[0], v = pq[1];
            Qp[0] = u.x; Qp[1] = u.y; Qp[2] = u.z; Qp[3] = v.x; Qp[4] = u.w;
            T = v.y;
        }
        float gQ[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, Ut = 0.f, U = 0.f;
        if (ray_ok) {
            const float4 st = ray_state[pidx], F = ray_feat[pidx];
            camera_gQ(g_rgb, g_alpha, g_depth, pidx, st.y, st.z, gQ);
            Ut = gQ[0] * F.x + gQ[1] * F.y + gQ[2] * F.z + gQ[3] * st.z + gQ[4] * st.y;
            U = gQ[0] * Qp[0] + gQ[1] * Qp[1] + gQ[2] * Qp[2] + gQ[3] * Qp[3] + gQ[4] * Qp[4];
        }
        uint32_t ncr = 0u, nid = 0u;    // the next batch's, one batch ahead
        if (lo + lane < hi) {
            ncr = crw[lo + lane];
            nid = ids[lo + lane];
        }
        for (uint32_t base = lo; base < hi; base += 32) {
            const uint32_t act = __ballot_sync(0xffffffffu, rg.x + last > base);
            const uint32_t idx = base + lane;
            const uint32_t g = nid;
            const uint32_t lm = word_lanes(ncr, sub) & act;
            if (idx + 32 < hi) {
                ncr = crw[idx + 32];
                nid = ids[idx + 32];
            } else {
                ncr = 0u;
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, lm != 0u);
            if (bal == 0u) continue;
            __syncwarp();
            if (lm) {
                const int pos = __popc(bal & ((1u << lane) - 1u));
                lidar_entry(rec[g], poses, sby, nrows, dh, dl, s, pos);
                s_lanes[wib][pos] = lm;
                s_pos[wib][pos] = idx + 1 - rg.x;
                s_gid[wib][pos] = g;
            }
            __syncwarp();
            const int cnt = __popc(bal);
            for (int j = 0; j < cnt; ++j) {
                PairEval pe;
                bool ok = lidar_pair_in(s, j, sb, (s_lanes[wib][j] >> lane) & 1u, dd, d,
                                        P.alpha_min, P.alpha_max, pe);
                ok = ok && s_pos[wib][j] <= last;
                if (!__any_sync(0xffffffffu, ok)) continue;
                float gg[kG];
#pragma unroll
                for (int k = 0; k < kG; ++k) gg[k] = 0.f;
                if (ok) {
                    const float4 m0 = s[0][j], m1 = s[1][j], m2 = s[2][j];
                    const float Mr[9] = {m0.x, m0.y, m0.z, m1.x, m1.y, m1.z, m2.x, m2.y, m2.z};
                    const float q[3] = {m1.w, m2.w, lid_u(s, j, sb).w};
                    composite_grads(pe, m0.w, q, gQ, T, U, Ut, Mr, d, gg);
                }
                warp_reduce_add16(gg, gacc + (int64_t)s_gid[wib][j] * kG);
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ LiDAR
__global__ void __launch_bounds__(32 * kBwWarps)
k_backward_lidar(LidRender P, const LidarItem *__restrict__ items,
                 const uint32_t *__restrict__ item_rays, const float4 *__restrict__ ray_e,
                 const double *__restrict__ item_u, const float *__restrict__ poses,
                 const uint2 *__restrict__ tile_items, const uint32_t *__restrict__ lmask,
                 int64_t lmask_stride, const GRec *__restrict__ rec,
                 const uint32_t *__restrict__ ids,
                 const uint2 *__restrict__ ranges, const uint2 *__restrict__ work,
                 const uint2 *__restrict__ unit_info, const uint32_t *__restrict__ counts,
                 uint32_t *__restrict__ counter, const float4 *__restrict__ partials,
                 const float4 *__restrict__ ray_state, const float4 *__restrict__ ray_feat,
                 const uint32_t *__restrict__ n_contrib, const float *__restrict__ g_range,
                 const float *__restrict__ g_int, const float *__restrict__ g_drop,
                 const float *__restrict__ g_alpha, float *__restrict__ gacc)
{
    __shared__ float4 s_all[kBwWarps][kLidPlanes][32];
    __shared__ uint32_t s_gid[kBwWarps][32], s_lanes[kBwWarps][32], s_pos[kBwWarps][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float4(*s)[32] = s_all[wib];
    const uint32_t n_work = counts[0];
    while (true) {
        uint32_t wi = 0;
        if (lane == 0) wi = atomicAdd(counter, 1u);
        wi = __shfl_sync(0xffffffffu, wi, 0);
        if (wi >= n_work) break;
        const uint2 w = work[wi];
        const int item_id = (int)w.x;
        const uint32_t seg = w.y;
        const uint2 ui = unit_info[item_id];
        const LidarItem it = items[item_id];
        const uint32_t ray = item_rays[it.ray_off + lane];
        const bool valid = ray != 0xffffffffu;
        const uint32_t last = valid ? n_contrib[ray] : 0u;
        const uint2 rg = ranges[it.tile];
        const uint32_t lo = rg.x + seg * kSegLen;
        uint32_t hi = min(rg.y, lo + kSegLen);
        uint32_t lim = rg.x + last;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lim = max(lim, __shfl_xor_sync(0xffffffffu, lim, o));
        hi = min(hi, lim);
        if (hi <= lo) continue;
        const int c = valid ? (int)(ray % (uint32_t)P.n_cols) : it.col0;
        const int sb = 3 + 4 * (c - it.col0);
        float dh[3], dl[3], dd[3], d[3];
        lidar_ray(it, item_u, item_id, poses, ray_e[it.ray_off + lane], c, dh, dl, dd, d);
        // the item's ray masks of the list entries (the forward's own)
        const uint32_t *lm = lmask + (int64_t)(item_id - (int)tile_items[it.tile].x) * lmask_stride;
        float T = 1.f, Qp[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (seg > 0) {
            const float4 *pq = partials + ((size_t)(ui.y + seg) * 32 + lane) * 2;
            const float4 u = pq[0], v = pq[1];
            Qp[0] = u.x; Qp[1] = u.y; Qp[2] = u.z; Qp[3] = v.x; Qp[4] = u.w;
            T = v.y;
        }
        float gQ[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, Ut = 0.f, U = 0.f;
        if (valid) {
            const float4 st = ray_state[ray], F = ray_feat[ray];
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
            Ut = gQ[0] * F.x + gQ[1] * F.y + gQ[2] * F.z + gQ[3] * Z + gQ[4] * W;
            U = gQ[0] * Qp[0] + gQ[1] * Qp[1] + gQ[2] * Qp[2] + gQ[3] * Qp[3] + gQ[4] * Qp[4];
        }
        uint32_t nid = 0u, nm = 0u;   // one batch ahead
        if (lo + lane < hi) {
            nid = ids[lo + lane];
            nm = lm[lo + lane];
        }
        for (uint32_t base = lo; base < hi; base += 32) {
            const uint32_t act = __ballot_sync(0xffffffffu, rg.x + last > base);
            const uint32_t idx = base + lane;
            const uint32_t g = nid;
            const uint32_t m = nm & act;
            if (idx + 32 < hi) {
                nid = ids[idx + 32];
                nm = lm[idx + 32];
            } else {
                nm = 0u;
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, m != 0u);
            if (bal == 0u) continue;
            __syncwarp();
            if (m) {
                const int pos = __popc(bal & ((1u << lane) - 1u));
                lidar_entry(rec[g], poses, it.col0, it.ncols, dh, dl, s, pos);
                s_lanes[wib][pos] = m;
                s_pos[wib][pos] = idx + 1 - rg.x;
                s_gid[wib][pos] = g;
            }
            __syncwarp();
            const int cnt = __popc(bal);
            for (int j = 0; j < cnt; ++j) {
                PairEval pe;
                bool ok = lidar_pair_in(s, j, sb, (s_lanes[wib][j] >> lane) & 1u, dd, d,
                                        P.alpha_min, P.alpha_max, pe);
                ok = ok && s_pos[wib][j] <= last;
                if (!__any_sync(0xffffffffu, ok)) continue;
                float g[kG];
#pragma unroll
                for (int k = 0; k < kG; ++k) g[k] = 0.f;
                if (ok) {
                    const float4 m0 = s[0][j], m1 = s[1][j], m2 = s[2][j];
                    const float Mr[9] = {m0.x, m0.y, m0.z, m1.x, m1.y, m1.z, m2.x, m2.y, m2.z};
                    const float q[3] = {m1.w, m2.w, lid_u(s, j, sb).w};
                    composite_grads(pe, m0.w, q, gQ, T, U, Ut, Mr, d, g);
                }
                warp_reduce_add16(g, gacc + (int64_t)s_gid[wib][j] * kG);
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

// SH origin: (ox, oy, oz) for cameras; for LiDAR SH^l features, the origin
// of the column pose that saw the mean, whose index the projection left in
// the record's feat.w.
__global__ void k_param_grads(const float *__restrict__ planes, int64_t pitch, int64_t n,
                              int feature_kind, int sh_degree, int F, float ox, float oy,
                              float oz, const GRec *__restrict__ rec,
                              const float *__restrict__ poses, ActorParams A, float beam,
                              int posed_origin,
                              const float *__restrict__ gacc, float *__restrict__ gm,
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
    // an actor's Gaussian: the accumulated gradients are in world
    // coordinates (M_w = S^-1 (Ra R)^T, mu_w = Ra mu + t); in its own frame
    // dL/dM_k becomes Ra^T dL/dM_k and dL/dmu becomes Ra^T dL/dmu
    float Ra[9] = {1.f, 0.f, 0.f, 0.f, 1.f, 0.f, 0.f, 0.f, 1.f}, ta[3] = {0.f, 0.f, 0.f};
    const int ak = A.of ? A.of[g] : -1;
    const bool actor = ak >= 0 && ak < A.n;
    if (actor) {
        const float *P = A.poses + 12 * ak;
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) Ra[3 * i + j] = P[4 * i + j];
            ta[i] = P[4 * i + 3];
        }
    }
    // Beam divergence (Eq. 6): the record holds M of the smoothed covariance
    // (rows m_k orthogonal), and the loss depends on M only through
    // A = M^T M = Sigma_hat^-1, so dL/dM = 2 M S with S = sym(dL/dA):
    // S = M^-1 dL/dM / 2, M^-1 = [m_k / |m_k|^2].  Then dL/dSigma_hat =
    // H = -A S A, and Sigma_hat = Sigma + beam^2 (|v|^2 I - v v^T), v = mu - o,
    // adds beam^2 (2 v tr(H) - 2 H v) to dL/dmu.
    float H[9];
    if (beam > 0.f) {
        const GRec &rc = rec[g];
        const float m[9] = {rc.m0.x, rc.m0.y, rc.m0.z, rc.m1.x, rc.m1.y, rc.m1.z,
                            rc.m2.x, rc.m2.y, rc.m2.z};
        float S[9], T[9], Am[9];
        for (int i = 0; i < 9; ++i) S[i] = 0.f;
        for (int k = 0; k < 3; ++k) {
            const float mk2 = m[3 * k] * m[3 * k] + m[3 * k + 1] * m[3 * k + 1] +
                              m[3 * k + 2] * m[3 * k + 2];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) S[3 * i + j] += 0.5f * m[3 * k + i] / mk2 * G[3 * k + j];
        }
        for (int i = 0; i < 3; ++i)
            for (int j = i + 1; j < 3; ++j) {
                const float a = 0.5f * (S[3 * i + j] + S[3 * j + i]);
                S[3 * i + j] = S[3 * j + i] = a;
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                Am[3 * i + j] = m[i] * m[j] + m[3 + i] * m[3 + j] + m[6 + i] * m[6 + j];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                T[3 * i + j] = S[3 * i] * Am[j] + S[3 * i + 1] * Am[3 + j] + S[3 * i + 2] * Am[6 + j];
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                H[3 * i + j] = -(Am[3 * i] * T[j] + Am[3 * i + 1] * T[3 + j] + Am[3 * i + 2] * T[6 + j]);
        const float *P = poses + 12 * __float_as_uint(rc.feat.w);
        float v[3];
        for (int i = 0; i < 3; ++i) {
            const float mw = Ra[3 * i] * planes[(Scene::kMean + 0) * pitch + g] +
                             Ra[3 * i + 1] * planes[(Scene::kMean + 1) * pitch + g] +
                             Ra[3 * i + 2] * planes[(Scene::kMean + 2) * pitch + g] + ta[i];
            v[i] = mw - P[4 * i + 3];
        }
        const float tr = H[0] + H[4] + H[8], b2 = beam * beam;
        for (int i = 0; i < 3; ++i)
            G[9 + i] += b2 * (2.f * v[i] * tr -
                              2.f * (H[3 * i] * v[0] + H[3 * i + 1] * v[1] + H[3 * i + 2] * v[2]));
        if (actor) {    // H in the Gaussian's own frame: Ra^T H Ra
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    T[3 * i + j] = H[3 * i] * Ra[j] + H[3 * i + 1] * Ra[3 + j] + H[3 * i + 2] * Ra[6 + j];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    H[3 * i + j] = Ra[i] * T[j] + Ra[3 + i] * T[3 + j] + Ra[6 + i] * T[6 + j];
        }
    }
    if (actor) {
        for (int k = beam > 0.f ? 3 : 0; k < 4; ++k) {   // the rows of dL/dM, then dL/dmu
            const float x = G[3 * k], y = G[3 * k + 1], z = G[3 * k + 2];
            G[3 * k] = Ra[0] * x + Ra[3] * y + Ra[6] * z;
            G[3 * k + 1] = Ra[1] * x + Ra[4] * y + Ra[7] * z;
            G[3 * k + 2] = Ra[2] * x + Ra[5] * y + Ra[8] * z;
        }
    }
    float q[4];
    for (int k = 0; k < 4; ++k) q[k] = planes[(Scene::kQuat + k) * pitch + g];
    const float qn = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float w = q[0] / qn, x = q[1] / qn, y = q[2] / qn, z = q[3] / qn;
    const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                        2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                        2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    float gR[9];
    if (beam > 0.f) {
        // Sigma = sum_k s_k^2 r_k r_k^T: dL/dls_k = 2 s_k^2 r_k^T H r_k,
        // dL/dr_k = 2 s_k^2 H r_k
        for (int k = 0; k < 3; ++k) {
            const float s = expf(planes[(Scene::kLogScale + k) * pitch + g]), s2 = s * s;
            const float rk[3] = {R[k], R[3 + k], R[6 + k]};
            float Hr[3];
            for (int i = 0; i < 3; ++i) Hr[i] = H[3 * i] * rk[0] + H[3 * i + 1] * rk[1] + H[3 * i + 2] * rk[2];
            if (gls) gls[3 * g + k] += 2.f * s2 * (rk[0] * Hr[0] + rk[1] * Hr[1] + rk[2] * Hr[2]);
            for (int i = 0; i < 3; ++i) gR[3 * i + k] = 2.f * s2 * Hr[i];
        }
    } else {
        // M_k = r_k / s_k (r_k = column k of R): dL/dls_k = -G_k . M_k,
        // dL/dr_k = G_k / s_k
        for (int k = 0; k < 3; ++k) {
            const float s = expf(planes[(Scene::kLogScale + k) * pitch + g]);
            const float rk[3] = {R[k], R[3 + k], R[6 + k]};
            const float Gk[3] = {G[3 * k], G[3 * k + 1], G[3 * k + 2]};
            if (gls) gls[3 * g + k] += -(Gk[0] * rk[0] + Gk[1] * rk[1] + Gk[2] * rk[2]) / s;
            for (int i = 0; i < 3; ++i) gR[3 * i + k] = Gk[i] / s;
        }
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
    if (sh_features(feature_kind)) {
        // the SH origin: for LiDAR and rolling-shutter cameras, the origin of
        // the pose (column, row) that saw the mean, whose index the projection
        // left in the record's feat.w
        const bool lidar = feature_kind == SG_FEATURES_LIDAR_SH;
        if (lidar || posed_origin) {
            const float *P = poses + 12 * __float_as_uint(rec[g].feat.w);
            ox = P[3];
            oy = P[7];
            oz = P[11];
        }
        // the view direction, in the Gaussian's own frame (Ra^T (mu_w - o))
        const float lx = planes[(Scene::kMean + 0) * pitch + g];
        const float ly = planes[(Scene::kMean + 1) * pitch + g];
        const float lz = planes[(Scene::kMean + 2) * pitch + g];
        const float wx = Ra[0] * lx + Ra[1] * ly + Ra[2] * lz + ta[0] - ox;
        const float wy = Ra[3] * lx + Ra[4] * ly + Ra[5] * lz + ta[1] - oy;
        const float wz = Ra[6] * lx + Ra[7] * ly + Ra[8] * lz + ta[2] - oz;
        const float mx = actor ? Ra[0] * wx + Ra[3] * wy + Ra[6] * wz : wx;
        const float my = actor ? Ra[1] * wx + Ra[4] * wy + Ra[7] * wz : wy;
        const float mz = actor ? Ra[2] * wx + Ra[5] * wy + Ra[8] * wz : wz;
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
            if (!lidar && acc + 0.5f < 0.f) continue;   // clamped colour channel
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

static sg_status finish(const Scene &sc, Frame &fr, const float o[3], float beam,
                        const sg_grads &g, cudaStream_t st)
{
    if (sc.n == 0) return SG_OK;
    k_param_grads<<<(unsigned)((sc.n + 127) / 128), 128, 0, st>>>(
        sc.d_planes, sc.pitch, sc.n, sc.feature_kind, sc.sh_degree, sc.F, o[0], o[1], o[2],
        (const GRec *)fr.rec.p, fr.d_lidar_poses, actor_params(sc), beam, fr.kind == 2 ? 1 : 0,
        (const float *)fr.gacc.p, g.d_g_means, g.d_g_log_scales, g.d_g_quats, g.d_g_opacity,
        g.d_g_features);
    SG_LAUNCHED();
    return SG_OK;
}

static int blocks_per_sm(const void *kern, int threads)
{
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, 0) != cudaSuccess ||
        nb < 1)
        nb = 4;
    return nb;
}

static sg_status persistent_grid(const void *kern, int64_t max_items, int64_t &grid)
{
    int dev = 0, sms = 0;
    SG_CUDA(cudaGetDevice(&dev));
    SG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t cap = (max_items + kBwWarps - 1) / kBwWarps;
    grid = (int64_t)sms * blocks_per_sm(kern, 32 * kBwWarps);
    grid = grid < cap ? grid : cap;
    if (grid < 1) grid = 1;
    return SG_OK;
}

sg_status backward_camera(const Scene &sc, const Camera &cam, Frame &fr, const float *g_rgb,
                          const float *g_alpha, const float *g_depth, const sg_grads &g,
                          cudaStream_t st)
{
    if (fr.seg_len != kSegLen) {
        set_error("sg_backward_camera: the frame's render used another list segment length");
        return SG_ERR_INVALID;
    }
    sg_status s = ensure(fr.gacc, sizeof(float) * kG * (sc.n > 0 ? sc.n : 1));
    if (s != SG_OK) return s;
    SG_CUDA(cudaMemsetAsync(fr.gacc.p, 0, sizeof(float) * kG * sc.n, st));
    const CamRender P = cam_render_params(cam, fr.opts);
    const int nt = cam.ntx * cam.nty;
    const WorkSize ws = work_size(nt, fr.n_pairs, kSegLen, 8);
    const unsigned char *cw = (const unsigned char *)fr.camwork.p;
    uint32_t *counter = (uint32_t *)fr.scalars.p + 6;
    SG_CUDA(cudaMemsetAsync(counter, 0, sizeof(uint32_t), st));
    int64_t grid = 0;
    if (fr.kind == 2) {     // rolling shutter: poses per pixel row
        if ((s = persistent_grid((const void *)k_backward_camera_rs, ws.max_items, grid)) != SG_OK)
            return s;
        k_backward_camera_rs<<<(unsigned)grid, 32 * kBwWarps, 0, st>>>(
            P, (const GRec *)fr.rec.p, (const uint32_t *)fr.pvals[fr.pair_buf].p,
            (const uint2 *)fr.ranges.p, (const uint2 *)(cw + ws.info_bytes + ws.off_bytes),
            (const uint2 *)cw, (const uint32_t *)fr.scalars.p + 4, (const uint32_t *)fr.submask.p,
            counter, (const float4 *)fr.partials.p, cam.d_pix, cam.d_tile_dir, fr.d_lidar_poses,
            (const float4 *)fr.ray_state.p, (const float4 *)fr.ray_feat.p,
            (const uint32_t *)fr.n_contrib.p, g_rgb, g_alpha, g_depth, (float *)fr.gacc.p);
        SG_LAUNCHED();
        const float o[3] = {0.f, 0.f, 0.f};
        return finish(sc, fr, o, 0.f, g, st);
    }
    if ((s = persistent_grid((const void *)k_backward_camera, ws.max_items, grid)) != SG_OK)
        return s;
    k_backward_camera<<<(unsigned)grid, 32 * kBwWarps, 0, st>>>(
        P, (const GRec *)fr.rec.p, (const uint32_t *)fr.pvals[fr.pair_buf].p,
        (const uint2 *)fr.ranges.p, (const uint2 *)(cw + ws.info_bytes + ws.off_bytes),
        (const uint2 *)cw, (const uint32_t *)fr.scalars.p + 4, (const uint32_t *)fr.submask.p,
        counter, (const float4 *)fr.partials.p, cam.d_pix, cam.d_tile_dir,
        (const RenderDesc *)fr.desc.p, (const float4 *)fr.ray_state.p,
        (const float4 *)fr.ray_feat.p, (const uint32_t *)fr.n_contrib.p, g_rgb, g_alpha,
        g_depth, (float *)fr.gacc.p);
    SG_LAUNCHED();
    const float o[3] = {fr.c2w[3], fr.c2w[7], fr.c2w[11]};
    return finish(sc, fr, o, 0.f, g, st);
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
        const WorkSize ws = work_size(L.n_items, fr.n_pairs * L.max_items_per_tile, kSegLen, 1);
        const unsigned char *cw = (const unsigned char *)fr.camwork.p;
        uint32_t *counter = (uint32_t *)fr.scalars.p + 6;
        SG_CUDA(cudaMemsetAsync(counter, 0, sizeof(uint32_t), st));
        int64_t grid = 0;
        if ((s = persistent_grid((const void *)k_backward_lidar, ws.max_items, grid)) != SG_OK)
            return s;
        k_backward_lidar<<<(unsigned)grid, 32 * kBwWarps, 0, st>>>(
            P, L.d_items, L.d_item_rays, L.d_ray_e, L.d_tile_u, fr.d_lidar_poses,
            L.d_tile_items, (const uint32_t *)fr.lmask.p, fr.lmask_stride,
            (const GRec *)fr.rec.p, (const uint32_t *)fr.pvals[fr.pair_buf].p,
            (const uint2 *)fr.ranges.p, (const uint2 *)(cw + ws.info_bytes + ws.off_bytes),
            (const uint2 *)cw, (const uint32_t *)fr.scalars.p + 4, counter,
            (const float4 *)fr.partials.p, (const float4 *)fr.ray_state.p,
            (const float4 *)fr.ray_feat.p, (const uint32_t *)fr.n_contrib.p, g_range, g_int,
            g_drop, g_alpha, (float *)fr.gacc.p);
        SG_LAUNCHED();
    }
    const float o[3] = {0.f, 0.f, 0.f};
    return finish(sc, fr, o, fr.opts.beam_divergence, g, st);
}

}  // namespace sg
