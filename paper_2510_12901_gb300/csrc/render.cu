// render.cu -- per-ray front-to-back compositing (Eq. 1) with the particle
// response evaluated in 3D at tau_max, the maximiser of rho along the ray
// (Sec. 3.2, following 3DGRT).
//
// For a Gaussian with M = S^-1 R^T (so Sigma^-1 = M^T M) and a ray o + t d:
//   tau_max = (M v) . (M d) / |M d|^2,    v = mu - o,
//   D^2     = |(M (o - mu)) x (M d)|^2 / |M d|^2
//           = |cof(M) (v x d)|^2 / |M d|^2,
// and cof(M) = det(M) M^-T has rows f_k M_k with f_k = s_k / (s_i s_j).
// v x d is the moment of the ray about the Gaussian centre; for a far, thin
// Gaussian it is tiny next to |v| |d| and a direct float evaluation loses
// most of its digits.  Each ray is therefore written as d = d_T + dd with a
// per-tile reference direction d_T (double, split into two floats) and a
// small float offset dd computed in double at set-up.  Per (tile, Gaussian)
// the moment v x d_T is evaluated once with error-free transformations
// (TwoSum, Kahan's difference of products); per (ray, Gaussian) only the
// well-conditioned part v x dd remains:
//   cof(M)(v x d) = a + P dd,  a = diag(f) M (v x d_T),  P = diag(f) M [v]_x.
// Float arithmetic throughout, no double-precision work in the per-pair loop.
//
// Camera: one 256-thread CTA per 16x16 tile, launched longest list first;
// batches of 256 list entries are staged through shared memory (one entry
// per thread, preprocessed); each warp walks only the entries overlapping its
// 8x4 sub-block; the CTA stops once every pixel's transmittance is below
// t_min.  LiDAR: one warp per work item (<= 32 rays of one tile, <= 4
// columns); batches of 32.
//
// Per ray the kernels save (T_final, omega, Z, drop) and the number of list
// entries up to the last composited one, which is all the backward needs.
#include <math.h>

#include "pairs.cuh"
#include "render.cuh"

namespace sg {

// Tile order for the camera kernels: tiles sorted (coarsely) by decreasing
// list length, so that the longest tiles start first and do not form the
// tail of the launch.  One CTA buckets the tiles by floor(log2(length)).
__global__ void __launch_bounds__(1024)
k_tile_order(const uint2 *__restrict__ ranges, int ntiles, uint32_t *__restrict__ order)
{
    __shared__ uint32_t s_cnt[33], s_off[33];
    if (threadIdx.x < 33) s_cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        const uint32_t len = ranges[t].y - ranges[t].x;
        const int b = len ? 32 - __clz(len) : 0;       // 0 (empty) .. 32
        atomicAdd(&s_cnt[32 - b], 1u);                   // longest bucket first
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int i = 0; i < 33; ++i) { s_off[i] = run; run += s_cnt[i]; }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        const uint32_t len = ranges[t].y - ranges[t].x;
        const int b = len ? 32 - __clz(len) : 0;
        order[atomicAdd(&s_off[32 - b], 1u)] = (uint32_t)t;
    }
}

// Camera compositing.  The 16x16 tile is split into eight 8x4 pixel
// sub-blocks, one per warp.  Each batch of up to 256 list entries is
// preprocessed into shared memory once (one entry per thread); each warp
// then compacts, in list order, the entries whose extent box overlaps its
// sub-block and walks only those, branch-free, so that a far Gaussian a
// pixel wide costs one warp instead of eight.
__global__ void __launch_bounds__(kCamThreads)
k_render_camera(CamRender P, const GRec *__restrict__ rec, const uint32_t *__restrict__ ids,
                const uint2 *__restrict__ ranges, const uint32_t *__restrict__ order,
                const float4 *__restrict__ pix, const double *__restrict__ tile_dir,
                float *__restrict__ out_rgb, float *__restrict__ out_alpha,
                float *__restrict__ out_depth, float4 *__restrict__ ray_state,
                uint32_t *__restrict__ n_contrib)
{
    __shared__ float4 s_e[9][kCamThreads];
    __shared__ uint8_t s_mask[kCamThreads];
    __shared__ uint8_t s_list[kCamThreads / 32][kCamThreads];
    __shared__ float s_ref[6];
    const int tile = (int)order[blockIdx.x];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = tile % P.ntx, ty = tile / P.ntx;
    // warp w: columns 8*(w&1) .. +7, rows 4*(w>>1) .. +3 of the tile
    const int sbx = tx * kTile + 8 * (warp & 1), sby = ty * kTile + 4 * (warp >> 1);
    const int px = sbx + (lane & 7), py = sby + (lane >> 3);
    if (tid == 0) cam_tile_ref(P, tile_dir, tile, s_ref);
    __syncthreads();
    const float dh[3] = {s_ref[0], s_ref[1], s_ref[2]};
    const float dl[3] = {s_ref[3], s_ref[4], s_ref[5]};
    const bool inside = px < P.W && py < P.H;
    const int64_t pidx = (int64_t)py * P.W + px;
    float4 e = inside ? pix[pidx] : make_float4(0.f, 0.f, 0.f, 0.f);
    bool done = !(inside && e.w > 0.f);
    float dd[3];
    cam_ray_offset(P, e, dd);
    const float rx = (float)px + 0.5f, ry = (float)py + 0.5f;
    float T = 1.f, W = 0.f, Z = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
    uint32_t last = 0;
    const uint2 rg = ranges[tile];
    for (uint32_t base = rg.x; base < rg.y; base += kCamThreads) {
        if (__syncthreads_count(done) == kCamThreads) break;
        const uint32_t idx = base + tid;
        uint8_t m = 0;
        if (idx < rg.y) {
            float4 ent[9];
            cam_entry(rec[ids[idx]], P.t, dh, dl, ent);
#pragma unroll
            for (int k = 0; k < 9; ++k) s_e[k][tid] = ent[k];
            // sub-blocks whose pixel centres the box can contain
            const float4 rc = ent[8];
#pragma unroll
            for (int w = 0; w < kCamThreads / 32; ++w) {
                const float x0 = (float)(tx * kTile + 8 * (w & 1)) + 0.5f;
                const float y0 = (float)(ty * kTile + 4 * (w >> 1)) + 0.5f;
                if (rc.x <= x0 + 7.f && rc.y >= x0 && rc.z <= y0 + 3.f && rc.w >= y0)
                    m |= (uint8_t)(1u << w);
            }
        }
        s_mask[tid] = m;
        __syncthreads();
        // this warp's entries, in list order
        int n = 0;
#pragma unroll
        for (int c = 0; c < kCamThreads / 32; ++c) {
            const bool mine = (s_mask[c * 32 + lane] >> warp) & 1u;
            const uint32_t bal = __ballot_sync(0xffffffffu, mine);
            if (mine) s_list[warp][n + __popc(bal & ((1u << lane) - 1u))] = (uint8_t)(c * 32 + lane);
            n += __popc(bal);
        }
        __syncwarp();
        for (int i = 0; i < n; ++i) {
            if (__all_sync(0xffffffffu, done)) break;
            const int j = s_list[warp][i];
            PairEval pe;
            bool ok = cam_pair(s_e[0][j], s_e[1][j], s_e[2][j], s_e[3][j], s_e[4][j], s_e[5][j],
                               s_e[6][j], s_e[8][j], dd, rx, ry, P.alpha_min, P.alpha_max, pe);
            ok = ok && !done;
            const float Tn = T * (1.f - pe.alpha);
            const bool stop = ok && Tn < P.t_min;
            done = done || stop;
            ok = ok && !stop;
            const float wgt = ok ? pe.alpha * T : 0.f;
            const float4 col = s_e[7][j];
            c0 += wgt * col.x;
            c1 += wgt * col.y;
            c2 += wgt * col.z;
            Z += wgt * pe.tau;
            W += wgt;
            T = ok ? Tn : T;
            last = ok ? base + j + 1 - rg.x : last;
        }
    }
    if (!inside) return;
    if (out_rgb) {
        out_rgb[3 * pidx] = c0;
        out_rgb[3 * pidx + 1] = c1;
        out_rgb[3 * pidx + 2] = c2;
    }
    if (out_alpha) out_alpha[pidx] = W;
    if (out_depth) out_depth[pidx] = W > 0.f ? Z / W : 0.f;
    ray_state[pidx] = make_float4(T, W, Z, 0.f);
    n_contrib[pidx] = last;
}

sg_status render_camera(const Camera &cam, const float c2w[12], const sg_render_opts &o,
                        Frame &fr, float *rgb, float *alpha, float *depth, cudaStream_t st)
{
    const CamRender P = cam_render_params(cam, c2w, o);
    const int nt = cam.ntx * cam.nty;
    sg_status s = ensure(fr.order, sizeof(uint32_t) * (nt > 0 ? nt : 1));
    if (s != SG_OK) return s;
    k_tile_order<<<1, 1024, 0, st>>>((const uint2 *)fr.ranges.p, nt, (uint32_t *)fr.order.p);
    SG_LAUNCHED();
    const uint32_t *ids = (const uint32_t *)fr.pvals[fr.pair_buf].p;
    k_render_camera<<<(unsigned)nt, kCamThreads, 0, st>>>(
        P, (const GRec *)fr.rec.p, ids, (const uint2 *)fr.ranges.p, (const uint32_t *)fr.order.p,
        cam.d_pix, cam.d_tile_dir, rgb, alpha, depth, (float4 *)fr.ray_state.p,
        (uint32_t *)fr.n_contrib.p);
    SG_LAUNCHED();
    return SG_OK;
}

// ------------------------------------------------------------------ LiDAR

__global__ void __launch_bounds__(32 * kLidarWarps)
k_render_lidar(LidRender P, const LidarItem *__restrict__ items,
               const uint32_t *__restrict__ item_rays, const float4 *__restrict__ ray_e,
               const double *__restrict__ item_u, const float *__restrict__ poses,
               const float *__restrict__ az_col, const float *__restrict__ elev,
               const GRec *__restrict__ rec, const uint32_t *__restrict__ ids,
               const uint2 *__restrict__ ranges, float *__restrict__ out_range,
               float *__restrict__ out_int, float *__restrict__ out_drop,
               float *__restrict__ out_alpha, float4 *__restrict__ ray_state,
               uint32_t *__restrict__ n_contrib)
{
    __shared__ float s_all[kLidarWarps][kLidEntry][32];
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
    bool done = !valid;
    float T = 1.f, W = 0.f, Z = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
    uint32_t last = 0;
    const uint2 rg = ranges[it.tile];
    for (uint32_t base = rg.x; base < rg.y; base += 32) {
        if (__all_sync(0xffffffffu, done)) break;
        const uint32_t idx = base + lane;
        __syncwarp();
        if (idx < rg.y) lidar_entry(rec[ids[idx]], poses, it.col0, it.ncols, dh, dl, s, lane);
        __syncwarp();
        const int cnt = min(32u, rg.y - base);
        for (int j = 0; j < cnt && !done; ++j) {
            PairEval pe;
            if (!lidar_pair(s, j, sb, raz, rel, dd, d, P.alpha_min, P.alpha_max, pe)) continue;
            const float Tn = T * (1.f - pe.alpha);
            if (Tn < P.t_min) { done = true; break; }
            const float wgt = pe.alpha * T;
            c0 += wgt * s[13][j];
            c1 += wgt * s[14][j];
            c2 += wgt * s[15][j];
            Z += wgt * pe.tau;
            W += wgt;
            T = Tn;
            last = base + j + 1 - rg.x;
        }
    }
    if (!valid) return;
    const float drop = 1.f / (1.f + expf(c1 - c2));
    if (out_range) out_range[ray] = W > 0.f ? Z / W : 0.f;
    if (out_int) out_int[ray] = c0;
    if (out_drop) out_drop[ray] = drop;
    if (out_alpha) out_alpha[ray] = W;
    ray_state[ray] = make_float4(T, W, Z, drop);
    n_contrib[ray] = last;
}

sg_status render_lidar(const Lidar &L, const float *d_poses, const sg_render_opts &o,
                       Frame &fr, float *range, float *intensity, float *drop, float *alpha,
                       cudaStream_t st)
{
    const LidRender P = lidar_render_params(L, o);
    if (L.n_items == 0) return SG_OK;
    const uint32_t *ids = (const uint32_t *)fr.pvals[fr.pair_buf].p;
    unsigned grid = (unsigned)((L.n_items + kLidarWarps - 1) / kLidarWarps);
    k_render_lidar<<<grid, 32 * kLidarWarps, 0, st>>>(
        P, L.d_items, L.d_item_rays, L.d_ray_e, L.d_tile_u, d_poses, L.d_az, L.d_elev,
        (const GRec *)fr.rec.p, ids, (const uint2 *)fr.ranges.p, range, intensity, drop, alpha,
        (float4 *)fr.ray_state.p, (uint32_t *)fr.n_contrib.p);
    SG_LAUNCHED();
    return SG_OK;
}

}  // namespace sg
