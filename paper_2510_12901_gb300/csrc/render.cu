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
// Camera: persistent independent warps, one 8x4 pixel sub-block of a 16x16
// tile per work item, densest tiles first (k_render_camera below).  LiDAR:
// one warp per work item (<= 32 rays of one tile, <= 4 columns); batches of
// 32 list entries staged through the warp's shared-memory slice.
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

// Per (tile, Gaussian) pair of a camera list: which of the tile's eight
// 8x4 pixel sub-blocks the Gaussian's extent box can reach (bit w: columns
// 8*(w&1).., rows 4*(w>>1)..).  One byte per pair, written after the tile
// sort, so that the compositing warps scan contiguous bytes instead of
// gathering every entry's box.
__global__ void k_submask(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ ids,
                          const GRec *__restrict__ rec, int64_t K, int ntx,
                          uint8_t *__restrict__ mask)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K) return;
    const uint32_t t = keys[i];
    const float4 rc = rec[ids[i]].rect;
    const int tx = (int)(t % (uint32_t)ntx), ty = (int)(t / (uint32_t)ntx);
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const float x0 = (float)(tx * kTile + 8 * (w & 1)) + 0.5f;
        const float y0 = (float)(ty * kTile + 4 * (w >> 1)) + 0.5f;
        if (rc.x <= x0 + 7.f && rc.y >= x0 && rc.z <= y0 + 3.f && rc.w >= y0) m |= 1u << w;
    }
    mask[i] = (uint8_t)m;
}

// Camera compositing, persistent and warp-independent.  A work item is one
// 8x4 pixel sub-block of a 16x16 tile (eight per tile); items are taken in
// order of decreasing tile-list length through an atomic counter, so the
// densest tiles start first and their eight sub-blocks run on different
// SMs.  A warp reads its tile's sub-block masks 32 at a time, keeps (in list
// order) the entries whose extent box can reach one of its pixel centres,
// preprocesses only those into its shared-memory slice, and composites them
// branch-free.  There is no block-level barrier.
constexpr int kCamWarps = 4;       // warps per block of the persistent grid

__global__ void __launch_bounds__(32 * kCamWarps, 6)
k_render_camera(CamRender P, const GRec *__restrict__ rec, const uint32_t *__restrict__ ids,
                const uint2 *__restrict__ ranges, const uint32_t *__restrict__ order,
                const uint8_t *__restrict__ submask, int n_items, uint32_t *__restrict__ counter,
                const float4 *__restrict__ pix,
                const double *__restrict__ tile_dir, float *__restrict__ out_rgb,
                float *__restrict__ out_alpha, float *__restrict__ out_depth,
                float4 *__restrict__ ray_state, uint32_t *__restrict__ n_contrib)
{
    __shared__ float4 s_all[kCamWarps][9][32];
    __shared__ uint32_t s_pos[kCamWarps][32];
    __shared__ float s_refs[kCamWarps][6];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float4(*s_e)[32] = s_all[wib];
    float *s_ref = s_refs[wib];
    while (true) {
        uint32_t item = 0;
        if (lane == 0) item = atomicAdd(counter, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= (uint32_t)n_items) break;
        const int tile = (int)order[item >> 3], sub = (int)(item & 7);
        const int tx = tile % P.ntx, ty = tile / P.ntx;
        const int sbx = tx * kTile + 8 * (sub & 1), sby = ty * kTile + 4 * (sub >> 1);
        const int px = sbx + (lane & 7), py = sby + (lane >> 3);
        if (lane == 0) cam_tile_ref(P, tile_dir, tile, s_ref);
        __syncwarp();
        const float dh[3] = {s_ref[0], s_ref[1], s_ref[2]};
        const float dl[3] = {s_ref[3], s_ref[4], s_ref[5]};
        const bool inside = px < P.W && py < P.H;
        const int64_t pidx = (int64_t)py * P.W + px;
        const float4 e = inside ? pix[pidx] : make_float4(0.f, 0.f, 0.f, 0.f);
        bool done = !(inside && e.w > 0.f);
        float dd[3];
        cam_ray_offset(P, e, dd);
        const float rx = (float)px + 0.5f, ry = (float)py + 0.5f;
        float T = 1.f, W = 0.f, Z = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f;
        uint32_t last = 0;
        const uint2 rg = ranges[tile];
        for (uint32_t base = rg.x; base < rg.y; base += 32) {
            if (__all_sync(0xffffffffu, done)) break;
            const uint32_t idx = base + lane;
            const bool ov = idx < rg.y && ((submask[idx] >> sub) & 1u);
            const uint32_t bal = __ballot_sync(0xffffffffu, ov);
            if (bal == 0u) continue;
            __syncwarp();
            if (ov) {
                const int pos = __popc(bal & ((1u << lane) - 1u));
                float4 ent[9];
                cam_entry(rec[ids[idx]], P.t, dh, dl, ent);
#pragma unroll
                for (int k = 0; k < 9; ++k) s_e[k][pos] = ent[k];
                s_pos[wib][pos] = idx + 1 - rg.x;
            }
            __syncwarp();
            const int n = __popc(bal);
            for (int j = 0; j < n; ++j) {
                PairEval pe;
                bool ok = cam_pair(s_e[0][j], s_e[1][j], s_e[2][j], s_e[3][j], s_e[4][j],
                                   s_e[5][j], s_e[6][j], s_e[8][j], dd, rx, ry, P.alpha_min,
                                   P.alpha_max, pe);
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
                last = ok ? s_pos[wib][j] : last;
            }
        }
        if (inside) {
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
        __syncwarp();
    }
}

static int cam_blocks_per_sm()
{
    static int cached = 0;
    if (!cached) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_camera, 32 * kCamWarps,
                                                          0) != cudaSuccess || nb < 1)
            nb = 4;
        cached = nb;
    }
    return cached;
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
    const int64_t K = fr.n_pairs;
    s = ensure(fr.submask, K > 0 ? (size_t)K : 1);
    if (s != SG_OK) return s;
    const uint32_t *ids = (const uint32_t *)fr.pvals[fr.pair_buf].p;
    if (K > 0) {
        k_submask<<<(unsigned)((K + 255) / 256), 256, 0, st>>>(
            (const uint32_t *)fr.pkeys[fr.pair_buf].p, ids, (const GRec *)fr.rec.p, K, cam.ntx,
            (uint8_t *)fr.submask.p);
        SG_LAUNCHED();
    }
    uint32_t *counter = (uint32_t *)fr.scalars.p + 2;
    SG_CUDA(cudaMemsetAsync(counter, 0, sizeof(uint32_t), st));
    int dev = 0, sms = 0;
    SG_CUDA(cudaGetDevice(&dev));
    SG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int n_items = 8 * nt;
    int grid = sms * cam_blocks_per_sm();
    grid = grid < (n_items + kCamWarps - 1) / kCamWarps ? grid : (n_items + kCamWarps - 1) / kCamWarps;
    if (grid < 1) grid = 1;
    k_render_camera<<<grid, 32 * kCamWarps, 0, st>>>(
        P, (const GRec *)fr.rec.p, ids, (const uint2 *)fr.ranges.p, (const uint32_t *)fr.order.p,
        (const uint8_t *)fr.submask.p, n_items, counter, cam.d_pix, cam.d_tile_dir, rgb, alpha, depth, (float4 *)fr.ray_state.p,
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
