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

// Exclusive sum over a block of 1024 threads; every thread calls it.
__device__ __forceinline__ uint32_t block_excl_scan_1024(uint32_t v, uint32_t *s_w, uint32_t &total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
        uint32_t x = s_w[lane];
        uint32_t xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= o) xi += t;
        }
        s_w[lane] = xi - x;
        if (lane == 31) s_w[32] = xi;
    }
    __syncthreads();
    const uint32_t r = s_w[w] + inc - v;
    total = s_w[32];
    __syncthreads();
    return r;
}

// Work items of the camera compositing.  Tiles are taken in (coarsely)
// decreasing list length, so the longest start first.  A tile whose list is
// longer than seg_len entries is split along the list into
// ceil(len / seg_len) segments; every (tile, segment) gives eight items, one
// per 8x4 sub-block.  k_camera_items (one CTA) orders the tiles and assigns
// per tile (segments, first partial slot) and its first item; k_emit_items
// (one warp per tile) writes the items (tile, 8 seg + sub) and resets the
// arrival counters of long tiles.  The item counter of the compositing
// kernel is reset here too.
__global__ void __launch_bounds__(1024)
k_camera_items(const uint2 *__restrict__ ranges, int ntiles, uint32_t seg_len,
               uint32_t *__restrict__ order, uint2 *__restrict__ tile_info,
               uint32_t *__restrict__ item_off, uint32_t *__restrict__ counts,
               uint32_t *__restrict__ counter)
{
    __shared__ uint32_t s_cnt[33], s_off[33], s_w[33];
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
    __syncthreads();
    uint32_t item_run = 0, part_run = 0;
    for (int c0 = 0; c0 < ntiles; c0 += blockDim.x) {
        const int k = c0 + threadIdx.x;
        uint32_t t = 0, nseg = 0;
        if (k < ntiles) {
            t = order[k];
            const uint32_t len = ranges[t].y - ranges[t].x;
            nseg = len > seg_len ? (len + seg_len - 1) / seg_len : 1u;
        }
        uint32_t tot_items, tot_parts;
        const uint32_t ib = item_run + block_excl_scan_1024(k < ntiles ? 8 * nseg : 0, s_w, tot_items);
        const uint32_t pb = part_run + block_excl_scan_1024(nseg > 1 ? nseg : 0, s_w, tot_parts);
        if (k < ntiles) {
            tile_info[t] = make_uint2(nseg, pb);
            item_off[k] = ib;
        }
        item_run += tot_items;
        part_run += tot_parts;
    }
    if (threadIdx.x == 0) {
        counts[0] = item_run;
        counts[1] = part_run;
        *counter = 0u;
    }
}

__global__ void k_emit_items(const uint32_t *__restrict__ order,
                             const uint2 *__restrict__ tile_info,
                             const uint32_t *__restrict__ item_off, int ntiles,
                             uint2 *__restrict__ items, uint32_t *__restrict__ arrive)
{
    const int k = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (k >= ntiles) return;
    const uint32_t t = order[k];
    const uint2 ti = tile_info[t];
    const uint32_t ib = item_off[k], n = 8 * ti.x;
    for (uint32_t i = lane; i < n; i += 32) items[ib + i] = make_uint2(t, i);
    if (ti.x > 1 && lane < 8) arrive[ti.y * 8 + lane] = 0u;
}

// Per (tile, Gaussian) pair of a camera list: which of the tile's eight
// 8x4 pixel sub-blocks hold a pixel centre inside the Gaussian's extent box
// (bit w: columns 8*(w&1).., rows 4*(w>>1)..), by the same float comparisons
// as the per-ray test.  One byte per pair, written after the tile sort, so
// that the compositing warps scan contiguous bytes and never stage an entry
// that no pixel of their sub-block can see.
__global__ void k_submask(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ ids,
                          const GRec *__restrict__ rec, const uint32_t *__restrict__ d_K, int ntx,
                          uint8_t *__restrict__ mask)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)*d_K) return;
    const uint32_t t = keys[i];
    const float4 rc = rec[ids[i]].rect;
    const int tx = (int)(t % (uint32_t)ntx), ty = (int)(t / (uint32_t)ntx);
    uint32_t cols = 0, rows = 0;
#pragma unroll
    for (int c = 0; c < kTile; ++c) {
        const float x = (float)(tx * kTile + c) + 0.5f;
        const float y = (float)(ty * kTile + c) + 0.5f;
        cols |= (uint32_t)(x >= rc.x && x <= rc.y) << c;
        rows |= (uint32_t)(y >= rc.z && y <= rc.w) << c;
    }
    uint32_t m = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
        const bool cx = ((cols >> (8 * (w & 1))) & 0xffu) != 0u;
        const bool cy = ((rows >> (4 * (w >> 1))) & 0xfu) != 0u;
        m |= (uint32_t)(cx && cy) << w;
    }
    mask[i] = (uint8_t)m;
}

// Camera compositing, persistent and warp-independent.  A work item is one
// 8x4 pixel sub-block of a 16x16 tile and one segment of that tile's list
// (k_camera_items); items are taken in order of decreasing tile-list length
// through an atomic counter, so the densest tiles start first and their
// sub-blocks and segments run on different SMs.  A warp reads its segment's
// sub-block masks 32 at a time, keeps (in list order) the entries whose
// extent box can reach one of its pixel centres, preprocesses only those into
// its shared-memory slice, and composites them branch-free.  There is no
// block-level barrier.
//
// Segments of a long tile are composited independently from T = 1.  Eq. 1
// is associative over consecutive runs of the list: with (C_s, omega_s, Z_s,
// T_s) the sums and the transmittance of run s started at T = 1, the whole
// list gives C = C_0 + T_0 C_1 + T_0 T_1 C_2 + ... and T = prod T_s, as long
// as the termination test (T_before * (1 - alpha) < T_min) never fires.  It
// fires inside run s exactly when the running product drops below T_min
// there, i.e. when T_<s * T_s < T_min or the run itself stopped (its local
// transmittance is an upper bound of the true one).  The last warp to finish
// a (tile, sub-block) combines the runs in order and re-walks, from the true
// transmittance, the one run in which a ray stops.  Run 0 starts from the
// true state, so its own stop is final.
constexpr int kCamWarps = 4;       // warps per block of the persistent grid

struct CamAcc {
    float T, W, Z, c0, c1, c2;
    uint32_t last;                 // list entries up to the last composited one
};

// Composite list entries [lo, hi) of a tile (first entry `begin`) that can
// reach sub-block `sub` into the lane's accumulator; lanes with done = true
// take part in the warp's staging but keep their state.  Returns whether the
// lane's ray stopped at T_min.
__device__ __forceinline__ bool cam_walk(const CamRender &P, const CamPose &pose,
                                         const GRec *__restrict__ rec,
                                         const uint32_t *__restrict__ ids,
                                         const uint8_t *__restrict__ submask, int sub,
                                         int sbx, int sby, uint32_t lo, uint32_t hi,
                                         uint32_t begin, const float dh[3], const float dl[3],
                                         const float dd[3], float4 (*s_e)[32],
                                         uint32_t *s_pos, uint32_t *s_lanes, CamAcc &a,
                                         bool done)
{
    const int lane = threadIdx.x & 31;
    const bool done0 = done;
    for (uint32_t base = lo; base < hi; base += 32) {
        if (__all_sync(0xffffffffu, done)) break;
        const uint32_t idx = base + lane;
        const bool ov = idx < hi && ((submask[idx] >> sub) & 1u);
        const uint32_t bal = __ballot_sync(0xffffffffu, ov);
        if (bal == 0u) continue;
        __syncwarp();
        if (ov) {
            const int pos = __popc(bal & ((1u << lane) - 1u));
            float4 ent[9];
            cam_entry(rec[ids[idx]], pose.t, dh, dl, ent);
#pragma unroll
            for (int k = 0; k < 8; ++k) s_e[k][pos] = ent[k];
            s_lanes[pos] = subblock_lanes(ent[8], sbx, sby);
            s_pos[pos] = idx + 1 - begin;
        }
        __syncwarp();
        const int n = __popc(bal);
        for (int j = 0; j < n; ++j) {
            PairEval pe;
            bool ok = cam_pair_in(s_e[0][j], s_e[1][j], s_e[2][j], s_e[3][j], s_e[4][j],
                                  s_e[5][j], s_e[6][j], (s_lanes[j] >> lane) & 1u, dd,
                                  P.alpha_min, P.alpha_max, pe);
            ok = ok && !done;
            const float Tn = a.T * (1.f - pe.alpha);
            const bool stop = ok && Tn < P.t_min;
            done = done || stop;
            ok = ok && !stop;
            const float wgt = ok ? pe.alpha * a.T : 0.f;
            const float4 col = s_e[7][j];
            a.c0 += wgt * col.x;
            a.c1 += wgt * col.y;
            a.c2 += wgt * col.z;
            a.Z += wgt * pe.tau;
            a.W += wgt;
            a.T = ok ? Tn : a.T;
            a.last = ok ? s_pos[j] : a.last;
        }
    }
    return done && !done0;   // the ray stopped at T_min in this walk
}

template <uint32_t kSeg>
__global__ void __launch_bounds__(32 * kCamWarps, 6)
k_render_camera(CamRender P, const GRec *__restrict__ rec, const uint32_t *__restrict__ ids,
                const uint2 *__restrict__ ranges, const uint2 *__restrict__ items,
                const uint2 *__restrict__ tile_info, const uint32_t *__restrict__ counts,
                const uint8_t *__restrict__ submask, uint32_t *__restrict__ counter,
                uint32_t *__restrict__ arrive, float4 *__restrict__ partials,
                const float4 *__restrict__ pix, const double *__restrict__ tile_dir,
                const RenderDesc *__restrict__ D, float4 *__restrict__ ray_state,
                uint32_t *__restrict__ n_contrib)
{
    __shared__ float4 s_all[kCamWarps][8][32];
    __shared__ uint32_t s_pos[kCamWarps][32];
    __shared__ uint32_t s_lanes[kCamWarps][32];
    __shared__ float s_refs[kCamWarps][6];
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
        const uint2 ti = tile_info[tile];            // (segments, first partial slot)
        const int tx = tile % P.ntx, ty = tile / P.ntx;
        const int sbx = tx * kTile + 8 * (sub & 1), sby = ty * kTile + 4 * (sub >> 1);
        const int px = sbx + (lane & 7), py = sby + (lane >> 3);
        if (lane == 0) cam_tile_ref(s_pose, tile_dir, tile, s_ref);
        __syncwarp();
        const float dh[3] = {s_ref[0], s_ref[1], s_ref[2]};
        const float dl[3] = {s_ref[3], s_ref[4], s_ref[5]};
        const bool inside = px < P.W && py < P.H;
        const int64_t pidx = (int64_t)py * P.W + px;
        const float4 e = inside ? pix[pidx] : make_float4(0.f, 0.f, 0.f, 0.f);
        const bool no_ray = !(inside && e.w > 0.f);
        float dd[3];
        cam_ray_offset(s_pose, e, dd);
        const uint2 rg = ranges[tile];
        const uint32_t lo = rg.x + (uint32_t)seg * kSeg;
        const uint32_t hi = min(rg.y, lo + kSeg);
        CamAcc a = {1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u};
        const bool stopped = cam_walk(P, s_pose, rec, ids, submask, sub, sbx, sby, lo, hi, rg.x,
                                      dh, dl, dd, s_e, s_pos[wib], s_lanes[wib], a, no_ray);
        if (ti.x > 1) {
            // long tile: publish this run, and combine if it is the last one
            float4 *pp = partials + ((size_t)(ti.y + seg) * 256 + sub * 32 + lane) * 2;
            pp[0] = make_float4(a.c0, a.c1, a.c2, a.W);
            pp[1] = make_float4(a.Z, a.T, __uint_as_float(a.last), stopped ? 1.f : 0.f);
            __threadfence();
            __syncwarp();
            uint32_t prev = 0;
            if (lane == 0) prev = atomicAdd(&arrive[ti.y * 8 + sub], 1u);
            prev = __shfl_sync(0xffffffffu, prev, 0);
            if (prev != ti.x - 1) {
                __syncwarp();
                continue;
            }
            __threadfence();
            const float4 *pq = partials + ((size_t)ti.y * 256 + sub * 32 + lane) * 2;
            float4 u = __ldcg(pq), v = __ldcg(pq + 1);
            a = {v.y, u.w, v.x, u.x, u.y, u.z, __float_as_uint(v.z)};
            bool fin = no_ray || v.w != 0.f;
            for (uint32_t sgi = 1; sgi < ti.x; ++sgi) {
                if (__all_sync(0xffffffffu, fin)) break;
                pq += 512;
                u = __ldcg(pq);
                v = __ldcg(pq + 1);
                const bool take = !fin && v.w == 0.f && a.T * v.y >= P.t_min;
                const bool redo = !fin && !take;
                if (take) {
                    a.c0 += a.T * u.x;
                    a.c1 += a.T * u.y;
                    a.c2 += a.T * u.z;
                    a.W += a.T * u.w;
                    a.Z += a.T * v.x;
                    a.T *= v.y;
                    const uint32_t l = __float_as_uint(v.z);
                    a.last = l ? l : a.last;
                }
                if (__any_sync(0xffffffffu, redo)) {
                    const uint32_t l0 = rg.x + sgi * kSeg;
                    cam_walk(P, s_pose, rec, ids, submask, sub, sbx, sby, l0,
                             min(rg.y, l0 + kSeg), rg.x, dh, dl, dd, s_e, s_pos[wib],
                             s_lanes[wib], a, !redo);
                }
                fin = fin || redo;
            }
        }
        if (inside) {
            float *const out_rgb = D->out[0], *const out_alpha = D->out[1];
            float *const out_depth = D->out[2];
            if (out_rgb) {
                out_rgb[3 * pidx] = a.c0;
                out_rgb[3 * pidx + 1] = a.c1;
                out_rgb[3 * pidx + 2] = a.c2;
            }
            if (out_alpha) out_alpha[pidx] = a.W;
            if (out_depth) out_depth[pidx] = a.W > 0.f ? a.Z / a.W : 0.f;
            ray_state[pidx] = make_float4(a.T, a.W, a.Z, 0.f);
            n_contrib[pidx] = a.last;
        }
        __syncwarp();
    }
}

template <uint32_t kSeg> static int cam_blocks_per_sm()
{
    static int cached = 0;
    if (!cached) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_camera<kSeg>,
                                                          32 * kCamWarps, 0) != cudaSuccess ||
            nb < 1)
            nb = 4;
        cached = nb;
    }
    return cached;
}

sg_status render_camera(const Camera &cam, const sg_render_opts &o, Frame &fr, cudaStream_t st)
{
    if (fr.seg_len != kSegLen && fr.seg_len != kSegLenStatic) {
        set_error("internal: camera list segment length %u not compiled", fr.seg_len);
        return SG_ERR_INVALID;
    }
    const CamRender P = cam_render_params(cam, o);
    const int nt = cam.ntx * cam.nty;
    const int64_t K = fr.n_pairs;
    const CamWorkSize ws = cam_work_size(nt, K, fr.seg_len);
    sg_status s = ensure(fr.order, sizeof(uint32_t) * (nt > 0 ? nt : 1));
    if (s == SG_OK) s = ensure(fr.camwork, ws.work_bytes);
    if (s == SG_OK) s = ensure(fr.partials, ws.partial_bytes);
    if (s == SG_OK) s = ensure(fr.submask, K > 0 ? (size_t)K : 1);
    if (s != SG_OK) return s;
    unsigned char *cw = (unsigned char *)fr.camwork.p;
    uint2 *tile_info = (uint2 *)cw;
    uint32_t *item_off = (uint32_t *)(cw + ws.info_bytes);
    uint2 *items = (uint2 *)(cw + ws.info_bytes + ws.off_bytes);
    uint32_t *arrive = (uint32_t *)(cw + ws.info_bytes + ws.off_bytes + ws.items_bytes);
    uint32_t *counts = (uint32_t *)fr.scalars.p + 4;    // [0] items [1] slots
    uint32_t *counter = (uint32_t *)fr.scalars.p + 2;
    k_camera_items<<<1, 1024, 0, st>>>((const uint2 *)fr.ranges.p, nt, fr.seg_len,
                                       (uint32_t *)fr.order.p, tile_info, item_off, counts,
                                       counter);
    SG_LAUNCHED();
    if (nt > 0) {
        k_emit_items<<<(unsigned)((nt + 7) / 8), 256, 0, st>>>(
            (const uint32_t *)fr.order.p, tile_info, item_off, nt, items, arrive);
        SG_LAUNCHED();
    }
    const uint32_t *ids = (const uint32_t *)fr.pvals[fr.pair_buf].p;
    if (K > 0) {
        k_submask<<<(unsigned)((K + 255) / 256), 256, 0, st>>>(
            (const uint32_t *)fr.pkeys[fr.pair_buf].p, ids, (const GRec *)fr.rec.p,
            (const uint32_t *)fr.scalars.p + 1, cam.ntx, (uint8_t *)fr.submask.p);
        SG_LAUNCHED();
    }
    int dev = 0, sms = 0;
    SG_CUDA(cudaGetDevice(&dev));
    SG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t cap = (ws.max_items + kCamWarps - 1) / kCamWarps;
    const bool dflt = fr.seg_len == kSegLen;
    int64_t grid = (int64_t)sms * (dflt ? cam_blocks_per_sm<kSegLen>()
                                        : cam_blocks_per_sm<kSegLenStatic>());
    grid = grid < cap ? grid : cap;
    if (grid < 1) grid = 1;
    auto kern = dflt ? k_render_camera<kSegLen> : k_render_camera<kSegLenStatic>;
    kern<<<(unsigned)grid, 32 * kCamWarps, 0, st>>>(
        P, (const GRec *)fr.rec.p, ids, (const uint2 *)fr.ranges.p, items, tile_info, counts,
        (const uint8_t *)fr.submask.p, counter, arrive, (float4 *)fr.partials.p, cam.d_pix,
        cam.d_tile_dir, (const RenderDesc *)fr.desc.p, (float4 *)fr.ray_state.p,
        (uint32_t *)fr.n_contrib.p);
    SG_LAUNCHED();
    return SG_OK;
}

// ------------------------------------------------------------------ LiDAR

__global__ void __launch_bounds__(32 * kLidarWarps)
k_render_lidar(LidRender P, const LidarItem *__restrict__ items,
               const uint32_t *__restrict__ item_rays, const float4 *__restrict__ ray_e,
               const double *__restrict__ item_u, const float *__restrict__ az_col,
               const float *__restrict__ elev, const GRec *__restrict__ rec,
               const uint32_t *__restrict__ ids, const uint2 *__restrict__ ranges,
               const RenderDesc *__restrict__ D, float4 *__restrict__ ray_state,
               uint32_t *__restrict__ n_contrib)
{
    __shared__ float s_all[kLidarWarps][kLidEntry][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int item_id = blockIdx.x * kLidarWarps + wib;
    if (item_id >= P.n_items) return;
    float(*s)[32] = s_all[wib];
    const float *__restrict__ poses = D->poses;
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
    float *const out_range = D->out[0], *const out_int = D->out[1];
    float *const out_drop = D->out[2], *const out_alpha = D->out[3];
    if (out_range) out_range[ray] = W > 0.f ? Z / W : 0.f;
    if (out_int) out_int[ray] = c0;
    if (out_drop) out_drop[ray] = drop;
    if (out_alpha) out_alpha[ray] = W;
    ray_state[ray] = make_float4(T, W, Z, drop);
    n_contrib[ray] = last;
}

sg_status render_lidar(const Lidar &L, const sg_render_opts &o, Frame &fr, cudaStream_t st)
{
    const LidRender P = lidar_render_params(L, o);
    if (L.n_items == 0) return SG_OK;
    const uint32_t *ids = (const uint32_t *)fr.pvals[fr.pair_buf].p;
    unsigned grid = (unsigned)((L.n_items + kLidarWarps - 1) / kLidarWarps);
    k_render_lidar<<<grid, 32 * kLidarWarps, 0, st>>>(
        P, L.d_items, L.d_item_rays, L.d_ray_e, L.d_tile_u, L.d_az, L.d_elev,
        (const GRec *)fr.rec.p, ids, (const uint2 *)fr.ranges.p, (const RenderDesc *)fr.desc.p,
        (float4 *)fr.ray_state.p, (uint32_t *)fr.n_contrib.p);
    SG_LAUNCHED();
    return SG_OK;
}

}  // namespace sg
