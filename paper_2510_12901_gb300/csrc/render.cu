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

// Per-ray state for the backward, written only by frames that keep it.
static float4 *saved_state(Frame &fr) { return fr.keep_state ? (float4 *)fr.ray_state.p : nullptr; }
static float4 *saved_feat(Frame &fr) { return fr.keep_state ? (float4 *)fr.ray_feat.p : nullptr; }
static uint32_t *saved_contrib(Frame &fr)
{
    return fr.keep_state ? (uint32_t *)fr.n_contrib.p : nullptr;
}

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

// Work items of the compositing.  A unit is a camera tile (units = tiles)
// or a LiDAR work item (up to 32 rays of one tile, unit_tile[u].tile).
// Units are taken in (coarsely) decreasing list length, so the longest start
// first.  A unit whose list is longer than seg_len entries is split along
// the list into ceil(len / seg_len) segments; every (unit, segment) gives
// `subs` work items (the eight 8x4 sub-blocks of a camera tile, or one).
// Two grid-wide kernels build them: k_work_count sums the work items of each
// length bucket (32 - floor(log2 len), longest first) and of the split
// units' partial slots, and its last block turns the bucket sums into the
// buckets' first items; k_work_emit (a warp per unit) takes its unit's run of
// items within its bucket and its first partial slot from atomic cursors,
// writes the items (unit, subs * seg + sub) and resets the arrival counters
// of a split unit.  The order of units within a bucket is immaterial: every
// item is independent and the merges combine segments in list order.  The
// work counter of the compositing kernel is reset here too.
__device__ __forceinline__ uint32_t unit_len(const uint2 *ranges, const LidarItem *unit_tile, int u)
{
    const uint2 r = ranges[unit_tile ? unit_tile[u].tile : (uint32_t)u];
    return r.y - r.x;
}

__device__ __forceinline__ uint32_t len_bucket(uint32_t len)
{
    return 32u - (len ? 32u - __clz(len) : 0u);        // longest first: 0 .. 32
}

__device__ __forceinline__ uint32_t unit_segments(uint32_t len, uint32_t seg_len)
{
    return len > seg_len ? (len + seg_len - 1) / seg_len : 1u;
}

// Scratch words (zeroed before k_work_count): the work items per bucket, the
// buckets' first items, the partial slots, the blocks done, the slot cursor
// and the buckets' item cursors.
constexpr int kWsBucketItems = 0, kWsBucketBase = 33, kWsSlots = 66, kWsDone = 67,
              kWsSlotCursor = 68, kWsBucketCursor = 69, kWsWords = 102;

__global__ void __launch_bounds__(256)
k_work_count(const uint2 *__restrict__ ranges, const LidarItem *__restrict__ unit_tile,
             int n_units, int subs, uint32_t seg_len, uint32_t *__restrict__ ws,
             uint32_t *__restrict__ counts, uint32_t *__restrict__ counter)
{
    __shared__ uint32_t s_b[33], s_slots;
    __shared__ bool s_last;
    const int t = threadIdx.x;
    if (t < 33) s_b[t] = 0u;
    if (t == 0) s_slots = 0u;
    __syncthreads();
    const int u = blockIdx.x * blockDim.x + t;
    if (u < n_units) {
        const uint32_t len = unit_len(ranges, unit_tile, u), nseg = unit_segments(len, seg_len);
        atomicAdd(&s_b[len_bucket(len)], (uint32_t)subs * nseg);
        if (nseg > 1) atomicAdd(&s_slots, nseg);
    }
    __syncthreads();
    if (t < 33 && s_b[t]) atomicAdd(&ws[kWsBucketItems + t], s_b[t]);
    if (t == 33 && s_slots) atomicAdd(&ws[kWsSlots], s_slots);
    __threadfence();
    __syncthreads();
    if (t == 0) s_last = atomicAdd(&ws[kWsDone], 1u) == gridDim.x - 1;
    __syncthreads();
    if (s_last && t == 0) {       // every block's sums are in: the buckets' first items
        __threadfence();
        uint32_t run = 0;
        for (int b = 0; b < 33; ++b) {
            const uint32_t c = __ldcg(&ws[kWsBucketItems + b]);
            ws[kWsBucketBase + b] = run;
            run += c;
        }
        counts[0] = run;
        counts[1] = __ldcg(&ws[kWsSlots]);
        counts[3] = 0u;      // deferred re-walks
        *counter = 0u;
    }
}

__global__ void __launch_bounds__(256)
k_work_emit(const uint2 *__restrict__ ranges, const LidarItem *__restrict__ unit_tile,
            int n_units, int subs, uint32_t seg_len, uint32_t *__restrict__ ws,
            uint2 *__restrict__ unit_info, uint2 *__restrict__ items, uint32_t *__restrict__ arrive)
{
    const int u = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    if (u >= n_units) return;
    const uint32_t len = unit_len(ranges, unit_tile, u), nseg = unit_segments(len, seg_len);
    const uint32_t n = (uint32_t)subs * nseg, b = len_bucket(len);
    uint32_t ib = 0, pb = 0;
    if (lane == 0) {
        ib = ws[kWsBucketBase + b] + atomicAdd(&ws[kWsBucketCursor + b], n);
        if (nseg > 1) pb = atomicAdd(&ws[kWsSlotCursor], nseg);
        unit_info[u] = make_uint2(nseg, pb);
    }
    ib = __shfl_sync(0xffffffffu, ib, 0);
    pb = __shfl_sync(0xffffffffu, pb, 0);
    for (uint32_t i = lane; i < n; i += 32) items[ib + i] = make_uint2((uint32_t)u, i);
    if (nseg > 1 && lane < subs) arrive[pb * subs + lane] = 0u;
}

// Launch both: the work items of `n_units` units into the frame's camwork
// buffer laid out by ws (its unit-offset region holds the scratch words).
sg_status launch_work_items(Frame &fr, const WorkSize &ws, const LidarItem *unit_tile,
                            int n_units, int subs, uint32_t seg_len, cudaStream_t st)
{
    unsigned char *cw = (unsigned char *)fr.camwork.p;
    uint2 *unit_info = (uint2 *)cw;
    uint32_t *scratch = (uint32_t *)(cw + ws.info_bytes);
    uint2 *items = (uint2 *)(cw + ws.info_bytes + ws.off_bytes);
    uint32_t *arrive = (uint32_t *)(cw + ws.info_bytes + ws.off_bytes + ws.items_bytes);
    if (ws.off_bytes < sizeof(uint32_t) * kWsWords) {
        set_error("internal: work-item scratch too small");
        return SG_ERR_INVALID;
    }
    SG_CUDA(cudaMemsetAsync(scratch, 0, sizeof(uint32_t) * kWsWords, st));
    const unsigned g1 = (unsigned)((n_units + 255) / 256);
    k_work_count<<<g1 > 0 ? g1 : 1, 256, 0, st>>>((const uint2 *)fr.ranges.p, unit_tile, n_units,
                                                  subs, seg_len, scratch,
                                                  (uint32_t *)fr.scalars.p + 4,
                                                  (uint32_t *)fr.scalars.p + 2);
    SG_LAUNCHED();
    if (n_units > 0) {
        k_work_emit<<<(unsigned)((n_units + 7) / 8), 256, 0, st>>>(
            (const uint2 *)fr.ranges.p, unit_tile, n_units, subs, seg_len, scratch, unit_info,
            items, arrive);
        SG_LAUNCHED();
    }
    return SG_OK;
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
// state, the run in which a ray stops (run 0 starts from the true state, so
// its own stop is final).  The pixels of a sub-block mostly stop in the same
// run or two, so the re-walks stay in the merge (LiDAR items, whose rays
// spread further, defer theirs: k_render_lidar).  As it goes, the merge
// overwrites each later run's partial with the state before that run
// (colour, omega, Z, T, last entry), from which the backward walks the run.
constexpr int kCamWarps = 4;       // warps per block of the persistent grid


struct CamAcc {
    float T, W, Z, c0, c1, c2;
    uint32_t last;                 // list entries up to the last composited one
};

// Composite the n entries staged in s_e into the lane's accumulator.
__device__ __forceinline__ void cam_composite(const CamRender &P, float4 (*s_e)[32],
                                              const uint32_t *s_pos, int n, const float dd[3],
                                              CamAcc &a, bool &done)
{
    const int lane = threadIdx.x & 31;
    int lastj = -1;            // the batch's last composited entry of this lane
    for (int j = 0; j < n; ++j) {
        PairEval pe;
        // plane 7: features, with the entry's lane mask in .w
        const float4 col = s_e[7][j];
        bool ok = cam_pair_scaled(s_e[0][j], s_e[1][j], s_e[2][j], s_e[3][j], s_e[4][j],
                                  s_e[5][j], s_e[6][j], (__float_as_uint(col.w) >> lane) & 1u,
                                  dd, P.alpha_min, P.alpha_max, pe);
        ok = ok && !done;
        const float Tn = a.T * (1.f - pe.alpha);
        const bool stop = ok && Tn < P.t_min;
        done = done || stop;
        ok = ok && !stop;
        const float wgt = ok ? pe.alpha * a.T : 0.f;
        a.c0 += wgt * col.x;
        a.c1 += wgt * col.y;
        a.c2 += wgt * col.z;
        a.Z += wgt * pe.tau;
        a.W += wgt;
        a.T = ok ? Tn : a.T;
        lastj = ok ? j : lastj;
    }
    if (lastj >= 0) a.last = s_pos[lastj];
}

// Composite list entries [lo, hi) of a tile (first entry `begin`) that can
// reach sub-block `sub` into the lane's accumulator; lanes with done = true
// take part in the warp's staging but keep their state; `rays` = the lanes
// that have a ray.  Returns whether the lane's ray stopped at T_min.
__device__ __forceinline__ bool cam_walk(const CamRender &P, const CamPose &pose,
                                         const GRec *__restrict__ rec,
                                         const uint32_t *__restrict__ ids,
                                         const uint32_t *__restrict__ crw, int sub,
                                         uint32_t lo, uint32_t hi,
                                         uint32_t begin, const float dh[3], const float dl[3],
                                         const float dd[3], float4 (*s_e)[32],
                                         uint32_t *s_pos, CamAcc &a, bool done)
{
    const int lane = threadIdx.x & 31;
    const bool done0 = done;
    // the next batch's mask byte and Gaussian id, loaded one batch ahead so
    // that staging waits for the record load alone
    uint32_t ncr = 0u, nid = 0u;
    if (lo + lane < hi) {
        ncr = crw[lo + lane];
        nid = ids[lo + lane];
    }
    for (uint32_t base = lo; base < hi; base += 32) {
        const uint32_t act = __ballot_sync(0xffffffffu, !done);
        if (act == 0u) break;
        const uint32_t idx = base + lane;
        const uint32_t gid = nid;
        // the entry's lanes in the sub-block, from its column/row word: only
        // entries that reach a ray still compositing are staged
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
            cam_entry(rec[gid], pose.t, dh, dl, ent, kResponseScale);
            ent[7].w = __uint_as_float(lm);
#pragma unroll
            for (int k = 0; k < 8; ++k) s_e[k][pos] = ent[k];
            s_pos[pos] = idx + 1 - begin;
        }
        __syncwarp();
        cam_composite(P, s_e, s_pos, __popc(bal), dd, a, done);
    }
    return done && !done0;   // the ray stopped at T_min in this walk
}

// Partial slot layout: (c0, c1, c2, W), (Z, T, last, stopped flag).
__device__ __forceinline__ void put_state(float4 *pq, const CamAcc &a, bool stopped)
{
    pq[0] = make_float4(a.c0, a.c1, a.c2, a.W);
    pq[1] = make_float4(a.Z, a.T, __uint_as_float(a.last), stopped ? 1.f : 0.f);
}
__device__ __forceinline__ CamAcc get_state(float4 u, float4 v)
{
    return {v.y, u.w, v.x, u.x, u.y, u.z, __float_as_uint(v.z)};
}

template <uint32_t kSeg>
__global__ void __launch_bounds__(32 * kCamWarps, 6)
k_render_camera(CamRender P, const GRec *__restrict__ rec, const uint32_t *__restrict__ ids,
                const uint2 *__restrict__ ranges, const uint2 *__restrict__ items,
                const uint2 *__restrict__ tile_info, const uint32_t *__restrict__ counts,
                const uint32_t *__restrict__ crw, uint32_t *__restrict__ counter,
                uint32_t *__restrict__ arrive, float4 *__restrict__ partials,
                const float4 *__restrict__ pix, const double *__restrict__ tile_dir,
                const RenderDesc *__restrict__ D, float4 *__restrict__ ray_state,
                float4 *__restrict__ ray_feat, uint32_t *__restrict__ n_contrib)
{
    __shared__ float4 s_all[kCamWarps][8][32];
    __shared__ uint32_t s_pos[kCamWarps][32];
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
        const bool stopped = cam_walk(P, s_pose, rec, ids, crw, sub, lo, hi, rg.x, dh, dl, dd,
                                      s_e, s_pos[wib], a, no_ray);
        if (ti.x > 1) {
            // long tile: publish this run, and combine if it is the last one
            put_state(partials + ((size_t)(ti.y + seg) * 256 + sub * 32 + lane) * 2, a, stopped);
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
            float4 *pq = partials + ((size_t)ti.y * 256 + sub * 32 + lane) * 2;
            const float4 u0 = __ldcg(pq), v0 = __ldcg(pq + 1);
            a = get_state(u0, v0);
            bool fin = no_ray || v0.w != 0.f;
            for (uint32_t sgi = 1; sgi < ti.x; ++sgi) {
                if (__all_sync(0xffffffffu, fin)) break;
                pq += 512;
                const float4 u = __ldcg(pq), v = __ldcg(pq + 1);
                // the state before run sgi replaces its partial
                put_state(pq, a, false);
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
                    cam_walk(P, s_pose, rec, ids, crw, sub, l0,
                             min(rg.y, l0 + kSeg), rg.x, dh, dl, dd, s_e, s_pos[wib],
                             a, !redo);
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
            if (ray_state) {   // the state the backward needs (frames that keep it)
                ray_state[pidx] = make_float4(a.T, a.W, a.Z, 0.f);
                ray_feat[pidx] = make_float4(a.c0, a.c1, a.c2, 0.f);
                n_contrib[pidx] = a.last;
            }
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
    if (camera_forward_only(cam, fr)) return render_camera_fwd(cam, o, fr, st);
    const CamRender P = cam_render_params(cam, o);
    const int nt = cam.ntx * cam.nty;
    const int64_t K = fr.n_pairs;
    const WorkSize ws = work_size(nt, K, fr.seg_len, 8);
    sg_status s = ensure(fr.order, sizeof(uint32_t) * (nt > 0 ? nt : 1));
    if (s == SG_OK) s = ensure(fr.camwork, ws.work_bytes);
    if (s == SG_OK) s = ensure(fr.partials, ws.partial_bytes);
    if (s == SG_OK && fr.submask.bytes < 4 * (size_t)(K > 0 ? K : 1)) {
        set_error("internal: sub-block masks of the camera list missing");
        s = SG_ERR_INVALID;
    }
    if (s != SG_OK) return s;
    unsigned char *cw = (unsigned char *)fr.camwork.p;
    const uint2 *tile_info = (const uint2 *)cw;
    const uint2 *items = (const uint2 *)(cw + ws.info_bytes + ws.off_bytes);
    uint32_t *arrive = (uint32_t *)(cw + ws.info_bytes + ws.off_bytes + ws.items_bytes);
    const uint32_t *counts = (const uint32_t *)fr.scalars.p + 4;    // [0] items [1] slots
    uint32_t *counter = (uint32_t *)fr.scalars.p + 2;
    if ((s = launch_work_items(fr, ws, nullptr, nt, 8, fr.seg_len, st)) != SG_OK) return s;
    const uint32_t *ids = (const uint32_t *)fr.pvals[fr.pair_buf].p;
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
        (const uint32_t *)fr.submask.p, counter, arrive, (float4 *)fr.partials.p, cam.d_pix,
        cam.d_tile_dir, (const RenderDesc *)fr.desc.p, saved_state(fr),
        saved_feat(fr), saved_contrib(fr));
    SG_LAUNCHED();
    return SG_OK;
}

// ------------------------------------------------------------------ rolling shutter
// Rolling-shutter camera compositing: the camera's work items, lists,
// segments and merges, with every pixel row under its own pose.  The four
// rows of an 8x4 sub-block are staged like the columns of a LiDAR work item
// (lidar_entry: per row slot the P rows, a and u = M v of the row's origin),
// and a ray's direction is its tile reference ray under the sub-block's
// first row's pose plus its offset under its own row's pose (sensor_ray).

// Composite entries [lo, hi) that reach sub-block `sub` (first pixel sbx,
// sby; rows r0 .. r0 + nrows - 1) into the lane's accumulator; sb: the
// lane's row slot.  As cam_walk.
__device__ __forceinline__ bool cam_walk_rs(const CamRender &P, const GRec *__restrict__ rec,
                                            const uint32_t *__restrict__ ids,
                                            const uint32_t *__restrict__ crw, int sub,
                                            int sbx, int sby, uint32_t lo, uint32_t hi,
                                            uint32_t begin, const float *__restrict__ poses,
                                            int nrows, int sb, const float dh[3],
                                            const float dl[3], const float dd[3],
                                            const float d[3], float4 (*s)[32], uint32_t *s_pos,
                                            uint32_t *s_lanes, CamAcc &a, bool done)
{
    const int lane = threadIdx.x & 31;
    const bool done0 = done;
    uint32_t ncr = 0u, nid = 0u;    // the next batch's, as in cam_walk
    if (lo + lane < hi) {
        ncr = crw[lo + lane];
        nid = ids[lo + lane];
    }
    for (uint32_t base = lo; base < hi; base += 32) {
        const uint32_t act = __ballot_sync(0xffffffffu, !done);
        if (act == 0u) break;
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
            s_lanes[pos] = lm;
            s_pos[pos] = idx + 1 - begin;
        }
        __syncwarp();
        const int n = __popc(bal);
        for (int j = 0; j < n; ++j) {
            PairEval pe;
            bool ok = lidar_pair_in(s, j, sb, (s_lanes[j] >> lane) & 1u, dd, d, P.alpha_min,
                                    P.alpha_max, pe);
            ok = ok && !done;
            const float Tn = a.T * (1.f - pe.alpha);
            const bool stop = ok && Tn < P.t_min;
            done = done || stop;
            ok = ok && !stop;
            const float wgt = ok ? pe.alpha * a.T : 0.f;
            a.c0 += wgt * s[1][j].w;
            a.c1 += wgt * s[2][j].w;
            a.c2 += wgt * lid_u(s, j, sb).w;
            a.Z += wgt * pe.tau;
            a.W += wgt;
            a.T = ok ? Tn : a.T;
            a.last = ok ? s_pos[j] : a.last;
        }
    }
    return done && !done0;
}

// The per-lane ray of a rolling-shutter sub-block: rows, the lane's slot,
// and its direction (see above).
__device__ __forceinline__ void cam_rs_ray(const float *__restrict__ poses,
                                           const double *__restrict__ tile_dir, int tile, int H,
                                           int sby, int py, const float4 e, int &nrows, int &sb,
                                           float dh[3], float dl[3], float dd[3], float d[3])
{
    nrows = min(4, H - sby);
    const int row = py < H ? py : sby;
    sb = 3 + 4 * (row - sby);
    const double *u = tile_dir + 3 * tile;
    sensor_ray(poses + 12 * sby, u[0], u[1], u[2], poses + 12 * row, e, dh, dl, dd, d);
}

template <uint32_t kSeg>
__global__ void __launch_bounds__(32 * kCamWarps)
k_render_camera_rs(CamRender P, const GRec *__restrict__ rec, const uint32_t *__restrict__ ids,
                   const uint2 *__restrict__ ranges, const uint2 *__restrict__ items,
                   const uint2 *__restrict__ tile_info, const uint32_t *__restrict__ counts,
                   const uint32_t *__restrict__ crw, uint32_t *__restrict__ counter,
                   uint32_t *__restrict__ arrive, float4 *__restrict__ partials,
                   const float4 *__restrict__ pix, const double *__restrict__ tile_dir,
                   const RenderDesc *__restrict__ D, float4 *__restrict__ ray_state,
                   float4 *__restrict__ ray_feat, uint32_t *__restrict__ n_contrib)
{
    __shared__ float4 s_all[kCamWarps][kLidPlanes][32];
    __shared__ uint32_t s_pos[kCamWarps][32];
    __shared__ uint32_t s_lanes[kCamWarps][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float4(*s_e)[32] = s_all[wib];
    const float *__restrict__ poses = D->poses;
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
        const bool no_ray = !(inside && e.w > 0.f);
        int nrows, sb;
        float dh[3], dl[3], dd[3], d[3];
        cam_rs_ray(poses, tile_dir, tile, P.H, sby, py, e, nrows, sb, dh, dl, dd, d);
        const uint2 rg = ranges[tile];
        const uint32_t lo = rg.x + (uint32_t)seg * kSeg;
        const uint32_t hi = min(rg.y, lo + kSeg);
        CamAcc a = {1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u};
        const bool stopped = cam_walk_rs(P, rec, ids, crw, sub, sbx, sby, lo, hi, rg.x, poses,
                                         nrows, sb, dh, dl, dd, d, s_e, s_pos[wib], s_lanes[wib],
                                         a, no_ray);
        if (ti.x > 1) {
            put_state(partials + ((size_t)(ti.y + seg) * 256 + sub * 32 + lane) * 2, a, stopped);
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
            float4 *pq = partials + ((size_t)ti.y * 256 + sub * 32 + lane) * 2;
            const float4 u0 = __ldcg(pq), v0 = __ldcg(pq + 1);
            a = get_state(u0, v0);
            bool fin = no_ray || v0.w != 0.f;
            for (uint32_t sgi = 1; sgi < ti.x; ++sgi) {
                if (__all_sync(0xffffffffu, fin)) break;
                pq += 512;
                const float4 u = __ldcg(pq), v = __ldcg(pq + 1);
                put_state(pq, a, false);
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
                    cam_walk_rs(P, rec, ids, crw, sub, sbx, sby, l0, min(rg.y, l0 + kSeg),
                                rg.x, poses, nrows, sb, dh, dl, dd, d, s_e, s_pos[wib],
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
            if (ray_state) {   // the state the backward needs (frames that keep it)
                ray_state[pidx] = make_float4(a.T, a.W, a.Z, 0.f);
                ray_feat[pidx] = make_float4(a.c0, a.c1, a.c2, 0.f);
                n_contrib[pidx] = a.last;
            }
        }
        __syncwarp();
    }
}

sg_status render_camera_rs(const Camera &cam, const sg_render_opts &o, Frame &fr,
                           cudaStream_t st)
{
    if (fr.seg_len != kSegLen) {
        set_error("internal: rolling-shutter renders use the default segment length");
        return SG_ERR_INVALID;
    }
    const CamRender P = cam_render_params(cam, o);
    const int nt = cam.ntx * cam.nty;
    const int64_t K = fr.n_pairs;
    const WorkSize ws = work_size(nt, K, fr.seg_len, 8);
    sg_status s = ensure(fr.order, sizeof(uint32_t) * (nt > 0 ? nt : 1));
    if (s == SG_OK) s = ensure(fr.camwork, ws.work_bytes);
    if (s == SG_OK) s = ensure(fr.partials, ws.partial_bytes);
    if (s == SG_OK && fr.submask.bytes < 4 * (size_t)(K > 0 ? K : 1)) {
        set_error("internal: sub-block masks of the camera list missing");
        s = SG_ERR_INVALID;
    }
    if (s != SG_OK) return s;
    unsigned char *cw = (unsigned char *)fr.camwork.p;
    const uint2 *tile_info = (const uint2 *)cw;
    const uint2 *items = (const uint2 *)(cw + ws.info_bytes + ws.off_bytes);
    uint32_t *arrive = (uint32_t *)(cw + ws.info_bytes + ws.off_bytes + ws.items_bytes);
    const uint32_t *counts = (const uint32_t *)fr.scalars.p + 4;
    uint32_t *counter = (uint32_t *)fr.scalars.p + 2;
    if ((s = launch_work_items(fr, ws, nullptr, nt, 8, fr.seg_len, st)) != SG_OK) return s;
    const uint32_t *ids = (const uint32_t *)fr.pvals[fr.pair_buf].p;
    int dev = 0, sms = 0, nb = 0;
    SG_CUDA(cudaGetDevice(&dev));
    SG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_camera_rs<kSegLen>,
                                                      32 * kCamWarps, 0) != cudaSuccess || nb < 1)
        nb = 4;
    const int64_t cap = (ws.max_items + kCamWarps - 1) / kCamWarps;
    int64_t grid = (int64_t)sms * nb;
    grid = grid < cap ? grid : cap;
    if (grid < 1) grid = 1;
    k_render_camera_rs<kSegLen><<<(unsigned)grid, 32 * kCamWarps, 0, st>>>(
        P, (const GRec *)fr.rec.p, ids, (const uint2 *)fr.ranges.p, items, tile_info, counts,
        (const uint32_t *)fr.submask.p, counter, arrive, (float4 *)fr.partials.p, cam.d_pix,
        cam.d_tile_dir, (const RenderDesc *)fr.desc.p, saved_state(fr),
        saved_feat(fr), saved_contrib(fr));
    SG_LAUNCHED();
    return SG_OK;
}

// ------------------------------------------------------------------ LiDAR
// LiDAR compositing, persistent warps over (work item, segment) units: a
// LiDAR work item holds up to 32 rays of one tile (at most kLidarColsMax
// columns, each with its own pose); lists longer than kSegLen entries are
// split and combined exactly as for the camera (see k_render_camera).
// Batches of 32 list entries are staged through the warp's shared-memory
// slice with their per-column moments.

// Per-warp shared state of a LiDAR work item: staged entries, their ray
// masks and list positions.
struct LidStage {
    float4 (*s)[32];
    uint32_t *lanes, *pos;
};

// Composite entries [lo, hi) of the item's list (first entry `begin`): the
// item's ray masks of a window of 32 entries (written with the tile ranges,
// lmask[i] for list entry i) select the entries that reach a ray still
// compositing; only those are staged.  The lanes of one column (a group)
// then evaluate, in list order, the staged entries whose box holds a ray of
// that column, while the other groups evaluate theirs.  Returns whether the
// lane's ray stopped at T_min.
__device__ __forceinline__ bool lidar_walk(const LidRender &P, const GRec *__restrict__ rec,
                                           const uint32_t *__restrict__ ids,
                                           const uint32_t *__restrict__ lmask,
                                           const float *__restrict__ poses, const LidarItem &it,
                                           int sb, const float dh[3], const float dl[3],
                                           const float dd[3], const float d[3], uint32_t lo,
                                           uint32_t hi, uint32_t begin, const LidStage &L,
                                           CamAcc &a, bool done)
{
    const int lane = threadIdx.x & 31;
    const bool done0 = done;
    const uint32_t gm = __match_any_sync(0xffffffffu, sb);   // lanes of this lane's column
    // the next batch's ray masks and ids, loaded one batch ahead
    uint32_t nm = 0u, nid = 0u;
    if (lo + lane < hi) {
        nm = lmask[lo + lane];
        nid = ids[lo + lane];
    }
    for (uint32_t base = lo; base < hi; base += 32) {
        // only entries that reach a ray still compositing
        const uint32_t act = __ballot_sync(0xffffffffu, !done);
        if (act == 0u) break;
        const uint32_t idx = base + lane;
        const uint32_t g = nid;
        const uint32_t m = nm & act;
        if (idx + 32 < hi) {
            nm = lmask[idx + 32];
            nid = ids[idx + 32];
        } else {
            nm = 0u;
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, m != 0u);
        if (bal == 0u) continue;
        __syncwarp();
        if (m) {
            const int pos = __popc(bal & ((1u << lane) - 1u));
            lidar_entry(rec[g], poses, it.col0, it.ncols, dh, dl, L.s, pos);
            L.lanes[pos] = m;
            L.pos[pos] = idx + 1 - begin;
        }
        __syncwarp();
        // the staged entries that reach a ray of this lane's column group:
        // the groups (lanes of one column) walk their own entries side by
        // side, so an entry whose box holds rays of one column takes one
        // step of that group only
        const int n = __popc(bal);
        const uint32_t lj = lane < n ? L.lanes[lane] : 0u;
        uint32_t G = 0u;
        for (uint32_t rest = 0xffffffffu; rest;) {
            const uint32_t gm_g = __shfl_sync(0xffffffffu, gm, __ffs(rest) - 1);
            const uint32_t Gg = __ballot_sync(0xffffffffu, (lj & gm_g) != 0u);
            G = gm == gm_g ? Gg : G;
            rest &= ~gm_g;
        }
        while (__any_sync(0xffffffffu, G != 0u)) {
            const bool has = G != 0u;
            const int j = has ? __ffs(G) - 1 : 0;
            G &= G - 1u;
            PairEval pe;
            bool ok = lidar_pair_in(L.s, j, sb, has && ((L.lanes[j] >> lane) & 1u), dd, d,
                                    P.alpha_min, P.alpha_max, pe);
            ok = ok && !done;
            const float Tn = a.T * (1.f - pe.alpha);
            const bool stop = ok && Tn < P.t_min;
            done = done || stop;
            ok = ok && !stop;
            const float wgt = ok ? pe.alpha * a.T : 0.f;
            a.c0 += wgt * L.s[1][j].w;
            a.c1 += wgt * L.s[2][j].w;
            a.c2 += wgt * lid_u(L.s, j, sb).w;
            a.Z += wgt * pe.tau;
            a.W += wgt;
            a.T = ok ? Tn : a.T;
            a.last = ok ? L.pos[j] : a.last;
        }
    }
    return done && !done0;
}

// The merge of a split item re-walks the first kLidarInlineRewalks segments
// in which some of its rays stop, as the camera merge does; the rays of a
// LiDAR item span several beams and columns and stop in up to 32 different
// segments, which one warp would walk one after another (this tail once held
// a third of the launch), so later ones are recorded as deferred re-walks
// (item, segment, lanes).  A second launch (kFix = true) walks those in
// parallel, each from the state before its segment, and writes their rays.
constexpr int kLidarInlineRewalks = 2;

template <bool kFix>
__global__ void __launch_bounds__(32 * kLidarWarps)
k_render_lidar(LidRender P, const LidarItem *__restrict__ items,
               const uint32_t *__restrict__ item_rays, const float4 *__restrict__ ray_e,
               const double *__restrict__ item_u, const uint2 *__restrict__ tile_items,
               const uint32_t *__restrict__ lmask, int64_t lmask_stride,
               const GRec *__restrict__ rec,
               const uint32_t *__restrict__ ids, const uint2 *__restrict__ ranges,
               const uint2 *__restrict__ work, const uint2 *__restrict__ unit_info,
               const uint32_t *__restrict__ counts, uint32_t *__restrict__ counter,
               uint32_t *__restrict__ arrive, float4 *__restrict__ partials, FixList F,
               const RenderDesc *__restrict__ D, float4 *__restrict__ ray_state,
               float4 *__restrict__ ray_feat, uint32_t *__restrict__ n_contrib)
{
    __shared__ float4 s_all[kLidarWarps][kLidPlanes][32];
    __shared__ uint32_t s_lanes[kLidarWarps][32], s_pos[kLidarWarps][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const LidStage stg = {s_all[wib], s_lanes[wib], s_pos[wib]};
    const float *__restrict__ poses = D->poses;
    const uint32_t n_work = kFix ? *F.n_fix : counts[0];
    uint32_t fix_next = blockIdx.x * kLidarWarps + wib;
    while (true) {
        uint2 w;
        uint32_t fix_lanes = 0u;
        if constexpr (kFix) {
            if (fix_next >= n_work || fix_next >= F.cap) break;
            const uint4 f = F.fix[fix_next];
            fix_next += gridDim.x * kLidarWarps;
            w = make_uint2(f.x, f.y);
            fix_lanes = f.z;
        } else {
            uint32_t wi = 0;
            if (lane == 0) wi = atomicAdd(counter, 1u);
            wi = __shfl_sync(0xffffffffu, wi, 0);
            if (wi >= n_work) break;
            w = work[wi];
        }
        const int item_id = (int)w.x;
        const uint32_t seg = w.y;
        const uint2 ui = unit_info[item_id];         // (segments, first partial slot)
        const LidarItem it = items[item_id];
        const uint32_t ray = item_rays[it.ray_off + lane];
        const bool valid = ray != 0xffffffffu;
        const int c = valid ? (int)(ray % (uint32_t)P.n_cols) : it.col0;
        const int sb = 3 + 4 * (c - it.col0);
        float dh[3], dl[3], dd[3], d[3];
        lidar_ray(it, item_u, item_id, poses, ray_e[it.ray_off + lane], c, dh, dl, dd, d);
        // this item's plane of ray masks
        const uint32_t *lm = lmask + (int64_t)(item_id - (int)tile_items[it.tile].x) * lmask_stride;
        const uint2 rg = ranges[it.tile];
        const uint32_t lo = rg.x + seg * kSegLen;
        const uint32_t hi = min(rg.y, lo + kSegLen);
        CamAcc a = {1.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u};
        bool write = valid;
        if constexpr (kFix) {
            const bool mine = (fix_lanes >> lane) & 1u;
            const float4 *pq = partials + ((size_t)(ui.y + seg) * 32 + lane) * 2;
            if (mine) a = get_state(pq[0], pq[1]);
            lidar_walk(P, rec, ids, lm, poses, it, sb, dh, dl, dd, d, lo, hi, rg.x, stg, a, !mine);
            write = mine;
        } else {
            const bool stopped = lidar_walk(P, rec, ids, lm, poses, it, sb, dh, dl, dd, d, lo,
                                            hi, rg.x, stg, a, !valid);
            if (ui.x > 1) {
                // split item: publish this segment, and combine if it is the last one
                put_state(partials + ((size_t)(ui.y + seg) * 32 + lane) * 2, a, stopped);
                __threadfence();
                __syncwarp();
                uint32_t prev = 0;
                if (lane == 0) prev = atomicAdd(&arrive[ui.y], 1u);
                prev = __shfl_sync(0xffffffffu, prev, 0);
                if (prev != ui.x - 1) {
                    __syncwarp();
                    continue;
                }
                __threadfence();
                float4 *pq = partials + ((size_t)ui.y * 32 + lane) * 2;
                const float4 u0 = __ldcg(pq), v0 = __ldcg(pq + 1);
                a = get_state(u0, v0);
                bool fin = !valid || v0.w != 0.f;
                int n_inline = 0;
                for (uint32_t sgi = 1; sgi < ui.x; ++sgi) {
                    if (__all_sync(0xffffffffu, fin)) break;
                    pq += 64;
                    const float4 u = __ldcg(pq), v = __ldcg(pq + 1);
                    // the state before segment sgi replaces its partial
                    put_state(pq, a, false);
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
                    const uint32_t rl = __ballot_sync(0xffffffffu, redo);
                    if (rl && n_inline < kLidarInlineRewalks) {
                        ++n_inline;
                        const uint32_t l0 = rg.x + sgi * kSegLen;
                        lidar_walk(P, rec, ids, lm, poses, it, sb, dh, dl, dd, d, l0,
                                   min(rg.y, l0 + kSegLen), rg.x, stg, a, !redo);
                    } else if (rl) {
                        push_fix(F, (uint32_t)item_id, sgi, rl);
                        write = write && !redo;  // the deferred re-walk writes this ray
                    }
                    fin = fin || redo;
                }
            }
        }
        if (write) {
            const float drop = 1.f / (1.f + expf(a.c1 - a.c2));
            float *const out_range = D->out[0], *const out_int = D->out[1];
            float *const out_drop = D->out[2], *const out_alpha = D->out[3];
            if (out_range) out_range[ray] = a.W > 0.f ? a.Z / a.W : 0.f;
            if (out_int) out_int[ray] = a.c0;
            if (out_drop) out_drop[ray] = drop;
            if (out_alpha) out_alpha[ray] = a.W;
            if (ray_state) {   // the state the backward needs (frames that keep it)
                ray_state[ray] = make_float4(a.T, a.W, a.Z, drop);
                ray_feat[ray] = make_float4(a.c0, a.c1, a.c2, 0.f);
                n_contrib[ray] = a.last;
            }
        }
        __syncwarp();
    }
}

static int lidar_blocks_per_sm()
{
    static int cached = 0;
    if (!cached) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_lidar<false>, 32 * kLidarWarps,
                                                          0) != cudaSuccess ||
            nb < 1)
            nb = 4;
        cached = nb;
    }
    return cached;
}

sg_status render_lidar(const Lidar &L, const sg_render_opts &o, Frame &fr, cudaStream_t st)
{
    if (lidar_forward_only(fr)) return render_lidar_fwd(L, o, fr, st);
    const LidRender P = lidar_render_params(L, o);
    if (L.n_items == 0) return SG_OK;
    const int64_t K = fr.n_pairs;
    // items that share a tile each walk its list: the entries of all units
    // add up to at most max_items_per_tile x K
    const WorkSize ws = work_size(L.n_items, K * L.max_items_per_tile, kSegLen, 1);
    sg_status s = ensure(fr.order, sizeof(uint32_t) * (size_t)L.n_items);
    if (s == SG_OK) s = ensure(fr.camwork, ws.work_bytes);
    if (s == SG_OK) s = ensure(fr.partials, ws.partial_bytes);
    if (s != SG_OK) return s;
    if ((s = launch_work_items(fr, ws, L.d_items, L.n_items, 1, kSegLen, st)) != SG_OK) return s;
    unsigned char *cw = (unsigned char *)fr.camwork.p;
    const uint2 *unit_info = (const uint2 *)cw;
    const uint2 *work = (const uint2 *)(cw + ws.info_bytes + ws.off_bytes);
    uint32_t *arrive = (uint32_t *)(cw + ws.info_bytes + ws.off_bytes + ws.items_bytes);
    const uint32_t *ids = (const uint32_t *)fr.pvals[fr.pair_buf].p;
    int dev = 0, sms = 0;
    SG_CUDA(cudaGetDevice(&dev));
    SG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t cap = (ws.max_items + kLidarWarps - 1) / kLidarWarps;
    int64_t grid = (int64_t)sms * lidar_blocks_per_sm();
    grid = grid < cap ? grid : cap;
    if (grid < 1) grid = 1;
    const FixList F = fix_list(fr, ws);
    k_render_lidar<false><<<(unsigned)grid, 32 * kLidarWarps, 0, st>>>(
        P, L.d_items, L.d_item_rays, L.d_ray_e, L.d_tile_u, L.d_tile_items,
        (const uint32_t *)fr.lmask.p, fr.lmask_stride,
        (const GRec *)fr.rec.p, ids, (const uint2 *)fr.ranges.p, work, unit_info,
        (const uint32_t *)fr.scalars.p + 4, (uint32_t *)fr.scalars.p + 2, arrive,
        (float4 *)fr.partials.p, F, (const RenderDesc *)fr.desc.p, saved_state(fr),
        saved_feat(fr), saved_contrib(fr));
    SG_LAUNCHED();
    if (ws.max_slots > 0) {       // some item may be split: the deferred re-walks
        const int64_t fcap = (ws.max_fixes + kLidarWarps - 1) / kLidarWarps;
        const int64_t fgrid = grid < fcap ? grid : fcap;
        k_render_lidar<true><<<(unsigned)fgrid, 32 * kLidarWarps, 0, st>>>(
            P, L.d_items, L.d_item_rays, L.d_ray_e, L.d_tile_u, L.d_tile_items,
            (const uint32_t *)fr.lmask.p, fr.lmask_stride,
            (const GRec *)fr.rec.p, ids, (const uint2 *)fr.ranges.p, work, unit_info,
            (const uint32_t *)fr.scalars.p + 4, (uint32_t *)fr.scalars.p + 2, arrive,
            (float4 *)fr.partials.p, F, (const RenderDesc *)fr.desc.p, saved_state(fr),
            saved_feat(fr), saved_contrib(fr));
        SG_LAUNCHED();
    }
    return SG_OK;
}

}  // namespace sg
