// render_lidar_fwd.cu -- LiDAR compositing (Eq. 1 at the response maximum,
// the quantities of Sec. 3.2: range, intensity, ray-drop and alpha, as
// k_render_lidar) for frames that keep no state for a backward: the LiDAR
// render of a serving loop or a benchmark.  The work decomposition is
// k_render_lidar's (persistent warps over (work item, segment) units, split
// items combined by the last arriving warp, deferred re-walks, per-entry ray
// masks from the tile ranges); what differs:
//
// Beam groups.  A staged entry is evaluated by the lanes of each beam it
// reaches (the lanes of one beam, one per column of the item, form a group;
// the groups walk their own entries side by side).  A Gaussian's box holds a
// few of an item's beams and columns; grouping by beam evaluates a pair on
// about two thirds in-box lanes, against under a third with groups by column.
//
// One parameter per ray.  The rays of column c (pose R_c, origin o_c) are,
// divided by the cosine of their elevation el,
//     d' = h_c + tan(el) z_c,   h_c = R_c (cos az_c, sin az_c, 0),  z_c = R_c e_z,
// an affine family in one parameter.  With the item's reference tan(el_r)
// and x = tan(el) - tan(el_r) (a per-ray constant, small within an item):
//     num_k = a_k + x p_k,  a_k = f_k M_k . (v x d_r),  p_k = f_k M_k . (v x z_c)
//     den_k = b_k + x m_k,  b_k = M_k . d_r,            m_k = M_k . z_c
//     (M v) . den = t_0 + x t_1
// d_r = h_c + tan(el_r) z_c in double, split in two floats, so a_k keeps the
// error-free moment of render.cu.  D^2 does not depend on the length of d',
// and tau_max along d' is the range along the unit ray divided by |d'| =
// 1 / cos(el).  A pair costs 7 FMAs for the affine parts (18 with the
// 3-vector offsets of k_render_lidar) and 5 shared-memory loads (7).
#include <math.h>

#include "pairs.cuh"
#include "render.cuh"

namespace sg {

constexpr int kLfWarps = 4;     // warps per block of the persistent grid
// blocks per SM: the staged entries take 8.5 KB of shared memory per warp
constexpr int kLfBlocks = 6;
// List entries a warp scans per window: kLfPer per lane.  The entries of the
// window that reach a live ray (about half of them on the street sweep) are
// staged 32 at a time, so that the staging pass, one entry per lane, runs
// with more of its lanes busy than over a 32-entry window.
#ifndef SG_LF_PER_LANE
#define SG_LF_PER_LANE 2
#endif
constexpr int kLfPer = SG_LF_PER_LANE;
constexpr int kLfWin = 32 * kLfPer;

// Per-warp shared state.  Quantities of entry j and column slot sl sit at
// 4 j + (sl ^ swizzle(j)): the four slots of an entry stay together (the
// lanes of a beam group read them in one piece), and the lanes staging 32
// entries at once write distinct banks.
struct LfShared {
    float4 q[3][32 * kLidarColsMax];   // (a0, p0, a1, p1) (a2, p2, b0, m0) (b1, m1, b2, m2)
    float2 t[32 * kLidarColsMax];      // (t0, t1)
    float4 e[32];                      // (sigma, f0, f1, f2)
    uint32_t lanes[32];                // staged entry's ray mask
    uint2 cand[kLfWin];                // a window's entries to stage: (Gaussian, ray mask)
    float ref[kLidarColsMax][12];      // per column slot: d_r (hi, lo), z_c, o_c
};

static_assert(kLidarColsMax == 4, "the slot swizzle below assumes four column slots");
__device__ __forceinline__ int lf_qi(int j, int sl) { return 4 * j + (sl ^ ((j >> 1) & 3)); }
__device__ __forceinline__ int lf_ti(int j, int sl) { return 4 * j + (sl ^ ((j >> 2) & 3)); }

// Stage entry `pos` (record r) for the item's ncols column slots.
__device__ __forceinline__ void lf_entry(const GRec &r, LfShared &S, int pos, int ncols)
{
    const float mu[3] = {r.mu_sigma.x, r.mu_sigma.y, r.mu_sigma.z};
    const float M[3][3] = {{r.m0.x, r.m0.y, r.m0.z}, {r.m1.x, r.m1.y, r.m1.z},
                           {r.m2.x, r.m2.y, r.m2.z}};
    const float f[3] = {kResponseScale * r.m0.w, kResponseScale * r.m1.w,
                        kResponseScale * r.m2.w};
    S.e[pos] = make_float4(r.mu_sigma.w, r.feat.x, r.feat.y, r.feat.z);
    for (int sl = 0; sl < ncols; ++sl) {
        const float *ref = S.ref[sl];
        const float dh[3] = {ref[0], ref[1], ref[2]}, dl[3] = {ref[3], ref[4], ref[5]};
        const float z[3] = {ref[6], ref[7], ref[8]}, o[3] = {ref[9], ref[10], ref[11]};
        float w[3], vh[3];
        precise_moment(mu, o, dh, dl, w, vh);
        const float g[3] = {vh[1] * z[2] - vh[2] * z[1], vh[2] * z[0] - vh[0] * z[2],
                            vh[0] * z[1] - vh[1] * z[0]};
        float a[3], p[3], b[3], m[3], mv[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            a[k] = f[k] * dot3(M[k], w);
            p[k] = f[k] * dot3(M[k], g);
            b[k] = dot3(M[k], dh);
            m[k] = dot3(M[k], z);
            mv[k] = dot3(M[k], vh);
        }
        const int qi = lf_qi(pos, sl);
        S.q[0][qi] = make_float4(a[0], p[0], a[1], p[1]);
        S.q[1][qi] = make_float4(a[2], p[2], b[0], m[0]);
        S.q[2][qi] = make_float4(b[1], m[1], b[2], m[2]);
        S.t[lf_ti(pos, sl)] = make_float2(dot3(mv, b), dot3(mv, m));
    }
}

// A ray's running sums.  T = 0 marks a ray that has stopped (or has none, or
// sits out a re-walk): every later weight alpha T is then 0.  A live ray's
// transmittance is >= t_min; it reaches 0 only where nothing more can add.
struct LfAcc {
    float T, W, Z, c0, c1, c2;
};

// Composite entries [lo, hi) of the item's list into the lane's sums: the
// item's ray masks (lm[i] for list entry i) select the entries of a window
// of kLfWin that reach a ray still compositing; only those are staged, 32 at
// a time.  Then each beam group (lanes gm) evaluates, in list order, the
// staged entries whose box holds a ray of its beam.  x: the lane's tan(el) -
// tan(el_r); sl: its column slot.
__device__ __forceinline__ void lf_walk(const LidRender &P, const GRec *__restrict__ rec,
                                        const uint32_t *__restrict__ ids,
                                        const uint32_t *__restrict__ lm, int ncols, float x,
                                        int sl, uint32_t gm, uint32_t lo, uint32_t hi,
                                        LfShared &S, LfAcc &a)
{
    const int lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    const uint32_t bit = 1u << lane;
    // the next window's ray masks and ids (entries lane + 32 w of it), loaded
    // one window ahead
    uint32_t nm[kLfPer], nid[kLfPer];
#pragma unroll
    for (int w = 0; w < kLfPer; ++w) {
        const uint32_t i = lo + 32 * w + lane;
        nm[w] = i < hi ? lm[i] : 0u;
        nid[w] = i < hi ? ids[i] : 0u;
    }
    for (uint32_t base = lo; base < hi; base += kLfWin) {
        const uint32_t act = __ballot_sync(0xffffffffu, a.T != 0.f);
        if (act == 0u) break;
        uint32_t g[kLfPer], m[kLfPer], bw[kLfPer];
#pragma unroll
        for (int w = 0; w < kLfPer; ++w) {
            g[w] = nid[w];
            m[w] = nm[w] & act;
            const uint32_t i = base + kLfWin + 32 * w + lane;
            nm[w] = 0u;
            if (i < hi) {
                nm[w] = lm[i];
                nid[w] = ids[i];
            }
        }
        int n = 0;
#pragma unroll
        for (int w = 0; w < kLfPer; ++w) {
            bw[w] = __ballot_sync(0xffffffffu, m[w] != 0u);
            n += __popc(bw[w]);
        }
        if (n == 0) continue;
        __syncwarp();
        int off = 0;
#pragma unroll
        for (int w = 0; w < kLfPer; ++w) {
            if (m[w]) S.cand[off + __popc(bw[w] & below)] = make_uint2(g[w], m[w]);
            off += __popc(bw[w]);
        }
        for (int c0 = 0; c0 < n; c0 += 32) {
            const int nb = n - c0 < 32 ? n - c0 : 32;
            __syncwarp();
            if (lane < nb) {
                const uint2 c = S.cand[c0 + lane];
                lf_entry(rec[c.x], S, lane, ncols);
                S.lanes[lane] = c.y;
            }
            __syncwarp();
            // per live beam group, the staged entries that reach one of its rays
            const uint32_t lj = lane < nb ? S.lanes[lane] : 0u;
            uint32_t G = 0u;
            for (uint32_t rest = __ballot_sync(0xffffffffu, a.T != 0.f); rest;) {
                const uint32_t gm_g = __shfl_sync(0xffffffffu, gm, __ffs(rest) - 1);
                const uint32_t Gg = __ballot_sync(0xffffffffu, (lj & gm_g) != 0u);
                G = gm == gm_g ? Gg : G;
                rest &= ~gm_g;
            }
            while (__any_sync(0xffffffffu, G != 0u)) {
                const bool has = G != 0u;
                const int j = has ? __ffs(G) - 1 : 0;
                G &= G - 1u;
                const int qi = lf_qi(j, sl);
                const float4 A = S.q[0][qi], B = S.q[1][qi], C = S.q[2][qi];
                const float2 U = S.t[lf_ti(j, sl)];
                const float4 E = S.e[j];
                const bool in = has && (S.lanes[j] & bit) != 0u;
                const float n0 = fmaf(A.y, x, A.x), n1 = fmaf(A.w, x, A.z);
                const float n2 = fmaf(B.y, x, B.x);
                const float d0 = fmaf(B.w, x, B.z), d1 = fmaf(C.y, x, C.x);
                const float d2 = fmaf(C.w, x, C.z);
                const float tn = fmaf(U.y, x, U.x);
                const float inv = __fdividef(1.f, d0 * d0 + d1 * d1 + d2 * d2);
                const float rho = ex2_approx(-((n0 * n0 + n1 * n1 + n2 * n2) * inv));
                const float alpha = fminf(E.x * rho, P.alpha_max);
                const bool ok = in && tn > 0.f && alpha >= P.alpha_min;
                const float w = (ok ? alpha : 0.f) * a.T;
                const float Tn = a.T - w;
                const bool stop = Tn < P.t_min;
                const float wgt = stop ? 0.f : w;
                a.T = stop ? 0.f : Tn;
                a.c0 += wgt * E.y;
                a.c1 += wgt * E.z;
                a.c2 += wgt * E.w;
                a.W += wgt;
                a.Z += wgt * (tn * inv);
            }
        }
    }
}

// Partial slot layout, as k_render_lidar's: (c0, c1, c2, W), (Z, T, 0,
// stopped flag).
__device__ __forceinline__ void lf_put(float4 *pq, const LfAcc &a, bool stopped)
{
    pq[0] = make_float4(a.c0, a.c1, a.c2, a.W);
    pq[1] = make_float4(a.Z, a.T, 0.f, stopped ? 1.f : 0.f);
}
__device__ __forceinline__ LfAcc lf_get(float4 u, float4 v) { return {v.y, u.w, v.x, u.x, u.y, u.z}; }

// Walk [lo, hi) for the lanes in `mine` only: the others sit it out with
// T = 0 and get their transmittance back.
__device__ __forceinline__ void lf_walk_for(const LidRender &P, const GRec *__restrict__ rec,
                                            const uint32_t *__restrict__ ids,
                                            const uint32_t *__restrict__ lm, int ncols, float x,
                                            int sl, uint32_t gm, uint32_t lo, uint32_t hi,
                                            LfShared &S, LfAcc &a, bool mine)
{
    const float keep_T = a.T;
    if (!mine) a.T = 0.f;
    lf_walk(P, rec, ids, lm, ncols, x, sl, gm, lo, hi, S, a);
    if (!mine) a.T = keep_T;
}

// Split items re-walk the first kLfInlineRewalks segments in which some of
// their rays stop; later ones are deferred to the kFix launch, as in
// k_render_lidar.
constexpr int kLfInlineRewalks = 2;
// Segment length of this kernel's work items: LiDAR lists are walked in
// runs of 512 entries, twice the camera's: fewer merges and deferred
// re-walks.  Measured (street sweep, render ms): 128 0.358, 256 0.346, 512
// 0.340, 1024 0.361, 2048 0.409.
constexpr uint32_t kLfSeg = 512;

template <bool kFix>
__global__ void __launch_bounds__(32 * kLfWarps, kLfBlocks)
k_render_lidar_fwd(LidRender P, const LidarItem *__restrict__ items,
                   const uint32_t *__restrict__ item_rays, const float2 *__restrict__ ray_tau,
                   const double *__restrict__ item_ref, const uint2 *__restrict__ tile_items,
                   const uint32_t *__restrict__ lmask, int64_t lmask_stride,
                   const GRec *__restrict__ rec, const uint32_t *__restrict__ ids,
                   const uint2 *__restrict__ ranges, const uint2 *__restrict__ work,
                   const uint2 *__restrict__ unit_info, const uint32_t *__restrict__ counts,
                   uint32_t *__restrict__ counter, uint32_t *__restrict__ arrive,
                   float4 *__restrict__ partials, FixList F, const RenderDesc *__restrict__ D)
{
    __shared__ LfShared s_all[kLfWarps];
    const int lane = threadIdx.x & 31;
    LfShared &S = s_all[threadIdx.x >> 5];
    const float *__restrict__ poses = D->poses;
    const uint32_t n_work = kFix ? *F.n_fix : counts[0];
    uint32_t fix_next = blockIdx.x * kLfWarps + (threadIdx.x >> 5);
    while (true) {
        uint2 w;
        uint32_t fix_lanes = 0u;
        if constexpr (kFix) {
            if (fix_next >= n_work || fix_next >= F.cap) break;
            const uint4 f = F.fix[fix_next];
            fix_next += gridDim.x * kLfWarps;
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
        const int sl = valid ? (int)(ray % (uint32_t)P.n_cols) - (int)it.col0 : 0;
        const float2 rt = ray_tau[it.ray_off + lane];        // (x, |d'|)
        const uint32_t gm = __match_any_sync(0xffffffffu, valid ? ray / (uint32_t)P.n_cols
                                                                : 0xffffffffu);
        // the column slots' reference rays, under each column's own pose
        __syncwarp();
        if (lane < (int)it.ncols) {
            const float *Pc = poses + 12 * (it.col0 + lane);
            const double *u = item_ref + 12 * (size_t)item_id + 3 * lane;
            float *ref = S.ref[lane];
#pragma unroll
            for (int i = 0; i < 3; ++i) {
                const double d = (double)Pc[4 * i] * u[0] + (double)Pc[4 * i + 1] * u[1] +
                                 (double)Pc[4 * i + 2] * u[2];
                const float h = (float)d;
                ref[i] = h;
                ref[3 + i] = (float)(d - (double)h);
                ref[6 + i] = Pc[4 * i + 2];
                ref[9 + i] = Pc[4 * i + 3];
            }
        }
        __syncwarp();
        const uint32_t *lm = lmask + (int64_t)(item_id - (int)tile_items[it.tile].x) * lmask_stride;
        const uint2 rg = ranges[it.tile];
        const uint32_t lo = rg.x + seg * kLfSeg;
        const uint32_t hi = min(rg.y, lo + kLfSeg);
        LfAcc a = {valid ? 1.f : 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        bool write = valid;
        if constexpr (kFix) {
            const bool mine = (fix_lanes >> lane) & 1u;
            const float4 *pq = partials + ((size_t)(ui.y + seg) * 32 + lane) * 2;
            if (mine) a = lf_get(pq[0], pq[1]);
            else a.T = 0.f;
            lf_walk(P, rec, ids, lm, it.ncols, rt.x, sl, gm, lo, hi, S, a);
            write = mine;
        } else {
            lf_walk(P, rec, ids, lm, it.ncols, rt.x, sl, gm, lo, hi, S, a);
            if (ui.x > 1) {
                // split item: publish this segment, and combine if it is the last one
                lf_put(partials + ((size_t)(ui.y + seg) * 32 + lane) * 2, a,
                       valid && a.T == 0.f);
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
                a = lf_get(u0, v0);
                bool fin = !valid || v0.w != 0.f;
                int n_inline = 0;
                for (uint32_t sgi = 1; sgi < ui.x; ++sgi) {
                    if (__all_sync(0xffffffffu, fin)) break;
                    pq += 64;
                    const float4 u = __ldcg(pq), v = __ldcg(pq + 1);
                    // the state before segment sgi replaces its partial
                    lf_put(pq, a, false);
                    const bool take = !fin && v.w == 0.f && a.T * v.y >= P.t_min;
                    const bool redo = !fin && !take;
                    if (take) {
                        a.c0 += a.T * u.x;
                        a.c1 += a.T * u.y;
                        a.c2 += a.T * u.z;
                        a.W += a.T * u.w;
                        a.Z += a.T * v.x;
                        a.T *= v.y;
                    }
                    const uint32_t rl = __ballot_sync(0xffffffffu, redo);
                    if (rl && n_inline < kLfInlineRewalks) {
                        ++n_inline;
                        const uint32_t l0 = rg.x + sgi * kLfSeg;
                        lf_walk_for(P, rec, ids, lm, it.ncols, rt.x, sl, gm, l0,
                                    min(rg.y, l0 + kLfSeg), S, a, redo);
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
            // Z sums tau' along d'; the range along the unit ray is tau' |d'|
            if (out_range) out_range[ray] = a.W > 0.f ? a.Z * rt.y / a.W : 0.f;
            if (out_int) out_int[ray] = a.c0;
            if (out_drop) out_drop[ray] = drop;
            if (out_alpha) out_alpha[ray] = a.W;
        }
        __syncwarp();
    }
}

static int lf_blocks_per_sm()
{
    static int cached = 0;
    if (!cached) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_lidar_fwd<false>,
                                                          32 * kLfWarps, 0) != cudaSuccess ||
            nb < 1)
            nb = 4;
        cached = nb;
    }
    return cached;
}

bool lidar_forward_only(const Frame &fr) { return !fr.keep_state; }

sg_status render_lidar_fwd(const Lidar &L, const sg_render_opts &o, Frame &fr, cudaStream_t st)
{
    const LidRender P = lidar_render_params(L, o);
    if (L.n_items == 0) return SG_OK;
    const int64_t K = fr.n_pairs;
    const WorkSize ws = work_size(L.n_items, K * L.max_items_per_tile, kLfSeg, 1);
    sg_status s = ensure(fr.order, sizeof(uint32_t) * (size_t)L.n_items);
    if (s == SG_OK) s = ensure(fr.camwork, ws.work_bytes);
    if (s == SG_OK) s = ensure(fr.partials, ws.partial_bytes);
    if (s != SG_OK) return s;
    if ((s = launch_work_items(fr, ws, L.d_items, L.n_items, 1, kLfSeg, st)) != SG_OK) return s;
    unsigned char *cw = (unsigned char *)fr.camwork.p;
    const uint2 *unit_info = (const uint2 *)cw;
    const uint2 *work = (const uint2 *)(cw + ws.info_bytes + ws.off_bytes);
    uint32_t *arrive = (uint32_t *)(cw + ws.info_bytes + ws.off_bytes + ws.items_bytes);
    const uint32_t *ids = (const uint32_t *)fr.pvals[fr.pair_buf].p;
    int dev = 0, sms = 0;
    SG_CUDA(cudaGetDevice(&dev));
    SG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t cap = (ws.max_items + kLfWarps - 1) / kLfWarps;
    int64_t grid = (int64_t)sms * lf_blocks_per_sm();
    grid = grid < cap ? grid : cap;
    if (grid < 1) grid = 1;
    const FixList F = fix_list(fr, ws);
    k_render_lidar_fwd<false><<<(unsigned)grid, 32 * kLfWarps, 0, st>>>(
        P, L.d_items, L.d_item_rays, L.d_ray_tau, L.d_item_ref, L.d_tile_items,
        (const uint32_t *)fr.lmask.p, fr.lmask_stride, (const GRec *)fr.rec.p, ids,
        (const uint2 *)fr.ranges.p, work, unit_info, (const uint32_t *)fr.scalars.p + 4,
        (uint32_t *)fr.scalars.p + 2, arrive, (float4 *)fr.partials.p, F,
        (const RenderDesc *)fr.desc.p);
    SG_LAUNCHED();
    if (ws.max_slots > 0) {       // some item may be split: the deferred re-walks
        const int64_t fcap = (ws.max_fixes + kLfWarps - 1) / kLfWarps;
        const int64_t fgrid = grid < fcap ? grid : fcap;
        k_render_lidar_fwd<true><<<(unsigned)fgrid, 32 * kLfWarps, 0, st>>>(
            P, L.d_items, L.d_item_rays, L.d_ray_tau, L.d_item_ref, L.d_tile_items,
            (const uint32_t *)fr.lmask.p, fr.lmask_stride, (const GRec *)fr.rec.p, ids,
            (const uint2 *)fr.ranges.p, work, unit_info, (const uint32_t *)fr.scalars.p + 4,
            (uint32_t *)fr.scalars.p + 2, arrive, (float4 *)fr.partials.p, F,
            (const RenderDesc *)fr.desc.p);
        SG_LAUNCHED();
    }
    return SG_OK;
}

}  // namespace sg
