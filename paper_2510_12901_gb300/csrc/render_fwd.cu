// render_fwd.cu -- camera compositing (Eq. 1, the response at tau_max as in
// render.cu) for frames that keep no state for a backward: images only, as
// rendered by a serving loop or a benchmark.  The work decomposition is
// k_render_camera's (persistent independent warps, tile lists split into
// segments merged by the last arriving warp, sub-block masks, live-ray
// staging) over 8x4 pixel sub-blocks; the rays are parameterised so that a
// (ray, Gaussian) pair costs fewer instructions, and no state for a backward
// (last composited entry, final sums) is tracked or written.
//
// Tangent-plane rays.  With d_T the tile's reference direction (double, split
// into two floats) and (e_1, e_2) an orthonormal basis of the plane normal to
// it, a pixel's unit direction d is written as d / (d . d_T) = d_T + u_1 e_1 +
// u_2 e_2, (u_1, u_2) computed once per camera in double.  D^2 does not depend
// on the length of the direction, and tau_max along d' = d / (d . d_T) is the
// distance along d times (d . d_T), so the distance is tau' |d'|.  With v =
// mu - o and f_k = s_k / (s_i s_j):
//   num_k = a_k + u_1 p_k1 + u_2 p_k2,  a_k = f_k M_k . (v x d_T),
//                                        p_kj = f_k M_k . (v x e_j)
//   den_k = b_k + u_1 m_k1 + u_2 m_k2,  b_k = M_k . d_T,  m_kj = M_k . e_j
//   (M v) . den = t_0 + u_1 t_1 + u_2 t_2
// so each of the seven is two FMAs per pair, against three with a 3-vector
// offset; a_k keeps the error-free moment of render.cu, and the u-terms are
// small corrections.
#include <math.h>

#include "pairs.cuh"
#include "render.cuh"

namespace sg {

constexpr int kFwdWarps = 4;        // warps per block of the persistent grid
// blocks per SM the register budget is set for (72 registers; a few bytes of
// the merge spill).  Measured on the street views, compositing alone / the
// two-view step: 6 blocks 0.387 / 0.547 ms, 3122 Mrays/s; 7 blocks 0.383 /
// 0.534 ms, 3189-3200 Mrays/s; 8 blocks 0.418 / 0.545 ms, 3237 Mrays/s.
constexpr int kFwdBlocks = 7;
// List entries a warp scans per batch: kFwdPer per lane.  The entries of
// the window that reach a live ray of the sub-block (about a third of them
// on the street views) are staged together, so that the staging pass, one
// entry per lane, runs with more of its lanes busy than over a 32-entry
// window.  Measured (street views, compositing alone / bench): 32 entries
// 0.374 / 0.528 ms, 3219 Mrays/s; 64 entries 0.364 / 0.519 ms, 3284; 96
// entries 0.362 / 0.514 ms, 3305; 128 entries 0.361 / 0.524 ms, 3265.
#ifndef SG_FWD_PER_LANE
#define SG_FWD_PER_LANE 3
#endif
constexpr int kFwdPer = SG_FWD_PER_LANE;
constexpr int kFwdWin = 32 * kFwdPer;
constexpr int kFwdStage = 64;
// Segment length of this kernel's work items (frames that keep no backward
// state need not match the segments of a backward).  Measured on the street
// views (compositing alone fisheye / pinhole, two-view step): 128 entries
// 0.390 / 0.562 ms, 3102 Mrays/s; 256 0.363 / 0.513 ms, 3310; 384 0.367 /
// 0.503 ms, 3364; 512 0.381 / 0.508 ms, 3384.  Longer runs mean fewer
// merges; shorter ones split the densest tiles (the fisheye's) finer.
constexpr uint32_t kFwdSeg = 384;   // staged entries held in shared memory at once

// The tile's reference frame in world coordinates: d_T = dh + dl (from the
// double direction, as cam_tile_ref) and e_1, e_2 rotated in float.
__device__ __forceinline__ void fwd_tile_ref(const CamPose &P, const double *tile_dir,
                                             const float *tile_basis, int tile, float *s_ref)
{
    cam_tile_ref(P, tile_dir, tile, s_ref);
    const float *b = tile_basis + 6 * tile;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        s_ref[6 + i] = P.R[3 * i] * b[0] + P.R[3 * i + 1] * b[1] + P.R[3 * i + 2] * b[2];
        s_ref[9 + i] = P.R[3 * i] * b[3] + P.R[3 * i + 1] * b[4] + P.R[3 * i + 2] * b[5];
    }
}

__device__ __forceinline__ void cross3(const float a[3], const float b[3], float c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

// A staged entry, 7 float4 (one per shared-memory plane):
//   0 (a0, p01, p02, a1)   1 (p11, p12, a2, p21)   2 (p22, b0, m01, m02)
//   3 (b1, m11, m12, b2)   4 (m21, m22, t0, t1)    5 (t2, sigma, c0, c1)
//   6 (c2, lane mask, 0, 0)
// with p_kj = f_k M_k . (v x e_j) and m_kj = M_k . e_j.  The P terms (a, p)
// carry the response scale sqrt(log2(e) / 2), as in cam_pair_scaled, so that
// |num|^2 / |den|^2 is the exponent of 2.  ref: the tile's reference frame
// (dh, dl, e_1, e_2), in the warp's shared memory.
__device__ __forceinline__ void fwd_entry(const GRec &r, const float o[3], const float *ref,
                                          float4 e[7])
{
    const float mu[3] = {r.mu_sigma.x, r.mu_sigma.y, r.mu_sigma.z};
    const float M[3][3] = {{r.m0.x, r.m0.y, r.m0.z}, {r.m1.x, r.m1.y, r.m1.z},
                           {r.m2.x, r.m2.y, r.m2.z}};
    const float f[3] = {kResponseScale * r.m0.w, kResponseScale * r.m1.w,
                        kResponseScale * r.m2.w};
    const float dh[3] = {ref[0], ref[1], ref[2]}, dl[3] = {ref[3], ref[4], ref[5]};
    const float e1[3] = {ref[6], ref[7], ref[8]}, e2[3] = {ref[9], ref[10], ref[11]};
    float w[3], vh[3], g1[3], g2[3];
    precise_moment(mu, o, dh, dl, w, vh);
    cross3(vh, e1, g1);
    cross3(vh, e2, g2);
    float a[3], p1[3], p2[3], b[3], m1[3], m2[3], mv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a[k] = f[k] * dot3(M[k], w);
        p1[k] = f[k] * dot3(M[k], g1);
        p2[k] = f[k] * dot3(M[k], g2);
        b[k] = dot3(M[k], dh);
        m1[k] = dot3(M[k], e1);
        m2[k] = dot3(M[k], e2);
        mv[k] = dot3(M[k], vh);
    }
    e[0] = make_float4(a[0], p1[0], p2[0], a[1]);
    e[1] = make_float4(p1[1], p2[1], a[2], p1[2]);
    e[2] = make_float4(p2[2], b[0], m1[0], m2[0]);
    e[3] = make_float4(b[1], m1[1], m2[1], b[2]);
    e[4] = make_float4(m1[2], m2[2], dot3(mv, b), dot3(mv, m1));
    e[5] = make_float4(dot3(mv, m2), r.mu_sigma.w, r.feat.x, r.feat.y);
    e[6] = make_float4(r.feat.z, 0.f, 0.f, 0.f);
}

struct FwdAcc {
    float T, W, Z, c0, c1, c2;
};

// Composite the n staged entries into the lane's accumulator (ray with
// tangent-plane coordinates (x, y)); done: the ray has stopped (or has none).
__device__ __forceinline__ void fwd_composite(const CamRender &P, float4 (*s)[kFwdStage], int n,
                                              float x, float y, FwdAcc &a, bool &done)
{
    const uint32_t bit = 1u << (threadIdx.x & 31);
    for (int j = 0; j < n; ++j) {
        const float4 A = s[0][j], B = s[1][j], C = s[2][j], D = s[3][j], E = s[4][j];
        const float4 F = s[5][j], G = s[6][j];
        const float n0 = fmaf(A.z, y, fmaf(A.y, x, A.x));
        const float n1 = fmaf(B.y, y, fmaf(B.x, x, A.w));
        const float n2 = fmaf(C.x, y, fmaf(B.w, x, B.z));
        const float d0 = fmaf(C.w, y, fmaf(C.z, x, C.y));
        const float d1 = fmaf(D.z, y, fmaf(D.y, x, D.x));
        const float d2 = fmaf(E.y, y, fmaf(E.x, x, D.w));
        const float tn = fmaf(F.x, y, fmaf(E.w, x, E.z));
        const float inv = __fdividef(1.f, d0 * d0 + d1 * d1 + d2 * d2);
        const float rho = ex2_approx(-((n0 * n0 + n1 * n1 + n2 * n2) * inv));
        const float alpha = fminf(F.y * rho, P.alpha_max);
        const bool in = (__float_as_uint(G.y) & bit) != 0u;
        const bool ok = in && tn > 0.f && alpha >= P.alpha_min && !done;
        const float w = alpha * a.T;
        const float Tn = a.T - w;
        const bool stop = ok && Tn < P.t_min;
        done = done || stop;
        const bool take = ok && !stop;
        const float wgt = take ? w : 0.f;
        a.c0 += wgt * F.z;
        a.c1 += wgt * F.w;
        a.c2 += wgt * G.x;
        a.Z += wgt * (tn * inv);
        a.W += wgt;
        a.T = take ? Tn : a.T;
    }
}

// Composite list entries [lo, hi) of a tile that can reach sub-block `sub`
// into the lane's accumulator.  Lanes whose ray is done take part in the
// staging and keep their state; only entries whose box holds a live ray are
// staged (their lane masks come from the column/row words, no record load).
// cand: the warp's (Gaussian, lane mask) list of a window's staged entries.
__device__ __forceinline__ void fwd_walk(const CamRender &P, const CamPose &pose,
                                         const GRec *__restrict__ rec,
                                         const uint32_t *__restrict__ ids,
                                         const uint32_t *__restrict__ crw, int sub, uint32_t lo,
                                         uint32_t hi, const float *ref, float x, float y,
                                         float4 (*s)[kFwdStage], uint2 *cand, FwdAcc &a,
                                         bool &done)
{
    const int lane = threadIdx.x & 31;
    const uint32_t below = (1u << lane) - 1u;
    // the next window's column/row words and Gaussian ids (entries lane + 32 w
    // of it), loaded one window ahead
    uint32_t ncr[kFwdPer], nid[kFwdPer];
#pragma unroll
    for (int w = 0; w < kFwdPer; ++w) {
        const uint32_t i = lo + 32 * w + lane;
        ncr[w] = i < hi ? crw[i] : 0u;
        nid[w] = i < hi ? ids[i] : 0u;
    }
    for (uint32_t base = lo; base < hi; base += kFwdWin) {
        const uint32_t act = __ballot_sync(0xffffffffu, !done);
        if (act == 0u) break;
        uint32_t g[kFwdPer], lm[kFwdPer], bw[kFwdPer];
#pragma unroll
        for (int w = 0; w < kFwdPer; ++w) {
            g[w] = nid[w];
            lm[w] = word_lanes(ncr[w], sub) & act;
            const uint32_t i = base + kFwdWin + 32 * w + lane;
            ncr[w] = 0u;
            if (i < hi) {
                ncr[w] = crw[i];
                nid[w] = ids[i];
            }
        }
        int n = 0;
#pragma unroll
        for (int w = 0; w < kFwdPer; ++w) {
            bw[w] = __ballot_sync(0xffffffffu, lm[w] != 0u);
            n += __popc(bw[w]);
        }
        if (n == 0) continue;
        __syncwarp();
        int off = 0;
#pragma unroll
        for (int w = 0; w < kFwdPer; ++w) {
            if (lm[w]) cand[off + __popc(bw[w] & below)] = make_uint2(g[w], lm[w]);
            off += __popc(bw[w]);
        }
        // stage and composite them, in list order, kFwdStage at a time
        for (int c0 = 0; c0 < n; c0 += kFwdStage) {
            const int m = n - c0 < kFwdStage ? n - c0 : kFwdStage;
            __syncwarp();
            for (int t = lane; t < m; t += 32) {
                const uint2 c = cand[c0 + t];
                float4 e[7];
                fwd_entry(rec[c.x], pose.t, ref, e);
                e[6].y = __uint_as_float(c.y);
#pragma unroll
                for (int k = 0; k < 7; ++k) s[k][t] = e[k];
            }
            __syncwarp();
            fwd_composite(P, s, m, x, y, a, done);
        }
    }
}

// Partial slot layout, as k_render_camera's: (c0, c1, c2, W), (Z, T, 0,
// stopped flag), at pixel slot 32 sub + lane of the tile's 8x4 sub-block sub.
__device__ __forceinline__ void fwd_put(float4 *pq, const FwdAcc &a, bool stopped)
{
    pq[0] = make_float4(a.c0, a.c1, a.c2, a.W);
    pq[1] = make_float4(a.Z, a.T, 0.f, stopped ? 1.f : 0.f);
}

template <uint32_t kSeg>
__global__ void __launch_bounds__(32 * kFwdWarps, kFwdBlocks)
k_render_camera_fwd(CamRender P, const GRec *__restrict__ rec, const uint32_t *__restrict__ ids,
                    const uint2 *__restrict__ ranges, const uint2 *__restrict__ items,
                    const uint2 *__restrict__ tile_info, const uint32_t *__restrict__ counts,
                    const uint32_t *__restrict__ crw, uint32_t *__restrict__ counter,
                    uint32_t *__restrict__ arrive, float4 *__restrict__ partials,
                    const float4 *__restrict__ pix2, const double *__restrict__ tile_dir,
                    const float *__restrict__ tile_basis, const RenderDesc *__restrict__ D)
{
    __shared__ float4 s_all[kFwdWarps][7][kFwdStage];
    __shared__ uint2 s_cand[kFwdWarps][kFwdWin];
    __shared__ float s_refs[kFwdWarps][12];
    __shared__ CamPose s_pose;
    load_cam_pose(D, s_pose);
    __syncthreads();
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float4(*s_e)[kFwdStage] = s_all[wib];
    uint2 *cand = s_cand[wib];
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
        if (lane == 0) fwd_tile_ref(s_pose, tile_dir, tile_basis, tile, s_ref);
        __syncwarp();
        const int px = sbx + (lane & 7), py = sby + (lane >> 3);
        const bool inside = px < P.W && py < P.H;
        const int64_t pidx = inside ? (int64_t)py * P.W + px : -1;
        const float4 e = inside ? pix2[pidx] : make_float4(0.f, 0.f, 0.f, 0.f);
        const bool no_ray = !(inside && e.w > 0.f);
        const uint2 rg = ranges[tile];
        const uint32_t lo = rg.x + (uint32_t)seg * kSeg;
        const uint32_t hi = min(rg.y, lo + kSeg);
        FwdAcc a = {1.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        bool done = no_ray;
        fwd_walk(P, s_pose, rec, ids, crw, sub, lo, hi, s_ref, e.x, e.y, s_e, cand, a, done);
        if (ti.x > 1) {
            // long tile: publish this run, and combine if it is the last one
            fwd_put(partials + ((size_t)(ti.y + seg) * 256 + sub * 32 + lane) * 2, a,
                    done && !no_ray);
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
            // combine the runs in list order, two runs' partials in flight at
            // a time and no walk in between: a ray that stops in run s > 0
            // keeps the state before it and its run number.  The re-walks of a
            // dense tile's sub-block (up to ~20 runs) are a serial chain of
            // the launch; keeping the partials' loads out of it shortens it ...
            const float4 *pq = partials + ((size_t)ti.y * 256 + sub * 32 + lane) * 2;
            const float4 u0 = __ldcg(pq), v0 = __ldcg(pq + 1);
            a = {v0.y, u0.w, v0.x, u0.x, u0.y, u0.z};
            bool fin = no_ray || v0.w != 0.f;
            uint32_t stop_run = 0u;
            for (uint32_t s0 = 1; s0 < ti.x; s0 += 2) {
                if (__all_sync(0xffffffffu, fin)) break;
                float4 u[2], v[2];
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (s0 + k < ti.x) {
                        u[k] = __ldcg(pq + 512 * (s0 + k));
                        v[k] = __ldcg(pq + 512 * (s0 + k) + 1);
                    }
                }
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    if (s0 + k >= ti.x) break;
                    const bool take = !fin && v[k].w == 0.f && a.T * v[k].y >= P.t_min;
                    if (take) {
                        a.c0 += a.T * u[k].x;
                        a.c1 += a.T * u[k].y;
                        a.c2 += a.T * u[k].z;
                        a.W += a.T * u[k].w;
                        a.Z += a.T * v[k].x;
                        a.T *= v[k].y;
                    } else if (!fin) {
                        stop_run = s0 + k;
                    }
                    fin = fin || !take;
                }
            }
            // ... then each run in which rays stop, walked again for them from
            // the true state before it, in list order
            bool pend = stop_run != 0u;
            while (true) {
                const uint32_t r = __reduce_min_sync(0xffffffffu, pend ? stop_run : 0xffffffffu);
                if (r == 0xffffffffu) break;
                const bool mine = pend && stop_run == r;
                bool dn = !mine;
                const uint32_t l0 = rg.x + r * kSeg;
                fwd_walk(P, s_pose, rec, ids, crw, sub, l0, min(rg.y, l0 + kSeg), s_ref, e.x, e.y,
                         s_e, cand, a, dn);
                pend = pend && !mine;
            }
        }
        if (pidx >= 0) {
            float *const out_rgb = D->out[0], *const out_alpha = D->out[1];
            float *const out_depth = D->out[2];
            if (out_rgb) {
                out_rgb[3 * pidx] = a.c0;
                out_rgb[3 * pidx + 1] = a.c1;
                out_rgb[3 * pidx + 2] = a.c2;
            }
            if (out_alpha) out_alpha[pidx] = a.W;
            // Z sums tau' along d'; the distance along the unit ray is tau' |d'|
            if (out_depth) out_depth[pidx] = a.W > 0.f ? a.Z * pix2[pidx].z / a.W : 0.f;
        }
        __syncwarp();
    }
}

static int fwd_blocks_per_sm()
{
    static int cached = 0;
    if (!cached) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_render_camera_fwd<kFwdSeg>,
                                                          32 * kFwdWarps, 0) != cudaSuccess ||
            nb < 1)
            nb = 4;
        cached = nb;
    }
    return cached;
}

bool camera_forward_only(const Camera &cam, const Frame &fr)
{
    return !fr.keep_state && fr.seg_len == kSegLen && cam.tangent_ok;
}

sg_status render_camera_fwd(const Camera &cam, const sg_render_opts &o, Frame &fr,
                            cudaStream_t st)
{
    const CamRender P = cam_render_params(cam, o);
    const int nt = cam.ntx * cam.nty;
    const int64_t K = fr.n_pairs;
    const WorkSize ws = work_size(nt, K, kFwdSeg, 8);
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
    if ((s = launch_work_items(fr, ws, nullptr, nt, 8, kFwdSeg, st)) != SG_OK) return s;
    const uint32_t *ids = (const uint32_t *)fr.pvals[fr.pair_buf].p;
    int dev = 0, sms = 0;
    SG_CUDA(cudaGetDevice(&dev));
    SG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t cap = (ws.max_items + kFwdWarps - 1) / kFwdWarps;
    int64_t grid = (int64_t)sms * fwd_blocks_per_sm();
    grid = grid < cap ? grid : cap;
    if (grid < 1) grid = 1;
    k_render_camera_fwd<kFwdSeg><<<(unsigned)grid, 32 * kFwdWarps, 0, st>>>(
        P, (const GRec *)fr.rec.p, ids, (const uint2 *)fr.ranges.p, items, tile_info, counts,
        (const uint32_t *)fr.submask.p, counter, arrive, (float4 *)fr.partials.p, cam.d_pix2,
        cam.d_tile_dir, cam.d_tile_basis, (const RenderDesc *)fr.desc.p);
    SG_LAUNCHED();
    return SG_OK;
}

}  // namespace sg
