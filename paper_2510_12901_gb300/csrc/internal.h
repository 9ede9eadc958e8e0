// internal.h -- types and helpers shared by the CUDA translation units of
// libsimgut.  Not part of the C-ABI (include/simgut.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/simgut.h"

namespace sg {

// Feature kinds a LiDAR render takes, and kinds whose features are SH.
__host__ __device__ inline bool lidar_features(int kind)
{
    return kind == SG_FEATURES_LIDAR || kind == SG_FEATURES_LIDAR_SH;
}
__host__ __device__ inline bool sh_features(int kind)
{
    return kind == SG_FEATURES_SH || kind == SG_FEATURES_LIDAR_SH;
}

constexpr int kTile = 16;                 // camera tile edge (pixels)
constexpr int kCamThreads = kTile * kTile;
constexpr int kLidarColsMax = 4;          // distinct columns per LiDAR work item
constexpr int kLidarWarps = 4;            // warps (work items) per LiDAR render block
// Camera tile lists longer than the segment length are composited in
// segments of that many entries, each an independent work item, and
// combined afterwards.  kSegLen is the default of a frame (a build may set
// SG_SEG_LEN to tune it); the allocation-free render uses kSegLenStatic,
// which needs less workspace.
#ifndef SG_SEG_LEN
#define SG_SEG_LEN 256
#endif
constexpr uint32_t kSegLen = SG_SEG_LEN;
constexpr uint32_t kSegLenStatic = 1024;

void set_error(const char *fmt, ...);
bool opts_ok(const sg_render_opts *o);   // render options in range (sets the message)
sg_status cuda_status(cudaError_t e, const char *what);
// Every cudaMalloc / cudaFree / cudaMallocHost / cudaFreeHost of the library
// goes through these, which count the calls (sg_alloc_count).
void note_alloc();
template <class T> inline cudaError_t dev_malloc(T **p, size_t bytes)
{
    note_alloc();
    return cudaMalloc((void **)p, bytes);
}
inline cudaError_t dev_free(void *p)
{
    if (!p) return cudaSuccess;
    note_alloc();
    return cudaFree(p);
}
template <class T> inline cudaError_t host_malloc(T **p, size_t bytes)
{
    note_alloc();
    return cudaMallocHost((void **)p, bytes);
}
inline cudaError_t host_free(void *p)
{
    if (!p) return cudaSuccess;
    note_alloc();
    return cudaFreeHost(p);
}
void count_launch();           // not counted while capture_guard() is set
void count_launches(int64_t n); // kernels run by a graph replay

// after every kernel launch: count it and surface launch errors
#define SG_LAUNCHED()                                                     \
    do {                                                                  \
        ::sg::count_launch();                                             \
        cudaError_t e_ = cudaGetLastError();                              \
        if (e_ != cudaSuccess) return ::sg::cuda_status(e_, "kernel launch"); \
    } while (0)

#define SG_CUDA(call)                                                     \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return ::sg::cuda_status(e_, #call);       \
    } while (0)

// ------------------------------------------------------------------ handles
struct Scene {
    int64_t n = 0;
    int feature_kind = 0, sh_degree = 0, F = 3;
    // planar SoA, plane k holds component k of all Gaussians (n floats each)
    float *d_planes = nullptr;  // [3 mean + 3 logscale + 4 quat + 1 opacity + F] * n
    int64_t pitch = 0;          // floats per plane (n rounded up to 32)
    float *plane(int k) const { return d_planes + (int64_t)k * pitch; }
    static constexpr int kMean = 0, kLogScale = 3, kQuat = 6, kOpacity = 10, kFeat = 11;
    // dynamic actors: per-Gaussian actor index (-1 static) and the actors'
    // poses [n_actors,12] (row-major [R | t], actor to world); none if n_actors = 0
    int32_t *d_actor_of = nullptr;
    float *d_actor_poses = nullptr;
    int n_actors = 0;
};

// What a kernel needs of the actors (of = nullptr: every Gaussian static).
struct ActorParams {
    const int32_t *of;
    const float *poses;
    int n;
};
inline ActorParams actor_params(const Scene &s)
{
    return {s.n_actors > 0 ? s.d_actor_of : nullptr, s.d_actor_poses, s.n_actors};
}

struct Camera {
    int model = 0, width = 0, height = 0;
    float fx = 0, fy = 0, cx = 0, cy = 0, k[4] = {0, 0, 0, 0};
    double theta_max = 0;
    int ntx = 0, nty = 0;
    // per pixel: camera-frame direction minus its tile's reference direction
    // (w = 1 valid, 0 no ray); per tile: reference direction (double)
    float4 *d_pix = nullptr;
    double *d_tile_dir = nullptr;  // [ntiles*3]
    // per pixel: tangent-plane coordinates (u1, u2) of the direction over its
    // cosine to the tile's reference direction, that length |d'|, valid;
    // per tile: the tangent basis e1, e2 (camera frame, float [ntiles*6]).
    // tangent_ok: every valid pixel is within 75 degrees of its tile's
    // reference direction (|d'| <= 4), which the forward-only kernel assumes.
    float4 *d_pix2 = nullptr;
    float *d_tile_basis = nullptr;
    bool tangent_ok = false;
};

struct LidarItem {       // one warp of LiDAR rendering
    uint32_t tile;       // elevation-major tile id e * n_theta + a
    uint16_t col0;       // first column of the item
    uint8_t ncols;       // distinct columns (<= kLidarColsMax)
    uint8_t nrays;       // rays (<= 32)
    uint32_t ray_off;    // offset into item_rays (32 slots per item)
    uint32_t ref_col;    // column whose rotation defines the tile reference ray
};

// The ray slots of a LiDAR work item, factorised: slot k holds the ray of
// column col0 + s (bit k of col_bits[s]) and of the beam at elevation
// beam_el[j] (bit k of beam_bits[j]); empty slots are in no mask.
struct LidarItemRays {
    int ncols, nbeams;
    float col_az[kLidarColsMax];
    uint32_t col_bits[kLidarColsMax];
    float beam_el[32];
    uint32_t beam_bits[32];
};

struct Lidar {
    int n_beams = 0, n_cols = 0;
    float az0 = 0;
    int nphi = 0, M = 0, n_theta = 0, cull_az = 0, cull_el = 0;
    std::vector<float> elev, T;
    int n_items = 0;
    int max_items_per_tile = 1;     // work items sharing one tile, at most
    float *d_T = nullptr;           // [nphi+1]
    float *d_elev = nullptr;        // [n_beams]
    float *d_az = nullptr;          // [n_cols] column azimuth (deg)
    int *d_sat = nullptr;           // [(A+1)*(E+1)]
    LidarItem *d_items = nullptr;   // [n_items]
    uint32_t *d_item_rays = nullptr;  // [n_items*32]: beam*n_cols + col, ~0u = none
    float4 *d_ray_e = nullptr;      // [n_beams*n_cols] sensor dir minus tile reference
    double *d_tile_u = nullptr;     // [ntiles*3] tile reference sensor direction
    uint2 *d_tile_items = nullptr;  // [ntiles] (first item, number of items) of each tile
    LidarItemRays *d_item_ray_tab = nullptr;   // [n_items] factorised ray slots
    // forward-only compositing (render_lidar_fwd.cu): per item and column
    // slot the sensor-frame reference (cos az, sin az, tan el_r), double; per
    // ray slot (tan el - tan el_r, 1 / cos el)
    double *d_item_ref = nullptr;   // [n_items * kLidarColsMax * 3]
    float2 *d_ray_tau = nullptr;    // [n_items * 32]
};

// ------------------------------------------------------------------ records
// Per-Gaussian render record written by the projection (96 bytes).
struct __align__(16) GRec {
    float4 mu_sigma;   // mean, opacity
    float4 m0;         // row 0 of M = S^-1 R^T, w = f_0 = s0^2/(s0 s1 s2)
    float4 m1;         // row 1, f_1
    float4 m2;         // row 2, f_2
    float4 feat;       // colour / LiDAR features (3), pad
    float4 rect;       // per-ray test box x_lo, x_hi, y_lo, y_hi
};

// ------------------------------------------------------------------ frame
// Per-render parameters that change from one render to the next, kept in
// device memory (copied from pinned host memory at the start of each render)
// so that a captured launch sequence can be replayed for a new pose and new
// output buffers.  The kernels read the pose and the output pointers here.
struct RenderDesc {
    float c2w[12];          // camera renders: row-major [R | t]
    const float *poses;     // LiDAR renders: per-column c2w [n_cols, 12] (device)
    float *out[4];          // outputs (device), NULL = not written
};

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
    bool borrowed = false;   // memory the frame does not own (a fixed workspace): never grown
};

struct Frame {
    // per-Gaussian
    Buf rec, rect, tiles, depth, count, mean2d, cov2d;
    // depth sort / offsets
    Buf dkeys[2], dvals[2], offsets, hist;
    // pairs; LiDAR: per (work item of the pair's tile, pair) the 32-bit mask
    // of the item's rays inside the Gaussian's box, planes of lmask_stride
    Buf pkeys[2], pvals[2], ranges, order, submask, lmask;
    int64_t lmask_stride = 0;
    // camera work items: per-tile (segments, first partial slot), items,
    // arrival counters of long tiles; per-pixel partials of their segments
    Buf camwork, partials;
    // per-ray saved state: (T_final, omega, Z, LiDAR drop) and contributor count
    Buf ray_state, n_contrib;
    Buf ray_feat;     // per ray: the final feature sums (F0, F1, F2, 0), for the backward
    // backward accumulators: per Gaussian dL/dM (9), dL/dmu (3), dL/dsigma,
    // dL/dfeature (3)
    Buf gacc;
    Buf scalars;      // device scalars: [0] valid Gaussians [1] pairs [2] work-item
                      // counter [3] pairs dropped over capacity [4..5] work-item counts
                      // [6] backward work counter [7] deferred re-walks
                      // [8] status: a look-back wait gave up (kScalStatus)
    Buf desc;         // RenderDesc of the current render (device)
    uint32_t *h_scalars = nullptr;  // pinned: scalars mirror (64 B), then the RenderDesc
    RenderDesc *h_desc = nullptr;   // pinned staging of desc
    // capacity mode: > 0 = the pair buffers hold this many pairs and no
    // step waits for the pair count (pairs beyond it are dropped and counted)
    int64_t k_cap = 0;
    uint32_t seg_len = kSegLen;     // camera list segment length
    bool keep_state = true;         // renders write the per-ray state the backward needs
    bool state_kept = false;        // the last render did
    int64_t n_pairs = 0, n_tiles = 0, n_rays = 0, n_gauss = 0;
    int pair_buf = 0;  // which of pkeys/pvals holds the sorted result
    int depth_buf = 0; // which of dkeys/dvals holds the depth-sorted Gaussians
    int kind = -1;     // 0 camera, 1 lidar, 2 rolling-shutter camera
    const void *scene = nullptr;
    const void *sensor = nullptr;
    float c2w[12];     // camera pose of the last render
    const float *d_lidar_poses = nullptr;   // per-ray poses of the last render (LiDAR
                                            // columns, rolling-shutter rows)
    sg_render_opts opts;
    bool timing = false;
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    float ms[4] = {0, 0, 0, 0};
    cudaEvent_t ev_count = nullptr;  // exact mode: the pair count has reached h_scalars
    Buf host_stage[3];               // device results of a render with host outputs
    cudaStream_t copy_st = nullptr;  // their copies to the host run here, off the view's stream
    cudaEvent_t ev_rendered = nullptr, ev_copied = nullptr;
    bool copy_pending = false;       // ev_copied marks the last copies queued
};

// Grow b to at least `bytes` (with head-room); growing frees the old buffer.
// While capture_guard() is set on the calling thread (a launch sequence is
// being captured), a call that would allocate fails with SG_ERR_BUSY.
sg_status ensure(Buf &b, size_t bytes);
bool &capture_guard();
uint64_t next_uid();            // identity of a scene / sensor handle

constexpr size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// Index of the status word in a frame's device scalars: non-zero once a
// bounded device wait has given up in the current render (a look-back wait
// of the sort stages, or the projection's wait for bulk copies).  The
// projection kernel clears it at the start of every render.  Kernels after
// the give-up stay in bounds: the binning and the tile ranges write nothing,
// so every list is empty.  The host reads it with the pair count (exact
// mode), with the scalars at the end of a capacity-mode render, and in
// sg_frame_status / with host outputs.
constexpr int kScalStatus = 8;
// Bits of the status word: a look-back wait of a sort pass gave up; a
// wait for the projection's bulk copies of feature planes gave up.
constexpr uint32_t kStatusLookback = 1u;
constexpr uint32_t kStatusBulkCopy = 2u;
// Pinned-mirror slots (frame h_scalars) of the status word read after the
// render: by sg_frame_status, and with the host-output copies.
constexpr int kHostStatusQuery = 12, kHostStatusOutputs = 13;

// Upper bounds of the compositing work-item buffers.  A unit (a camera
// tile, or a LiDAR work item of up to 32 rays of one tile) whose list holds
// len entries gives 1 segment if len <= L and ceil(len / L) above; each
// segment gives `subs` work items (8 sub-blocks of a camera tile, 1 for
// LiDAR).  So with `units` units and `n_pairs` list entries in all, the
// work items are at most subs (units + n_pairs / L) and the partial slots
// (segments of split units) at most min(2 n_pairs / L, units + n_pairs / L).
// Buffers: per unit (segments, first partial slot) and its first work item
// in launch order, the work items, arrival counters (subs per slot), the
// deferred re-walks (one uint4 per slot and sub-unit at most) and the
// per-ray partials (32 subs rays per slot, two float4 each).
struct WorkSize {
    int64_t max_items = 0, max_slots = 0, max_fixes = 0;
    size_t info_bytes = 0, off_bytes = 0, items_bytes = 0, arrive_bytes = 0, fix_bytes = 0,
           work_bytes = 0, partial_bytes = 0;
};
constexpr WorkSize work_size(int64_t units, int64_t n_pairs, uint32_t seg_len, int subs)
{
    WorkSize w;
    const int64_t per = n_pairs / (int64_t)seg_len;
    const int64_t u1 = units > 0 ? units : 1;
    w.max_items = subs * (units + per);
    w.max_slots = 2 * per < units + per ? 2 * per : units + per;
    const int64_t items1 = w.max_items > 0 ? w.max_items : 1;
    const int64_t slots1 = w.max_slots > 0 ? w.max_slots : 1;
    w.info_bytes = al256(8 * (size_t)u1);
    w.off_bytes = al256(4 * (size_t)(u1 > 128 ? u1 : 128));   // >= the work-item scratch
    w.items_bytes = al256(8 * (size_t)items1);
    w.arrive_bytes = al256(4 * (size_t)subs * (size_t)slots1);
    // deferred re-walks: at most one per (split unit, sub-unit, segment >= 1)
    w.max_fixes = subs * slots1;
    w.fix_bytes = al256(16 * (size_t)w.max_fixes);
    w.work_bytes = w.info_bytes + w.off_bytes + w.items_bytes + w.arrive_bytes + w.fix_bytes;
    w.partial_bytes = 2 * 16 * 32 * (size_t)subs * (size_t)slots1;
    return w;
}

// ------------------------------------------------------------------ launchers
// sort.cu
// Scratch words (fr.hist) of a radix sort of up to n_max pairs in `passes`
// 8-bit passes: digit counts and offsets (256 per pass), per-pass tile
// tickets, and the look-back words (256 per tile of kRadixTile pairs and pass).
#ifndef SG_RADIX_TILE
#define SG_RADIX_TILE 8192
#endif
constexpr int kRadixTile = SG_RADIX_TILE;
constexpr int64_t radix_scratch_words(int64_t n_max, int passes)
{
    const int64_t tiles = (n_max + kRadixTile - 1) / kRadixTile;
    return 2 * 256 * (int64_t)passes + 16 + (int64_t)passes * (tiles > 0 ? tiles : 1) * 256;
}
// The depth stage's scratch (fr.hist): the radix scratch of its 4 passes,
// then two tickets and a 64-bit look-back word per tile of kChainTile
// entries for each of its two chained scans.
constexpr int kChainTile = 4096;
constexpr int64_t depth_stage_words(int64_t n)
{
    return radix_scratch_words(n, 4) + 2 * (2 + 2 * ((n + kChainTile - 1) / kChainTile));
}
sg_status radix_prepare(int64_t n_max, int passes, Frame &fr, cudaStream_t st, uint32_t **hist,
                        int64_t extra);
// Stable sort of up to n pairs (*d_n of them) by key bits [begin_bit,
// end_bit); the digit counts are in the scratch that radix_prepare returned.
// site: SG_LOOKBACK_DEPTH_SORT or SG_LOOKBACK_TILE_SORT (the test hook's site).
sg_status radix_sort_pairs(uint32_t *keys[2], uint32_t *vals[2], int64_t n,
                           const uint32_t *d_n, int begin_bit, int end_bit, Frame &fr,
                           cudaStream_t st, int *result_buf, int site);
// The depth stage: the Gaussians with a non-zero tile count sorted by depth
// (keys/vals[*result_buf]: depth bits, ids), d_scal[0] = their number,
// d_offsets = exclusive scan of their tile counts in that order, d_scal[1]
// = the pair total.
sg_status depth_stage(const uint32_t *d_count, const float *d_depth, int64_t n, uint32_t *keys[2],
                      uint32_t *vals[2], uint32_t *d_scal, uint32_t *d_offsets, Frame &fr,
                      cudaStream_t st, int *result_buf);
// With d_hist (zeroed by radix_prepare), k_bin also counts the digits of
// the tile sort over end_bit bits, for radix_sort_pairs.  d_err: the frame's
// status word (nothing is written once it is set).
sg_status bin_pairs(const uint32_t *d_ids, const uint32_t *d_offsets, const uint32_t *d_nvalid,
                    const int4 *d_tiles, int ntx, int wrap_x, int64_t cap, uint32_t *d_keys,
                    uint32_t *d_vals, cudaStream_t st, const uint32_t *d_err,
                    uint32_t *d_hist = nullptr, int end_bit = 0);
// Per-tile ranges of the sorted pairs; with d_mask (camera lists), also the
// per-pair sub-block masks (d_ids, d_rects, ntx: the pairs' Gaussians, the
// per-Gaussian extent boxes, tiles per row).
sg_status tile_ranges(const uint32_t *d_keys, const uint32_t *d_K, int64_t K_max, uint2 *d_ranges,
                      int64_t ntiles, cudaStream_t st, const uint32_t *d_err,
                      const uint32_t *d_ids = nullptr, const float4 *d_rects = nullptr,
                      int ntx = 0, uint32_t *d_words = nullptr);
// LiDAR lists: ranges, and for every pair and every work item of its tile
// the item's rays inside the Gaussian's extent box (lmask[k * K_max + i]
// for the k-th item of the tile, by the compositing's own float test).
sg_status lidar_tile_ranges(const uint32_t *d_keys, const uint32_t *d_K, int64_t K_max,
                            uint2 *d_ranges, int64_t ntiles, cudaStream_t st,
                            const uint32_t *d_err, const uint32_t *d_ids,
                            const float4 *d_rects, const Lidar &L, uint32_t *d_lmask);
sg_status clamp_pairs(uint32_t *d_K, int64_t cap, uint32_t *d_dropped, cudaStream_t st);

// project.cu
// The pose and the outputs of a render are read from fr.desc (RenderDesc).
// rolling: the RenderDesc's poses are per pixel row (rolling shutter)
sg_status project_camera(const Scene &sc, const Camera &cam, const sg_render_opts &o, Frame &fr,
                         cudaStream_t st, bool rolling = false);
sg_status project_lidar(const Scene &sc, const Lidar &L, const sg_render_opts &o, Frame &fr,
                        cudaStream_t st);

// render.cu
sg_status render_camera(const Camera &cam, const sg_render_opts &o, Frame &fr, cudaStream_t st);
// render_fwd.cu: the compositing of frames that keep no backward state
// (tangent-plane rays); render_camera dispatches to it when
// camera_forward_only holds.
bool camera_forward_only(const Camera &cam, const Frame &fr);
sg_status render_camera_fwd(const Camera &cam, const sg_render_opts &o, Frame &fr,
                            cudaStream_t st);
// render.cu: the compositing's work items (k_work_count, k_work_emit) of
// n_units units with `subs` sub-units each, in the camwork layout of ws.

sg_status launch_work_items(Frame &fr, const WorkSize &ws, const LidarItem *unit_tile,
                            int n_units, int subs, uint32_t seg_len, cudaStream_t st);
// rolling shutter: the RenderDesc's poses are per pixel row
sg_status render_camera_rs(const Camera &cam, const sg_render_opts &o, Frame &fr,
                           cudaStream_t st);
sg_status render_lidar(const Lidar &L, const sg_render_opts &o, Frame &fr, cudaStream_t st);
// render_lidar_fwd.cu: the LiDAR compositing of frames that keep no backward
// state (beam groups, one ray parameter); render_lidar dispatches to it when
// lidar_forward_only holds.
bool lidar_forward_only(const Frame &fr);
sg_status render_lidar_fwd(const Lidar &L, const sg_render_opts &o, Frame &fr,
                           cudaStream_t st);

// sensors.cu
sg_status build_camera(Camera &cam);
sg_status build_lidar(Lidar &L);

// backward.cu
sg_status backward_camera(const Scene &sc, const Camera &cam, Frame &fr,
                          const float *g_rgb, const float *g_alpha, const float *g_depth,
                          const sg_grads &g, cudaStream_t st);
sg_status backward_lidar(const Scene &sc, const Lidar &L, Frame &fr, const float *g_range,
                         const float *g_int, const float *g_drop, const float *g_alpha,
                         const sg_grads &g, cudaStream_t st);

}  // namespace sg

// the opaque handle types of the C-ABI
// Every device buffer of a frame (for release, and for recognising captured
// launch sequences whose buffers have since been reallocated).
namespace sg {
template <class Fn> inline void for_each_buf(Frame &f, Fn fn)
{
    Buf *bufs[] = {&f.rec, &f.rect, &f.tiles, &f.depth, &f.count, &f.mean2d, &f.cov2d,
                   &f.dkeys[0], &f.dkeys[1], &f.dvals[0], &f.dvals[1], &f.offsets, &f.hist,
                   &f.pkeys[0], &f.pkeys[1], &f.pvals[0], &f.pvals[1], &f.ranges, &f.order, &f.submask,
                   &f.lmask, &f.camwork,
                   &f.partials, &f.ray_state, &f.n_contrib, &f.ray_feat, &f.gacc, &f.scalars,
                   &f.desc, &f.host_stage[0], &f.host_stage[1], &f.host_stage[2]};
    for (Buf *b : bufs) fn(*b);
}
}  // namespace sg

struct sg_scene_s { sg::Scene s; uint64_t uid = sg::next_uid(); };
struct sg_camera_s { sg::Camera c; uint64_t uid = sg::next_uid(); };
struct sg_lidar_s { sg::Lidar l; uint64_t uid = sg::next_uid(); };
struct sg_frame_s { sg::Frame f; };

// ---------------------------------------------------------------- device math
#ifdef __CUDACC__
namespace sgd {

// a - b as an unevaluated sum hi + lo, exactly (Knuth's TwoSum of a and -b).
__device__ __forceinline__ void two_diff(float a, float b, float &hi, float &lo)
{
    float s = __fsub_rn(a, b);
    float bb = __fsub_rn(s, a);
    lo = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(-b, bb));
    hi = s;
}

// a*b - c*d with an error near one ulp of the result (Kahan's algorithm
// with fused multiply-adds).
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d)
{
    float w = __fmul_rn(c, d);
    float e = __fmaf_rn(-c, d, w);       // w - c*d exactly
    float f = __fmaf_rn(a, b, -w);
    return __fadd_rn(f, e);
}

}  // namespace sgd
#endif
