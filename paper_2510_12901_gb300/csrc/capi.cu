// capi.cu -- the extern "C" entry points of libsimgut (declared in
// include/simgut.h): handle management, argument checks and the order of
// the render stages.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>

#include <vector>

#include "internal.h"

namespace sg {

static thread_local char g_err[512] = "";
static std::atomic<int64_t> g_launches{0};

static thread_local bool g_capture_guard = false;
static std::atomic<uint64_t> g_uid{1};
static std::atomic<int64_t> g_allocs{0};

void note_alloc() { g_allocs.fetch_add(1, std::memory_order_relaxed); }

void count_launch()
{
    if (!g_capture_guard) g_launches.fetch_add(1, std::memory_order_relaxed);
}
void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
bool &capture_guard() { return g_capture_guard; }
uint64_t next_uid() { return g_uid.fetch_add(1, std::memory_order_relaxed); }

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

sg_status cuda_status(cudaError_t e, const char *what)
{
    set_error("%s: %s", what, cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? SG_ERR_OOM : SG_ERR_CUDA;
}

sg_status ensure(Buf &b, size_t bytes)
{
    if (bytes <= b.bytes && b.p) return SG_OK;
    if (b.borrowed) {   // a fixed workspace (the allocation-free render): never freed here
        set_error("a buffer of the static workspace (%zu bytes) is too small for %zu bytes",
                  b.bytes, bytes);
        return SG_ERR_OVERFLOW;
    }
    if (g_capture_guard) {
        set_error("workspace of %zu bytes would grow to %zu during launch capture", b.bytes, bytes);
        return SG_ERR_BUSY;
    }
    size_t nb = bytes < 256 ? 256 : bytes + bytes / 4;   // grow with head-room
    if (b.p) {
        dev_free(b.p);   // implicitly waits for work that may still use it
        b.p = nullptr;
        b.bytes = 0;
    }
    cudaError_t e = dev_malloc(&b.p, nb);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation of %zu bytes failed", nb);
        return SG_ERR_OOM;
    }
    b.bytes = nb;
    return SG_OK;
}

static void release(Buf &b)
{
    if (b.p && !b.borrowed) dev_free(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

// AoS [n, comps] -> planes
// Flags (bad = 1) an actor index outside -1..n_actors-1.
__global__ void k_check_actors(const int32_t *__restrict__ of, int64_t n, int n_actors,
                               uint32_t *__restrict__ bad)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && (of[i] < -1 || of[i] >= n_actors)) *bad = 1u;
}

__global__ void k_to_planes(const float *__restrict__ src, int64_t n, int comps, int plane0,
                            int64_t pitch, float *__restrict__ planes)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * comps) return;
    int64_t g = i / comps;
    int c = (int)(i % comps);
    planes[(int64_t)(plane0 + c) * pitch + g] = src[i];
}

static sg_status check_desc(const sg_gaussians_desc *d, int *F)
{
    if (!d) { set_error("desc is NULL"); return SG_ERR_INVALID; }
    if (d->n < 0 || d->n > (int64_t)1 << 31) {
        set_error("n = %lld out of range [0, 2^31]", (long long)d->n);
        return SG_ERR_INVALID;
    }
    if (sh_features(d->feature_kind)) {
        if (d->sh_degree < 0 || d->sh_degree > 3) {
            set_error("sh_degree %d not in 0..3", d->sh_degree);
            return SG_ERR_INVALID;
        }
        *F = 3 * (d->sh_degree + 1) * (d->sh_degree + 1);
    } else if (d->feature_kind == SG_FEATURES_RGB || d->feature_kind == SG_FEATURES_LIDAR) {
        *F = 3;
    } else {
        set_error("feature_kind %d unknown", d->feature_kind);
        return SG_ERR_INVALID;
    }
    if (d->n > 0 && (!d->d_means || !d->d_log_scales || !d->d_quats || !d->d_opacity ||
                     !d->d_features)) {
        set_error("a parameter array is NULL");
        return SG_ERR_INVALID;
    }
    return SG_OK;
}

static sg_status upload_planes(Scene &s, const sg_gaussians_desc *d, cudaStream_t st)
{
    struct { const float *p; int comps, plane0; } parts[5] = {
        {d->d_means, 3, Scene::kMean}, {d->d_log_scales, 3, Scene::kLogScale},
        {d->d_quats, 4, Scene::kQuat}, {d->d_opacity, 1, Scene::kOpacity},
        {d->d_features, s.F, Scene::kFeat}};
    for (auto &p : parts) {
        int64_t tot = s.n * p.comps;
        if (tot == 0) continue;
        k_to_planes<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(p.p, s.n, p.comps, p.plane0,
                                                                    s.pitch, s.d_planes);
        SG_LAUNCHED();
    }
    return SG_OK;
}

bool opts_ok(const sg_render_opts *o)
{
    if (!o) { set_error("opts is NULL"); return false; }
    if (!(o->alpha_min > 0.f && o->alpha_min < 1.f) || !(o->alpha_max > 0.f && o->alpha_max <= 1.f) ||
        !(o->t_min >= 0.f && o->t_min < 1.f) || !(o->near_dist > 0.f) ||
        !(o->ut_alpha > 0.f) || !(o->ut_kappa > -3.f) || !isfinite(o->ut_beta) ||
        o->pose_iters < 0 || o->pose_iters > 8 ||
        !(o->beam_divergence >= 0.f && o->beam_divergence <= 0.1f)) {
        set_error("render options out of range");
        return false;
    }
    return true;
}

// Per-Gaussian and per-ray buffers of a render.
static sg_status frame_prepare(Frame &fr, int64_t n, int64_t nrays, int64_t ntiles)
{
    sg_status s;
#define SG_ENS(buf, by) if ((s = ensure(buf, by)) != SG_OK) return s
    SG_ENS(fr.rec, sizeof(GRec) * (n > 0 ? n : 1));
    SG_ENS(fr.rect, sizeof(float4) * (n > 0 ? n : 1));
    SG_ENS(fr.tiles, sizeof(int4) * (n > 0 ? n : 1));
    SG_ENS(fr.depth, sizeof(float) * (n > 0 ? n : 1));
    SG_ENS(fr.count, sizeof(uint32_t) * (n > 0 ? n : 1));
    SG_ENS(fr.mean2d, sizeof(float2) * (n > 0 ? n : 1));
    SG_ENS(fr.cov2d, sizeof(float4) * (n > 0 ? n : 1));
    for (int i = 0; i < 2; ++i) {
        SG_ENS(fr.dkeys[i], sizeof(uint32_t) * (n > 0 ? n : 1));
        SG_ENS(fr.dvals[i], sizeof(uint32_t) * (n > 0 ? n : 1));
    }
    SG_ENS(fr.offsets, sizeof(uint32_t) * (n > 0 ? n : 1));
    SG_ENS(fr.ranges, sizeof(uint2) * (ntiles > 0 ? ntiles : 1));
    SG_ENS(fr.ray_state, sizeof(float4) * (nrays > 0 ? nrays : 1));
    SG_ENS(fr.ray_feat, sizeof(float4) * (nrays > 0 ? nrays : 1));
    SG_ENS(fr.n_contrib, sizeof(uint32_t) * (nrays > 0 ? nrays : 1));
    SG_ENS(fr.scalars, 64);
    SG_ENS(fr.desc, sizeof(RenderDesc));
#undef SG_ENS
    if (!fr.h_scalars) {
        static_assert(sizeof(RenderDesc) <= 256, "RenderDesc outgrew its pinned slot");
        if (host_malloc(&fr.h_scalars, 512) != cudaSuccess) {
            cudaGetLastError();
            set_error("pinned allocation failed");
            return SG_ERR_OOM;
        }
        fr.h_desc = (RenderDesc *)((char *)fr.h_scalars + 256);
    }
    if (!fr.ev_count && cudaEventCreateWithFlags(&fr.ev_count, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        set_error("event creation failed");
        return SG_ERR_CUDA;
    }
    fr.n_gauss = n;
    fr.n_rays = nrays;
    fr.n_tiles = ntiles;
    fr.state_kept = fr.keep_state;
    return SG_OK;
}

static void tmark(Frame &fr, int i, cudaStream_t st)
{
    if (fr.timing) cudaEventRecord(fr.ev[i], st);
}

// The render's RenderDesc (written to fr.h_desc by the caller) to the device.
static sg_status upload_desc(Frame &fr, cudaStream_t st)
{
    SG_CUDA(cudaMemcpyAsync(fr.desc.p, fr.h_desc, sizeof(RenderDesc), cudaMemcpyHostToDevice, st));
    return SG_OK;
}

// Stages shared by both sensors after projection, in two halves so that
// several renders on their own streams can each have their pair count on
// the way before any of them waits for one.
// sort_and_count: depth sort, offsets and the pair count.  In exact mode the
// count is copied to h_scalars and ev_count recorded; in capacity mode
// (fr.k_cap > 0) the count stays on the device, clamped to k_cap (the excess
// in scalars[3]).
static sg_status sort_and_count(Frame &fr, int64_t n, cudaStream_t st)
{
    uint32_t *sc = (uint32_t *)fr.scalars.p;   // [0] valid Gaussians, [1] pairs
    uint32_t *dk[2] = {(uint32_t *)fr.dkeys[0].p, (uint32_t *)fr.dkeys[1].p};
    uint32_t *dv[2] = {(uint32_t *)fr.dvals[0].p, (uint32_t *)fr.dvals[1].p};
    int rb = 0;
    sg_status s = depth_stage((const uint32_t *)fr.count.p, (const float *)fr.depth.p, n, dk, dv,
                              sc, (uint32_t *)fr.offsets.p, fr, st, &rb);
    if (s != SG_OK) return s;
    fr.depth_buf = rb;
    tmark(fr, 2, st);
    if (fr.k_cap > 0) return clamp_pairs(sc + 1, fr.k_cap, sc + 3, st);
    // the counts and the status word in one copy
    SG_CUDA(cudaMemcpyAsync(fr.h_scalars, sc, 4 * (kScalStatus + 1), cudaMemcpyDeviceToHost, st));
    SG_CUDA(cudaEventRecord(fr.ev_count, st));
    return SG_OK;
}

// The message of a non-zero device status word (kStatus* bits).
static const char *status_cause(uint32_t w)
{
    if ((w & kStatusLookback) && (w & kStatusBulkCopy))
        return "a look-back wait of the sort and a bulk-copy wait of the projection gave up";
    if (w & kStatusBulkCopy) return "a bulk-copy wait of the projection gave up";
    return "a look-back wait of the sort gave up";
}

// bin_and_sort: waits for the pair count (exact mode), which sizes the pair
// buffers, then binning, tile sort and ranges; in capacity mode nothing
// waits and the scalars are copied to h_scalars at the end for the caller
// to check.
static sg_status bin_and_sort(Frame &fr, int64_t n, int ntx, int64_t ntiles, int wrap,
                              cudaStream_t st)
{
    uint32_t *sc = (uint32_t *)fr.scalars.p;
    int64_t K = 0;
    if (fr.k_cap > 0) {
        K = fr.k_cap;
    } else {
        SG_CUDA(cudaEventSynchronize(fr.ev_count));
        if (fr.h_scalars[kScalStatus]) {
            set_error("%s before the pair count (device status word set)",
                      status_cause(fr.h_scalars[kScalStatus]));
            return SG_ERR_TIMEOUT;
        }
        K = fr.h_scalars[1];
        if (K > 0x7fffffffLL) {
            set_error("%lld (tile, Gaussian) pairs exceed 2^31-1", (long long)K);
            return SG_ERR_OVERFLOW;
        }
    }
    fr.n_pairs = K;
    sg_status s;
    for (int i = 0; i < 2; ++i) {
        if ((s = ensure(fr.pkeys[i], sizeof(uint32_t) * (K > 0 ? K : 1))) != SG_OK) return s;
        if ((s = ensure(fr.pvals[i], sizeof(uint32_t) * (K > 0 ? K : 1))) != SG_OK) return s;
    }
    uint32_t *pk[2] = {(uint32_t *)fr.pkeys[0].p, (uint32_t *)fr.pkeys[1].p};
    uint32_t *pv[2] = {(uint32_t *)fr.pvals[0].p, (uint32_t *)fr.pvals[1].p};
    int bits = 1;
    while (((int64_t)1 << bits) < ntiles) ++bits;
    // binning counts the tile sort's digits as it writes the pairs
    uint32_t *hist = nullptr;
    if (K > 0 && (s = radix_prepare(K, (bits + 7) / 8, fr, st, &hist, 0)) != SG_OK) return s;
    const uint32_t *err = sc + kScalStatus;
    s = bin_pairs((const uint32_t *)fr.dvals[fr.depth_buf].p, (const uint32_t *)fr.offsets.p, sc,
                  (const int4 *)fr.tiles.p, ntx, wrap, K, pk[0], pv[0], st, err, hist, bits);
    if (s != SG_OK) return s;
    int pb = 0;
    s = radix_sort_pairs(pk, pv, K, sc + 1, 0, bits, fr, st, &pb, SG_LOOKBACK_TILE_SORT);
    if (s != SG_OK) return s;
    fr.pair_buf = pb;
    if (fr.kind == 1) {   // LiDAR lists also get their per-item ray masks
        const Lidar &L = static_cast<const sg_lidar_s *>(fr.sensor)->l;
        const size_t by = sizeof(uint32_t) * (size_t)(K > 0 ? K : 1) * L.max_items_per_tile;
        if ((s = ensure(fr.lmask, by)) != SG_OK) return s;
        fr.lmask_stride = K;
        s = lidar_tile_ranges(pk[pb], sc + 1, K, (uint2 *)fr.ranges.p, ntiles, st, err, pv[pb],
                              (const float4 *)fr.rect.p, L, (uint32_t *)fr.lmask.p);
    } else {   // camera lists also get their column/row words
        if ((s = ensure(fr.submask, 4 * (size_t)(K > 0 ? K : 1))) != SG_OK) return s;
        s = tile_ranges(pk[pb], sc + 1, K, (uint2 *)fr.ranges.p, ntiles, st, err, pv[pb],
                        (const float4 *)fr.rect.p, ntx, (uint32_t *)fr.submask.p);
    }
    if (s != SG_OK) return s;
    if (fr.k_cap > 0)   // counts, dropped pairs and the status word, for the caller
        SG_CUDA(cudaMemcpyAsync(fr.h_scalars, sc, 4 * (kScalStatus + 1), cudaMemcpyDeviceToHost,
                                st));
    tmark(fr, 3, st);
    return SG_OK;
}

static sg_status sort_and_bin(Frame &fr, int64_t n, int ntx, int64_t ntiles, int wrap,
                              cudaStream_t st)
{
    sg_status s = sort_and_count(fr, n, st);
    return s != SG_OK ? s : bin_and_sort(fr, n, ntx, ntiles, wrap, st);
}

// A camera render in two halves (see sort_and_count): camera_begin checks
// the arguments, projects and starts the pair count; camera_finish bins,
// sorts and composites.
static sg_status camera_begin(sg_scene scene, sg_camera cam, const float h_c2w[12],
                              const sg_render_opts *opts, sg_frame frame, float *d_rgb,
                              float *d_alpha, float *d_depth, cudaStream_t st,
                              const float *d_row_c2w = nullptr)
{
    if (!scene || !cam || !frame || !h_c2w) { set_error("NULL handle or pose"); return SG_ERR_INVALID; }
    if (!opts_ok(opts)) return SG_ERR_INVALID;
    const Scene &sc = scene->s;
    if (lidar_features(sc.feature_kind)) {
        set_error("sg_render_camera: scene carries LiDAR features");
        return SG_ERR_INVALID;
    }
    for (int i = 0; i < 12; ++i)
        if (!isfinite(h_c2w[i])) { set_error("pose is not finite"); return SG_ERR_INVALID; }
    const Camera &c = cam->c;
    Frame &fr = frame->f;
    int64_t nt = (int64_t)c.ntx * c.nty, nr = (int64_t)c.width * c.height;
    sg_status s = frame_prepare(fr, sc.n, nr, nt);
    if (s != SG_OK) return s;
    fr.kind = d_row_c2w ? 2 : 0;
    fr.scene = scene;
    fr.sensor = cam;
    fr.opts = *opts;
    fr.d_lidar_poses = d_row_c2w;
    memcpy(fr.c2w, h_c2w, sizeof(fr.c2w));
    RenderDesc &D = *fr.h_desc;
    memcpy(D.c2w, h_c2w, sizeof(D.c2w));
    D.poses = d_row_c2w;
    D.out[0] = d_rgb;
    D.out[1] = d_alpha;
    D.out[2] = d_depth;
    D.out[3] = nullptr;
    if (fr.timing) cudaEventRecord(fr.ev[0], st);
    if ((s = upload_desc(fr, st)) != SG_OK) return s;
    if ((s = project_camera(sc, c, *opts, fr, st, d_row_c2w != nullptr)) != SG_OK) return s;
    if (fr.timing) cudaEventRecord(fr.ev[1], st);
    return sort_and_count(fr, sc.n, st);
}

static sg_status camera_finish(sg_camera cam, sg_frame frame, cudaStream_t st)
{
    const Camera &c = cam->c;
    Frame &fr = frame->f;
    sg_status s = bin_and_sort(fr, fr.n_gauss, c.ntx, (int64_t)c.ntx * c.nty, 0, st);
    if (s != SG_OK) return s;
    s = fr.kind == 2 ? render_camera_rs(c, fr.opts, fr, st) : render_camera(c, fr.opts, fr, st);
    if (s != SG_OK) return s;
    if (fr.timing) cudaEventRecord(fr.ev[4], st);
    return SG_OK;
}

}  // namespace sg

using namespace sg;


extern "C" {

int sg_version(void) { return 100; }
int64_t sg_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }
int64_t sg_alloc_count(void) { return g_allocs.load(std::memory_order_relaxed); }
int sg_cuda_arch(void) { return 103; }
const char *sg_last_error(void) { return g_err; }

sg_render_opts sg_default_opts(void)
{
    sg_render_opts o;
    o.alpha_min = 1.0f / 255.0f;
    o.alpha_max = 0.99f;
    o.t_min = 1e-4f;
    o.near_dist = 0.2f;
    o.ut_alpha = 1.0f;
    o.ut_beta = 2.0f;
    o.ut_kappa = 0.0f;
    o.pose_iters = 2;
    o.cull = 1;
    o.beam_divergence = 0.0f;   // the paper does not state delta: off by default
    return o;
}

sg_status sg_create_scene(const sg_gaussians_desc *desc, void *stream, sg_scene *out)
{
    if (!out) { set_error("out is NULL"); return SG_ERR_INVALID; }
    *out = nullptr;
    int F = 0;
    sg_status s = check_desc(desc, &F);
    if (s != SG_OK) return s;
    sg_scene h = new (std::nothrow) sg_scene_s;
    if (!h) { set_error("host allocation failed"); return SG_ERR_OOM; }
    Scene &sc = h->s;
    sc.n = desc->n;
    sc.feature_kind = desc->feature_kind;
    sc.sh_degree = sh_features(desc->feature_kind) ? desc->sh_degree : 0;
    sc.F = F;
    sc.pitch = ((desc->n + 31) / 32) * 32;
    if (sc.pitch == 0) sc.pitch = 32;
    size_t bytes = sizeof(float) * (size_t)sc.pitch * (Scene::kFeat + F);
    if (dev_malloc(&sc.d_planes, bytes) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        set_error("scene allocation of %zu bytes failed", bytes);
        return SG_ERR_OOM;
    }
    s = upload_planes(sc, desc, (cudaStream_t)stream);
    if (s != SG_OK) {
        dev_free(sc.d_planes);
        delete h;
        return s;
    }
    *out = h;
    return SG_OK;
}

sg_status sg_update_scene(sg_scene scene, const sg_gaussians_desc *desc, void *stream)
{
    if (!scene) { set_error("scene is NULL"); return SG_ERR_INVALID; }
    int F = 0;
    sg_status s = check_desc(desc, &F);
    if (s != SG_OK) return s;
    if (desc->n != scene->s.n || F != scene->s.F || desc->feature_kind != scene->s.feature_kind) {
        set_error("sg_update_scene: size or feature layout differs from the scene");
        return SG_ERR_INVALID;
    }
    return upload_planes(scene->s, desc, (cudaStream_t)stream);
}

void sg_destroy_scene(sg_scene scene)
{
    if (!scene) return;
    cudaDeviceSynchronize();   // renders still queued may read the scene
    dev_free(scene->s.d_planes);
    dev_free(scene->s.d_actor_of);
    dev_free(scene->s.d_actor_poses);
    delete scene;
}

sg_status sg_scene_set_actors(sg_scene scene, const int32_t *d_actor_of, int n_actors,
                              void *stream)
{
    if (!scene) { set_error("scene is NULL"); return SG_ERR_INVALID; }
    if (capture_guard()) { set_error("sg_scene_set_actors during a graph capture"); return SG_ERR_BUSY; }
    Scene &sc = scene->s;
    if (n_actors < 0 || (n_actors > 0 && sc.n > 0 && !d_actor_of)) {
        set_error("n_actors = %d with %s actor list", n_actors, d_actor_of ? "an" : "no");
        return SG_ERR_INVALID;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // the scene's old buffers may still be read by renders queued on `stream`
    SG_CUDA(cudaStreamSynchronize(st));
    dev_free(sc.d_actor_of);
    dev_free(sc.d_actor_poses);
    sc.d_actor_of = nullptr;
    sc.d_actor_poses = nullptr;
    sc.n_actors = 0;
    scene->uid = next_uid();   // captured launch sequences of this scene are stale
    if (n_actors == 0) return SG_OK;
    int32_t *of = nullptr;
    float *poses = nullptr;
    uint32_t *bad = nullptr;
    if (dev_malloc(&of, sizeof(int32_t) * (size_t)(sc.n > 0 ? sc.n : 1)) != cudaSuccess ||
        dev_malloc(&poses, sizeof(float) * 12 * (size_t)n_actors) != cudaSuccess ||
        dev_malloc(&bad, sizeof(uint32_t)) != cudaSuccess) {
        cudaGetLastError();
        dev_free(of);
        dev_free(poses);
        dev_free(bad);
        set_error("device allocation failed");
        return SG_ERR_OOM;
    }
    std::vector<float> eye((size_t)n_actors * 12, 0.f);
    for (int a = 0; a < n_actors; ++a) eye[12 * a] = eye[12 * a + 5] = eye[12 * a + 10] = 1.f;
    uint32_t h_bad = 0;
    cudaError_t e = cudaMemcpyAsync(poses, eye.data(), sizeof(float) * eye.size(),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && sc.n > 0)
        e = cudaMemcpyAsync(of, d_actor_of, sizeof(int32_t) * (size_t)sc.n,
                            cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess && sc.n > 0) {
        k_check_actors<<<(unsigned)((sc.n + 255) / 256), 256, 0, st>>>(of, sc.n, n_actors, bad);
        e = cudaGetLastError();
        if (e == cudaSuccess) count_launch();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(bad);
    if (e != cudaSuccess || h_bad) {
        dev_free(of);
        dev_free(poses);
        if (e != cudaSuccess) return cuda_status(e, "sg_scene_set_actors");
        set_error("an actor index is outside -1..%d", n_actors - 1);
        return SG_ERR_INVALID;
    }
    sc.d_actor_of = of;
    sc.d_actor_poses = poses;
    sc.n_actors = n_actors;
    return SG_OK;
}

sg_status sg_scene_set_actor_poses(sg_scene scene, const float *h_poses, void *stream)
{
    if (!scene || !h_poses) { set_error("NULL scene or poses"); return SG_ERR_INVALID; }
    Scene &sc = scene->s;
    if (sc.n_actors == 0) { set_error("the scene has no actors"); return SG_ERR_INVALID; }
    for (int i = 0; i < 12 * sc.n_actors; ++i)
        if (!isfinite(h_poses[i])) { set_error("actor pose %d is not finite", i / 12); return SG_ERR_INVALID; }
    SG_CUDA(cudaMemcpyAsync(sc.d_actor_poses, h_poses, sizeof(float) * 12 * (size_t)sc.n_actors,
                            cudaMemcpyHostToDevice, (cudaStream_t)stream));
    return SG_OK;
}

int64_t sg_scene_size(sg_scene scene) { return scene ? scene->s.n : -1; }

sg_status sg_create_camera(int model, int width, int height, float fx, float fy, float cx,
                           float cy, const float k[4], sg_camera *out)
{
    if (!out) { set_error("out is NULL"); return SG_ERR_INVALID; }
    *out = nullptr;
    if ((model != SG_CAMERA_PINHOLE && model != SG_CAMERA_FISHEYE) || width <= 0 ||
        height <= 0 || width > 16384 || height > 16384 || !(fx > 0.f) || !(fy > 0.f) ||
        !isfinite(cx) || !isfinite(cy)) {
        set_error("sg_create_camera: bad model, size or intrinsics");
        return SG_ERR_INVALID;
    }
    sg_camera h = new (std::nothrow) sg_camera_s;
    if (!h) { set_error("host allocation failed"); return SG_ERR_OOM; }
    Camera &c = h->c;
    c.model = model;
    c.width = width;
    c.height = height;
    c.fx = fx; c.fy = fy; c.cx = cx; c.cy = cy;
    for (int i = 0; i < 4; ++i) c.k[i] = (model == SG_CAMERA_FISHEYE && k) ? k[i] : 0.f;
    sg_status s = build_camera(c);
    if (s != SG_OK) {
        dev_free(c.d_pix);
        dev_free(c.d_tile_dir);
        dev_free(c.d_pix2);
        dev_free(c.d_tile_basis);
        delete h;
        return s;
    }
    *out = h;
    return SG_OK;
}

void sg_destroy_camera(sg_camera cam)
{
    if (!cam) return;
    cudaDeviceSynchronize();   // renders still queued may read its ray tables
    dev_free(cam->c.d_pix);
    dev_free(cam->c.d_tile_dir);
    dev_free(cam->c.d_pix2);
    dev_free(cam->c.d_tile_basis);
    delete cam;
}

sg_status sg_create_lidar(const float *h_elev_deg, int n_beams, int n_cols, float az0_deg,
                          int max_rays_per_tile, int n_elev_tiles, int cull_az,
                          int cull_el_per_tile, sg_lidar *out)
{
    if (!out) { set_error("out is NULL"); return SG_ERR_INVALID; }
    *out = nullptr;
    if (!h_elev_deg || n_beams <= 0 || n_beams > 65535 || n_cols <= 0 || n_cols > 65535 ||
        n_elev_tiles < 1 || n_elev_tiles > 1024 || max_rays_per_tile <= 0 || cull_az <= 0 ||
        cull_el_per_tile <= 0 || !isfinite(az0_deg)) {
        set_error("sg_create_lidar: bad arguments");
        return SG_ERR_INVALID;
    }
    for (int b = 0; b < n_beams; ++b)
        if (!(h_elev_deg[b] > -90.f && h_elev_deg[b] < 90.f)) {
            set_error("sg_create_lidar: elevation %d out of (-90, 90)", b);
            return SG_ERR_INVALID;
        }
    sg_lidar h = new (std::nothrow) sg_lidar_s;
    if (!h) { set_error("host allocation failed"); return SG_ERR_OOM; }
    Lidar &L = h->l;
    L.n_beams = n_beams;
    L.n_cols = n_cols;
    L.az0 = az0_deg;
    L.nphi = n_elev_tiles;
    L.M = max_rays_per_tile;
    L.cull_az = cull_az;
    L.cull_el = cull_el_per_tile;
    L.elev.assign(h_elev_deg, h_elev_deg + n_beams);
    sg_status s = build_lidar(L);
    if (s != SG_OK) {
        sg_destroy_lidar(h);
        return s;
    }
    *out = h;
    return SG_OK;
}

void sg_destroy_lidar(sg_lidar lidar)
{
    if (!lidar) return;
    cudaDeviceSynchronize();   // renders still queued may read its tables
    Lidar &L = lidar->l;
    dev_free(L.d_T);
    dev_free(L.d_elev);
    dev_free(L.d_az);
    dev_free(L.d_sat);
    dev_free(L.d_items);
    dev_free(L.d_item_rays);
    dev_free(L.d_ray_e);
    dev_free(L.d_item_ref);
    dev_free(L.d_ray_tau);
    dev_free(L.d_tile_u);
    dev_free(L.d_tile_items);
    dev_free(L.d_item_ray_tab);
    delete lidar;
}

sg_status sg_lidar_tiling(sg_lidar lidar, float *h_T, int *n_theta)
{
    if (!lidar) { set_error("lidar is NULL"); return SG_ERR_INVALID; }
    if (h_T) memcpy(h_T, lidar->l.T.data(), sizeof(float) * lidar->l.T.size());
    if (n_theta) *n_theta = lidar->l.n_theta;
    return SG_OK;
}

sg_status sg_frame_create(sg_frame *out)
{
    if (!out) { set_error("out is NULL"); return SG_ERR_INVALID; }
    sg_frame h = new (std::nothrow) sg_frame_s;
    if (!h) { set_error("host allocation failed"); return SG_ERR_OOM; }
    *out = h;
    return SG_OK;
}

void sg_frame_destroy(sg_frame frame)
{
    if (!frame) return;
    cudaDeviceSynchronize();   // work queued on the frame must finish first
    Frame &f = frame->f;
    for_each_buf(f, [](Buf &b) { release(b); });
    if (f.h_scalars) host_free(f.h_scalars);
    for (auto &e : f.ev)
        if (e) cudaEventDestroy(e);
    if (f.ev_count) cudaEventDestroy(f.ev_count);
    if (f.ev_rendered) cudaEventDestroy(f.ev_rendered);
    if (f.ev_copied) cudaEventDestroy(f.ev_copied);
    if (f.copy_st) cudaStreamDestroy(f.copy_st);
    delete frame;
}

sg_status sg_frame_set_backward_state(sg_frame frame, int keep)
{
    if (!frame) { set_error("frame is NULL"); return SG_ERR_INVALID; }
    frame->f.keep_state = keep != 0;
    return SG_OK;
}

sg_status sg_frame_set_timing(sg_frame frame, int on)
{
    if (!frame) { set_error("frame is NULL"); return SG_ERR_INVALID; }
    Frame &f = frame->f;
    if (on && !f.ev[0])
        for (auto &e : f.ev) SG_CUDA(cudaEventCreate(&e));
    f.timing = on != 0;
    return SG_OK;
}

sg_status sg_frame_timing(sg_frame frame, float ms[4])
{
    if (!frame || !ms) { set_error("NULL argument"); return SG_ERR_INVALID; }
    Frame &f = frame->f;
    if (!f.timing) { set_error("timing is off for this frame"); return SG_ERR_INVALID; }
    SG_CUDA(cudaEventSynchronize(f.ev[4]));
    for (int i = 0; i < 4; ++i) SG_CUDA(cudaEventElapsedTime(&ms[i], f.ev[i], f.ev[i + 1]));
    return SG_OK;
}

sg_status sg_frame_marks(sg_frame frame, sg_frame ref, float ms[5])
{
    if (!frame || !ref || !ms) { set_error("NULL argument"); return SG_ERR_INVALID; }
    Frame &f = frame->f, &r = ref->f;
    if (!f.timing || !r.timing) { set_error("timing is off for a frame"); return SG_ERR_INVALID; }
    SG_CUDA(cudaEventSynchronize(f.ev[4]));
    SG_CUDA(cudaEventSynchronize(r.ev[0]));
    for (int i = 0; i < 5; ++i) SG_CUDA(cudaEventElapsedTime(&ms[i], r.ev[0], f.ev[i]));
    return SG_OK;
}

}  // extern "C"

// Pairs of the last render: the exact count, or in capacity mode the pairs
// kept (read back at the end of the render, valid once it has completed).
static int64_t pairs_kept(const Frame &f)
{
    return f.k_cap > 0 && f.h_scalars ? (int64_t)f.h_scalars[1] : f.n_pairs;
}

extern "C" {

sg_status sg_frame_set_capacity(sg_frame frame, int64_t max_pairs)
{
    if (!frame || max_pairs < 0 || max_pairs > 0x7fffffffLL) {
        set_error("sg_frame_set_capacity: NULL frame or capacity out of range");
        return SG_ERR_INVALID;
    }
    frame->f.k_cap = max_pairs;
    return SG_OK;
}

sg_status sg_frame_dropped_pairs(sg_frame frame, int64_t *dropped, int64_t *pairs)
{
    if (!frame || !dropped) { set_error("NULL argument"); return SG_ERR_INVALID; }
    const Frame &f = frame->f;
    if (f.k_cap <= 0 || !f.h_scalars) {
        set_error("sg_frame_dropped_pairs: the frame is not in capacity mode");
        return SG_ERR_INVALID;
    }
    *dropped = f.h_scalars[3];
    if (pairs) *pairs = f.h_scalars[1];
    return SG_OK;
}

// timing marks: ev0 | project | ev1 | depth sort + offsets | ev2 | bin + tile
// sort + ranges | ev3 | render | ev4

sg_status sg_render_camera(sg_scene scene, sg_camera cam, const float h_c2w[12],
                           const sg_render_opts *opts, sg_frame frame, float *d_rgb,
                           float *d_alpha, float *d_depth, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    sg_status s = camera_begin(scene, cam, h_c2w, opts, frame, d_rgb, d_alpha, d_depth, st);
    return s != SG_OK ? s : camera_finish(cam, frame, st);
}

sg_status sg_render_camera_rs(sg_scene scene, sg_camera cam, const float *d_row_c2w,
                              const sg_render_opts *opts, sg_frame frame, float *d_rgb,
                              float *d_alpha, float *d_depth, void *stream)
{
    if (!d_row_c2w || !cam) { set_error("NULL camera or row poses"); return SG_ERR_INVALID; }
    if (!frame) { set_error("frame is NULL"); return SG_ERR_INVALID; }
    if (frame->f.seg_len != kSegLen) {
        set_error("sg_render_camera_rs: the frame belongs to the allocation-free render");
        return SG_ERR_INVALID;
    }
    // the global pose of the frame (the middle row's) is read from the device
    // only by the projection of a global-shutter render: any finite pose does
    const float eye[12] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0};
    cudaStream_t st = (cudaStream_t)stream;
    sg_status s = camera_begin(scene, cam, eye, opts, frame, d_rgb, d_alpha, d_depth, st,
                               d_row_c2w);
    return s != SG_OK ? s : camera_finish(cam, frame, st);
}

sg_status sg_render_cameras(sg_scene scene, int n_views, const sg_camera_view *views,
                            const sg_render_opts *opts, int host_outputs)
{
    if (n_views < 0 || (n_views > 0 && !views)) {
        set_error("sg_render_cameras: bad view list");
        return SG_ERR_INVALID;
    }
    if (host_outputs < 0 || host_outputs > 2) {
        set_error("sg_render_cameras: host_outputs %d is not 0, 1 or 2", host_outputs);
        return SG_ERR_INVALID;
    }
    for (int i = 0; i < n_views; ++i) {
        if (!views[i].camera || !views[i].frame) {
            set_error("view %d: NULL camera or frame", i);
            return SG_ERR_INVALID;
        }
        for (int j = 0; j < i; ++j)
            if (views[j].frame == views[i].frame) {
                set_error("views %d and %d share a frame", j, i);
                return SG_ERR_INVALID;
            }
    }
    sg_status s;
    for (int i = 0; i < n_views; ++i) {
        const sg_camera_view &v = views[i];
        float *out[3] = {v.rgb, v.alpha, v.depth};
        if (host_outputs) {
            Frame &f = v.frame->f;
            const int64_t np = (int64_t)v.camera->c.width * v.camera->c.height;
            for (int k = 0; k < 3; ++k) {
                if (!out[k]) continue;
                const size_t by = sizeof(float) * (size_t)np * (k == 0 ? 3 : 1);
                // growing frees the staging buffer, which the copies of the
                // frame's previous render may still be reading
                if (by > f.host_stage[k].bytes && f.copy_pending)
                    SG_CUDA(cudaEventSynchronize(f.ev_copied));
                if ((s = ensure(f.host_stage[k], by)) != SG_OK) return s;
                out[k] = (float *)f.host_stage[k].p;
            }
        }
        if (host_outputs && v.frame->f.copy_pending)   // the staging is free once copied
            SG_CUDA(cudaStreamWaitEvent((cudaStream_t)v.stream, v.frame->f.ev_copied, 0));
        if (v.row_c2w && v.frame->f.seg_len != kSegLen) {
            set_error("view %d: a rolling-shutter view cannot use an allocation-free frame", i);
            return SG_ERR_INVALID;
        }
        s = camera_begin(scene, v.camera, v.c2w, opts, v.frame, out[0], out[1], out[2],
                         (cudaStream_t)v.stream, v.row_c2w);
        if (s != SG_OK) return s;
    }
    for (int i = 0; i < n_views; ++i) {
        const sg_camera_view &v = views[i];
        cudaStream_t st = (cudaStream_t)v.stream;
        if ((s = camera_finish(v.camera, v.frame, st)) != SG_OK) return s;
        if (!host_outputs) continue;
        // the copies run on the frame's own stream, so that the view's next
        // work does not queue behind them
        Frame &f = v.frame->f;
        if (!f.copy_st) {
            SG_CUDA(cudaStreamCreateWithFlags(&f.copy_st, cudaStreamNonBlocking));
            SG_CUDA(cudaEventCreateWithFlags(&f.ev_rendered, cudaEventDisableTiming));
            SG_CUDA(cudaEventCreateWithFlags(&f.ev_copied, cudaEventDisableTiming));
        }
        SG_CUDA(cudaEventRecord(f.ev_rendered, st));
        SG_CUDA(cudaStreamWaitEvent(f.copy_st, f.ev_rendered, 0));
        const int64_t np = (int64_t)v.camera->c.width * v.camera->c.height;
        float *h[3] = {v.rgb, v.alpha, v.depth};
        for (int k = 0; k < 3; ++k)
            if (h[k])
                SG_CUDA(cudaMemcpyAsync(h[k], f.host_stage[k].p,
                                        sizeof(float) * (size_t)np * (k == 0 ? 3 : 1),
                                        cudaMemcpyDeviceToHost, f.copy_st));
        // the render's status word travels with its outputs
        SG_CUDA(cudaMemcpyAsync(f.h_scalars + kHostStatusOutputs,
                                (const uint32_t *)f.scalars.p + kScalStatus, 4,
                                cudaMemcpyDeviceToHost, f.copy_st));
        SG_CUDA(cudaEventRecord(f.ev_copied, f.copy_st));
        f.copy_pending = true;
    }
    if (host_outputs == 1)
        for (int i = 0; i < n_views; ++i)
            if ((s = sg_frame_sync_outputs(views[i].frame)) != SG_OK) return s;
    return SG_OK;
}

sg_status sg_frame_sync_outputs(sg_frame frame)
{
    if (!frame) { set_error("frame is NULL"); return SG_ERR_INVALID; }
    Frame &f = frame->f;
    if (!f.copy_pending) return SG_OK;
    SG_CUDA(cudaEventSynchronize(f.ev_copied));
    if (f.h_scalars[kHostStatusOutputs]) {
        set_error("%s in the frame's last render", status_cause(f.h_scalars[kHostStatusOutputs]));
        return SG_ERR_TIMEOUT;
    }
    return SG_OK;
}

sg_status sg_frame_status(sg_frame frame, void *stream)
{
    if (!frame) { set_error("frame is NULL"); return SG_ERR_INVALID; }
    Frame &f = frame->f;
    if (f.kind < 0 || !f.h_scalars) { set_error("frame has not been rendered"); return SG_ERR_INVALID; }
    cudaStream_t st = (cudaStream_t)stream;
    SG_CUDA(cudaMemcpyAsync(f.h_scalars + kHostStatusQuery,
                            (const uint32_t *)f.scalars.p + kScalStatus, 4,
                            cudaMemcpyDeviceToHost, st));
    SG_CUDA(cudaStreamSynchronize(st));
    if (f.h_scalars[kHostStatusQuery]) {
        set_error("%s in the frame's last render", status_cause(f.h_scalars[kHostStatusQuery]));
        return SG_ERR_TIMEOUT;
    }
    return SG_OK;
}

sg_status sg_render_lidar(sg_scene scene, sg_lidar lidar, const float *d_col_c2w,
                          const sg_render_opts *opts, sg_frame frame, float *d_range,
                          float *d_intensity, float *d_drop, float *d_alpha, void *stream)
{
    if (!scene || !lidar || !frame || !d_col_c2w) { set_error("NULL handle or poses"); return SG_ERR_INVALID; }
    if ((uintptr_t)d_col_c2w % 16 != 0) {
        set_error("sg_render_lidar: d_col_c2w must be 16-byte aligned");
        return SG_ERR_INVALID;
    }
    if (!opts_ok(opts)) return SG_ERR_INVALID;
    const Scene &sc = scene->s;
    if (!lidar_features(sc.feature_kind)) {
        set_error("sg_render_lidar: scene does not carry LiDAR features");
        return SG_ERR_INVALID;
    }
    const Lidar &L = lidar->l;
    Frame &fr = frame->f;
    cudaStream_t st = (cudaStream_t)stream;
    int64_t nt = (int64_t)L.n_theta * L.nphi, nr = (int64_t)L.n_beams * L.n_cols;
    sg_status s = frame_prepare(fr, sc.n, nr, nt);
    if (s != SG_OK) return s;
    fr.kind = 1;
    fr.scene = scene;
    fr.sensor = lidar;
    fr.opts = *opts;
    fr.d_lidar_poses = d_col_c2w;
    RenderDesc &D = *fr.h_desc;
    memset(D.c2w, 0, sizeof(D.c2w));
    D.poses = d_col_c2w;
    D.out[0] = d_range;
    D.out[1] = d_intensity;
    D.out[2] = d_drop;
    D.out[3] = d_alpha;
    if (fr.timing) cudaEventRecord(fr.ev[0], st);
    if ((s = upload_desc(fr, st)) != SG_OK) return s;
    if ((s = project_lidar(sc, L, *opts, fr, st)) != SG_OK) return s;
    if (fr.timing) cudaEventRecord(fr.ev[1], st);
    if ((s = sort_and_bin(fr, sc.n, L.n_theta, nt, 1, st)) != SG_OK) return s;
    if ((s = render_lidar(L, *opts, fr, st)) != SG_OK) return s;
    if (fr.timing) cudaEventRecord(fr.ev[4], st);
    return SG_OK;
}

// Host-output variants: render into library-owned device buffers, then copy
// (cameras: the frame's own staging buffers, through sg_render_cameras;
// LiDAR: per-thread buffers).
static thread_local Buf g_host_out[4];
static thread_local Buf g_host_poses;

sg_status sg_render_camera_host(sg_scene scene, sg_camera cam, const float h_c2w[12],
                                const sg_render_opts *opts, sg_frame frame, float *h_rgb,
                                float *h_alpha, float *h_depth, void *stream)
{
    if (!h_c2w) { set_error("pose is NULL"); return SG_ERR_INVALID; }
    sg_camera_view v{};   // zero: no row poses (global shutter)
    v.camera = cam;
    memcpy(v.c2w, h_c2w, sizeof(v.c2w));
    v.frame = frame;
    v.rgb = h_rgb;
    v.alpha = h_alpha;
    v.depth = h_depth;
    v.stream = stream;
    return sg_render_cameras(scene, 1, &v, opts, 1);
}

sg_status sg_render_lidar_host(sg_scene scene, sg_lidar lidar, const float *h_col_c2w,
                               const sg_render_opts *opts, sg_frame frame, float *h_range,
                               float *h_intensity, float *h_drop, float *h_alpha, void *stream)
{
    if (!lidar || !h_col_c2w) { set_error("NULL lidar or poses"); return SG_ERR_INVALID; }
    const Lidar &L = lidar->l;
    int64_t nr = (int64_t)L.n_beams * L.n_cols;
    sg_status s;
    cudaStream_t st = (cudaStream_t)stream;
    if ((s = ensure(g_host_poses, sizeof(float) * 12 * L.n_cols)) != SG_OK) return s;
    SG_CUDA(cudaMemcpyAsync(g_host_poses.p, h_col_c2w, sizeof(float) * 12 * L.n_cols,
                            cudaMemcpyHostToDevice, st));
    float *h[4] = {h_range, h_intensity, h_drop, h_alpha};
    float *d[4];
    for (int i = 0; i < 4; ++i) {
        if ((s = ensure(g_host_out[i], sizeof(float) * nr)) != SG_OK) return s;
        d[i] = h[i] ? (float *)g_host_out[i].p : nullptr;
    }
    s = sg_render_lidar(scene, lidar, (const float *)g_host_poses.p, opts, frame, d[0], d[1],
                        d[2], d[3], stream);
    if (s != SG_OK) return s;
    for (int i = 0; i < 4; ++i)
        if (h[i]) SG_CUDA(cudaMemcpyAsync(h[i], d[i], sizeof(float) * nr, cudaMemcpyDeviceToHost, st));
    return sg_frame_status(frame, stream);   // also waits for the copies
}

// The frame bytes one render asks for, buffer by buffer as frame_prepare,
// bin_and_sort, the sorts and the compositing launchers size them, each
// grown with ensure()'s head-room.
static size_t grown(size_t bytes) { return bytes < 256 ? 256 : bytes + bytes / 4; }

sg_status sg_workspace_bytes(sg_scene scene, int sensor_kind, int64_t n_rays, size_t *bytes)
{
    if (!scene || !bytes || n_rays < 0 ||
        (sensor_kind != SG_REQ_CAMERA && sensor_kind != SG_REQ_LIDAR)) {
        set_error("sg_workspace_bytes: NULL argument, unknown sensor kind or n_rays < 0");
        return SG_ERR_INVALID;
    }
    const bool cam = sensor_kind == SG_REQ_CAMERA;
    const int64_t n = scene->s.n > 0 ? scene->s.n : 1, nr = n_rays > 0 ? n_rays : 1;
    // units of the compositing: camera tiles (16x16 pixels, images >= 256 px
    // a side: at most (17/16)^2 n_rays / 256 of them) or LiDAR work items
    const int64_t units = cam ? (nr * 289 + 65535) / 65536 + 16
                              : (nr + SG_ADMIT_LIDAR_RAYS_PER_TILE - 1) / SG_ADMIT_LIDAR_RAYS_PER_TILE;
    const int64_t K = SG_ADMIT_PAIRS_PER_GAUSSIAN * n;
    const int per_tile = cam ? 1 : 2;   // LiDAR work items sharing one tile's list
    size_t b = 0;
    // per Gaussian: record, box, tile range, depth, count, UT mean and
    // covariance, depth keys and ids (x2), offsets
    const size_t g[] = {sizeof(GRec), 16, 16, 4, 4, 8, 16, 4, 4, 4, 4, 4};
    for (size_t by : g) b += grown(by * (size_t)n);
    // per ray: state, features, contributor count; per unit: ranges, order
    b += grown(16 * (size_t)nr) * 2 + grown(4 * (size_t)nr);
    b += grown(8 * (size_t)units) + grown(4 * (size_t)units);
    // pairs: keys and ids (x2), camera column/row masks or LiDAR ray masks
    b += 4 * grown(4 * (size_t)K) + grown(4 * (size_t)K * per_tile);
    // sort scratch: the larger of the depth stage's and the tile sort's
    const int64_t hd = depth_stage_words(n), ht = radix_scratch_words(K, 3);
    b += grown(4 * (size_t)(hd > ht ? hd : ht));
    const WorkSize ws = work_size(units, K * per_tile, kSegLen, cam ? 8 : 1);
    b += grown(ws.work_bytes) + grown(ws.partial_bytes);
    b += grown(64) + grown(sizeof(RenderDesc));   // scalars, descriptor
    *bytes = b;
    return SG_OK;
}

sg_status sg_frame_workspace_bytes(sg_frame frame, size_t *bytes)
{
    if (!frame || !bytes) { set_error("NULL argument"); return SG_ERR_INVALID; }
    size_t b = 0;
    for_each_buf(frame->f, [&](Buf &x) { if (!x.borrowed) b += x.bytes; });
    *bytes = b;
    return SG_OK;
}

sg_status sg_frame_field(sg_frame frame, int field, const void **d_ptr, int64_t *count)
{
    if (!frame || !d_ptr || !count) { set_error("NULL argument"); return SG_ERR_INVALID; }
    Frame &f = frame->f;
    if (f.kind < 0) { set_error("frame has not been rendered"); return SG_ERR_INVALID; }
    switch (field) {
    case SG_FIELD_RECT: *d_ptr = f.rect.p; *count = f.n_gauss; break;
    case SG_FIELD_TILES: *d_ptr = f.tiles.p; *count = f.n_gauss; break;
    case SG_FIELD_DEPTH: *d_ptr = f.depth.p; *count = f.n_gauss; break;
    case SG_FIELD_COUNT: *d_ptr = f.count.p; *count = f.n_gauss; break;
    case SG_FIELD_PAIR_IDS: *d_ptr = f.pvals[f.pair_buf].p; *count = pairs_kept(f); break;
    case SG_FIELD_PAIR_TILES: *d_ptr = f.pkeys[f.pair_buf].p; *count = pairs_kept(f); break;
    case SG_FIELD_RANGES: *d_ptr = f.ranges.p; *count = f.n_tiles; break;
    case SG_FIELD_RAY_STATE: *d_ptr = f.ray_state.p; *count = f.n_rays; break;
    case SG_FIELD_N_CONTRIB: *d_ptr = f.n_contrib.p; *count = f.n_rays; break;
    case SG_FIELD_MEAN2D: *d_ptr = f.mean2d.p; *count = f.n_gauss; break;
    case SG_FIELD_COV2D: *d_ptr = f.cov2d.p; *count = f.n_gauss; break;
    default: set_error("unknown field %d", field); return SG_ERR_INVALID;
    }
    return SG_OK;
}

sg_status sg_frame_stats(sg_frame frame, int64_t *n_pairs, int64_t *n_tiles, int64_t *n_rays)
{
    if (!frame) { set_error("frame is NULL"); return SG_ERR_INVALID; }
    if (n_pairs) *n_pairs = pairs_kept(frame->f);
    if (n_tiles) *n_tiles = frame->f.n_tiles;
    if (n_rays) *n_rays = frame->f.n_rays;
    return SG_OK;
}

sg_status sg_backward_camera(sg_scene scene, sg_frame frame, const float *d_g_rgb,
                             const float *d_g_alpha, const float *d_g_depth,
                             const sg_grads *grads, void *stream)
{
    if (!scene || !frame || !grads) { set_error("NULL argument"); return SG_ERR_INVALID; }
    Frame &f = frame->f;
    if ((f.kind != 0 && f.kind != 2) || f.scene != scene) {
        set_error("sg_backward_camera: the frame's last render is not a camera render of this scene");
        return SG_ERR_INVALID;
    }
    if (!f.state_kept) {
        set_error("sg_backward_camera: the frame kept no state for the backward "
                  "(sg_frame_set_backward_state)");
        return SG_ERR_INVALID;
    }
    return backward_camera(scene->s, ((sg_camera)f.sensor)->c, f, d_g_rgb, d_g_alpha, d_g_depth,
                           *grads, (cudaStream_t)stream);
}

sg_status sg_backward_lidar(sg_scene scene, sg_frame frame, const float *d_g_range,
                            const float *d_g_intensity, const float *d_g_drop,
                            const float *d_g_alpha, const sg_grads *grads, void *stream)
{
    if (!scene || !frame || !grads) { set_error("NULL argument"); return SG_ERR_INVALID; }
    Frame &f = frame->f;
    if (f.kind != 1 || f.scene != scene) {
        set_error("sg_backward_lidar: the frame's last render is not a LiDAR render of this scene");
        return SG_ERR_INVALID;
    }
    if (!f.state_kept) {
        set_error("sg_backward_lidar: the frame kept no state for the backward "
                  "(sg_frame_set_backward_state)");
        return SG_ERR_INVALID;
    }
    return backward_lidar(scene->s, ((sg_lidar)f.sensor)->l, f, d_g_range, d_g_intensity,
                          d_g_drop, d_g_alpha, *grads, (cudaStream_t)stream);
}

}  // extern "C"
