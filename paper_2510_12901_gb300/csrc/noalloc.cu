// noalloc.cu -- sg_render_camera_static: the camera render for small
// workloads with every byte of its workspace in one file-scope device array,
// for callers that must not allocate device memory while they run (their
// device memory is held by another allocator, or a cudaMalloc / cudaFree,
// which can block on the whole device, is not acceptable in their loop).
// The paper has no counterpart; this is a deployment variant of the same
// kernels.
#include <math.h>
#include <string.h>

#include <mutex>

#include "internal.h"

namespace sg {

// Stated limits of the static workspace.
constexpr int64_t kStMaxGauss = 32768;     // Gaussians in the scene
constexpr int64_t kStMaxRays = 65536;      // pixels (width x height)
constexpr int64_t kStMaxTiles = 256;       // 16x16 tiles
constexpr int64_t kStMaxPairs = 262144;    // (tile, Gaussian) pairs

// byte layout of the workspace (every piece 256-byte aligned)
constexpr size_t al(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kStRec = al(sizeof(GRec) * kStMaxGauss);
constexpr size_t kStG16 = al(16 * kStMaxGauss);       // float4 / int4 per Gaussian
constexpr size_t kStG8 = al(8 * kStMaxGauss);
constexpr size_t kStG4 = al(4 * kStMaxGauss);
constexpr size_t kStP4 = al(4 * kStMaxPairs);
constexpr size_t kStHist = al(4 * (radix_scratch_words(kStMaxPairs, 4) > depth_stage_words(kStMaxGauss)
                                       ? radix_scratch_words(kStMaxPairs, 4)
                                       : depth_stage_words(kStMaxGauss)));
constexpr WorkSize kStWork = work_size(kStMaxTiles, kStMaxPairs, kSegLenStatic, 8);
constexpr size_t kStBytes = kStRec + 3 * kStG16 + kStG8 +       // rec, rect, tiles, cov2d, mean2d
                            2 * kStG4 +                          // depth, count
                            4 * kStG4 +                          // depth-sort keys/values x2
                            kStG4 +                              // offsets
                            4 * kStP4 +                          // pair keys/values x2
                            kStHist +
                            al(8 * kStMaxTiles) + al(4 * kStMaxTiles) +  // ranges, order
                            2 * al(16 * kStMaxRays) + al(4 * kStMaxRays) + // ray state, features,
                                                                         // contributors
                            kStP4 +                                      // column/row words
                            kStWork.work_bytes + kStWork.partial_bytes + // work items, partials
                            al(64) +                                     // device scalars
                            al(sizeof(RenderDesc));                      // render descriptor

static __device__ __align__(256) unsigned char g_static_ws[kStBytes];

// Device address of the array, looked up once per device (under a lock)
// with that device current.
static std::mutex g_ws_mu;
static void *g_ws_addr[128];

static sg_status static_workspace(unsigned char **out)
{
    int dev = 0;
    SG_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) {
        set_error("device ordinal %d out of range", dev);
        return SG_ERR_INVALID;
    }
    std::lock_guard<std::mutex> lk(g_ws_mu);
    if (!g_ws_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_ws);
        if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(static workspace)");
        g_ws_addr[dev] = p;
    }
    *out = (unsigned char *)g_ws_addr[dev];
    return SG_OK;
}

// A frame buffer inside the array: borrowed, so that a launcher asking for
// more than its size gets SG_ERR_OVERFLOW instead of a reallocation.
static void carve(Buf &b, unsigned char *&cur, size_t bytes)
{
    b.p = cur;
    b.bytes = bytes;
    b.borrowed = true;
    cur += bytes;
}

}  // namespace sg

using namespace sg;

extern "C" sg_status sg_render_camera_static(sg_scene scene, sg_camera cam,
                                             const float h_c2w[12], const sg_render_opts *opts,
                                             float *d_rgb, float *d_alpha, float *d_depth,
                                             void *stream)
{
    if (!scene || !cam || !h_c2w || !opts) {
        set_error("sg_render_camera_static: NULL argument");
        return SG_ERR_INVALID;
    }
    const Scene &sc = scene->s;
    const Camera &c = cam->c;
    const int64_t nr = (int64_t)c.width * c.height, nt = (int64_t)c.ntx * c.nty;
    if (lidar_features(sc.feature_kind)) {
        set_error("sg_render_camera_static: scene carries LiDAR features");
        return SG_ERR_INVALID;
    }
    if (sc.n > kStMaxGauss || nr > kStMaxRays || nt > kStMaxTiles) {
        set_error("sg_render_camera_static: %lld Gaussians / %lld pixels / %lld tiles exceed the "
                  "static workspace (at most %lld / %lld / %lld)",
                  (long long)sc.n, (long long)nr, (long long)nt, (long long)kStMaxGauss,
                  (long long)kStMaxRays, (long long)kStMaxTiles);
        return SG_ERR_INVALID;
    }
    if (!opts_ok(opts)) return SG_ERR_INVALID;
    for (int i = 0; i < 12; ++i)
        if (!isfinite(h_c2w[i])) {
            set_error("sg_render_camera_static: pose is not finite");
            return SG_ERR_INVALID;
        }
    unsigned char *base = nullptr;
    sg_status s = static_workspace(&base);
    if (s != SG_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;

    // a frame whose buffers all point into the static array; every buffer
    // is sized for the limits above, so no launcher ever needs to grow one
    Frame fr;
    unsigned char *cur = base;
    carve(fr.rec, cur, kStRec);
    carve(fr.rect, cur, kStG16);
    carve(fr.tiles, cur, kStG16);
    carve(fr.cov2d, cur, kStG16);
    carve(fr.mean2d, cur, kStG8);
    carve(fr.depth, cur, kStG4);
    carve(fr.count, cur, kStG4);
    for (int i = 0; i < 2; ++i) {
        carve(fr.dkeys[i], cur, kStG4);
        carve(fr.dvals[i], cur, kStG4);
    }
    carve(fr.offsets, cur, kStG4);
    for (int i = 0; i < 2; ++i) {
        carve(fr.pkeys[i], cur, kStP4);
        carve(fr.pvals[i], cur, kStP4);
    }
    carve(fr.hist, cur, kStHist);
    carve(fr.ranges, cur, al(8 * kStMaxTiles));
    carve(fr.order, cur, al(4 * kStMaxTiles));
    carve(fr.ray_state, cur, al(16 * kStMaxRays));
    carve(fr.ray_feat, cur, al(16 * kStMaxRays));
    carve(fr.n_contrib, cur, al(4 * kStMaxRays));
    carve(fr.submask, cur, kStP4);
    carve(fr.camwork, cur, kStWork.work_bytes);
    carve(fr.partials, cur, kStWork.partial_bytes);
    fr.seg_len = kSegLenStatic;
    carve(fr.scalars, cur, al(64));
    carve(fr.desc, cur, al(sizeof(RenderDesc)));
    fr.n_gauss = sc.n;
    fr.n_rays = nr;
    fr.n_tiles = nt;
    fr.kind = 0;
    fr.opts = *opts;
    memcpy(fr.c2w, h_c2w, sizeof(fr.c2w));

    // the stages of sg_render_camera: project, depth sort, offsets, pair
    // count, binning, tile sort, ranges, compositing
    const int64_t n = sc.n;
    // the descriptor goes from pageable host memory: the copy has taken its
    // source by the time cudaMemcpyAsync returns
    RenderDesc D;
    memcpy(D.c2w, h_c2w, sizeof(D.c2w));
    D.poses = nullptr;
    D.out[0] = d_rgb;
    D.out[1] = d_alpha;
    D.out[2] = d_depth;
    D.out[3] = nullptr;
    SG_CUDA(cudaMemcpyAsync(fr.desc.p, &D, sizeof(D), cudaMemcpyHostToDevice, st));
    if ((s = project_camera(sc, c, *opts, fr, st)) != SG_OK) return s;
    uint32_t *scal = (uint32_t *)fr.scalars.p;
    uint32_t *dk[2] = {(uint32_t *)fr.dkeys[0].p, (uint32_t *)fr.dkeys[1].p};
    uint32_t *dv[2] = {(uint32_t *)fr.dvals[0].p, (uint32_t *)fr.dvals[1].p};
    int rb = 0;
    if ((s = depth_stage((const uint32_t *)fr.count.p, (const float *)fr.depth.p, n, dk, dv, scal,
                         (uint32_t *)fr.offsets.p, fr, st, &rb)) != SG_OK)
        return s;
    // the counts and the status word (pageable: the copy is synchronous here)
    uint32_t hs[kScalStatus + 1] = {};
    SG_CUDA(cudaMemcpyAsync(hs, scal, sizeof(hs), cudaMemcpyDeviceToHost, st));
    SG_CUDA(cudaStreamSynchronize(st));
    if (hs[kScalStatus]) {
        set_error("sg_render_camera_static: a bounded device wait (sort look-back or projection bulk copy) gave up");
        return SG_ERR_TIMEOUT;
    }
    const int64_t K = hs[1];
    if (K > kStMaxPairs) {
        set_error("sg_render_camera_static: %lld (tile, Gaussian) pairs exceed the static "
                  "workspace (at most %lld)", (long long)K, (long long)kStMaxPairs);
        return SG_ERR_OVERFLOW;
    }
    fr.n_pairs = K;
    uint32_t *pk[2] = {(uint32_t *)fr.pkeys[0].p, (uint32_t *)fr.pkeys[1].p};
    uint32_t *pv[2] = {(uint32_t *)fr.pvals[0].p, (uint32_t *)fr.pvals[1].p};
    int bits = 1;
    while (((int64_t)1 << bits) < nt) ++bits;
    uint32_t *hist = nullptr;
    if (K > 0 && (s = radix_prepare(K, (bits + 7) / 8, fr, st, &hist, 0)) != SG_OK) return s;
    const uint32_t *err = scal + kScalStatus;
    if ((s = bin_pairs(dv[rb], (const uint32_t *)fr.offsets.p, scal, (const int4 *)fr.tiles.p,
                       c.ntx, 0, K, pk[0], pv[0], st, err, hist, bits)) != SG_OK)
        return s;
    int pb = 0;
    if ((s = radix_sort_pairs(pk, pv, K, scal + 1, 0, bits, fr, st, &pb,
                              SG_LOOKBACK_TILE_SORT)) != SG_OK)
        return s;
    fr.pair_buf = pb;
    if ((s = tile_ranges(pk[pb], scal + 1, K, (uint2 *)fr.ranges.p, nt, st, err, pv[pb],
                         (const float4 *)fr.rect.p, c.ntx, (uint32_t *)fr.submask.p)) != SG_OK)
        return s;
    return render_camera(c, *opts, fr, st);
}
