// sensors.cu -- once-per-sensor set-up: camera ray tables and the LiDAR
// tiling of App. A (Proc. 1 ElevationTiling) with the ray-mask summed-area
// table of App. B.
//
// Ray directions are produced in double precision and stored relative to a
// per-tile reference direction.  The renderer rebuilds each ray as
// reference (double, rotated per render) + small float offset, which keeps
// the closest-approach distance of far, thin Gaussians accurate in float
// arithmetic (see render.cu).
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include <string.h>

#include "internal.h"

namespace sg {

// ------------------------------------------------------------------ camera

// Largest valid incidence angle of the OpenCV fisheye model: the first
// stationary point of theta_d(theta) = theta (1 + k1 t^2 + k2 t^4 + k3 t^6 +
// k4 t^8), at most pi/2.  d theta_d / d theta is a quartic in x = theta^2:
// 1 + 3 k1 x + 5 k2 x^2 + 7 k3 x^3 + 9 k4 x^4; its first sign change on
// (0, (pi/2)^2] is bracketed on a grid and refined by bisection on x.
static double fisheye_theta_limit(const float k[4])
{
    auto deriv = [&](double x) {
        return 1.0 + x * (3.0 * k[0] + x * (5.0 * k[1] + x * (7.0 * k[2] + x * 9.0 * k[3])));
    };
    const double cap = M_PI / 2.0;
    const double xmax = cap * cap;
    const int n = 40000;
    double prev = 0.0;
    for (int i = 1; i <= n; ++i) {
        double x = xmax * i / n;
        if (deriv(x) <= 0.0) {
            double lo = prev, hi = x;
            for (int it = 0; it < 200 && hi - lo > 0; ++it) {
                double m = 0.5 * (lo + hi);
                if (m <= lo || m >= hi) break;
                if (deriv(m) > 0.0) lo = m; else hi = m;
            }
            return sqrt(lo);
        }
        prev = x;
    }
    return cap;
}

__device__ double fisheye_forward(const double k[4], double t)
{
    double t2 = t * t;
    return t * (1.0 + t2 * (k[0] + t2 * (k[1] + t2 * (k[2] + t2 * k[3]))));
}

// Per-pixel camera-frame unit direction in double.  Fisheye inverse by
// safeguarded Newton iteration on [0, theta_max] (the model is increasing
// there).
__global__ void k_camera_dirs(int model, int W, int H, double fx, double fy, double cx,
                              double cy, double k0, double k1, double k2, double k3,
                              double tmax, double *dirs, unsigned char *valid)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (int64_t)W * H) return;
    int px = (int)(p % W), py = (int)(p / W);
    double mx = ((double)px + 0.5 - cx) / fx;
    double my = ((double)py + 0.5 - cy) / fy;
    double d0, d1, d2;
    unsigned char ok = 1;
    if (model == SG_CAMERA_PINHOLE) {
        double inv = 1.0 / sqrt(mx * mx + my * my + 1.0);
        d0 = mx * inv; d1 = my * inv; d2 = inv;
    } else {
        const double k[4] = {k0, k1, k2, k3};
        double rd = sqrt(mx * mx + my * my);
        if (rd > fisheye_forward(k, tmax)) {
            ok = 0;
            d0 = 0; d1 = 0; d2 = 1;
        } else {
            double lo = 0.0, hi = tmax, t = fmin(rd, tmax);
            for (int it = 0; it < 100; ++it) {
                double t2 = t * t;
                double f = fisheye_forward(k, t) - rd;
                if (f < 0) lo = t; else hi = t;
                double df = 1.0 + t2 * (3.0 * k0 + t2 * (5.0 * k1 + t2 * (7.0 * k2 + t2 * 9.0 * k3)));
                double tn = t - f / df;
                if (!(tn > lo && tn < hi)) tn = 0.5 * (lo + hi);
                if (fabs(tn - t) <= 1e-17 * fmax(1.0, t)) { t = tn; break; }
                t = tn;
            }
            double st = sin(t);
            if (rd > 0) { d0 = st * mx / rd; d1 = st * my / rd; }
            else { d0 = 0; d1 = 0; }
            d2 = cos(t);
        }
    }
    dirs[3 * p] = d0;
    dirs[3 * p + 1] = d1;
    dirs[3 * p + 2] = d2;
    valid[p] = ok;
}

// Smallest cosine between a pixel's direction and its tile's reference
// direction for which the tangent-plane table is used (|d'| <= 4).
constexpr double kTangentMinCos = 0.25;

// One block per tile: reference direction = normalised mean of the tile's
// valid pixel directions; each pixel stores its offset from it.  Also the
// tile's tangent basis (e1 normal to the reference direction and to the
// coordinate axis least aligned with it, e2 = reference x e1) and each
// pixel's direction over its cosine to the reference, in that basis; `far`
// is set when a cosine is below kTangentMinCos.
__global__ void k_camera_tile_ref(int W, int H, int ntx, const double *dirs,
                                  const unsigned char *valid, double *tile_dir, float4 *pix,
                                  float *tile_basis, float4 *pix2, int *far)
{
    __shared__ double red[3][kCamThreads];
    int t = blockIdx.x;
    int tx = t % ntx, ty = t / ntx;
    int lx = threadIdx.x % kTile, ly = threadIdx.x / kTile;
    int px = tx * kTile + lx, py = ty * kTile + ly;
    bool in = px < W && py < H;
    int64_t p = (int64_t)py * W + px;
    bool ok = in && valid[p];
    for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = ok ? dirs[3 * p + c] : 0.0;
    __syncthreads();
    for (int s = kCamThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
        __syncthreads();
    }
    double r0 = red[0][0], r1 = red[1][0], r2 = red[2][0];
    double nr = sqrt(r0 * r0 + r1 * r1 + r2 * r2);
    if (nr > 0) { r0 /= nr; r1 /= nr; r2 /= nr; }
    else { r0 = 0; r1 = 0; r2 = 1; }
    if (threadIdx.x == 0) {
        tile_dir[3 * t] = r0;
        tile_dir[3 * t + 1] = r1;
        tile_dir[3 * t + 2] = r2;
    }
    if (in)
        pix[p] = ok ? make_float4((float)(dirs[3 * p] - r0), (float)(dirs[3 * p + 1] - r1),
                                  (float)(dirs[3 * p + 2] - r2), 1.0f)
                    : make_float4(0.f, 0.f, 0.f, 0.f);
    const double a0 = fabs(r0), a1 = fabs(r1), a2 = fabs(r2);
    const double x0 = (a0 <= a1 && a0 <= a2) ? 1.0 : 0.0;
    const double x1 = x0 == 0.0 && a1 <= a2 ? 1.0 : 0.0;
    const double x2 = x0 == 0.0 && x1 == 0.0 ? 1.0 : 0.0;
    double e10 = x1 * r2 - x2 * r1, e11 = x2 * r0 - x0 * r2, e12 = x0 * r1 - x1 * r0;
    const double ne = sqrt(e10 * e10 + e11 * e11 + e12 * e12);
    e10 /= ne; e11 /= ne; e12 /= ne;
    const double e20 = r1 * e12 - r2 * e11, e21 = r2 * e10 - r0 * e12, e22 = r0 * e11 - r1 * e10;
    if (threadIdx.x == 0) {
        float *b = tile_basis + 6 * t;
        b[0] = (float)e10; b[1] = (float)e11; b[2] = (float)e12;
        b[3] = (float)e20; b[4] = (float)e21; b[5] = (float)e22;
    }
    if (in) {
        float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ok) {
            const double d0 = dirs[3 * p], d1 = dirs[3 * p + 1], d2 = dirs[3 * p + 2];
            const double c = d0 * r0 + d1 * r1 + d2 * r2;
            if (!(c >= kTangentMinCos)) {
                atomicOr(far, 1);
            } else {
                q = make_float4((float)((d0 * e10 + d1 * e11 + d2 * e12) / c),
                                (float)((d0 * e20 + d1 * e21 + d2 * e22) / c), (float)(1.0 / c),
                                1.0f);
            }
        }
        pix2[p] = q;
    }
}

sg_status build_camera(Camera &cam)
{
    cam.theta_max = cam.model == SG_CAMERA_FISHEYE ? fisheye_theta_limit(cam.k) : 0.0;
    cam.ntx = (cam.width + kTile - 1) / kTile;
    cam.nty = (cam.height + kTile - 1) / kTile;
    int64_t np = (int64_t)cam.width * cam.height;
    int64_t nt = (int64_t)cam.ntx * cam.nty;
    double *dirs = nullptr;
    unsigned char *valid = nullptr;
    int *far = nullptr;
    if (dev_malloc(&dirs, sizeof(double) * 3 * np) != cudaSuccess ||
        dev_malloc(&valid, np) != cudaSuccess || dev_malloc(&far, sizeof(int)) != cudaSuccess ||
        dev_malloc(&cam.d_pix, sizeof(float4) * np) != cudaSuccess ||
        dev_malloc(&cam.d_tile_dir, sizeof(double) * 3 * nt) != cudaSuccess ||
        dev_malloc(&cam.d_pix2, sizeof(float4) * np) != cudaSuccess ||
        dev_malloc(&cam.d_tile_basis, sizeof(float) * 6 * nt) != cudaSuccess) {
        dev_free(dirs);
        dev_free(valid);
        dev_free(far);
        set_error("sg_create_camera: device allocation failed");
        return SG_ERR_OOM;
    }
    cudaMemset(far, 0, sizeof(int));
    k_camera_dirs<<<(unsigned)((np + 255) / 256), 256>>>(
        cam.model, cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, cam.k[0], cam.k[1],
        cam.k[2], cam.k[3], cam.theta_max, dirs, valid);
    count_launch();
    k_camera_tile_ref<<<(unsigned)nt, kCamThreads>>>(cam.width, cam.height, cam.ntx, dirs,
                                                     valid, cam.d_tile_dir, cam.d_pix,
                                                     cam.d_tile_basis, cam.d_pix2, far);
    count_launch();
    cudaError_t e = cudaDeviceSynchronize();
    int h_far = 1;
    if (e == cudaSuccess) e = cudaMemcpy(&h_far, far, sizeof(int), cudaMemcpyDeviceToHost);
    dev_free(dirs);
    dev_free(valid);
    dev_free(far);
    if (e != cudaSuccess) return cuda_status(e, "camera ray table");
    cam.tangent_ok = h_far == 0;
    return SG_OK;
}

// ------------------------------------------------------------------ LiDAR

// Elevation tile of an angle: number of interior boundaries T_1..T_{nphi-1}
// not above it (float comparisons, as on the device).
static int host_elev_tile(const std::vector<float> &T, int nphi, float el)
{
    int lo = 1, hi = nphi - 1, e = 0;   // last j with T[j] <= el
    while (lo <= hi) {
        int m = (lo + hi) / 2;
        if (T[m] <= el) { e = m; lo = m + 1; } else hi = m - 1;
    }
    return e;
}

static int host_elev_cell(const std::vector<float> &T, int nphi, int per, float el)
{
    int e = host_elev_tile(T, nphi, el);
    float f = (el - T[e]) / (T[e + 1] - T[e]) * (float)per;
    int sub = !(f >= 0.f) ? 0 : (f >= (float)per ? per - 1 : (int)floorf(f));
    return e * per + std::min(sub, per - 1);
}

sg_status build_lidar(Lidar &L)
{
    const int nb = L.n_beams, nc = L.n_cols, nphi = L.nphi;
    // Proc. 1: histogram of the ray elevations (each beam once per column)
    // over r = 400 bins; boundaries where the normalised CDF reaches each
    // integer 1..N_phi (integer test cum * N_phi >= b * total); mapped back
    // to degrees; N_theta = ceil(max rays per elevation tile / M).
    const int r = 400;
    double pmin = 1e300, pmax = -1e300;
    for (float e : L.elev) { pmin = std::min(pmin, (double)e); pmax = std::max(pmax, (double)e); }
    if (!(pmax > pmin)) {
        set_error("sg_create_lidar: the beam elevations must not all be equal");
        return SG_ERR_INVALID;
    }
    std::vector<int64_t> hist(r, 0);
    for (float e : L.elev) {
        int b = (int)floor(((double)e - pmin) / (pmax - pmin) * r);
        hist[std::min(std::max(b, 0), r - 1)] += nc;
    }
    const int64_t total = (int64_t)nb * nc;
    std::vector<double> edges(1, 0.0);
    int64_t cum = 0, next = 1;
    for (int i = 0; i < r; ++i) {
        cum += hist[i];
        for (; next <= nphi && cum * nphi >= next * total; ++next) edges.push_back(i + 1.0);
    }
    L.T.resize(nphi + 1);
    for (int j = 0; j <= nphi; ++j) L.T[j] = (float)(pmin + edges[j] / r * (pmax - pmin));
    std::vector<int> beam_tile(nb);
    std::vector<int64_t> per_tile(nphi, 0);
    for (int b = 0; b < nb; ++b) {
        beam_tile[b] = host_elev_tile(L.T, nphi, L.elev[b]);
        per_tile[beam_tile[b]] += nc;
    }
    int64_t hmax = *std::max_element(per_tile.begin(), per_tile.end());
    int64_t nth = (hmax + L.M - 1) / L.M;
    if (nth < 1) nth = 1;
    if (nth * nphi > 65535 || nth > 65535) {
        set_error("sg_create_lidar: %lld tiles exceed 65535", (long long)(nth * nphi));
        return SG_ERR_INVALID;
    }
    L.n_theta = (int)nth;

    // column azimuths (deg, rounded to float) and their azimuth tiles
    std::vector<float> az(nc);
    std::vector<int> col_tile(nc);
    for (int c = 0; c < nc; ++c) {
        az[c] = (float)((double)L.az0 + (c + 0.5) * 360.0 / nc);
        int a = (int)floorf((az[c] - L.az0) * ((float)L.n_theta / 360.0f));
        col_tile[c] = ((a % L.n_theta) + L.n_theta) % L.n_theta;
    }

    // ray mask on the dense grid and its summed-area table (zero first row
    // and column), App. B
    const int A = L.cull_az, E = nphi * L.cull_el;
    std::vector<unsigned char> mask((size_t)A * E, 0);
    std::vector<int> beam_cell(nb);
    for (int b = 0; b < nb; ++b) beam_cell[b] = host_elev_cell(L.T, nphi, L.cull_el, L.elev[b]);
    for (int c = 0; c < nc; ++c) {
        int x = (int)floorf((az[c] - L.az0) * ((float)A / 360.0f));
        x = ((x % A) + A) % A;
        for (int b = 0; b < nb; ++b) mask[(size_t)x * E + beam_cell[b]] = 1;
    }
    std::vector<int> sat((size_t)(A + 1) * (E + 1), 0);
    for (int x = 0; x < A; ++x) {
        int rowsum = 0;
        for (int y = 0; y < E; ++y) {
            rowsum += mask[(size_t)x * E + y];
            sat[(size_t)(x + 1) * (E + 1) + y + 1] = sat[(size_t)x * (E + 1) + y + 1] + rowsum;
        }
    }

    // warp work items: per tile, columns in groups of <= kLidarColsMax and
    // rays in chunks of <= 32; each item's reference direction points at the
    // middle of its elevation tile and column group (double precision)
    std::vector<std::vector<int>> tile_beams(nphi);
    for (int b = 0; b < nb; ++b) tile_beams[beam_tile[b]].push_back(b);
    std::vector<int> tile_c0(L.n_theta, -1), tile_c1(L.n_theta, -2);
    for (int c = 0; c < nc; ++c) {
        int a = col_tile[c];
        if (tile_c0[a] < 0) tile_c0[a] = c;
        tile_c1[a] = c;
    }
    std::vector<LidarItem> items;
    std::vector<uint32_t> rays;
    std::vector<float4> ray_e;
    std::vector<double> item_u;
    std::vector<double> item_ref;     // per item and column slot: cos az, sin az, tan el_r
    std::vector<float2> ray_tau;      // per ray slot: tan el - tan el_r, 1 / cos el
    const double d2r = M_PI / 180.0;
    for (int e = 0; e < nphi; ++e) {
        const std::vector<int> &bs = tile_beams[e];
        if (bs.empty()) continue;
        double el_ref = 0;
        for (int b : bs) el_ref += L.elev[b];
        el_ref /= (double)bs.size();
        for (int a = 0; a < L.n_theta; ++a) {
            if (tile_c0[a] < 0) continue;
            for (int g0 = tile_c0[a]; g0 <= tile_c1[a]; g0 += kLidarColsMax) {
                int g1 = std::min(g0 + kLidarColsMax - 1, tile_c1[a]);
                double az_ref = 0.5 * ((double)az[g0] + (double)az[g1]);
                double u0 = cos(el_ref * d2r) * cos(az_ref * d2r);
                double u1 = cos(el_ref * d2r) * sin(az_ref * d2r);
                double u2 = sin(el_ref * d2r);
                std::vector<uint32_t> rr;
                for (int c = g0; c <= g1; ++c)
                    for (int b : bs) rr.push_back((uint32_t)b * nc + c);
                for (size_t k0 = 0; k0 < rr.size(); k0 += 32) {
                    LidarItem it;
                    it.tile = (uint32_t)(e * L.n_theta + a);
                    it.col0 = (uint16_t)g0;
                    it.ncols = (uint8_t)(g1 - g0 + 1);
                    size_t k1 = std::min(rr.size(), k0 + 32);
                    it.nrays = (uint8_t)(k1 - k0);
                    it.ray_off = (uint32_t)rays.size();
                    it.ref_col = (uint32_t)g0;
                    items.push_back(it);
                    item_u.push_back(u0);
                    item_u.push_back(u1);
                    item_u.push_back(u2);
                    // the forward-only kernel's rays: d / cos el = h_c + tan el z_c
                    // around tan el_r, the middle of the item's range of tan el
                    double t_lo = 1e300, t_hi = -1e300;
                    for (size_t k = k0; k < k1; ++k) {
                        const double t = tan((double)L.elev[rr[k] / (uint32_t)nc] * d2r);
                        t_lo = std::min(t_lo, t);
                        t_hi = std::max(t_hi, t);
                    }
                    const double t_ref = 0.5 * (t_lo + t_hi);
                    for (int sl = 0; sl < kLidarColsMax; ++sl) {
                        // column azimuth in double, as the ray definition has it
                        const double azc =
                            ((double)L.az0 + (g0 + sl + 0.5) * 360.0 / nc) * d2r;
                        item_ref.push_back(sl <= g1 - g0 ? cos(azc) : 0.0);
                        item_ref.push_back(sl <= g1 - g0 ? sin(azc) : 0.0);
                        item_ref.push_back(sl <= g1 - g0 ? t_ref : 0.0);
                    }
                    for (size_t k = k0; k < k0 + 32; ++k) {
                        if (k < k1) {
                            uint32_t ray = rr[k];
                            int b = (int)(ray / nc), c = (int)(ray % nc);
                            double el = (double)L.elev[b] * d2r, azr = (double)az[c] * d2r;
                            double w0 = cos(el) * cos(azr), w1 = cos(el) * sin(azr), w2 = sin(el);
                            rays.push_back(ray);
                            ray_e.push_back(make_float4((float)(w0 - u0), (float)(w1 - u1),
                                                        (float)(w2 - u2), 1.0f));
                            ray_tau.push_back(make_float2((float)(tan(el) - t_ref),
                                                          (float)(1.0 / cos(el))));
                        } else {
                            rays.push_back(0xffffffffu);
                            ray_e.push_back(make_float4(0.f, 0.f, 0.f, 0.f));
                            ray_tau.push_back(make_float2(0.f, 1.f));
                        }
                    }
                }
            }
        }
    }
    L.n_items = (int)items.size();
    // a tile wider than kLidarColsMax columns or holding more than 32 rays
    // gives several items, each walking the tile's whole list; the items of
    // a tile are consecutive (first item, count per tile)
    std::vector<uint2> tile_items((size_t)nphi * L.n_theta, make_uint2(0u, 0u));
    for (size_t i = 0; i < items.size(); ++i) {
        uint2 &ti = tile_items[items[i].tile];
        if (ti.y == 0) ti.x = (uint32_t)i;
        ++ti.y;
    }
    L.max_items_per_tile = 1;
    for (const uint2 &ti : tile_items) L.max_items_per_tile = std::max(L.max_items_per_tile, (int)ti.y);
    // per item, its ray slots factorised into columns and beams (a ray is in
    // a box iff its column's azimuth and its beam's elevation are): the
    // azimuths of its (at most kLidarColsMax) columns and the elevations of
    // its distinct beams (at most 32), each with the mask of its ray slots
    std::vector<LidarItemRays> item_rays(items.size());
    for (size_t i = 0; i < items.size(); ++i) {
        LidarItemRays &R = item_rays[i];
        memset(&R, 0, sizeof(R));
        const LidarItem &it = items[i];
        R.ncols = it.ncols;
        for (int sl = 0; sl < kLidarColsMax; ++sl)
            R.col_az[sl] = sl < it.ncols ? az[it.col0 + sl] : 0.f;
        for (int k = 0; k < 32; ++k) {
            const uint32_t ray = rays[(size_t)it.ray_off + k];
            if (ray == 0xffffffffu) continue;
            const int c = (int)(ray % (uint32_t)nc), b = (int)(ray / (uint32_t)nc);
            R.col_bits[c - it.col0] |= 1u << k;
            int j = 0;
            while (j < R.nbeams && R.beam_el[j] != L.elev[b]) ++j;
            if (j == R.nbeams) R.beam_el[R.nbeams++] = L.elev[b];
            R.beam_bits[j] |= 1u << k;
        }
    }

#define SG_ALLOC_COPY(dst, vec)                                                         \
    do {                                                                                \
        size_t by_ = sizeof((vec)[0]) * (vec).size();                                   \
        if (dev_malloc((void **)&(dst), by_ ? by_ : 16) != cudaSuccess) {               \
            set_error("sg_create_lidar: device allocation failed");                     \
            return SG_ERR_OOM;                                                          \
        }                                                                               \
        if (by_) SG_CUDA(cudaMemcpy((dst), (vec).data(), by_, cudaMemcpyHostToDevice)); \
    } while (0)
    SG_ALLOC_COPY(L.d_T, L.T);
    SG_ALLOC_COPY(L.d_elev, L.elev);
    SG_ALLOC_COPY(L.d_az, az);
    SG_ALLOC_COPY(L.d_sat, sat);
    SG_ALLOC_COPY(L.d_items, items);
    SG_ALLOC_COPY(L.d_item_rays, rays);
    SG_ALLOC_COPY(L.d_ray_e, ray_e);
    SG_ALLOC_COPY(L.d_tile_u, item_u);
    SG_ALLOC_COPY(L.d_tile_items, tile_items);
    SG_ALLOC_COPY(L.d_item_ray_tab, item_rays);
    SG_ALLOC_COPY(L.d_item_ref, item_ref);
    SG_ALLOC_COPY(L.d_ray_tau, ray_tau);
#undef SG_ALLOC_COPY
    return SG_OK;
}

}  // namespace sg
