// render.cuh -- launch parameters and per-ray set-up shared by the forward
// (render.cu, render_fwd.cu) and backward (backward.cu) kernels.
#pragma once

#include "internal.h"

namespace sg {

struct CamRender {
    int W, H, ntx;
    float alpha_min, alpha_max, t_min;
};

// The camera pose of a render, read from its RenderDesc into shared memory
// by every block that needs it.
struct CamPose {
    double Rd[9];        // rotation in double, for the tile reference rays
    float R[9], t[3];    // rotation (camera to world, row-major) and centre
};

// Cooperative load by the block's threads; the caller synchronises.
__device__ __forceinline__ void load_cam_pose(const RenderDesc *__restrict__ D, CamPose &p)
{
    const int i = threadIdx.x;
    if (i < 12) {
        const float v = D->c2w[i];
        const int r = i >> 2, c = i & 3;
        if (c < 3) {
            p.R[3 * r + c] = v;
            p.Rd[3 * r + c] = (double)v;
        } else {
            p.t[r] = v;
        }
    }
}

struct LidRender {
    int n_cols, n_items;
    float alpha_min, alpha_max, t_min;
};

inline CamRender cam_render_params(const Camera &cam, const sg_render_opts &o)
{
    CamRender P;
    P.W = cam.width;
    P.H = cam.height;
    P.ntx = cam.ntx;
    P.alpha_min = o.alpha_min;
    P.alpha_max = o.alpha_max;
    P.t_min = o.t_min;
    return P;
}

inline LidRender lidar_render_params(const Lidar &L, const sg_render_opts &o)
{
    LidRender P;
    P.n_cols = L.n_cols;
    P.n_items = L.n_items;
    P.alpha_min = o.alpha_min;
    P.alpha_max = o.alpha_max;
    P.t_min = o.t_min;
    return P;
}

// reference direction of a camera tile in world coordinates, split in two
// floats: d_T = R r_T computed in double
__device__ __forceinline__ void cam_tile_ref(const CamPose &P, const double *tile_dir, int tile,
                                             float *s_ref)
{
    const double *r = tile_dir + 3 * tile;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        double d = P.Rd[3 * i] * r[0] + P.Rd[3 * i + 1] * r[1] + P.Rd[3 * i + 2] * r[2];
        float h = (float)d;
        s_ref[i] = h;
        s_ref[3 + i] = (float)(d - (double)h);
    }
}

// world-frame offset of a pixel's ray direction from its tile reference
__device__ __forceinline__ void cam_ray_offset(const CamPose &P, const float4 e, float dd[3])
{
#pragma unroll
    for (int i = 0; i < 3; ++i) dd[i] = P.R[3 * i] * e.x + P.R[3 * i + 1] * e.y + P.R[3 * i + 2] * e.z;
}

// Deferred re-walks of the compositing (scalars[7] of them): (unit, work
// code, lane mask, 0), the work code as in the work items.
struct FixList {
    uint4 *fix;
    uint32_t *n_fix;
    uint32_t cap;
};

__device__ __forceinline__ void push_fix(const FixList &F, uint32_t unit, uint32_t code,
                                         uint32_t lanes)
{
    if ((threadIdx.x & 31) == 0) {
        const uint32_t k = atomicAdd(F.n_fix, 1u);
        if (k < F.cap) F.fix[k] = make_uint4(unit, code, lanes, 0u);   // < cap by construction
    }
}

// The deferred re-walks' list in the frame's camwork buffer laid out by ws.
inline FixList fix_list(Frame &fr, const WorkSize &ws)
{
    unsigned char *cw = (unsigned char *)fr.camwork.p;
    return {(uint4 *)(cw + ws.info_bytes + ws.off_bytes + ws.items_bytes + ws.arrive_bytes),
            (uint32_t *)fr.scalars.p + 7, (uint32_t)ws.max_fixes};
}

}  // namespace sg
