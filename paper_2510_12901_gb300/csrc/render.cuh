// render.cuh -- launch parameters and per-ray set-up shared by the forward
// (render.cu) and backward (backward.cu) kernels.
#pragma once

#include "internal.h"

namespace sg {

struct CamRender {
    int W, H, ntx;
    float R[9], t[3];
    double Rd[9];
    float alpha_min, alpha_max, t_min;
};

struct LidRender {
    int n_cols, n_items;
    float alpha_min, alpha_max, t_min;
};

inline CamRender cam_render_params(const Camera &cam, const float c2w[12],
                                   const sg_render_opts &o)
{
    CamRender P;
    P.W = cam.width;
    P.H = cam.height;
    P.ntx = cam.ntx;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            P.R[3 * r + c] = c2w[4 * r + c];
            P.Rd[3 * r + c] = (double)c2w[4 * r + c];
        }
        P.t[r] = c2w[4 * r + 3];
    }
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
__device__ __forceinline__ void cam_tile_ref(const CamRender &P, const double *tile_dir, int tile,
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
__device__ __forceinline__ void cam_ray_offset(const CamRender &P, const float4 e, float dd[3])
{
#pragma unroll
    for (int i = 0; i < 3; ++i) dd[i] = P.R[3 * i] * e.x + P.R[3 * i + 1] * e.y + P.R[3 * i + 2] * e.z;
}

}  // namespace sg
