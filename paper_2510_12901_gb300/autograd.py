"""torch.autograd.Function wrappers around the hand-written backward.

``render_camera(params, scene, cam, c2w)`` and ``render_lidar(...)`` copy the
parameter tensors into the library's resident scene (sg_update_scene),
render through the C-ABI and return outputs whose backward calls
sg_backward_camera / sg_backward_lidar.  Gradients flow to ``means``,
``log_scales``, ``quats``, ``opacity`` and ``features``; the unscented
projection only selects tiles and carries no gradient (Sec. 3.2).
"""
from __future__ import annotations

import torch

from . import simgut as sg

_PARAMS = ("means", "log_scales", "quats", "opacity", "features")


def _ptr(t):
    return 0 if t is None else t.data_ptr()


class _RenderCamera(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity, features, scene, cam, c2w, opts, frame):
        ts = [t.detach().contiguous() for t in (means, log_scales, quats, opacity, features)]
        stream = torch.cuda.current_stream().cuda_stream
        scene.update(*ts)
        h, w = cam.height, cam.width
        rgb = torch.empty((h, w, 3), device=means.device)
        alpha = torch.empty((h, w), device=means.device)
        depth = torch.empty((h, w), device=means.device)
        sg.sg_render_camera(scene.handle, cam.handle, c2w, opts, frame.handle, rgb.data_ptr(),
                            alpha.data_ptr(), depth.data_ptr(), stream)
        ctx.scene, ctx.frame = scene, frame
        ctx.shapes = [t.shape for t in ts]
        return rgb, alpha, depth

    @staticmethod
    def backward(ctx, g_rgb, g_alpha, g_depth):
        dev = g_rgb.device if g_rgb is not None else g_alpha.device
        grads = [torch.zeros(s, device=dev) for s in ctx.shapes]
        gs = sg.sg_grads(*[g.data_ptr() for g in grads])
        ups = [None if g is None else g.contiguous() for g in (g_rgb, g_alpha, g_depth)]
        sg.sg_backward_camera(ctx.scene.handle, ctx.frame.handle, *[_ptr(u) for u in ups], gs,
                              torch.cuda.current_stream().cuda_stream)
        return (*grads, None, None, None, None, None)


class _RenderLidar(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity, features, scene, lid, poses, opts, frame):
        ts = [t.detach().contiguous() for t in (means, log_scales, quats, opacity, features)]
        stream = torch.cuda.current_stream().cuda_stream
        scene.update(*ts)
        shape = (lid.n_beams, lid.n_cols)
        outs = [torch.empty(shape, device=means.device) for _ in range(4)]
        sg.sg_render_lidar(scene.handle, lid.handle, poses.data_ptr(), opts, frame.handle,
                           *[o.data_ptr() for o in outs], stream)
        ctx.scene, ctx.frame, ctx.poses = scene, frame, poses
        ctx.shapes = [t.shape for t in ts]
        return tuple(outs)

    @staticmethod
    def backward(ctx, g_range, g_int, g_drop, g_alpha):
        ref = next(g for g in (g_range, g_int, g_drop, g_alpha) if g is not None)
        grads = [torch.zeros(s, device=ref.device) for s in ctx.shapes]
        gs = sg.sg_grads(*[g.data_ptr() for g in grads])
        ups = [None if g is None else g.contiguous() for g in (g_range, g_int, g_drop, g_alpha)]
        sg.sg_backward_lidar(ctx.scene.handle, ctx.frame.handle, *[_ptr(u) for u in ups], gs,
                             torch.cuda.current_stream().cuda_stream)
        return (*grads, None, None, None, None, None)


def render_camera(params: dict, scene: "sg.Scene", cam: "sg.Camera", c2w, opts=None,
                  frame: "sg.Frame | None" = None):
    """Differentiable camera render: (rgb [H,W,3], alpha [H,W], depth [H,W])."""
    opts = opts or sg.sg_default_opts()
    frame = frame or sg.Frame()
    return _RenderCamera.apply(*[params[k] for k in _PARAMS], scene, cam, c2w, opts, frame)


def render_lidar(params: dict, scene: "sg.Scene", lid: "sg.Lidar", col_c2w, opts=None,
                 frame: "sg.Frame | None" = None):
    """Differentiable LiDAR render: (range, intensity, drop, alpha), [beams, cols]."""
    opts = opts or sg.sg_default_opts()
    frame = frame or sg.Frame()
    poses = col_c2w if isinstance(col_c2w, torch.Tensor) else torch.as_tensor(col_c2w)
    poses = poses.to("cuda", torch.float32).contiguous()
    return _RenderLidar.apply(*[params[k] for k in _PARAMS], scene, lid, poses, opts, frame)
