"""Backward pass on the GPU (hand-written kernels, through the C-ABI and the
autograd wrapper) against the oracle's analytic gradients (themselves pinned
to central finite differences on the CPU).

Upstream gradients are random on rays whose forward decisions the oracle
reports as unambiguous, and zero elsewhere (a cutoff flip there would change
the function itself, not only its gradient).  Tolerance per element, the
gradient check's stated bar: relative 1e-3, or absolute 1e-5 times the
array's gradient scale max|g_oracle|.  A few elements per hundred thousand
may exceed it, none by more than 10x: the kernels form dL/dalpha_i front to
back from a float difference of the ray's final sum and its prefix, divided
by 1 - alpha_i, so an opaque entry (alpha near 0.99) amplifies the float
rounding of the ray's sums up to 100-fold, and where an element's
contributions cancel that rounding is not small next to the result.  The
quaternion and log-scale gradients share one scale (the larger of the two):
a step delta in either changes M = S^-1 R^T by O(delta) |M|, so both are
bounded by |dL/dM| |M|, and the float rounding of dL/dM reaches both; an
isotropic Gaussian's quaternion gradient is zero exactly, its float value
is that rounding.
"""
import numpy as np
import pytest

from paper_2510_12901_gb300 import synthetic as syn
from tests import parity as par

pytestmark = pytest.mark.gpu
NAMES = ("means", "log_scales", "quats", "opacity", "features")


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_12901_gb300 import _build
    _build.build()
    from paper_2510_12901_gb300 import simgut
    simgut.load()
    return simgut


def compare_grads(G_gpu, G_orc, label, rel=1e-3, absf=1e-5, outlier_frac=1e-4,
                  outlier_factor=10.0):
    out = {}
    shape_scale = max(np.abs(np.asarray(G_orc[k], np.float64)).max()
                      for k in ("quats", "log_scales"))
    for k in NAMES:
        a = np.asarray(G_gpu[k], np.float64).reshape(-1)
        b = np.asarray(G_orc[k], np.float64).reshape(-1)
        scale = shape_scale if k in ("quats", "log_scales") else np.abs(b).max()
        err = np.abs(a - b)
        tol = np.maximum(rel * np.abs(b), absf * scale)
        over = err > tol
        out[k] = (float(scale), float((err / max(scale, 1e-30)).max()), int(over.sum()))
        assert over.sum() <= max(1, int(outlier_frac * len(a))), (
            label, k, out[k], np.nonzero(over)[0][:5], a[over][:5], b[over][:5])
        far = err > outlier_factor * tol
        assert not far.any(), (label, k, out[k], np.nonzero(far)[0][:5], a[far][:5], b[far][:5])
    return out


def camera_backward(sg, S, C, cam, g_rgb, g_alpha, g_depth, n, F):
    import torch
    out = sg.render_camera(S, C, cam.c2w)
    grads = {k: torch.zeros(s, device="cuda") for k, s in
             zip(NAMES, [(n, 3), (n, 3), (n, 4), (n,), (n, F)])}
    ups = [torch.from_numpy(np.ascontiguousarray(u, np.float32)).cuda() for u in
           (g_rgb, g_alpha, g_depth)]
    gs = sg.sg_grads(*[grads[k].data_ptr() for k in NAMES])
    sg.sg_backward_camera(S.handle, out["frame"].handle, *[u.data_ptr() for u in ups], gs,
                          torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in grads.items()}


def upstream(orc, rng, lidar=False, scale_depth=0.05, rays=None):
    n = len(orc)
    ok = ~par.ambiguous_rays(orc, lidar=lidar)
    g = [rng.normal(size=(n, 3)).astype(np.float32), rng.normal(size=n).astype(np.float32),
         (scale_depth * rng.normal(size=n)).astype(np.float32)]
    if lidar:
        g.append(rng.normal(size=n).astype(np.float32))
        g[0] = g[0][:, 0].copy()
    for a in g:
        a[~ok] = 0
    return g


def scatter(vals, rays, total, shape):
    out = np.zeros((total,) + shape[1:], np.float32)
    out[rays] = vals
    return out


def test_camera_backward_tiny(sg, O64):
    sc, cam = syn.tiny_scene(), syn.tiny_camera()
    orc = O64.render_camera(sc, cam)
    g = upstream(orc, np.random.default_rng(0))
    Go = O64.backward_camera(sc, cam, *g)
    Gg = camera_backward(sg, sg.Scene(sc), sg.Camera(cam), cam, *g, sc.n, 3)
    compare_grads(Gg, Go, "tiny")


def test_camera_backward_long_segmented_lists(sg, O64):
    # lists of 14-31 segments of 256 entries, rays stopping in most of them
    sc, cam = syn.layered_scene(), syn.tiny_camera()
    orc = O64.render_camera(sc, cam)
    g = upstream(orc, np.random.default_rng(2))
    Go = O64.backward_camera(sc, cam, *g)
    Gg = camera_backward(sg, sg.Scene(sc), sg.Camera(cam), cam, *g, sc.n, 3)
    compare_grads(Gg, Go, "layered")


def _street_crop(n=30000, seed=5):
    sc = syn.street_scene(n, seed=seed, kind="camera", length=40.0)
    fish, _ = syn.street_cameras()
    cam = syn.Camera(fish.model, 240, 160, 80.0, 80.0, 120.0, 80.0, fish.k, fish.c2w)
    return sc, cam


def test_camera_backward_sh_fisheye(sg, O64):
    sc, cam = _street_crop()
    orc = O64.render_camera(sc, cam)
    g = upstream(orc, np.random.default_rng(1))
    Go = O64.backward_camera(sc, cam, *g)
    Gg = camera_backward(sg, sg.Scene(sc), sg.Camera(cam), cam, *g, sc.n, sc.features.shape[1])
    compare_grads(Gg, Go, "sh-fisheye")


def lidar_backward(sg, S, Ld, L, g, n, F=3):
    import torch
    out = sg.render_lidar(S, Ld, L.col_c2w)
    grads = {k: torch.zeros(s, device="cuda") for k, s in
             zip(NAMES, [(n, 3), (n, 3), (n, 4), (n,), (n, F)])}
    ups = [torch.from_numpy(np.ascontiguousarray(u, np.float32)).cuda() for u in g]
    gs = sg.sg_grads(*[grads[k].data_ptr() for k in NAMES])
    sg.sg_backward_lidar(S.handle, out["frame"].handle, *[u.data_ptr() for u in ups], gs,
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in grads.items()}


@pytest.mark.parametrize("kind", ["lidar", "lidar_sh"])
def test_lidar_backward_toy(sg, O64, kind):
    """Raw LiDAR features, and degree-3 SH^l features (feature gradients
    Y_k(dir) times the channel gradients, and the direction term in the
    mean gradients)."""
    L = syn.street_lidar(n_cols=256)
    sc = syn.street_scene(1500, seed=0, kind=kind, length=60.0)
    orc = O64.render_lidar(sc, L)
    rng = np.random.default_rng(2)
    ok = ~par.ambiguous_rays(orc, lidar=True)
    n = len(orc)
    g = [(0.05 * rng.normal(size=n)).astype(np.float32) for _ in range(1)] + \
        [rng.normal(size=n).astype(np.float32) for _ in range(3)]
    for a in g:
        a[~ok] = 0
    Go = O64.backward_lidar(sc, L, *g)
    Gg = lidar_backward(sg, sg.Scene(sc), sg.Lidar(L), L, g, sc.n, sc.features.shape[1])
    compare_grads(Gg, Go, f"{kind}-toy")


def test_differentiable_step_full_size_sampled(sg, O64):
    """The differentiable step's shapes: 1M-Gaussian scene, 1920x1280
    fisheye and a 2M-Gaussian 128x2048 LiDAR sweep; upstream on 1500 sampled
    rays per sensor, compared with the oracle's backward over those rays."""
    rng = np.random.default_rng(3)
    sc = syn.street_scene(1_000_000, seed=0, kind="camera")
    fish, _ = syn.street_cameras()
    rays = np.unique(rng.choice(fish.width * fish.height, 1500, replace=False))
    orc = O64.render_camera(sc, fish, rays=rays)
    g = upstream(orc, rng)
    tot = fish.width * fish.height
    gfull = [scatter(g[0], rays, tot, (tot, 3)), scatter(g[1], rays, tot, (tot,)),
             scatter(g[2], rays, tot, (tot,))]
    Go = O64.backward_camera(sc, fish, *gfull, rays=rays)
    Gg = camera_backward(sg, sg.Scene(sc), sg.Camera(fish), fish, *gfull, sc.n,
                         sc.features.shape[1])
    compare_grads(Gg, Go, "fisheye-1M")

    lsc = syn.street_scene(2_000_000, seed=10, kind="lidar")
    L = syn.street_lidar()
    tot = L.n_beams * L.n_cols
    rays = np.unique(rng.choice(tot, 1500, replace=False))
    lorc = O64.render_lidar(lsc, L, rays=rays)
    ok = ~par.ambiguous_rays(lorc, lidar=True)
    gl = [(0.05 * rng.normal(size=len(rays))).astype(np.float32)] + \
         [rng.normal(size=len(rays)).astype(np.float32) for _ in range(3)]
    for a in gl:
        a[~ok] = 0
    glf = [scatter(a, rays, tot, (tot,)) for a in gl]
    Go = O64.backward_lidar(lsc, L, *glf, rays=rays)
    Gg = lidar_backward(sg, sg.Scene(lsc), sg.Lidar(L), L, glf, lsc.n)
    compare_grads(Gg, Go, "lidar-2M")


def test_autograd_function_matches_oracle(sg, O64):
    import torch
    from paper_2510_12901_gb300 import autograd as ag
    sc, cam = _street_crop(8000, seed=7)
    S, C = sg.Scene(sc), sg.Camera(cam)
    params = {k: torch.tensor(getattr(sc, k), device="cuda", requires_grad=True) for k in NAMES}
    orc = O64.render_camera(sc, cam)
    g = upstream(orc, np.random.default_rng(4))
    rgb, alpha, depth = ag.render_camera(params, S, C, cam.c2w)
    w = [torch.from_numpy(a).cuda() for a in g]
    loss = (rgb.reshape(-1, 3) * w[0]).sum() + (alpha.reshape(-1) * w[1]).sum() + \
        (depth.reshape(-1) * w[2]).sum()
    loss.backward()
    Go = O64.backward_camera(sc, cam, *g)
    compare_grads({k: params[k].grad.cpu().numpy() for k in NAMES}, Go, "autograd")
    # the L1 training loss of the differentiable step runs end to end
    tgt = torch.from_numpy(syn.noisy_targets((cam.height, cam.width, 3))).cuda()
    for p in params.values():
        p.grad = None
    rgb, alpha, depth = ag.render_camera(params, S, C, cam.c2w)
    (rgb - tgt).abs().mean().backward()
    assert all(torch.isfinite(p.grad).all() for p in params.values())
    assert params["features"].grad.abs().sum() > 0


def test_lidar_backward_beam_divergence(sg, O64):
    """Gradients through the smoothed covariance of Eq. 6 (delta = 0.01):
    dL/dA -> dL/dSigma_hat -> (log-scales, quaternion) and the mean's term
    from |v|^2 I - v v^T."""
    import torch
    L = syn.street_lidar(n_cols=256)
    sc = syn.street_scene(1500, seed=3, kind="lidar", length=60.0)
    delta = 0.01
    orc = O64.render_lidar(sc, L, O64.opts(beam_divergence=delta))
    rng = np.random.default_rng(5)
    ok = ~par.ambiguous_rays(orc, lidar=True)
    n = len(orc)
    g = [(0.05 * rng.normal(size=n)).astype(np.float32)] + \
        [rng.normal(size=n).astype(np.float32) for _ in range(3)]
    for a in g:
        a[~ok] = 0
    Go = O64.backward_lidar(sc, L, *g, opts=O64.opts(beam_divergence=delta))
    S, Ld = sg.Scene(sc), sg.Lidar(L)
    out = sg.render_lidar(S, Ld, L.col_c2w, sg.sg_default_opts(beam_divergence=delta))
    grads = {k: torch.zeros(s, device="cuda") for k, s in
             zip(NAMES, [(sc.n, 3), (sc.n, 3), (sc.n, 4), (sc.n,), (sc.n, 3)])}
    ups = [torch.from_numpy(np.ascontiguousarray(u, np.float32)).cuda() for u in g]
    gs = sg.sg_grads(*[grads[k].data_ptr() for k in NAMES])
    sg.sg_backward_lidar(S.handle, out["frame"].handle, *[u.data_ptr() for u in ups], gs,
                         torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    compare_grads({k: v.cpu().numpy() for k, v in grads.items()}, Go, "beam")
