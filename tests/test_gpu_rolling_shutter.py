"""Rolling-shutter camera (Sec. 3.2, time-dependent effects) on the GPU
against the oracle: each pixel row has its own pose; the projection takes
for every point the pose of the row it falls in, and every ray is
evaluated with its own row's origin and rotation."""
import dataclasses

import numpy as np
import pytest

from paper_2510_12901_gb300 import synthetic as syn
from tests import parity as par
from tests.test_gpu_backward import NAMES, compare_grads, upstream

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_12901_gb300 import _build
    _build.build()
    from paper_2510_12901_gb300 import simgut
    simgut.load()
    return simgut


def _crop(cam, w, h, f):
    return syn.Camera(cam.model, w, h, f, f, w / 2, h / 2, cam.k, cam.c2w)


def rs_render(sg, sc, cam, S=None):
    import torch
    S = S or sg.Scene(sc)
    C = sg.Camera(cam)          # the frame refers to the camera: keep it alive
    out = sg.render_camera_rs(S, C, cam.row_c2w)
    torch.cuda.synchronize()
    return dict(rgb=out["rgb"].cpu().numpy(), alpha=out["alpha"].cpu().numpy(),
                depth=out["depth"].cpu().numpy(), out=out, scene=S, cam=C)


@pytest.mark.parametrize("which,motion", [(0, "drive"), (1, "drive"), (1, "swerve")])
def test_rolling_shutter_every_pixel(sg, O64, which, motion):
    sc = syn.street_scene(60000, seed=18, length=40.0)
    fish, pin = syn.street_cameras()
    cam = _crop(fish, 320, 214, 107.0) if which == 0 else _crop(pin, 320, 180, 170.0)
    kw = dict(speed=15.0, readout_s=0.03, yaw_rate=0.1) if motion == "drive" else \
        dict(speed=30.0, readout_s=0.05, yaw_rate=1.0)
    cam = syn.rolling_shutter(cam, **kw)
    g = rs_render(sg, sc, cam)
    orc = O64.render_camera(sc, cam)
    # pixels in the box of a Gaussian whose sigma points' row choice is within
    # rounding (its box differs by up to a row's motion between the two)
    P64, _ = O64.project_camera(sc, cam)
    row_amb = (P64["ut"] == 1) & (P64["pmargin"] < par.MARGIN_POSE_COLS)
    fr = g["out"]["frame"]
    seen = par.camera_rays_seeing(np.arange(cam.width * cam.height), cam.width, row_amb,
                                  fr.field(sg.FIELD_RECT, np.float32, 4), P64["rect"])
    info = par.compare_camera_rays(g["rgb"].reshape(-1, 3), g["alpha"].reshape(-1),
                                   g["depth"].reshape(-1), orc, max_excluded=0.02,
                                   label=f"rs-{which}-{motion}", posed=True, also_excluded=seen)
    assert (orc["alpha"] > 0).mean() > 0.3, info


def test_equal_rows_match_the_global_shutter(sg):
    """All rows at the camera's pose: the rolling-shutter kernels render the
    global-shutter image (up to float rounding: another staging layout)."""
    import torch
    sc = syn.street_scene(60000, seed=19, length=40.0)
    cam = _crop(syn.street_cameras()[1], 320, 180, 170.0)
    rs = dataclasses.replace(cam, row_c2w=np.tile(cam.c2w, (cam.height, 1)))
    S = sg.Scene(sc)
    a = rs_render(sg, sc, rs, S)
    C = sg.Camera(cam)
    b = sg.render_camera(S, C, cam.c2w)
    torch.cuda.synchronize()
    # another staging layout rounds differently: a cutoff (alpha_min, T_min)
    # may flip at a few pixels, elsewhere the images agree to float rounding
    d = np.abs(a["rgb"] - b["rgb"].cpu().numpy()).max(axis=-1)
    da = np.abs(a["alpha"] - b["alpha"].cpu().numpy())
    assert (d > 1e-4).mean() < 1e-3 and (da > 1e-4).mean() < 1e-3
    assert np.median(d) < 1e-6


def test_rolling_shutter_backward(sg, O64):
    import torch
    sc = syn.street_scene(30000, seed=20, length=40.0)
    fish, _ = syn.street_cameras()
    cam = syn.rolling_shutter(_crop(fish, 240, 160, 80.0), speed=30.0, readout_s=0.05,
                              yaw_rate=1.0)
    orc = O64.render_camera(sc, cam)
    g = upstream(orc, np.random.default_rng(6))
    amb = par.ambiguous_rays(orc, lidar=True)
    for a in g:
        a[amb] = 0
    Go = O64.backward_camera(sc, cam, *g)
    S = sg.Scene(sc)
    C = sg.Camera(cam)          # the frame refers to the camera until the backward
    out = sg.render_camera_rs(S, C, cam.row_c2w)
    n, F = sc.n, sc.features.shape[1]
    grads = {k: torch.zeros(s, device="cuda") for k, s in
             zip(NAMES, [(n, 3), (n, 3), (n, 4), (n,), (n, F)])}
    ups = [torch.from_numpy(np.ascontiguousarray(u, np.float32)).cuda() for u in g]
    gs = sg.sg_grads(*[grads[k].data_ptr() for k in NAMES])
    sg.sg_backward_camera(S.handle, out["frame"].handle, *[u.data_ptr() for u in ups], gs,
                          torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    compare_grads({k: v.cpu().numpy() for k, v in grads.items()}, Go, "rs-backward")


def test_rolling_shutter_views_in_one_call(sg):
    """sg_render_cameras with a rolling-shutter and a global-shutter view on
    two streams gives each view's result alone, bit for bit."""
    import torch
    sc = syn.street_scene(60000, seed=21, length=40.0)
    fish, pin = syn.street_cameras()
    rs = syn.rolling_shutter(_crop(fish, 320, 214, 107.0), speed=30.0, readout_s=0.05,
                             yaw_rate=1.0)
    gl = _crop(pin, 320, 180, 170.0)
    S = sg.Scene(sc)
    a = rs_render(sg, sc, rs, S)
    Cg = sg.Camera(gl)
    b = sg.render_camera(S, Cg, gl.c2w)
    torch.cuda.synchronize()
    Cr = sg.Camera(rs)
    rows = torch.from_numpy(np.ascontiguousarray(rs.row_c2w, np.float32)).cuda()
    ss = [torch.cuda.Stream(), torch.cuda.Stream()]
    frames = [sg.Frame(), sg.Frame()]
    outs = []
    for c in (rs, gl):
        outs.append([torch.full((c.height, c.width, 3), -7.0, device="cuda"),
                     torch.full((c.height, c.width), -7.0, device="cuda"),
                     torch.full((c.height, c.width), -7.0, device="cuda")])
    torch.cuda.synchronize()
    views = sg.sg_camera_views([
        (Cr.handle, rs.c2w, frames[0].handle, *[t.data_ptr() for t in outs[0]], ss[0].cuda_stream,
         rows.data_ptr()),
        (Cg.handle, gl.c2w, frames[1].handle, *[t.data_ptr() for t in outs[1]], ss[1].cuda_stream)])
    sg.sg_render_cameras(S.handle, views, sg.sg_default_opts(), 0)
    torch.cuda.synchronize()
    assert np.array_equal(outs[0][0].cpu().numpy(), a["rgb"])
    assert np.array_equal(outs[0][2].cpu().numpy(), a["depth"])
    assert np.array_equal(outs[1][0].cpu().numpy(), b["rgb"].cpu().numpy())
