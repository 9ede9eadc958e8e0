"""sg_render_camera_static: the camera render that allocates no device
memory (its workspace is a fixed array inside the library), for callers that
cannot allocate while they run.  Called through the C-ABI twice in a row on
the same inputs; each result must match sg_render_camera's within the
tolerances of the other parity tests, and sizes beyond the array's limits
must be refused with a clear error.  The calls make no allocation of any
kind (the library's allocation counter and the device's free memory stay
put).  This file is collected last."""
import numpy as np
import pytest

from paper_2510_12901_gb300 import synthetic as syn
from tests import parity as par

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


def _static_render(sg, S, C, cam):
    import torch
    rgb = torch.full((cam.height, cam.width, 3), -1.0, device="cuda")
    alpha = torch.full((cam.height, cam.width), -1.0, device="cuda")
    depth = torch.full((cam.height, cam.width), -1.0, device="cuda")
    sg.sg_render_camera_static(S.handle, C.handle, cam.c2w, sg.sg_default_opts(),
                               rgb.data_ptr(), alpha.data_ptr(), depth.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return rgb.cpu().numpy(), alpha.cpu().numpy(), depth.cpu().numpy()


@pytest.mark.parametrize("kind", ["tiny", "fisheye-sh", "layered"])
def test_static_render_matches_allocating_render_twice(sg, kind):
    import torch
    if kind == "tiny":
        sc, cam = syn.tiny_scene(), syn.tiny_camera()
    elif kind == "layered":      # tile lists long enough to be split into segments
        sc, cam = syn.layered_scene(), syn.tiny_camera()
    else:
        sc = syn.street_scene(20000, seed=3, kind="camera", length=40.0)
        fish, _ = syn.street_cameras()
        cam = syn.Camera(fish.model, 256, 200, 90.0, 90.0, 128.0, 100.0, fish.k, fish.c2w)
    S, C = sg.Scene(sc), sg.Camera(cam)
    ref = sg.render_camera(S, C, cam.c2w)
    torch.cuda.synchronize()
    r_rgb, r_a, r_d = (ref[k].cpu().numpy() for k in ("rgb", "alpha", "depth"))
    for _ in range(2):
        rgb, a, d = _static_render(sg, S, C, cam)
        assert np.abs(rgb - r_rgb).max() <= par.TOL_ABS
        assert np.abs(a - r_a).max() <= par.TOL_ABS
        hit = r_a > 0
        assert np.all(np.abs(d - r_d)[hit] <= par.TOL_DEPTH_REL * r_d[hit])
        assert np.all(d[~hit] == 0)
        assert r_a.max() > 0.5     # the image is not empty


def test_static_render_refuses_oversized_inputs(sg):
    sc = syn.tiny_scene()
    cam = syn.tiny_camera()
    cam.width, cam.height, cam.cx, cam.cy = 300, 300, 150.0, 150.0
    S, C = sg.Scene(sc), sg.Camera(cam)
    with pytest.raises(sg.SimgutError) as e:
        _static_render(sg, S, C, cam)
    assert e.value.status == -1 and "static workspace" in str(e.value)
    big = syn.street_scene(40000, seed=1, kind="camera")
    with pytest.raises(sg.SimgutError) as e:
        _static_render(sg, sg.Scene(big), sg.Camera(syn.tiny_camera()), syn.tiny_camera())
    assert "static workspace" in str(e.value)


def test_static_render_allocates_nothing(sg):
    import torch
    sc, cam = syn.tiny_scene(), syn.tiny_camera()
    S, C = sg.Scene(sc), sg.Camera(cam)
    outs = [torch.zeros((cam.height, cam.width, 3), device="cuda"),
            torch.zeros((cam.height, cam.width), device="cuda"),
            torch.zeros((cam.height, cam.width), device="cuda")]
    st = torch.cuda.current_stream().cuda_stream
    ptrs = [t.data_ptr() for t in outs]
    # the first call may load the module that holds the array
    sg.sg_render_camera_static(S.handle, C.handle, cam.c2w, sg.sg_default_opts(), *ptrs, st)
    torch.cuda.synchronize()
    n0 = sg.sg_alloc_count()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        sg.sg_render_camera_static(S.handle, C.handle, cam.c2w, sg.sg_default_opts(), *ptrs, st)
    torch.cuda.synchronize()
    assert sg.sg_alloc_count() == n0
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_render_refuses_bad_options_and_poses(sg):
    sc, cam = syn.tiny_scene(), syn.tiny_camera()
    S, C = sg.Scene(sc), sg.Camera(cam)
    bad = [dict(ut_beta=float("nan")), dict(pose_iters=9), dict(beam_divergence=0.5),
           dict(alpha_min=0.0)]
    for kw in bad:
        with pytest.raises(sg.SimgutError) as e:
            sg.sg_render_camera_static(S.handle, C.handle, cam.c2w, sg.sg_default_opts(**kw),
                                       None, None, None, 0)
        assert e.value.status == -1, kw
    pose = np.array(cam.c2w, np.float32)
    pose[3] = np.inf
    with pytest.raises(sg.SimgutError) as e:
        sg.sg_render_camera_static(S.handle, C.handle, pose, sg.sg_default_opts(),
                                   None, None, None, 0)
    assert e.value.status == -1 and "finite" in str(e.value)


def test_static_render_refuses_too_many_pairs_then_recovers(sg):
    """Few Gaussians inside the size limits whose footprints cover most of a
    256x256 image: more pairs than the array holds.  The call stops after
    the depth stage with SG_ERR_OVERFLOW and writes no pairs; the next call
    within the limits still matches sg_render_camera."""
    import torch
    rng = np.random.default_rng(8)
    n = 3000
    big = syn.tiny_scene(n=n, seed=8)
    big.means[:] = np.stack([rng.uniform(-2, 2, n), rng.uniform(-4, -1, n),
                             rng.uniform(-2, 2, n)], 1).astype(np.float32)
    big.log_scales[:] = np.log(2.5)
    big.opacity[:] = 0.9
    cam = syn.tiny_camera()
    cam.width, cam.height, cam.cx, cam.cy, cam.fx, cam.fy = 256, 256, 128.0, 128.0, 90.0, 90.0
    S, C = sg.Scene(big), sg.Camera(cam)
    ref_fr = sg.Frame()
    sg.render_camera(S, C, cam.c2w, frame=ref_fr)
    torch.cuda.synchronize()
    assert ref_fr.stats()[0] > 262144
    with pytest.raises(sg.SimgutError) as e:
        _static_render(sg, S, C, cam)
    assert e.value.status == -4 and "static workspace" in str(e.value)
    sc, cam2 = syn.tiny_scene(), syn.tiny_camera()
    S2, C2 = sg.Scene(sc), sg.Camera(cam2)
    ref = sg.render_camera(S2, C2, cam2.c2w)
    torch.cuda.synchronize()
    rgb, a, d = _static_render(sg, S2, C2, cam2)
    assert np.abs(rgb - ref["rgb"].cpu().numpy()).max() <= par.TOL_ABS
    assert np.abs(a - ref["alpha"].cpu().numpy()).max() <= par.TOL_ABS
