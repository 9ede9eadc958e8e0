"""sg_render_camera_static: the camera render that allocates no device
memory (its workspace is a fixed array inside the library), for callers that
cannot allocate while they run.  Called through the C-ABI twice in a row on
the same inputs; each result must match sg_render_camera's within the
tolerances of the other parity tests, and sizes beyond the array's limits
must be refused with a clear error.  This file is collected last."""
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
