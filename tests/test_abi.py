"""The C-ABI library loads and exports every entry point of include/simgut.h
(no GPU needed: only argument checks that return before any CUDA work)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sg():
    from paper_2510_12901_gb300 import _build
    _build.build()
    from paper_2510_12901_gb300 import simgut
    simgut.load()
    return simgut


def header_functions():
    src = open(os.path.join(ROOT, "include", "simgut.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sg_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(sg):
    names = header_functions()
    assert len(names) >= 25
    lib = C.CDLL(sg.LIB_PATH)
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the Python binding mirrors the same names
    assert sorted(sg.exported_symbols()) == names


def test_version_and_defaults(sg):
    assert sg.sg_cuda_arch() == 103
    assert sg.sg_version() >= 100
    o = sg.sg_default_opts()
    assert abs(o.alpha_min - 1 / 255) < 1e-9 and abs(o.alpha_max - 0.99) < 1e-7
    assert abs(o.t_min - 1e-4) < 1e-10 and o.pose_iters == 2 and o.cull == 1
    assert (o.ut_alpha, o.ut_beta, o.ut_kappa) == (1.0, 2.0, 0.0)


def test_invalid_arguments_are_rejected_before_any_cuda_work(sg):
    with pytest.raises(sg.SimgutError) as e:
        sg.sg_create_camera(7, 64, 64, 60, 60, 32, 32, [0, 0, 0, 0])
    assert e.value.status == -1
    with pytest.raises(sg.SimgutError):
        sg.sg_create_camera(0, 0, 64, 60, 60, 32, 32, [0, 0, 0, 0])
    with pytest.raises(sg.SimgutError):
        sg.sg_create_camera(1, 64, 64, -1.0, 60, 32, 32, [0, 0, 0, 0])
    with pytest.raises(sg.SimgutError):
        sg.sg_create_lidar([0.0, 1.0], 0, -180.0, 32, 16, 1600, 8)
    with pytest.raises(sg.SimgutError):
        sg.sg_create_lidar([0.0, 95.0], 64, -180.0, 32, 16, 1600, 8)
    # sensor limits, checked on the host before any device allocation
    with pytest.raises(sg.SimgutError):
        sg.sg_create_camera(0, 16385, 64, 60, 60, 32, 32, [0, 0, 0, 0])
    assert "size" in sg.sg_last_error()
    with pytest.raises(sg.SimgutError):       # Proc. 1 needs an elevation range
        sg.sg_create_lidar([5.0, 5.0, 5.0], 64, -180.0, 32, 16, 1600, 8)
    assert "equal" in sg.sg_last_error()
    with pytest.raises(sg.SimgutError):       # 64 x 65535 rays at one ray per tile
        sg.sg_create_lidar(np.linspace(-20.0, 10.0, 64), 65535, -180.0, 1, 1, 1600, 8)
    assert "65535" in sg.sg_last_error()
    lib = sg.load()
    h = C.c_void_p()
    assert lib.sg_create_scene(None, None, C.byref(h)) == -1
    d = sg.sg_gaussians_desc(10, None, None, None, None, None, sg.FEATURES_SH, 5)
    assert lib.sg_create_scene(C.byref(d), None, C.byref(h)) == -1
    assert "sh_degree" in sg.sg_last_error()
    d = sg.sg_gaussians_desc(10, None, None, None, None, None, sg.FEATURES_RGB, 0)
    assert lib.sg_create_scene(C.byref(d), None, C.byref(h)) == -1
    assert "NULL" in sg.sg_last_error()
    # frames are host objects until the first render
    fr = sg.sg_frame_create()
    with pytest.raises(sg.SimgutError):
        sg.sg_frame_field(fr, sg.FIELD_RECT)
    sg.sg_frame_destroy(fr)
    # render with NULL handles
    o = sg.sg_default_opts()
    assert lib.sg_render_camera(None, None, None, C.byref(o), None, None, None, None, None) == -1
    bad = sg.sg_default_opts(alpha_min=0.0)
    assert lib.sg_render_lidar(None, None, None, C.byref(bad), None, None, None, None, None,
                               None) == -1


def test_camera_view_lists_are_checked_before_any_cuda_work(sg):
    lib = sg.load()
    o = sg.sg_default_opts()
    assert lib.sg_render_cameras(None, -1, None, C.byref(o), 0) == -1
    assert lib.sg_render_cameras(None, 2, None, C.byref(o), 0) == -1
    fr = sg.sg_frame_create()
    v = sg.sg_camera_views([(None, np.eye(3, 4), fr, 0, 0, 0, 0)])
    assert lib.sg_render_cameras(None, 1, v, C.byref(o), 0) == -1     # NULL camera
    assert "NULL camera" in sg.sg_last_error()
    sg.sg_frame_destroy(fr)
    assert lib.sg_render_cameras(None, 0, None, C.byref(o), 0) == 0   # nothing to render


def test_camera_view_struct_layout(sg):
    # the C struct: handle, float[12], handle, three pointers, stream
    f = sg.sg_camera_view
    assert C.sizeof(f) == 104
    assert [getattr(f, n).offset for n in ("camera", "c2w", "frame", "rgb", "alpha", "depth",
                                           "stream", "row_c2w")] \
        == [0, 8, 56, 64, 72, 80, 88, 96]


def test_status_workspace_and_hook_arguments_are_checked(sg):
    lib = sg.load()
    # NULL scene, unknown kind, negative rays: refused before any CUDA work
    b = C.c_size_t()
    assert lib.sg_workspace_bytes(None, sg.REQ_CAMERA, 100, C.byref(b)) == -1
    assert lib.sg_frame_workspace_bytes(None, C.byref(b)) == -1
    assert lib.sg_frame_status(None, None) == -1
    fr = sg.sg_frame_create()
    assert lib.sg_frame_status(fr, None) == -1          # never rendered
    assert "not been rendered" in sg.sg_last_error()
    sg.sg_frame_destroy(fr)
    assert lib.sg_debug_lookback(0, 9, 0) == -1         # unknown site
    assert lib.sg_debug_lookback(0, sg.LOOKBACK_COMPACT, -2) == -1
    assert sg.sg_alloc_count() >= 0
