"""Device status channel and workspace queries, through the C-ABI.

The sort stages wait on one another's published counts (decoupled
look-back); every such wait is bounded.  The tests make a wait run out
without faulting anything: a testing hook withholds one tile's published
counts, so the next tile's wait is certain to end at a short polling limit.
The render must then report SG_ERR_TIMEOUT (from the call itself when the
depth stage gave up in exact mode, otherwise from sg_frame_status, the
host-output paths and the server), stay in bounds, and leave the context
usable: the next render, with the hook off, equals a render made before.
"""
import numpy as np
import pytest

from paper_2510_12901_gb300 import synthetic as syn

pytestmark = pytest.mark.gpu
TIMEOUT = -5
SPINS = 2000          # polling rounds before a wait gives up in these tests


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_12901_gb300 import _build
    _build.build()
    from paper_2510_12901_gb300 import simgut
    simgut.load()
    yield simgut
    simgut.sg_debug_lookback(0, simgut.LOOKBACK_NONE, -1)


@pytest.fixture()
def hook(sg):
    def set_(site, tile=0):
        sg.sg_debug_lookback(SPINS, site, tile)
    yield set_
    sg.sg_debug_lookback(0, sg.LOOKBACK_NONE, -1)


def _scene(sg):
    # 20000 Gaussians (5 compaction tiles) seen by a 256x256 camera with the
    # tiny camera's field of view: several radix tiles of pairs
    sc = syn.tiny_scene(n=20000, seed=2)
    cam = syn.tiny_camera()
    cam.width, cam.height, cam.cx, cam.cy, cam.fx, cam.fy = 256, 256, 128.0, 128.0, 240.0, 240.0
    return sc, cam


def _render(sg, S, C, cam, frame):
    import torch
    out = sg.render_camera(S, C, cam.c2w, frame=frame)
    torch.cuda.synchronize()
    return {k: out[k].cpu().numpy() for k in ("rgb", "alpha", "depth")}


def _same(a, b):
    return all(np.array_equal(a[k], b[k]) for k in ("rgb", "alpha", "depth"))


@pytest.mark.parametrize("site", ["COMPACT", "DEPTH_SORT", "OFFSETS"])
def test_depth_stage_timeout_is_returned_by_the_render(sg, hook, site):
    sc, cam = _scene(sg)
    S, C = sg.Scene(sc), sg.Camera(cam)
    fr = sg.Frame()
    ref = _render(sg, S, C, cam, fr)
    K, _, _ = fr.stats()
    assert K > 2 * 8192 and ref["alpha"].max() > 0.5
    hook(getattr(sg, "LOOKBACK_" + site), 0)
    with pytest.raises(sg.SimgutError) as e:
        _render(sg, S, C, cam, fr)
    assert e.value.status == TIMEOUT and "gave up" in str(e.value)
    sg.sg_debug_lookback(0, sg.LOOKBACK_NONE, -1)
    # the context is intact and the frame renders as before
    assert _same(_render(sg, S, C, cam, fr), ref)
    sg.sg_frame_status(fr.handle)


def test_tile_sort_timeout_is_reported_by_frame_status(sg, hook):
    import torch
    sc, cam = _scene(sg)
    S, C = sg.Scene(sc), sg.Camera(cam)
    fr = sg.Frame()
    ref = _render(sg, S, C, cam, fr)
    hook(sg.LOOKBACK_TILE_SORT, 0)
    out = _render(sg, S, C, cam, fr)          # the call itself cannot know yet
    with pytest.raises(sg.SimgutError) as e:
        sg.sg_frame_status(fr.handle, torch.cuda.current_stream().cuda_stream)
    assert e.value.status == TIMEOUT
    # every list was left empty: the render shows nothing, and stayed in bounds
    assert out["alpha"].max() == 0.0 and out["rgb"].max() == 0.0
    sg.sg_debug_lookback(0, sg.LOOKBACK_NONE, -1)
    assert _same(_render(sg, S, C, cam, fr), ref)
    sg.sg_frame_status(fr.handle, torch.cuda.current_stream().cuda_stream)


def test_host_output_render_reports_timeout(sg, hook):
    sc, cam = _scene(sg)
    S, C = sg.Scene(sc), sg.Camera(cam)
    fr = sg.Frame()
    opts = sg.sg_default_opts()
    rgb = np.zeros((cam.height, cam.width, 3), np.float32)
    alpha = np.zeros((cam.height, cam.width), np.float32)
    depth = np.zeros((cam.height, cam.width), np.float32)
    ptrs = [a.ctypes.data for a in (rgb, alpha, depth)]
    sg.sg_render_camera_host(S.handle, C.handle, cam.c2w, opts, fr.handle, *ptrs)
    ref = alpha.copy()
    hook(sg.LOOKBACK_TILE_SORT, 0)
    with pytest.raises(sg.SimgutError) as e:
        sg.sg_render_camera_host(S.handle, C.handle, cam.c2w, opts, fr.handle, *ptrs)
    assert e.value.status == TIMEOUT
    sg.sg_debug_lookback(0, sg.LOOKBACK_NONE, -1)
    sg.sg_render_camera_host(S.handle, C.handle, cam.c2w, opts, fr.handle, *ptrs)
    assert np.array_equal(alpha, ref)


def test_capacity_mode_timeout_is_reported_after_the_render(sg, hook):
    import torch
    sc, cam = _scene(sg)
    S, C = sg.Scene(sc), sg.Camera(cam)
    fr = sg.Frame()
    ref = _render(sg, S, C, cam, fr)
    K, _, _ = fr.stats()
    sg.sg_frame_set_capacity(fr.handle, K + 1000)
    hook(sg.LOOKBACK_COMPACT, 1)
    _render(sg, S, C, cam, fr)                # capacity mode: no host wait in the call
    with pytest.raises(sg.SimgutError) as e:
        sg.sg_frame_status(fr.handle, torch.cuda.current_stream().cuda_stream)
    assert e.value.status == TIMEOUT
    sg.sg_debug_lookback(0, sg.LOOKBACK_NONE, -1)
    assert _same(_render(sg, S, C, cam, fr), ref)
    dropped, kept = sg.sg_frame_dropped_pairs(fr.handle)
    assert dropped == 0 and kept == K
    sg.sg_frame_status(fr.handle, torch.cuda.current_stream().cuda_stream)


def test_lidar_timeout(sg, hook):
    import torch
    L = syn.street_lidar(n_cols=256)
    sc = syn.street_scene(20000, seed=1, kind="lidar", length=60.0)
    S, D = sg.Scene(sc), sg.Lidar(L)
    fr = sg.Frame()
    ref = sg.render_lidar(S, D, L.col_c2w, frame=fr)
    torch.cuda.synchronize()
    r_range = ref["range"].cpu().numpy()
    hook(sg.LOOKBACK_OFFSETS, 0)
    with pytest.raises(sg.SimgutError) as e:
        sg.render_lidar(S, D, L.col_c2w, frame=fr)
    assert e.value.status == TIMEOUT
    hook(sg.LOOKBACK_TILE_SORT, 0)
    out = sg.render_lidar(S, D, L.col_c2w, frame=fr)
    with pytest.raises(sg.SimgutError):
        sg.sg_frame_status(fr.handle, torch.cuda.current_stream().cuda_stream)
    assert out["alpha"].max().item() == 0.0
    sg.sg_debug_lookback(0, sg.LOOKBACK_NONE, -1)
    again = sg.render_lidar(S, D, L.col_c2w, frame=fr)
    torch.cuda.synchronize()
    assert np.array_equal(again["range"].cpu().numpy(), r_range)


def test_server_request_fails_with_timeout_and_the_next_one_succeeds(sg, hook):
    import torch
    from paper_2510_12901_gb300 import serve
    sc, cam = _scene(sg)
    S, C = sg.Scene(sc), sg.Camera(cam)
    fr = sg.Frame()
    sg.sg_frame_set_backward_state(fr.handle, 0)      # as the server's frames
    ref = _render(sg, S, C, cam, fr)
    outs = [torch.zeros((cam.height, cam.width, 3), device="cuda"),
            torch.zeros((cam.height, cam.width), device="cuda"),
            torch.zeros((cam.height, cam.width), device="cuda")]
    for graphs in (False, True):
        srv = serve.Server(n_slots=1, use_graphs=graphs)
        req = serve.Server.camera_request(S, C, cam.c2w, outs)
        for _ in range(3):          # graphs: exact, capacity + capture, then replays
            srv.wait(srv.submit(req))
        hook(sg.LOOKBACK_COMPACT, 0)
        with pytest.raises(sg.SimgutError) as e:
            srv.wait(srv.submit(req))
        assert e.value.status == TIMEOUT
        sg.sg_debug_lookback(0, sg.LOOKBACK_NONE, -1)
        srv.wait(srv.submit(req))
        assert np.array_equal(outs[1].cpu().numpy(), ref["alpha"])
        st = srv.stats()
        assert st["failed"] == 1
        srv.close()


def test_workspace_estimate_bounds_the_frame(sg):
    import torch
    cases = []
    sc, _ = _scene(sg)
    cases.append(("camera", sc, syn.tiny_camera()))
    street = syn.street_scene(200000, seed=4, kind="camera")
    fish, pin = syn.street_cameras()
    cases.append(("camera", street, fish))
    cases.append(("camera", street, pin))
    lsc = syn.street_scene(200000, seed=5, kind="lidar")
    cases.append(("lidar", lsc, syn.street_lidar()))
    cases.append(("lidar", lsc, syn.street_lidar(n_beams=64, n_cols=1024)))
    for kind, s, sensor in cases:
        S = sg.Scene(s)
        fr = sg.Frame()
        if kind == "camera":
            C = sg.Camera(sensor)
            sg.render_camera(S, C, sensor.c2w, frame=fr)
            rays = sensor.width * sensor.height
        else:
            D = sg.Lidar(sensor)
            sg.render_lidar(S, D, sensor.col_c2w, frame=fr)
            rays = sensor.n_beams * sensor.n_cols
        torch.cuda.synchronize()
        K, _, _ = fr.stats()
        assert K <= 4 * s.n       # inside the estimate's pair allowance
        est = sg.sg_workspace_bytes(S.handle, sg.REQ_CAMERA if kind == "camera" else
                                    sg.REQ_LIDAR, rays)
        have = sg.sg_frame_workspace_bytes(fr.handle)
        assert have <= est, (kind, have, est)
        assert est < 4 * have + (64 << 20), (kind, have, est)   # and not absurdly loose
    with pytest.raises(sg.SimgutError):
        sg.sg_workspace_bytes(S.handle, 7, 100)


def test_projection_bulk_copy_wait_reports_timeout(sg):
    """The camera projection stages the SH planes by bulk copies and waits for
    them with a bounded wait.  The hook makes the first wait give up at once:
    the render must report SG_ERR_TIMEOUT naming the bulk copy (a second,
    full wait still precedes every read, so nothing runs out of bounds), and
    the next render, hook off, equals one made before."""
    import torch
    sc = syn.street_scene(60000, seed=3, kind="camera")       # degree-3 SH features
    _, cam = syn.street_cameras()
    S, C = sg.Scene(sc), sg.Camera(cam)
    for forward_only in (False, True):
        fr = sg.Frame()
        if forward_only:
            sg.sg_frame_set_backward_state(fr.handle, 0)
        ref = _render(sg, S, C, cam, fr)
        assert ref["alpha"].max() > 0.5
        sg.sg_debug_bulk_wait(True)
        try:
            with pytest.raises(sg.SimgutError) as e:
                _render(sg, S, C, cam, fr)
        finally:
            sg.sg_debug_bulk_wait(False)
        assert e.value.status == TIMEOUT and "bulk-copy" in str(e.value)
        assert _same(_render(sg, S, C, cam, fr), ref)
        sg.sg_frame_status(fr.handle, torch.cuda.current_stream().cuda_stream)
