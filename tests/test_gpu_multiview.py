"""Several camera views of one scene in one call (sg_render_cameras): every
view's result equals the same view rendered alone by sg_render_camera, bit
for bit (the forward pass is deterministic), whether the views run on
separate streams or one, with device or host outputs."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rig():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_12901_gb300 import _build
    _build.build()
    from paper_2510_12901_gb300 import simgut as sg
    from paper_2510_12901_gb300 import synthetic as syn
    sc = syn.street_scene(150_000, seed=3, kind="camera")
    S = sg.Scene(sc)
    fish, pin = syn.street_cameras()
    # three views: the two street cameras and the pinhole moved and yawed
    specs = [fish, pin, syn.random_street_pose_camera(np.random.default_rng(5), pin)]
    cams = [sg.Camera(c) for c in specs]
    opts = sg.sg_default_opts()
    alone = []
    fr = sg.Frame()
    for ch, c in zip(cams, specs):
        o = [torch.full((c.height, c.width, 3), -7.0, device="cuda"),
             torch.full((c.height, c.width), -7.0, device="cuda"),
             torch.full((c.height, c.width), -7.0, device="cuda")]
        sg.sg_render_camera(S.handle, ch.handle, c.c2w, opts, fr.handle, o[0].data_ptr(),
                            o[1].data_ptr(), o[2].data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        alone.append([t.cpu().numpy() for t in o])
    return dict(sg=sg, S=S, specs=specs, cams=cams, opts=opts, alone=alone)


@pytest.mark.parametrize("streams", [1, 3])
def test_views_equal_alone_renders_device_outputs(rig, streams):
    import torch
    sg = rig["sg"]
    ss = [torch.cuda.Stream() for _ in range(streams)]
    frames = [sg.Frame() for _ in rig["cams"]]
    for rep in range(2):       # twice: the second reuses the frames' buffers
        outs, views = [], []
        for i, (ch, c, f) in enumerate(zip(rig["cams"], rig["specs"], frames)):
            o = [torch.full((c.height, c.width, 3), -7.0, device="cuda"),
                 torch.full((c.height, c.width), -7.0, device="cuda"),
                 torch.full((c.height, c.width), -7.0, device="cuda")]
            outs.append(o)
            views.append((ch.handle, c.c2w, f.handle, o[0].data_ptr(), o[1].data_ptr(),
                          o[2].data_ptr(), ss[i % streams].cuda_stream))
        torch.cuda.synchronize()
        sg.sg_render_cameras(rig["S"].handle, sg.sg_camera_views(views), rig["opts"], 0)
        torch.cuda.synchronize()
        for o, a in zip(outs, rig["alone"]):
            for t, ref in zip(o, a):
                assert np.array_equal(t.cpu().numpy(), ref)


def test_views_equal_alone_renders_host_outputs(rig):
    import torch
    sg = rig["sg"]
    ss = [torch.cuda.Stream() for _ in rig["cams"]]
    frames = [sg.Frame() for _ in rig["cams"]]
    host, views = [], []
    for i, (ch, c, f) in enumerate(zip(rig["cams"], rig["specs"], frames)):
        n = c.width * c.height
        # pinned rgb and depth, pageable alpha; depth of view 1 not asked for
        h = [torch.full((3 * n,), -7.0).pin_memory(), np.full(n, -7.0, np.float32),
             torch.full((n,), -7.0).pin_memory()]
        host.append(h)
        views.append((ch.handle, c.c2w, f.handle, h[0].data_ptr(), h[1].ctypes.data,
                      0 if i == 1 else h[2].data_ptr(), ss[i].cuda_stream))
    sg.sg_render_cameras(rig["S"].handle, sg.sg_camera_views(views), rig["opts"], 1)
    for i, (h, a) in enumerate(zip(host, rig["alone"])):
        assert np.array_equal(h[0].numpy(), a[0].reshape(-1))
        assert np.array_equal(h[1], a[1].reshape(-1))
        if i == 1:
            assert (h[2].numpy() == -7.0).all()
        else:
            assert np.array_equal(h[2].numpy(), a[2].reshape(-1))


def test_asynchronous_host_outputs_pipelined(rig):
    """host_outputs = 2: the call returns with the copies queued; three
    calls in a row on two frame sets (the host buffers of a call are read
    after the next call is queued, as a pipelined caller does) give every
    view's alone render, bit for bit; a bad mode is refused."""
    import torch
    sg = rig["sg"]
    ss = [torch.cuda.Stream() for _ in rig["cams"]]
    sets = []
    for _ in range(2):
        frames = [sg.Frame() for _ in rig["cams"]]
        host, views = [], []
        for i, (ch, c, f) in enumerate(zip(rig["cams"], rig["specs"], frames)):
            n = c.width * c.height
            h = [torch.full((3 * n,), -7.0).pin_memory(), torch.full((n,), -7.0).pin_memory(),
                 torch.full((n,), -7.0).pin_memory()]
            host.append(h)
            views.append((ch.handle, c.c2w, f.handle, h[0].data_ptr(), h[1].data_ptr(),
                          h[2].data_ptr(), ss[i].cuda_stream))
        sets.append((frames, host, sg.sg_camera_views(views)))
    for step in range(3):
        frames, host, views = sets[step % 2]
        sg.sg_render_cameras(rig["S"].handle, views, rig["opts"], 2)
        if step > 0:
            prev = (step - 1) % 2
            for f in sets[prev][0]:
                sg.sg_frame_sync_outputs(f.handle)
            for h, a in zip(sets[prev][1], rig["alone"]):
                for t, ref in zip(h, a):
                    assert np.array_equal(t.numpy(), ref.reshape(-1))
                    t.fill_(-7.0)
    for f in sets[0][0]:
        sg.sg_frame_sync_outputs(f.handle)
    for h, a in zip(sets[0][1], rig["alone"]):      # the third call's results
        for t, ref in zip(h, a):
            assert np.array_equal(t.numpy(), ref.reshape(-1))
    with pytest.raises(sg.SimgutError):
        sg.sg_render_cameras(rig["S"].handle, sets[0][2], rig["opts"], 3)


def test_single_view_host_call_matches(rig):
    import torch
    sg = rig["sg"]
    c, ch = rig["specs"][0], rig["cams"][0]
    n = c.width * c.height
    h = [torch.empty(3 * n).pin_memory(), torch.empty(n).pin_memory(), torch.empty(n).pin_memory()]
    f = sg.Frame()
    sg.sg_render_camera_host(rig["S"].handle, ch.handle, c.c2w, rig["opts"], f.handle,
                             h[0].data_ptr(), h[1].data_ptr(), h[2].data_ptr(),
                             torch.cuda.current_stream().cuda_stream)
    for t, ref in zip(h, rig["alone"][0]):
        assert np.array_equal(t.numpy(), ref.reshape(-1))


def test_bad_view_lists_are_refused(rig):
    sg = rig["sg"]
    ch, c = rig["cams"][0], rig["specs"][0]
    f = sg.Frame()
    shared = sg.sg_camera_views([(ch.handle, c.c2w, f.handle, 0, 0, 0, 0)] * 2)
    with pytest.raises(sg.SimgutError):
        sg.sg_render_cameras(rig["S"].handle, shared, rig["opts"], 0)
    sg.sg_render_cameras(rig["S"].handle, sg.sg_camera_views([]), rig["opts"], 0)   # no views: no-op


def test_stage_marks_place_views_on_one_time_line(rig):
    """sg_frame_marks: each view's five stage boundaries are non-decreasing,
    their differences are the view's sg_frame_timing stages, a frame against
    itself starts at 0, and views on two streams fall within the call."""
    import torch
    sg = rig["sg"]
    ss = [torch.cuda.Stream() for _ in range(2)]
    frames = [sg.Frame() for _ in rig["cams"][:2]]
    for f in frames:
        sg.sg_frame_set_timing(f.handle, 1)
    outs, views = [], []
    for i, (ch, c, f) in enumerate(zip(rig["cams"][:2], rig["specs"][:2], frames)):
        o = [torch.empty((c.height, c.width, 3), device="cuda"),
             torch.empty((c.height, c.width), device="cuda"),
             torch.empty((c.height, c.width), device="cuda")]
        outs.append(o)
        views.append((ch.handle, c.c2w, f.handle, o[0].data_ptr(), o[1].data_ptr(),
                      o[2].data_ptr(), ss[i].cuda_stream))
    torch.cuda.synchronize()
    sg.sg_render_cameras(rig["S"].handle, sg.sg_camera_views(views), rig["opts"], 0)
    torch.cuda.synchronize()
    m0 = sg.sg_frame_marks(frames[0].handle, frames[0].handle)
    m1 = sg.sg_frame_marks(frames[1].handle, frames[0].handle)
    assert m0[0] == 0.0
    for m, f in ((m0, frames[0]), (m1, frames[1])):
        assert all(b >= a for a, b in zip(m, m[1:]))
        st = sg.sg_frame_timing(f.handle)
        assert np.allclose(np.diff(m), st, atol=2e-3)
    # both views ran within one call: neither starts after the other ends
    assert m1[0] < m0[4] and m1[4] > 0.0
