"""The request server: requests that arrive while others run are admitted as
slots and memory free up, run concurrently on separate streams (waiting
requests of the same combination batched into one launch sequence), and
each result equals the same request rendered alone (bit for bit: the forward
pass is deterministic)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def W():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_12901_gb300 import _build
    _build.build()
    from paper_2510_12901_gb300 import serve
    return serve.ServingWorkload(sizes=(20_000, 60_000), n_requests=48, seed=11, ring=1,
                                 pinhole=(320, 240), fisheye=(256, 192))


def _outs(W, i):
    import torch
    name = W.KINDS[W.kinds[i]]
    if name in W.cams:
        c = W.cams[name][0]
        return [torch.full((c.height, c.width, 3), -7.0, device="cuda"),
                torch.full((c.height, c.width), -7.0, device="cuda"),
                torch.full((c.height, c.width), -7.0, device="cuda")]
    L = W.lidars[name][0]
    return [torch.full((L.n_beams, L.n_cols), -7.0, device="cuda") for _ in range(4)]


@pytest.fixture(scope="module")
def alone(W):
    """Every request rendered alone through the plain render call, into a
    frame that keeps no backward state, as the server's frames."""
    import torch
    from paper_2510_12901_gb300 import simgut as sg
    out = []
    fr = sg.Frame()
    sg.sg_frame_set_backward_state(fr.handle, 0)
    for i in range(len(W.kinds)):
        o = _outs(W, i)
        W.render_plain(i, fr, torch.cuda.current_stream().cuda_stream, outs=o)
        out.append(o)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("graphs,max_batch", [(False, 1), (True, 1), (False, 4), (True, 4)])
def test_results_identical_alone_and_in_the_mix(W, alone, graphs, max_batch):
    """Three bursts of the whole request stream.  With graphs, the first
    batch of each combination on a slot renders exactly, the second
    captures, the rest replay; with batching, requests of one combination
    that wait together render as one batch.  Every result must equal the
    alone render."""
    import torch
    from paper_2510_12901_gb300 import serve
    n = len(W.kinds)
    srv = serve.Server(n_slots=4, use_graphs=graphs, max_batch=max_batch)
    for burst in range(3):
        mixed = [_outs(W, i) for i in range(n)]
        tickets = [srv.submit(W.request(i, outs=mixed[i])) for i in range(n)]
        for t in tickets:
            srv.wait(t, 120.0)
        for i in range(n):
            for a, b in zip(alone[i], mixed[i]):
                assert torch.equal(a, b), (burst, i, W.KINDS[W.kinds[i]])
    st = srv.stats()
    srv.close()
    assert st["completed"] == 3 * n and st["failed"] == 0
    assert st["peak_in_flight"] > 1            # requests really overlapped
    if max_batch > 1:                          # bursts queue up: batches form
        assert st["batches"] > 0 and st["batched_requests"] >= 2 * st["batches"]
    else:
        assert st["batches"] == 0
    assert st["latency_p99_ms"] >= st["latency_p50_ms"] > 0
    if graphs:
        # one graph per slot, combination and batch size: with batching,
        # three bursts capture many and replay a few of them
        assert st["graph_captures"] >= 8
        assert st["graph_replays"] >= (n if max_batch == 1 else 1)
        assert st["overflow_rerenders"] == 0
    else:
        assert st["graph_captures"] == 0 and st["graph_replays"] == 0


def test_capacity_mode_matches_exact_and_reports_overflow(W):
    """A render in capacity mode (no wait for the pair count) equals the
    exact render when the pairs fit, and reports the dropped pairs, without
    touching memory beyond its buffers, when they do not."""
    import torch
    from paper_2510_12901_gb300 import simgut as sg
    i = next(i for i in range(len(W.kinds)) if W.KINDS[W.kinds[i]] == "fisheye")
    st = torch.cuda.current_stream().cuda_stream
    fr = sg.Frame()
    ref = _outs(W, i)
    W.render_plain(i, fr, st, outs=ref)
    torch.cuda.synchronize()
    K = sg.sg_frame_stats(fr.handle)[0]
    with pytest.raises(sg.SimgutError):
        sg.sg_frame_dropped_pairs(fr.handle)       # exact mode: nothing to report
    sg.sg_frame_set_capacity(fr.handle, K + 1000)
    o = _outs(W, i)
    W.render_plain(i, fr, st, outs=o)
    torch.cuda.synchronize()
    assert sg.sg_frame_dropped_pairs(fr.handle) == (0, K)
    for a, b in zip(ref, o):
        assert torch.equal(a, b)
    sg.sg_frame_set_capacity(fr.handle, K // 2)
    o = _outs(W, i)
    W.render_plain(i, fr, st, outs=o)
    torch.cuda.synchronize()
    assert sg.sg_frame_dropped_pairs(fr.handle) == (K - K // 2, K // 2)
    assert all(torch.isfinite(t).all() for t in o)
    sg.sg_frame_set_capacity(fr.handle, 0)
    o = _outs(W, i)
    W.render_plain(i, fr, st, outs=o)
    torch.cuda.synchronize()
    for a, b in zip(ref, o):
        assert torch.equal(a, b)


def test_graph_replay_that_outgrows_its_capacity_is_rendered_exactly():
    """One slot, one (scene, camera) combination.  Two requests see nothing
    (the camera looks away), so the graph is captured with the minimum pair
    capacity; the next request looks at the scene, overflows that capacity
    on replay and must be rendered again exactly; the graph is then
    recaptured larger and replayed.  Every result equals the alone render."""
    import torch
    from paper_2510_12901_gb300 import serve
    from paper_2510_12901_gb300 import simgut as sg
    from paper_2510_12901_gb300 import synthetic as syn
    sc = syn.layered_scene()
    cam = syn.Camera(syn.CAMERA_PINHOLE, 320, 240, 300.0, 300.0, 160.0, 120.0,
                     np.zeros(4, np.float32), syn.tiny_camera().c2w)
    away = syn._look_c2w([0.0, -10.0, 0.0], [0.0, -1.0, 0.0], [0.0, 0.0, -1.0])
    S, C = sg.Scene(sc), sg.Camera(cam)
    poses = [away, away, cam.c2w, cam.c2w, cam.c2w]

    def outs():
        return [torch.full((240, 320, 3), -7.0, device="cuda"),
                torch.full((240, 320), -7.0, device="cuda"),
                torch.full((240, 320), -7.0, device="cuda")]

    alone = []
    fr = sg.Frame()
    sg.sg_frame_set_backward_state(fr.handle, 0)      # as the server's frames
    st = torch.cuda.current_stream().cuda_stream
    for p in poses:
        o = outs()
        sg.sg_render_camera(S.handle, C.handle, p, sg.sg_default_opts(), fr.handle,
                            *[t.data_ptr() for t in o], st)
        alone.append(o)
    torch.cuda.synchronize()
    assert sg.sg_frame_stats(fr.handle)[0] > 200_000      # far above the minimum capacity
    srv = serve.Server(n_slots=1)
    for p, ref in zip(poses, alone):
        o = outs()
        srv.wait(srv.submit(serve.Server.camera_request(S, C, p, o)), 60.0)
        for a, b in zip(ref, o):
            assert torch.equal(a, b)
    stt = srv.stats()
    srv.close()
    assert stt["completed"] == 5 and stt["failed"] == 0
    assert stt["overflow_rerenders"] == 1
    assert stt["graph_captures"] == 2 and stt["graph_replays"] == 1


def test_memory_admission_serialises_and_completes(W):
    from paper_2510_12901_gb300 import serve
    from paper_2510_12901_gb300 import simgut as sg
    # pinhole requests on the larger scene, with a budget of 1.5 times one
    # request's workspace (sg_workspace_bytes, the server's admission
    # estimate): one at a time is admitted even with four free slots
    idx = [i for i in range(len(W.kinds)) if W.kinds[i] == 0 and W.scene_of[i] == 1]
    assert len(idx) >= 3
    cs, _ = W.scenes[1]
    pin = W.cams["pinhole"][0]
    one = sg.sg_workspace_bytes(cs.handle, sg.REQ_CAMERA, pin.width * pin.height)
    srv = serve.Server(n_slots=4, memory_budget=int(1.5 * one))
    tickets = [srv.submit(W.request(i)) for i in idx]
    for t in tickets:
        srv.wait(t, 120.0)
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(idx) and st["peak_in_flight"] == 1
    # twice the budget admits two at a time
    srv = serve.Server(n_slots=4, memory_budget=int(2.5 * one))
    tickets = [srv.submit(W.request(i)) for i in idx]
    for t in tickets:
        srv.wait(t, 120.0)
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(idx) and st["peak_in_flight"] <= 2


def test_queue_full_and_wait_timeout(W):
    from paper_2510_12901_gb300 import serve
    from paper_2510_12901_gb300 import simgut as sg
    srv = serve.Server(n_slots=1, queue_capacity=1)
    t0 = srv.submit(W.request(0))
    busy = 0
    tickets = [t0]
    for i in range(1, 12):
        try:
            tickets.append(srv.submit(W.request(i)))
        except sg.SimgutError as e:
            assert e.status == -6            # SG_ERR_BUSY
            busy += 1
    assert busy > 0
    with pytest.raises(sg.SimgutError) as e:
        srv.wait(tickets[-1], 1e-6)          # not done within a microsecond
    assert e.value.status == -5              # SG_ERR_TIMEOUT
    for t in tickets:
        srv.wait(t, 120.0)
    srv.drain(60.0)
    srv.close()
