"""Camera path on the GPU (through the C-ABI) against the CPU oracle.

Tiny cube scene: every pixel, every Gaussian, every tile list.  Street
scene (1M Gaussians, 1920x1280 OpenCV fisheye and 1920x1080 pinhole, the
benchmark's workload and launch configuration): every Gaussian's projection
and tile range, sampled tile lists and sampled rays (random pixels plus the
pixels of the longest tiles).  Plus edge cases.
"""
import numpy as np
import pytest

from paper_2510_12901_gb300 import synthetic as syn
from tests import parity as par

pytestmark = pytest.mark.gpu
SEG_LEN = 256       # the compositing's segment length (kSegLen in the library)


@pytest.fixture(scope="module")
def sg():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2510_12901_gb300 import _build
    _build.build()
    from paper_2510_12901_gb300 import simgut
    simgut.load()
    return simgut


# Frames that keep the state for a backward run k_render_camera; frames that
# keep none (serving, the benchmark) run k_render_camera_fwd, a different
# kernel (tangent-plane rays).  The parity tests run both.
MODES = ["saved", "forward"]


def gpu_render(sg, sc, cam, opts=None, scene=None, mode="saved"):
    import torch
    S = scene or sg.Scene(sc)
    C = sg.Camera(cam)
    fr = sg.Frame()
    if mode == "forward":
        sg.sg_frame_set_backward_state(fr.handle, 0)
    out = sg.render_camera(S, C, cam.c2w, opts, frame=fr)
    torch.cuda.synchronize()
    return dict(rgb=out["rgb"].cpu().numpy(), alpha=out["alpha"].cpu().numpy(),
                depth=out["depth"].cpu().numpy(), frame=out["frame"], cam=C, scene=S)


def check_projection(sg, fr, sc, cam, O32, O64, label):
    """Every Gaussian: box edges within the rounding band of the float32
    oracle's, tile count and range equal except where an edge lies within
    that band of a tile boundary (at most 0.01% of the Gaussians), sort
    keys within 2 float32 ulps."""
    P32, (ntx, nty) = O32.project_camera(sc, cam)
    P64, _ = O64.project_camera(sc, cam)
    count = fr.field(sg.FIELD_COUNT, np.uint32)
    tiles = fr.field(sg.FIELD_TILES, np.int32, 4)
    rect = fr.field(sg.FIELD_RECT, np.float32, 4)
    key = fr.field(sg.FIELD_DEPTH, np.float32)
    amb, band = par.tile_ambiguous_camera(P32, P64, cam.width, cam.height)
    v = (P64["ut"] == 1) & (P32["ut"] == 1)
    d = np.abs(rect[v].astype(np.float64) - P32["rect"][v])
    assert np.all(d <= band[v]), (label, d.max(), (d / band[v]).max())
    mism = par.range_mismatch(count, tiles, P32)
    assert not (mism & ~amb).any(), (label, np.nonzero(mism & ~amb)[0][:10])
    assert mism.mean() <= par.MAX_RANGE_MISMATCH, (label, int(mism.sum()))
    binned = (count > 0) | (P32["valid"] == 1)
    ku = par.key_ulps(key[binned], P32["depth"][binned])
    assert ku.max() <= par.MAX_KEY_ULPS, (label, int(ku.max()))
    return P32, mism, key, (ntx, nty)


def check_lists(sg, fr, sc, P32, mism, ntx, nty, O32, label):
    """Policy (i) on every tile, and the pair count against the oracle's
    own lists: equal up to the tiles of the Gaussians whose ranges differ."""
    K = par.rebin_exact(O32, sg, fr, sc.n, ntx, nty, False, label)
    assert K > 0
    o_count = np.where(P32["valid"] == 1, P32["count"], 0).astype(np.int64)
    g_count = fr.field(sg.FIELD_COUNT, np.uint32).astype(np.int64)
    assert K - o_count.sum() == (g_count - o_count)[mism].sum(), label


# ---------------------------------------------------------------- tiny cube
@pytest.mark.parametrize("mode", MODES)
def test_tiny_scene_every_pixel_and_list(sg, O32, O64, mode):
    sc, cam = syn.tiny_scene(), syn.tiny_camera()
    g = gpu_render(sg, sc, cam, mode=mode)
    orc = O64.render_camera(sc, cam)
    info = par.compare_camera_rays(g["rgb"].reshape(-1, 3), g["alpha"].reshape(-1),
                                   g["depth"].reshape(-1), orc, label="tiny")
    assert info["excluded"] <= 0.01 * len(orc)
    P32, mism, key, (ntx, nty) = check_projection(sg, g["frame"], sc, cam, O32, O64, "tiny")
    check_lists(sg, g["frame"], sc, P32, mism, ntx, nty, O32, "tiny")
    if mode == "forward":
        return
    # the saved state for the backward pass: T_final and omega = 1 - T_final
    st = g["frame"].field(sg.FIELD_RAY_STATE, np.float32, 4)
    assert np.allclose(1.0 - st[:, 0], g["alpha"].reshape(-1), atol=2e-6)
    assert np.array_equal(st[:, 1], g["alpha"].reshape(-1))


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("w,h", [(37, 23), (16, 16), (1, 1), (100, 3), (24, 13)])
def test_ragged_image_sizes(sg, O64, w, h, mode):
    sc, cam = syn.tiny_scene(), syn.tiny_camera()
    cam.width, cam.height, cam.cx, cam.cy = w, h, w / 2, h / 2
    g = gpu_render(sg, sc, cam, mode=mode)
    orc = O64.render_camera(sc, cam)
    par.compare_camera_rays(g["rgb"].reshape(-1, 3), g["alpha"].reshape(-1),
                            g["depth"].reshape(-1), orc, max_excluded=0.05,
                            label=f"{w}x{h}")


@pytest.mark.parametrize("mode", MODES)
def test_small_fisheye_with_rayless_corners(sg, O64, mode):
    sc = syn.tiny_scene()
    cam = syn.tiny_camera()
    cam.model = syn.CAMERA_FISHEYE
    cam.width, cam.height, cam.cx, cam.cy = 72, 56, 36.0, 28.0
    cam.fx = cam.fy = 18.0
    cam.k = np.array([0.03, -0.01, 0.004, -0.002], np.float32)
    g = gpu_render(sg, sc, cam, mode=mode)
    orc = O64.render_camera(sc, cam)
    corner = orc["n_visited"] == 0
    assert g["alpha"].reshape(-1)[0] == 0.0
    par.compare_camera_rays(g["rgb"].reshape(-1, 3), g["alpha"].reshape(-1),
                            g["depth"].reshape(-1), orc, label="fisheye-small")
    assert corner.any()


def test_forward_only_frame_falls_back_for_wide_tiles(sg, O64):
    """A fisheye whose single 16x16 tile spans nearly a hemisphere: some pixel
    is more than 75 degrees from the tile's reference direction, so the
    camera keeps no tangent-plane table and forward-only frames composite
    with the state-keeping kernel: bit-identical to a frame that keeps the
    state, and both match the oracle."""
    import torch
    sc = syn.tiny_scene()
    cam = syn.tiny_camera()
    cam.model = syn.CAMERA_FISHEYE
    cam.width, cam.height, cam.cx, cam.cy = 16, 16, 8.0, 8.0
    cam.fx = cam.fy = 2.5
    cam.k = np.zeros(4, np.float32)
    a = gpu_render(sg, sc, cam, mode="saved")
    b = gpu_render(sg, sc, cam, mode="forward", scene=a["scene"])
    for k in ("rgb", "alpha", "depth"):
        assert np.array_equal(a[k], b[k]), k
    orc = O64.render_camera(sc, cam)
    assert (orc["n_visited"] > 0).any()
    par.compare_camera_rays(b["rgb"].reshape(-1, 3), b["alpha"].reshape(-1),
                            b["depth"].reshape(-1), orc, max_excluded=0.05, label="wide-fisheye")


def test_empty_and_fully_culled_scenes(sg):
    sc, cam = syn.tiny_scene(), syn.tiny_camera()
    empty = sc.subset(np.zeros(0, np.int64))
    g = gpu_render(sg, empty, cam)
    assert not g["rgb"].any() and not g["alpha"].any() and not g["depth"].any()
    assert g["frame"].stats()[0] == 0
    behind = sc.subset(np.arange(100))
    behind.means[:, 1] = -30.0           # behind the camera at y = -10
    g = gpu_render(sg, behind, cam)
    assert not g["alpha"].any() and g["frame"].stats()[0] == 0
    faint = sc.subset(np.arange(100))
    faint.opacity[:] = 1.0 / 256.0        # below alpha_min: culled
    g = gpu_render(sg, faint, cam)
    assert not g["alpha"].any()


@pytest.mark.parametrize("mode", MODES)
def test_single_gaussian_on_axis(sg, O64, mode):
    cam = syn.tiny_camera()
    ok, o, d = O64.camera_ray(cam, 40, 21)
    sc = syn.tiny_scene(n=1)
    sc.means[0] = (o + 9.0 * d).astype(np.float32)
    sc.log_scales[0] = [-1, -1.2, -0.8]
    sc.opacity[0] = 0.9
    sc.features[0] = [0.2, 0.5, 0.9]
    g = gpu_render(sg, sc, cam, mode=mode)
    a = np.float32(0.9)
    assert np.allclose(g["rgb"][21, 40], a * sc.features[0], atol=1e-6)
    assert abs(g["depth"][21, 40] - np.linalg.norm(sc.means[0] - o)) < 1e-4


def test_host_output_path_matches_device_path(sg):
    import torch
    sc, cam = syn.tiny_scene(), syn.tiny_camera()
    g = gpu_render(sg, sc, cam)
    n = cam.width * cam.height
    h_rgb = np.zeros(3 * n, np.float32)
    h_a = np.zeros(n, np.float32)
    h_d = np.zeros(n, np.float32)
    fr = sg.Frame()
    sg.sg_render_camera_host(g["scene"].handle, g["cam"].handle, cam.c2w, sg.sg_default_opts(),
                             fr.handle, h_rgb.ctypes.data, h_a.ctypes.data, h_d.ctypes.data,
                             torch.cuda.current_stream().cuda_stream)
    assert np.array_equal(h_rgb.reshape(cam.height, cam.width, 3), g["rgb"])
    assert np.array_equal(h_a.reshape(cam.height, cam.width), g["alpha"])
    assert np.array_equal(h_d.reshape(cam.height, cam.width), g["depth"])


@pytest.mark.parametrize("mode", MODES)
def test_long_lists_composited_in_segments(sg, O64, mode):
    """Tile lists of 3.5k-7.7k entries: the compositing splits lists longer
    than SEG_LEN entries into independent segments (14 to 31 per tile) and
    combines them.  Rays stop at T_min in the first segment and in 20 or more
    later ones; others never stop."""
    sc, cam = syn.layered_scene(), syn.tiny_camera()
    g = gpu_render(sg, sc, cam, mode=mode)
    ranges = g["frame"].field(sg.FIELD_RANGES, np.uint32, 2)
    lens = ranges[:, 1].astype(np.int64) - ranges[:, 0]
    assert lens.max() > 28 * SEG_LEN and lens.min() > 12 * SEG_LEN
    orc = O64.render_camera(sc, cam)
    px = np.arange(cam.width * cam.height)
    tile = (px // cam.width // 16) * ((cam.width + 15) // 16) + (px % cam.width) // 16
    visited = orc["n_visited"].astype(np.int64)
    stopped = visited < lens[tile]
    seg = (visited - 1) // SEG_LEN
    per_seg = np.bincount(seg[stopped], minlength=32)
    assert per_seg[0] >= 500 and (per_seg[1:] >= 20).sum() >= 20, per_seg
    assert (~stopped & (visited > SEG_LEN)).sum() >= 500
    # thousands of threshold decisions per ray: 6.5% of the rays see one
    # within rounding of its threshold (3.1% alpha_min, 3.3% a box edge,
    # 0.1% T_min)
    par.compare_camera_rays(g["rgb"].reshape(-1, 3), g["alpha"].reshape(-1),
                            g["depth"].reshape(-1), orc, max_excluded=0.07, label="layered")
    if mode == "forward":
        return
    ok = ~par.ambiguous_rays(orc)
    st = g["frame"].field(sg.FIELD_RAY_STATE, np.float32, 4)
    assert np.abs(st[ok, 0] - orc["t_final"][ok]).max() <= par.TOL_ABS
    # the list position of the last composited entry: before the stopping
    # entry, and within the list
    last = g["frame"].field(sg.FIELD_N_CONTRIB, np.uint32).astype(np.int64)
    assert np.all(last[ok & stopped] < visited[ok & stopped])
    assert np.all(last <= lens[tile])


def test_forward_only_frame_agrees_and_refuses_the_backward(sg):
    import torch
    sc, cam = syn.tiny_scene(), syn.tiny_camera()
    a = gpu_render(sg, sc, cam)
    fr = sg.Frame()
    sg.sg_frame_set_backward_state(fr.handle, 0)
    b = sg.render_camera(a["scene"], a["cam"], cam.c2w, frame=fr)
    torch.cuda.synchronize()
    # another kernel and another ray parameterisation: equal up to rounding
    # away from threshold decisions (each is checked against the oracle above)
    for k in ("rgb", "alpha", "depth"):
        d = np.abs(a[k] - b[k].cpu().numpy())
        assert np.quantile(d, 0.99) <= 1e-5 and d.max() <= 0.05, (k, d.max())
    # a second forward-only render is bit-identical
    c = sg.render_camera(a["scene"], a["cam"], cam.c2w, frame=fr)
    torch.cuda.synchronize()
    for k in ("rgb", "alpha", "depth"):
        assert torch.equal(b[k], c[k]), k
    n = cam.width * cam.height
    grads = {k: torch.zeros(s, device="cuda") for k, s in
             (("m", (sc.n, 3)), ("l", (sc.n, 3)), ("q", (sc.n, 4)), ("o", (sc.n,)), ("f", (sc.n, 3)))}
    gs = sg.sg_grads(*[t.data_ptr() for t in grads.values()])
    up = torch.zeros(n * 3, device="cuda")
    with pytest.raises(sg.SimgutError) as e:
        sg.sg_backward_camera(a["scene"].handle, fr.handle, up.data_ptr(), None, None, gs,
                              torch.cuda.current_stream().cuda_stream)
    assert e.value.status == -1 and "kept no state" in str(e.value)
    sg.sg_frame_set_backward_state(fr.handle, 1)       # back on: the backward runs
    sg.render_camera(a["scene"], a["cam"], cam.c2w, frame=fr)
    sg.sg_backward_camera(a["scene"].handle, fr.handle, up.data_ptr(), None, None, gs,
                          torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()


def test_repeated_renders_are_deterministic(sg):
    sc, cam = syn.tiny_scene(), syn.tiny_camera()
    a = gpu_render(sg, sc, cam)
    b = gpu_render(sg, sc, cam, scene=a["scene"])
    assert np.array_equal(a["rgb"], b["rgb"]) and np.array_equal(a["depth"], b["depth"])


# ------------------------------------------------------------ street scene
@pytest.fixture(scope="module")
def street(sg):
    sc = syn.street_scene(1_000_000, seed=0, kind="camera")
    fish, pin = syn.street_cameras()
    S = sg.Scene(sc)
    return sc, S, {"fisheye": fish, "pinhole": pin}


def _sample_rays(sg, cam, g, n=3000, seed=0, heavy_tiles=3):
    rng = np.random.default_rng(seed)
    rays = rng.choice(cam.width * cam.height, n, replace=False)
    ranges = g["frame"].field(sg.FIELD_RANGES, np.uint32, 2)
    lens = ranges[:, 1].astype(np.int64) - ranges[:, 0]
    ntx = (cam.width + 15) // 16
    extra = []
    for t in np.argsort(-lens)[:heavy_tiles]:
        tx, ty = t % ntx, t // ntx
        for y in range(ty * 16, min(ty * 16 + 16, cam.height)):
            for x in range(tx * 16, min(tx * 16 + 16, cam.width)):
                extra.append(y * cam.width + x)
    return np.unique(np.concatenate([rays, np.array(extra, np.int64)])), lens


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("which", ["fisheye", "pinhole"])
def test_street_scene_sampled_parity(sg, O32, O64, street, which, mode):
    sc, S, cams = street
    cam = cams[which]
    g = gpu_render(sg, sc, cam, scene=S, mode=mode)
    rays, lens = _sample_rays(sg, cam, g)
    assert lens.max() > 256             # several shared-memory batches per tile
    orc = O64.render_camera(sc, cam, rays=rays)
    # the sample includes the three densest tiles (up to ~20k entries): a few
    # per cent of their rays see a decision within rounding of its threshold
    info = par.compare_camera_rays(g["rgb"].reshape(-1, 3)[rays], g["alpha"].reshape(-1)[rays],
                                   g["depth"].reshape(-1)[rays], orc, max_excluded=0.01,
                                   label=which)
    assert (orc["alpha"] > 0.5).mean() > 0.3, info     # the sample sees the scene
    if mode == "forward":
        return                  # the projection and the lists are the same stages
    P32, mism, key, (ntx, nty) = check_projection(sg, g["frame"], sc, cam, O32, O64, which)
    check_lists(sg, g["frame"], sc, P32, mism, ntx, nty, O32, which)
