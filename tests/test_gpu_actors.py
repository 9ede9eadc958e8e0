"""Dynamic actors (Sec. 3.1 scene graph) on the GPU against the oracle: the
Gaussians of car-sized actors have their means and rotations in the actor's
frame and are placed in the world by the actor's pose before projection;
their SH turn with the actor.  Forward (camera and LiDAR), backward (the
gradients in each Gaussian's own frame), and pose updates between renders."""
import numpy as np
import pytest

from paper_2510_12901_gb300 import synthetic as syn
from tests import parity as par
from tests.test_gpu_backward import (camera_backward, compare_grads, lidar_backward,
                                     upstream)
from tests.test_gpu_camera import check_projection
from tests.test_gpu_camera import gpu_render as cam_render
from tests.test_gpu_lidar import gpu_render as lid_render

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


def _actor_scene(n=60000, seed=8, kind="camera"):
    return syn.with_actors(syn.street_scene(n, seed=seed, kind=kind, length=40.0),
                           n_actors=8, frac=0.3, seed=seed)


@pytest.mark.parametrize("which", [0, 1])
def test_camera_with_actors_every_pixel(sg, O32, O64, which):
    sc = _actor_scene()
    fish, pin = syn.street_cameras()
    cam = _crop(fish, 320, 214, 107.0) if which == 0 else _crop(pin, 320, 180, 170.0)
    g = cam_render(sg, sc, cam)
    orc = O64.render_camera(sc, cam)
    info = par.compare_camera_rays(g["rgb"].reshape(-1, 3), g["alpha"].reshape(-1),
                                   g["depth"].reshape(-1), orc, label=f"actors-{which}")
    # the actors are in view and composite
    assert (orc["alpha"] > 0).mean() > 0.2, info
    check_projection(sg, g["frame"], sc, cam, O32, O64, f"actors-{which}")


@pytest.mark.parametrize("mode", ["saved", "forward"])
def test_lidar_with_actors_every_ray(sg, O64, mode):
    sc = _actor_scene(20000, seed=9, kind="lidar_sh")
    L = syn.street_lidar(n_cols=256, start_xyz=(20.0, 0.0, 1.8))
    g = lid_render(sg, sc, L, mode=mode)
    orc = O64.render_lidar(sc, L)
    info = par.compare_lidar_rays(g["range"], g["intensity"], g["drop"], g["alpha"], orc,
                                  max_excluded=0.02, label=f"actors-lidar-{mode}")
    assert (orc["alpha"] > 0).mean() > 0.2, info


def test_backward_with_actors(sg, O64):
    sc = _actor_scene(30000, seed=10)
    fish, _ = syn.street_cameras()
    cam = _crop(fish, 240, 160, 80.0)
    orc = O64.render_camera(sc, cam)
    g = upstream(orc, np.random.default_rng(3))
    Go = O64.backward_camera(sc, cam, *g)
    Gg = camera_backward(sg, sg.Scene(sc), sg.Camera(cam), cam, *g, sc.n, sc.features.shape[1])
    compare_grads(Gg, Go, "actors-camera")
    # LiDAR, SH^l features
    sc = _actor_scene(1500, seed=11, kind="lidar_sh")
    L = syn.street_lidar(n_cols=256, start_xyz=(20.0, 0.0, 1.8))
    orc = O64.render_lidar(sc, L)
    rng = np.random.default_rng(4)
    ok = ~par.ambiguous_rays(orc, lidar=True)
    n = len(orc)
    gl = [(0.05 * rng.normal(size=n)).astype(np.float32)] + \
         [rng.normal(size=n).astype(np.float32) for _ in range(3)]
    for a in gl:
        a[~ok] = 0
    Go = O64.backward_lidar(sc, L, *gl)
    Gg = lidar_backward(sg, sg.Scene(sc), sg.Lidar(L), L, gl, sc.n, sc.features.shape[1])
    compare_grads(Gg, Go, "actors-lidar")


def test_pose_updates_and_removing_actors(sg):
    """New poses take effect for the next render on the stream; the result
    equals a scene created with those poses.  Removing the actors gives the
    static scene."""
    import torch
    import dataclasses
    sc = _actor_scene(40000, seed=12)
    cam = _crop(syn.street_cameras()[1], 320, 180, 170.0)
    S = sg.Scene(sc)
    a = cam_render(sg, sc, cam, scene=S)
    moved = sc.actor_poses.copy()
    moved[:, 3] += 2.0                     # every actor 2 m further down the street
    S.set_actor_poses(moved)
    b = cam_render(sg, sc, cam, scene=S)
    fresh = cam_render(sg, dataclasses.replace(sc, actor_poses=moved), cam)
    assert not np.array_equal(a["rgb"], b["rgb"])
    for k in ("rgb", "alpha", "depth"):
        assert np.array_equal(b[k], fresh[k]), k
    S.set_actors(None, 0)
    c = cam_render(sg, sc, cam, scene=S)
    static = cam_render(sg, dataclasses.replace(sc, actor_of=None, actor_poses=None), cam)
    for k in ("rgb", "alpha", "depth"):
        assert np.array_equal(c[k], static[k]), k
    with pytest.raises(sg.SimgutError):
        S.set_actor_poses(moved)           # no actors any more
    bad = np.full(sc.n, 5, np.int32)
    with pytest.raises(sg.SimgutError):
        S.set_actors(bad, 3)               # index 5 >= 3 actors
    torch.cuda.synchronize()
