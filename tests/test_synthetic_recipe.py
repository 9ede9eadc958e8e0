"""The synthetic inputs that stand in for the paper's driving captures
(Sec. 4.1, 4.2) follow the stated recipe: seeded and reproducible, with the
sizes, layouts and value distributions the benchmark and the parity tests
are quoted on.  CPU only."""
import math

import numpy as np

from paper_2510_12901_gb300 import synthetic as syn


def test_street_scene_layout_scales_and_features():
    n = 100_000
    sc = syn.street_scene(n, seed=0, kind="camera")
    assert sc.n == n and sc.feature_kind == syn.FEATURES_SH and sc.sh_degree == 3
    assert sc.features.shape == (n, 48)
    ng = nf = int(round(0.45 * n))
    ground, facade = sc.means[:ng], sc.means[ng:ng + nf]
    assert np.abs(ground[:, 2]).max() < 0.35 and np.abs(ground[:, 1]).max() < 10.35
    assert np.abs(np.abs(facade[:, 1]) - 12.0).max() < 0.35
    assert sc.means[:, 0].min() > -0.35 and sc.means[:, 0].max() < 150.35
    # scales log-normal around 5 cm; the surface normal's axis x 0.2 on ground and facades
    s = np.exp(sc.log_scales.astype(np.float64))
    assert abs(np.median(s[:, 0]) / 0.05 - 1.0) < 0.02
    assert abs(np.median(s[:ng + nf, 2]) / 0.01 - 1.0) < 0.03
    assert np.allclose(np.linalg.norm(sc.quats, axis=1), 1.0, atol=1e-5)
    assert abs(sc.features.std() - 0.3) < 0.005
    assert np.all((sc.opacity > 0) & (sc.opacity < 1))


def test_street_lidar_scene_opacity_is_bimodal():
    sc = syn.street_scene(50_000, seed=0, kind="lidar")
    assert sc.feature_kind == syn.FEATURES_LIDAR and sc.features.shape == (50_000, 3)
    assert abs((sc.opacity > 0.5).mean() - 0.7) < 0.01
    assert sc.features[:, 0].min() >= 0.0 and sc.features[:, 0].max() <= 1.0
    sh = syn.street_scene(5_000, seed=0, kind="lidar_sh")
    assert sh.feature_kind == syn.FEATURES_LIDAR_SH and sh.features.shape == (5_000, 48)


def test_inputs_are_reproducible_from_their_seeds():
    a, b = syn.street_scene(2000, seed=4), syn.street_scene(2000, seed=4)
    c = syn.street_scene(2000, seed=5)
    for f in ("means", "log_scales", "quats", "opacity", "features"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert not np.array_equal(a.means, c.means)
    t1, t2 = syn.tiny_scene(), syn.tiny_scene()
    assert np.array_equal(t1.means, t2.means) and t1.n == 4096


def test_street_cameras():
    fish, pin = syn.street_cameras()
    assert (fish.model, fish.width, fish.height, fish.fx) == (syn.CAMERA_FISHEYE, 1920, 1280, 640.0)
    assert (pin.model, pin.width, pin.height, pin.fx) == (syn.CAMERA_PINHOLE, 1920, 1080, 1000.0)
    assert np.all(np.abs(fish.k) <= 0.05) and not np.any(pin.k)
    for cam in (fish, pin):
        M = np.asarray(cam.c2w, np.float64).reshape(3, 4)
        assert np.allclose(M[:, 3], [0.0, 0.0, 1.6])
        assert np.allclose(M[:, 2], [1.0, 0.0, 0.0])        # looking +x along the street
        assert np.allclose(M[:, :3].T @ M[:, :3], np.eye(3), atol=1e-6)


def test_street_lidar_beams_and_sweep():
    L = syn.street_lidar()
    el = np.asarray(L.elevations_deg, np.float64)
    assert L.n_beams == 128 and L.n_cols == 2048 and L.az0_deg == -180.0
    assert el.min() == -25.0 and el.max() == 15.0 and np.all(np.diff(el) > 0)
    assert ((el >= -6.0) & (el <= 2.0)).sum() == 64
    assert (el < -6.0).sum() == 40 and (el > 2.0).sum() == 24
    assert (L.max_rays_per_tile, L.n_elev_tiles) == (32, 16)
    P = np.asarray(L.col_c2w, np.float64).reshape(-1, 3, 4)
    # 0.1 s sweep at 15 m/s and 0.1 rad/s: 1.5 m and 0.01 rad from the first column to the last
    moved = P[-1, :, 3] - P[0, :, 3]
    assert abs(np.linalg.norm(moved) - 1.5 * (2047 / 2048)) < 1e-3
    yaw = math.atan2(P[-1, 1, 0], P[-1, 0, 0]) - math.atan2(P[0, 1, 0], P[0, 0, 0])
    assert abs(yaw - 0.01 * (2047 / 2048)) < 1e-5
    assert np.allclose(P[0, :, 3], [30.0 + 15.0 * 0.1 * 0.5 / 2048, 0.0, 1.8], atol=1e-5)
    static = syn.street_lidar(static=True)
    assert np.array_equal(static.col_c2w[0], static.col_c2w[-1])
    L64 = syn.street_lidar(n_beams=64, n_cols=1024)
    assert L64.n_beams == 64 and L64.n_cols == 1024
