"""Seeded synthetic inputs shaped like the driving captures of the paper.

This module holds no arithmetic of the rendering method itself: it only draws
Gaussian parameters, sensor intrinsics, beam tables and per-column poses.
Both the CUDA path (through the C-ABI) and the CPU oracle read the arrays it
returns, so the two sides always see bit-identical float32 inputs.

Workloads (the paper's Waymo / PandaSet scenes are not available; these stand
in for them, Sec. 4.1 and Sec. 4.2 of the paper):

* ``tiny_scene`` / ``tiny_camera``: 4096 Gaussians in a 20 m cube seen by a
  64x64 pinhole camera.
* ``street_scene``: a synthetic street (ground plane, two facade slabs,
  clutter) with surface-aligned, flattened Gaussians, 0.1 m-voxel-like scales
  (Sec. D initialises from 0.1 m voxels).  ``kind="camera"`` carries degree-3
  SH colour; ``kind="lidar"`` carries (intensity, beta_hit, beta_drop).
* ``street_cameras``: one 1920x1280 OpenCV-fisheye and one 1920x1080 pinhole
  camera at 1.6 m looking down the street.
* ``street_lidar``: a 128-beam spinning LiDAR with a nonuniform elevation table
  over -25..+15 deg, 2048 columns, and a per-column ego pose moving at 15 m/s
  with a 0.1 rad/s yaw rate over a 0.1 s sweep.

Seeds: 0 scenes, 1 sensors, 2 poses, 3 request streams, 4 loss targets.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

FEATURES_RGB = 0      # 3 floats per Gaussian, used directly as colour
FEATURES_SH = 1       # 3*(d+1)^2 floats per Gaussian, [n, (d+1)^2, 3]
FEATURES_LIDAR = 2    # 3 floats per Gaussian: intensity, beta_hit, beta_drop
FEATURES_LIDAR_SH = 3  # 3*(d+1)^2 floats: SH coefficients of those channels, [n, (d+1)^2, 3]

CAMERA_PINHOLE = 0
CAMERA_FISHEYE = 1


@dataclasses.dataclass
class Scene:
    means: np.ndarray        # [n, 3] float32, world metres
    log_scales: np.ndarray   # [n, 3] float32, log of the per-axis std-dev
    quats: np.ndarray        # [n, 4] float32, (w, x, y, z), not normalised
    opacity: np.ndarray      # [n] float32, already in (0, 1)
    features: np.ndarray     # [n, F] float32
    feature_kind: int
    sh_degree: int = 0
    # dynamic actors: per-Gaussian actor index (-1: static) and the actors'
    # poses [n_actors, 12] (row-major [R | t], actor to world), or None
    actor_of: Optional[np.ndarray] = None
    actor_poses: Optional[np.ndarray] = None

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.means[idx].copy(), self.log_scales[idx].copy(),
                     self.quats[idx].copy(), self.opacity[idx].copy(),
                     self.features[idx].copy(), self.feature_kind,
                     self.sh_degree,
                     None if self.actor_of is None else self.actor_of[idx].copy(),
                     None if self.actor_poses is None else self.actor_poses.copy())


@dataclasses.dataclass
class Camera:
    model: int
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    k: np.ndarray            # [4] float32, OpenCV fisheye k1..k4 (unused for pinhole)
    c2w: np.ndarray          # [12] float32, row-major 3x4 [R | t], OpenCV axes
    row_c2w: Optional[np.ndarray] = None   # [height, 12] per-row poses (rolling shutter)


@dataclasses.dataclass
class Lidar:
    elevations_deg: np.ndarray   # [n_beams] float32
    n_cols: int
    az0_deg: float               # azimuth of the left edge of column 0
    col_c2w: np.ndarray          # [n_cols, 12] float32, sensor-to-world per column
    max_rays_per_tile: int = 32  # M of the elevation-tiling procedure
    n_elev_tiles: int = 16       # N_phi
    cull_az: int = 1600          # dense culling cells over 360 deg of azimuth
    cull_el_per_tile: int = 8    # dense culling cells per elevation tile

    @property
    def n_beams(self) -> int:
        return int(self.elevations_deg.shape[0])


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _random_unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def _quat_mul(a, b):
    aw, ax, ay, az = a[..., 0], a[..., 1], a[..., 2], a[..., 3]
    bw, bx, by, bz = b[..., 0], b[..., 1], b[..., 2], b[..., 3]
    return np.stack([
        aw * bw - ax * bx - ay * by - az * bz,
        aw * bx + ax * bw + ay * bz - az * by,
        aw * by - ax * bz + ay * bw + az * bx,
        aw * bz + ax * by - ay * bx + az * bw,
    ], axis=-1)


def _small_rotation_quats(rng, n, sigma_rad):
    axis = rng.standard_normal((n, 3))
    axis /= np.linalg.norm(axis, axis=1, keepdims=True)
    ang = rng.normal(0.0, sigma_rad, size=n)
    q = np.empty((n, 4))
    q[:, 0] = np.cos(ang / 2)
    q[:, 1:] = axis * np.sin(ang / 2)[:, None]
    return q


def tiny_scene(seed: int = 0, n: int = 4096) -> Scene:
    """4096 Gaussians, means U([-10,10]^3), log-scales N(-1.5,0.5), random unit
    quaternions, opacity sigmoid(N(0,1)), RGB colour U[0,1]."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-10.0, 10.0, size=(n, 3))
    log_scales = rng.normal(-1.5, 0.5, size=(n, 3))
    quats = _random_unit_quats(rng, n)
    opacity = _sigmoid(rng.standard_normal(n))
    rgb = rng.uniform(0.0, 1.0, size=(n, 3))
    return Scene(means.astype(np.float32), log_scales.astype(np.float32),
                 quats.astype(np.float32), opacity.astype(np.float32),
                 rgb.astype(np.float32), FEATURES_RGB, 0)


def layered_scene(seed: int = 5, n: int = 20000) -> Scene:
    """Translucent layers in front of tiny_camera, for tile lists of several
    thousand entries whose rays reach T_min at different depths.

    n Gaussians at distances 3 + 27 (k + 1/2) / n m from the camera centre
    (k a random permutation of 0..n-1, so that no two depth keys are within
    rounding of each other), in directions (u, 1, -v) with u, v ~
    U(-0.55, 0.55); std-dev 0.15 x distance x U(0.6, 1.4) (second axis
    x U(0.7, 1.3)), random rotation, opacity 0.006 + 0.003 w U(0.5, 1.5) with
    w = (u + 0.55) / 1.1 rising from the left edge to the right; plus n/50
    opaque (U(0.8, 0.99)) small Gaussians at depth U(3, 4) over the upper-left
    quarter.  RGB colour U[0,1]."""
    rng = np.random.default_rng(seed)
    r = 3.0 + 27.0 * (rng.permutation(n) + 0.5) / n
    u = rng.uniform(-0.55, 0.55, n)
    v = rng.uniform(-0.55, 0.55, n)
    dirs = np.stack([u, np.ones(n), -v], 1)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    means = dirs * r[:, None] + np.array([0.0, -10.0, 0.0])
    s = 0.15 * r * rng.uniform(0.6, 1.4, n)
    log_scales = np.log(np.stack([s, s * rng.uniform(0.7, 1.3, n), s], 1))
    quats = _random_unit_quats(rng, n)
    w = (u + 0.55) / 1.1
    opacity = 0.006 + 0.003 * w * rng.uniform(0.5, 1.5, n)
    m = n // 50
    d2 = rng.uniform(3.0, 4.0, m)
    u2 = rng.uniform(-0.5, -0.1, m)
    v2 = rng.uniform(0.1, 0.5, m)
    means = np.concatenate([means, np.stack([u2 * d2, d2 - 10.0, -v2 * d2], 1)])
    s2 = np.log(0.05 * d2)
    log_scales = np.concatenate([log_scales, np.stack([s2, s2, s2], 1)])
    quats = np.concatenate([quats, _random_unit_quats(rng, m)])
    opacity = np.concatenate([opacity, rng.uniform(0.8, 0.99, m)])
    rgb = rng.uniform(0.0, 1.0, size=(n + m, 3))
    return Scene(means.astype(np.float32), log_scales.astype(np.float32),
                 quats.astype(np.float32), opacity.astype(np.float32),
                 rgb.astype(np.float32), FEATURES_RGB, 0)


def _look_c2w(eye, forward, down):
    """OpenCV camera-to-world: columns are the camera x (right), y (down) and
    z (forward) axes expressed in world coordinates."""
    z = np.asarray(forward, np.float64)
    z = z / np.linalg.norm(z)
    y = np.asarray(down, np.float64)
    y = y - z * np.dot(y, z)
    y = y / np.linalg.norm(y)
    x = np.cross(y, z)
    R = np.stack([x, y, z], axis=1)
    M = np.concatenate([R, np.asarray(eye, np.float64)[:, None]], axis=1)
    return M.reshape(12).astype(np.float32)


def tiny_camera() -> Camera:
    """64x64 pinhole, fx=fy=60, principal point at the image centre, on the
    y=-10 face of the cube looking +y with world +z up."""
    return Camera(CAMERA_PINHOLE, 64, 64, 60.0, 60.0, 32.0, 32.0,
                  np.zeros(4, np.float32),
                  _look_c2w([0.0, -10.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, -1.0]))


def street_scene(n: int, seed: int = 0, kind: str = "camera",
                 sh_degree: int = 3, length: float = 150.0) -> Scene:
    """Synthetic street along +x: 45% ground plane z=0 (|y|<=10), 45% facade
    slabs at y=+-12 (z in [0,15]), 10% clutter; positions jittered N(0,0.05).
    Scales log-normal around 5 cm with the surface-normal axis x0.2; rotations
    aligned with the surface plus N(0, 0.1 rad) jitter (clutter: random)."""
    rng = np.random.default_rng(seed)
    n_ground = int(round(0.45 * n))
    n_facade = int(round(0.45 * n))
    n_clutter = n - n_ground - n_facade
    means = np.empty((n, 3))
    base_q = np.empty((n, 4))
    flat = np.zeros(n, bool)
    # ground: local z axis = world z (normal)
    g = slice(0, n_ground)
    means[g, 0] = rng.uniform(0.0, length, n_ground)
    means[g, 1] = rng.uniform(-10.0, 10.0, n_ground)
    means[g, 2] = 0.0
    base_q[g] = [1.0, 0.0, 0.0, 0.0]
    flat[g] = True
    # facades: local z axis -> world y (rotate 90 deg about x)
    f = slice(n_ground, n_ground + n_facade)
    means[f, 0] = rng.uniform(0.0, length, n_facade)
    means[f, 1] = np.where(rng.uniform(size=n_facade) < 0.5, -12.0, 12.0)
    means[f, 2] = rng.uniform(0.0, 15.0, n_facade)
    c = math.cos(math.pi / 4)
    base_q[f] = [c, c, 0.0, 0.0]
    flat[f] = True
    # clutter
    cl = slice(n_ground + n_facade, n)
    means[cl, 0] = rng.uniform(0.0, length, n_clutter)
    means[cl, 1] = rng.uniform(-12.0, 12.0, n_clutter)
    means[cl, 2] = rng.uniform(0.0, 15.0, n_clutter)
    base_q[cl] = _random_unit_quats(rng, n_clutter)
    means += rng.normal(0.0, 0.05, size=(n, 3))

    quats = _quat_mul(base_q, _small_rotation_quats(rng, n, 0.1))
    quats[cl] = base_q[cl]
    log_scales = rng.normal(math.log(0.05), 0.5, size=(n, 3))
    log_scales[flat, 2] += math.log(0.2)

    if kind == "camera":
        opacity = _sigmoid(rng.standard_normal(n))
        nc = (sh_degree + 1) ** 2
        feats = rng.normal(0.0, 0.3, size=(n, nc * 3))
        scene = Scene(means, log_scales, quats, opacity, feats,
                      FEATURES_SH, sh_degree)
    elif kind in ("lidar", "lidar_sh"):
        hi = rng.uniform(size=n) < 0.7
        opacity = np.where(hi, _sigmoid(rng.normal(4.0, 1.0, n)),
                           _sigmoid(rng.normal(-4.0, 1.0, n)))
        feats = np.empty((n, 3))
        feats[:, 0] = rng.uniform(0.0, 1.0, n)
        feats[:, 1:] = rng.standard_normal((n, 2))
        if kind == "lidar":
            scene = Scene(means, log_scales, quats, opacity, feats,
                          FEATURES_LIDAR, 0)
        else:
            # SH^l: constant term about 3.5x the raw features (the degree-0
            # basis function is about 0.28), higher bands N(0, 0.3)
            nc = (sh_degree + 1) ** 2
            sh = rng.normal(0.0, 0.3, size=(n, nc, 3))
            sh[:, 0, :] = 3.5 * feats
            scene = Scene(means, log_scales, quats, opacity, sh.reshape(n, nc * 3),
                          FEATURES_LIDAR_SH, sh_degree)
    else:
        raise ValueError(kind)
    return Scene(scene.means.astype(np.float32),
                 scene.log_scales.astype(np.float32),
                 scene.quats.astype(np.float32),
                 scene.opacity.astype(np.float32),
                 scene.features.astype(np.float32),
                 scene.feature_kind, scene.sh_degree)


def actor_pose(x: float, y: float, yaw: float, z: float = 0.0) -> np.ndarray:
    """Row-major [R | t] of a rotation by `yaw` about +z and a translation."""
    c, s = math.cos(yaw), math.sin(yaw)
    return np.array([c, -s, 0.0, x, s, c, 0.0, y, 0.0, 0.0, 1.0, z], np.float32)


def with_actors(scene: Scene, n_actors: int = 16, frac: float = 0.1, seed: int = 3) -> Scene:
    """A copy of a street scene in which `frac` of the Gaussians belong to
    `n_actors` car-sized rigid actors: their means are redrawn on the surface
    of a 4.5 x 1.8 x 1.5 m box in the actor's frame (origin at the box's
    bottom centre), and the actors stand on the road at random headings."""
    rng = np.random.default_rng(seed)
    n = scene.n
    k = int(round(frac * n))
    idx = rng.choice(n, k, replace=False)
    actor_of = np.full(n, -1, np.int32)
    actor_of[idx] = rng.integers(0, n_actors, k)
    half = np.array([2.25, 0.9, 0.75])
    face = rng.integers(0, 3, k)
    side = np.where(rng.uniform(size=k) < 0.5, -1.0, 1.0)
    local = rng.uniform(-1.0, 1.0, (k, 3)) * half
    local[np.arange(k), face] = side * half[face]
    local[:, 2] += half[2]
    means = scene.means.copy()
    means[idx] = local.astype(np.float32)
    poses = np.stack([actor_pose(float(rng.uniform(5.0, 140.0)),
                                 float(rng.choice([-1.0, 1.0]) * rng.uniform(1.5, 6.0)),
                                 float(rng.uniform(-math.pi, math.pi)))
                      for _ in range(n_actors)])
    return dataclasses.replace(scene, means=means, actor_of=actor_of, actor_poses=poses)


def street_cameras(seed: int = 1, x: float = 0.0, y: float = 0.0):
    """(fisheye 1920x1280 fx=fy=640, k ~ U(-0.05,0.05); pinhole 1920x1080
    fx=fy=1000), both at (x, y, 1.6) looking +x along the street."""
    rng = np.random.default_rng(seed)
    k = rng.uniform(-0.05, 0.05, 4).astype(np.float32)
    c2w = _look_c2w([x, y, 1.6], [1.0, 0.0, 0.0], [0.0, 0.0, -1.0])
    fish = Camera(CAMERA_FISHEYE, 1920, 1280, 640.0, 640.0, 960.0, 640.0, k,
                  c2w.copy())
    pin = Camera(CAMERA_PINHOLE, 1920, 1080, 1000.0, 1000.0, 960.0, 540.0,
                 np.zeros(4, np.float32), c2w.copy())
    return fish, pin


def beam_table_128() -> np.ndarray:
    """128 beams over -25..+15 deg: 64 uniform in [-6,+2], 40 in [-25,-6),
    24 in (+2,+15]."""
    mid = np.linspace(-6.0, 2.0, 64)
    low = np.linspace(-25.0, -6.0, 41)[:-1]
    high = np.linspace(2.0, 15.0, 25)[1:]
    return np.sort(np.concatenate([low, mid, high])).astype(np.float32)


def beam_table_64() -> np.ndarray:
    """64 beams over -25..+15 deg: 32 uniform in [-6,+2], 20 below, 12 above."""
    mid = np.linspace(-6.0, 2.0, 32)
    low = np.linspace(-25.0, -6.0, 21)[:-1]
    high = np.linspace(2.0, 15.0, 13)[1:]
    return np.sort(np.concatenate([low, mid, high])).astype(np.float32)


def sweep_poses(n_cols: int, start_xyz, speed: float = 15.0,
                yaw0: float = 0.0, yaw_rate: float = 0.1,
                sweep_s: float = 0.1) -> np.ndarray:
    """Per-column sensor-to-world poses over one sweep: translation moves
    linearly along the heading at `speed`, heading turns at `yaw_rate`.
    Column c is taken at t = sweep_s * (c + 0.5) / n_cols.  Sensor axes:
    x forward, y left, z up."""
    t = sweep_s * (np.arange(n_cols) + 0.5) / n_cols
    yaw = yaw0 + yaw_rate * t
    out = np.zeros((n_cols, 12))
    cy, sy = np.cos(yaw), np.sin(yaw)
    out[:, 0], out[:, 1] = cy, -sy
    out[:, 4], out[:, 5] = sy, cy
    out[:, 10] = 1.0
    heading = np.array([math.cos(yaw0), math.sin(yaw0), 0.0])
    pos = np.asarray(start_xyz, np.float64)[None, :] + speed * t[:, None] * heading[None, :]
    out[:, 3], out[:, 7], out[:, 11] = pos[:, 0], pos[:, 1], pos[:, 2]
    return out.astype(np.float32)


def street_lidar(n_beams: int = 128, n_cols: int = 2048, seed: int = 2,
                 start_xyz=(30.0, 0.0, 1.8), static: bool = False,
                 max_rays_per_tile: int = 32, n_elev_tiles: int = 16) -> Lidar:
    """Spinning LiDAR on the street.  `static=True` repeats the first pose in
    every column (a sensor that does not move during the sweep)."""
    elev = beam_table_128() if n_beams == 128 else beam_table_64()
    poses = sweep_poses(n_cols, start_xyz)
    if static:
        poses[:] = poses[0]
    return Lidar(elev, n_cols, -180.0, poses, max_rays_per_tile, n_elev_tiles)


def rolling_shutter(cam: Camera, speed: float = 15.0, readout_s: float = 0.03,
                    yaw_rate: float = 0.1) -> Camera:
    """A copy of `cam` with a rolling shutter: row r is exposed at
    t_r = ((r + 0.5) / height - 0.5) readout_s around the frame's time, while
    the vehicle drives along +x at `speed` and turns about +z at `yaw_rate`."""
    base = np.asarray(cam.c2w, np.float64).reshape(3, 4)
    rows = np.empty((cam.height, 12), np.float32)
    for r in range(cam.height):
        t = ((r + 0.5) / cam.height - 0.5) * readout_s
        c, s_ = math.cos(yaw_rate * t), math.sin(yaw_rate * t)
        Rz = np.array([[c, -s_, 0.0], [s_, c, 0.0], [0.0, 0.0, 1.0]])
        P = np.concatenate([Rz @ base[:, :3], (base[:, 3] + np.array([speed * t, 0.0, 0.0]))[:, None]], 1)
        rows[r] = P.reshape(12)
    return dataclasses.replace(cam, row_c2w=rows)


def random_street_pose_camera(rng, cam: Camera) -> Camera:
    """A copy of `cam` moved to a random spot along the street (serving)."""
    x = float(rng.uniform(0.0, 100.0))
    y = float(rng.uniform(-3.0, 3.0))
    yaw = float(rng.uniform(-0.3, 0.3))
    c2w = _look_c2w([x, y, 1.6], [math.cos(yaw), math.sin(yaw), 0.0],
                    [0.0, 0.0, -1.0])
    return dataclasses.replace(cam, c2w=c2w)


def random_street_pose_lidar(rng, lidar: Lidar) -> Lidar:
    x = float(rng.uniform(10.0, 120.0))
    y = float(rng.uniform(-3.0, 3.0))
    yaw0 = float(rng.uniform(-math.pi, math.pi))
    poses = sweep_poses(lidar.n_cols, (x, y, 1.8), yaw0=yaw0)
    return dataclasses.replace(lidar, col_c2w=poses)


def noisy_targets(shape, seed: int = 4, lo: float = 0.0, hi: float = 1.0):
    """Seeded loss targets for the differentiable step (uniform noise)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=shape).astype(np.float32)
