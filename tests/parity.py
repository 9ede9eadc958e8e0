"""Helpers shared by the GPU parity tests: run the CUDA path through the
C-ABI binding, run the oracle on the same seeded inputs, and compare.

Tolerances (floating point), from the accuracy target of the renderer:
  RGB, alpha, LiDAR intensity, drop probability: max abs 1e-4
  depth / range: relative 1e-3 where alpha > 0
Integer work (tile ranges, counts, sorted lists) is compared bit-exactly
against the float32 oracle, the precision in which the kernels take those
decisions.  A ray or a Gaussian is excluded only when the oracle itself
reports that a decision lies within rounding distance of its threshold
(margins below); the excluded fraction is asserted to stay small.
"""
from __future__ import annotations

import numpy as np

# Decision margins under which float rounding may legitimately flip a choice.
# Each is about 10x the largest disagreement measured between the kernels
# and the double-precision oracle for the quantity it guards (alpha and T to
# ~1e-6 relative, tau to ~1e-6 m, box edges to 5e-4 px / 5e-5 deg).
MARGIN_ALPHA = 1e-5     # |alpha - alpha_min| / alpha_min
MARGIN_TMIN = 1e-5      # |T' - t_min| / t_min
MARGIN_TAU = 1e-5       # |tau_max| (metres)
MARGIN_ORDER = 5e-7     # relative gap of consecutive float32 sort keys (4 ulp)
MARGIN_RECT_PX = 1e-3   # pixels
MARGIN_RECT_DEG = 1e-4  # degrees
MARGIN_VALID = 1e-4     # relative margin of near / theta_max / opacity tests

TOL_ABS = 1e-4
TOL_DEPTH_REL = 1e-3


def ambiguous_rays(orc, lidar=False):
    mr = MARGIN_RECT_DEG if lidar else MARGIN_RECT_PX
    return ((orc["m_alpha"] < MARGIN_ALPHA) | (orc["m_tmin"] < MARGIN_TMIN) |
            (orc["m_rect"] < mr) | (orc["m_tau"] < MARGIN_TAU) |
            (orc["m_order"] < MARGIN_ORDER))


def compare_camera_rays(rgb, alpha, depth, orc, max_excluded=0.01, label=""):
    """rgb [n,3], alpha [n], depth [n] from the GPU for the rays of `orc`."""
    amb = ambiguous_rays(orc)
    ok = ~amb
    e_rgb = np.abs(rgb.astype(np.float64) - orc["out"]).max(axis=1)
    e_a = np.abs(alpha.astype(np.float64) - orc["alpha"])
    hit = orc["alpha"] > 0
    e_d = np.where(hit, np.abs(depth.astype(np.float64) - orc["depth"]) /
                   np.maximum(orc["depth"], 1e-12), np.abs(depth))
    bad = ok & ((e_rgb > TOL_ABS) | (e_a > TOL_ABS) | (e_d > TOL_DEPTH_REL))
    info = dict(rays=len(orc), excluded=int(amb.sum()), max_rgb=float(e_rgb[ok].max(initial=0)),
                max_alpha=float(e_a[ok].max(initial=0)), max_depth_rel=float(e_d[ok].max(initial=0)),
                bad=int(bad.sum()))
    assert amb.mean() <= max_excluded, (label, info)
    assert not bad.any(), (label, info, np.nonzero(bad)[0][:10])
    return info


def compare_lidar_rays(rng, inten, drop, alpha, orc, max_excluded=0.01, label=""):
    amb = ambiguous_rays(orc, lidar=True)
    ok = ~amb
    o_rng = orc["depth"]
    o_int = orc["out"][:, 0]
    o_drop = 1.0 / (1.0 + np.exp(orc["out"][:, 1] - orc["out"][:, 2]))
    hit = orc["alpha"] > 0
    e_r = np.where(hit, np.abs(rng - o_rng) / np.maximum(o_rng, 1e-12), np.abs(rng))
    e_i = np.abs(inten - o_int)
    e_p = np.abs(drop - o_drop)
    e_a = np.abs(alpha - orc["alpha"])
    bad = ok & ((e_r > TOL_DEPTH_REL) | (e_i > TOL_ABS) | (e_p > TOL_ABS) | (e_a > TOL_ABS))
    info = dict(rays=len(orc), excluded=int(amb.sum()), max_range_rel=float(e_r[ok].max(initial=0)),
                max_int=float(e_i[ok].max(initial=0)), max_drop=float(e_p[ok].max(initial=0)),
                max_alpha=float(e_a[ok].max(initial=0)), bad=int(bad.sum()))
    assert amb.mean() <= max_excluded, (label, info)
    assert not bad.any(), (label, info, np.nonzero(bad)[0][:10])
    return info


def _near_multiple(x, step, offset, tol):
    r = (x - offset) / step
    return np.abs(r - np.round(r)) * step < tol


def rect_band(P32, P64, floor, ulps):
    """Per-Gaussian, per-edge band within which two float32 implementations
    of the box may disagree: the larger of 8x the disagreement between the
    oracle's float32 and double builds and `ulps` float32 ulps of the edge's
    magnitude plus the box's spread (sigma points far from the axis and near
    Gaussians amplify rounding), plus a small floor."""
    r32 = P32["rect"].astype(np.float64)
    r64 = P64["rect"]
    d = np.abs(r32 - r64)
    both = (P32["ut"] == 1) & (P64["ut"] == 1)
    d[~both] = 0.0
    sx = np.sqrt(np.maximum(P64["cov2d"][:, 0], 0.0))
    sy = np.sqrt(np.maximum(P64["cov2d"][:, 2], 0.0))
    spread = np.stack([sx, sx, sy, sy], 1)
    return floor + np.maximum(8.0 * d, ulps * 2.0 ** -24 * (np.abs(r64) + spread))


MARGIN_POSE_COLS = 3e-4   # LiDAR: sigma point within ~4 float32 ulps (at 180 deg) of a column boundary


def _near(x, step, offset, tol):
    r = (x - offset) / step
    return np.abs(r - np.round(r)) * step < tol


def tile_ambiguous_camera(P32, P64, W, H, tile=16):
    """Gaussians whose tile range or cull decision could flip under rounding."""
    rect = P32["rect"].astype(np.float64)
    band = rect_band(P32, P64, 2e-4, 128)
    amb = (P32["ut"] != P64["ut"]) | (P32["vmargin"] < MARGIN_VALID)
    ut = P64["ut"] == 1
    for k in range(4):
        x, t = rect[:, k], band[:, k]
        lim = W if k < 2 else H
        amb |= ut & (_near(x, tile, 0.0, t) | (np.abs(x - lim) < t) | (np.abs(x) < t))
    return amb, band


def tile_ambiguous_lidar(P32, P64, T, n_theta, az0, A, per):
    rect = P32["rect"].astype(np.float64)
    band = rect_band(P32, P64, 2e-5, 16)
    amb = (P32["ut"] != P64["ut"]) | (P32["vmargin"] < MARGIN_VALID)
    ut = P64["ut"] == 1
    amb |= ut & (P64["pmargin"] < MARGIN_POSE_COLS)
    for k in (0, 1):
        x, t = rect[:, k], band[:, k]
        amb |= ut & (_near(x, 360.0 / n_theta, az0, t) | _near(x, 360.0 / A, az0, t))
    Tb = T.astype(np.float64)
    for k in (2, 3):
        x, t = rect[:, k], band[:, k]
        amb |= ut & (np.abs(x[:, None] - Tb[None, :]).min(axis=1) < t)
        for j in range(len(Tb) - 1):     # dense sub-cells within each elevation tile
            w = Tb[j + 1] - Tb[j]
            if w <= 0:
                continue
            inside = (x >= Tb[j]) & (x <= Tb[j + 1])
            amb |= ut & inside & _near(x, w / per, Tb[j], t)
    amb |= ut & (np.abs(rect[:, 1] - rect[:, 0] - 360.0) < band[:, 0] + band[:, 1])
    return amb, band


def compare_lists(gpu_ids, gpu_ranges, orc_ids, orc_ranges, tiles, amb_gauss, depth_key,
                  label=""):
    """Per tile: same Gaussians (ambiguous ones removed) in the same order
    (near-tied float32 keys may swap)."""
    checked = 0
    for t in tiles:
        g = gpu_ids[gpu_ranges[t, 0]:gpu_ranges[t, 1]]
        o = orc_ids[orc_ranges[t, 0]:orc_ranges[t, 1]]
        g = g[~amb_gauss[g]]
        o = o[~amb_gauss[o]]
        assert np.array_equal(np.sort(g), np.sort(o)), (label, t, len(g), len(o))
        if not np.array_equal(g, o):
            # allowed only between keys within 4 float32 ulps of each other (the
            # kernels' keys agree with the oracle's to that)
            k = depth_key[o].astype(np.float32)
            pos_g = {int(x): i for i, x in enumerate(g)}
            for i in range(len(o)):
                if pos_g[int(o[i])] != i:
                    near = np.abs(k.view(np.int32).astype(np.int64) -
                                  np.int64(k[i].view(np.int32))) <= 4
                    assert near.sum() > 1, (label, t, i)
        checked += len(g)
    return checked
