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
    amb = ((orc["m_alpha"] < MARGIN_ALPHA) | (orc["m_tmin"] < MARGIN_TMIN) |
           (orc["m_rect"] < mr) | (orc["m_tau"] < MARGIN_TAU) |
           (orc["m_order"] < MARGIN_ORDER))
    if lidar:   # a sort key whose column pose is within rounding of flipping
        amb |= orc["m_kpose"] < MARGIN_POSE_COLS
    return amb


def compare_camera_rays(rgb, alpha, depth, orc, max_excluded=0.01, label="", posed=False,
                        also_excluded=None):
    """rgb [n,3], alpha [n], depth [n] from the GPU for the rays of `orc`.
    posed: a rolling shutter (per-row poses), whose sort keys can flip with
    the row chosen for a mean, as for LiDAR columns."""
    amb = ambiguous_rays(orc, lidar=posed)
    if also_excluded is not None:
        amb = amb | also_excluded
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


def camera_rays_seeing(rays, W, gauss, rect_a, rect_b, pad=MARGIN_RECT_PX):
    """Which pixels (indices into the row-major image of width W) have
    their centre in the box of one of the Gaussians `gauss` by one of the
    rect arrays and not by the other (boxes padded by `pad` for "in" and
    shrunk by it for "out"): e.g. where the GPU and the oracle took
    different row poses for a sigma point."""
    rays = np.asarray(rays, np.int64)
    x = (rays % W).astype(np.float64) + 0.5
    y = (rays // W).astype(np.float64) + 0.5
    A = np.asarray(rect_a, np.float64)[gauss]
    B = np.asarray(rect_b, np.float64)[gauss]
    out = np.zeros(len(rays), bool)

    def inside(r, p):
        return ((x[:, None] >= r[None, :, 0] - p) & (x[:, None] <= r[None, :, 1] + p) &
                (y[:, None] >= r[None, :, 2] - p) & (y[:, None] <= r[None, :, 3] + p))

    for lo in range(0, len(A), 1024):
        a, b = A[lo:lo + 1024], B[lo:lo + 1024]
        out |= ((inside(a, pad) & ~inside(b, -pad)) | (inside(b, pad) & ~inside(a, -pad))).any(axis=1)
    return out


def lidar_rays_seeing(rays, L, gauss, rect_a, rect_b, pad=MARGIN_RECT_DEG):
    """Which rays (indices of the beam-major [n_beams, n_cols] grid) fall in
    the box of one of the Gaussians `gauss` by one of the two rect arrays
    [n, 4] and not by the other (any azimuth alias, boxes padded by `pad`
    for "in" and shrunk by it for "out"): the rays whose extent test such a
    Gaussian could decide either way, e.g. where the GPU and the oracle
    took different column poses for it."""
    rays = np.asarray(rays, np.int64)
    c = rays % L.n_cols
    az = L.az0_deg + (c + 0.5) * 360.0 / L.n_cols
    el = np.asarray(L.elevations_deg, np.float64)[rays // L.n_cols]
    A = np.asarray(rect_a, np.float64)[gauss]
    B = np.asarray(rect_b, np.float64)[gauss]
    out = np.zeros(len(rays), bool)

    def inside(r, p):
        m = (el[:, None] >= r[None, :, 2] - p) & (el[:, None] <= r[None, :, 3] + p)
        hit = np.zeros(m.shape, bool)
        for shift in (-360.0, 0.0, 360.0):
            a = az[:, None] + shift
            hit |= (a >= r[None, :, 0] - p) & (a <= r[None, :, 1] + p)
        return m & hit

    for lo in range(0, len(A), 2048):
        a, b = A[lo:lo + 2048], B[lo:lo + 2048]
        out |= ((inside(a, pad) & ~inside(b, -pad)) | (inside(b, pad) & ~inside(a, -pad))).any(axis=1)
    return out


def compare_lidar_rays(rng, inten, drop, alpha, orc, max_excluded=0.01, label="",
                       also_excluded=None):
    """also_excluded: rays whose result depends on a Gaussian whose
    projection is itself ambiguous (see lidar_rays_seeing)."""
    amb = ambiguous_rays(orc, lidar=True)
    if also_excluded is not None:
        amb = amb | also_excluded
    ok = ~amb
    from oracle import Oracle
    o_rng, o_int, o_drop = Oracle(64).lidar_decode(orc)     # Sec. 3.2 decode
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


def rect_band(P32, P64, floor, ulps, cond=None):
    """Per-Gaussian, per-edge band within which two float32 implementations
    of the box may disagree: the larger of 8x the disagreement between the
    oracle's float32 and double builds and `ulps` float32 ulps of the edge's
    magnitude plus the box's spread (sigma points far from the axis and near
    Gaussians amplify rounding), times an optional per-Gaussian condition
    factor, plus a small floor."""
    r32 = P32["rect"].astype(np.float64)
    r64 = P64["rect"]
    d = np.abs(r32 - r64)
    both = (P32["ut"] == 1) & (P64["ut"] == 1)
    d[~both] = 0.0
    sx = np.sqrt(np.maximum(P64["cov2d"][:, 0], 0.0))
    sy = np.sqrt(np.maximum(P64["cov2d"][:, 2], 0.0))
    spread = np.stack([sx, sx, sy, sy], 1)
    u = ulps * 2.0 ** -24 * (np.abs(r64) + spread)
    if cond is not None:
        u = u * cond[:, None]
    return floor + np.maximum(8.0 * d, u)


def lidar_condition(P64):
    """Amplification of rounding in a LiDAR box: sigma points at elevation e
    go through asin, whose slope is 1 / cos(e); the box's largest |elevation|
    (capped at 89 deg) bounds it.  About 1.1 in the beams' range, large only
    for Gaussians that reach towards the sensor's vertical axis."""
    e = np.minimum(np.maximum(np.abs(P64["rect"][:, 2]), np.abs(P64["rect"][:, 3])), 89.0)
    return 1.0 / np.cos(np.radians(e))


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
    band = rect_band(P32, P64, 2e-5, 16, lidar_condition(P64))
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


# Policy for the integer work, end to end (GPU against the float32 oracle):
# a Gaussian's tile range or count may differ only where the oracle reports a
# box edge within rounding of a tile (or culling-cell) boundary, and at most
# for MAX_RANGE_MISMATCH of the Gaussians; sort keys agree within
# MAX_KEY_ULPS float32 ulps.  The key is |mu - o| in float32: a difference,
# three squares, two sums and a square root, each rounded once, leave each
# implementation within about 1.5 ulps of the exact distance, so two of them
# may differ by 3.  The binning and sort are then checked bit-exactly on the
# GPU's own per-Gaussian results (rebin_exact).
MAX_RANGE_MISMATCH = 1e-4
MAX_KEY_ULPS = 3


def key_ulps(a, b):
    """Distance in float32 ulps between two arrays of positive floats."""
    ia = np.asarray(a, np.float32).view(np.int32).astype(np.int64)
    ib = np.asarray(b, np.float32).view(np.int32).astype(np.int64)
    return np.abs(ia - ib)


def range_mismatch(count, tiles, P32):
    """Gaussians whose GPU tile count or range differs from the oracle's."""
    o_count = np.where(P32["valid"] == 1, P32["count"], 0)
    return (count.astype(np.int64) != o_count) | ((o_count > 0) & (tiles != P32["tiles"]).any(1))


def rebin_exact(O32, sg, fr, n, ntx, nty, wrap, label=""):
    """Policy (i): the oracle's binning and (tile, depth, id) sort, fed the
    GPU's own per-Gaussian results (count, tile range, float32 key), must
    reproduce the GPU's pair list and every tile's range bit for bit."""
    P = np.zeros(n, dtype=O32.Proj)
    count = fr.field(sg.FIELD_COUNT, np.uint32)
    P["valid"] = (count > 0).astype(np.int32)
    P["count"] = count.astype(np.int32)
    P["tiles"] = fr.field(sg.FIELD_TILES, np.int32, 4)
    P["depth"] = fr.field(sg.FIELD_DEPTH, np.float32)
    ids = fr.field(sg.FIELD_PAIR_IDS, np.uint32)
    tl = fr.field(sg.FIELD_PAIR_TILES, np.uint32)
    rg = fr.field(sg.FIELD_RANGES, np.uint32, 2)
    o_ids, o_tl, o_rg = O32.bin_sort(P, ntx, nty, wrap)
    assert len(ids) == len(o_ids), (label, len(ids), len(o_ids))
    assert np.array_equal(ids, o_ids), label
    assert np.array_equal(tl, o_tl), label
    assert np.array_equal(rg, o_rg), label
    return len(ids)
