"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each checks a closed form, an
invariant, a textbook special case, a sampling estimate or a brute force.
Section / equation numbers refer to arXiv 2510.12901.
"""
import dataclasses
import math

import numpy as np
import pytest

from paper_2510_12901_gb300 import synthetic as syn


def rand_quats(rng, n):
    q = rng.standard_normal((n, 4)).astype(np.float32)
    return q


# ---------------------------------------------------------------- Sec. 3.1
def test_activation_rotation_is_proper(O64):
    rng = np.random.default_rng(5)
    q = rand_quats(rng, 200) * rng.uniform(0.2, 3.0, (200, 1)).astype(np.float32)
    ls = rng.normal(-1, 1, (200, 3)).astype(np.float32)
    R, s = O64.activate(ls, q)
    eye = np.einsum("nij,nkj->nik", R, R)
    assert np.abs(eye - np.eye(3)).max() < 1e-12
    assert np.abs(np.linalg.det(R) - 1).max() < 1e-12
    assert np.allclose(s, np.exp(ls.astype(np.float64)), rtol=1e-15)
    # rotation about z by 90 degrees (textbook)
    c = math.cos(math.pi / 4)
    R1, _ = O64.activate(np.zeros((1, 3), np.float32), np.array([[c, 0, 0, c]], np.float32))
    assert np.allclose(R1[0], [[0, -1, 0], [1, 0, 0], [0, 0, 1]], atol=1e-7)


# ------------------------------------------------- real spherical harmonics
def _sphere_quadrature(nt=24, nphi=48):
    x, w = np.polynomial.legendre.leggauss(nt)           # cos(theta) nodes
    phi = (np.arange(nphi) + 0.5) * 2 * np.pi / nphi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    wts = (w[:, None] * np.full(nphi, 2 * np.pi / nphi)[None, :]).reshape(-1)
    return dirs, wts


def test_sh_orthonormal_on_sphere(O64):
    dirs, wts = _sphere_quadrature()
    Y = np.stack([O64.sh_basis(d) for d in dirs])
    G = (Y * wts[:, None]).T @ Y
    assert np.abs(G - np.eye(16)).max() < 1e-12
    assert abs(Y[0, 0] - 0.5 / math.sqrt(math.pi)) < 1e-15   # Y_0^0 = 1/(2 sqrt(pi))


def test_sh_homogeneous_harmonic_and_gradient(O64):
    rng = np.random.default_rng(1)
    degree = np.array([0] + [1] * 3 + [2] * 5 + [3] * 7)
    h = 1e-3
    for _ in range(20):
        p = rng.normal(size=3)
        Y = O64.sh_basis(p)
        # homogeneous of degree l
        assert np.allclose(O64.sh_basis(2.0 * p), Y * 2.0 ** degree, rtol=1e-12, atol=1e-12)
        # Laplacian zero (central second differences are exact on cubics)
        lap = np.zeros(16)
        grad = np.zeros((16, 3))
        for k in range(3):
            e = np.zeros(3)
            e[k] = h
            lap += (O64.sh_basis(p + e) - 2 * Y + O64.sh_basis(p - e)) / h ** 2
            grad[:, k] = (O64.sh_basis(p + e) - O64.sh_basis(p - e)) / (2 * h)
        assert np.abs(lap).max() < 1e-6
        assert np.abs(grad - O64.sh_basis_grad(p)).max() < 1e-5


def test_sh_degree1_proportional_to_coordinates(O64):
    # Y_1^m = sqrt(3/(4 pi)) * (-y, z, -x)
    d = np.array([0.36, -0.48, 0.8])
    Y = O64.sh_basis(d)
    k = math.sqrt(3 / (4 * math.pi))
    assert np.allclose(Y[1:4], k * np.array([-d[1], d[2], -d[0]]), rtol=1e-14)


# ---------------------------------------------------------- camera models
def _cam(model, k=(0, 0, 0, 0), w=64, h=48, f=40.0):
    c = syn.tiny_camera()
    c.model, c.width, c.height = model, w, h
    c.fx = c.fy = f
    c.cx, c.cy = w / 2, h / 2
    c.k = np.array(k, np.float32)
    return c


def test_fisheye_k0_is_equidistant(O64):
    cam = _cam(1)
    # camera looks +y (world), x right; point at angle theta off-axis in x
    for th in [0.1, 0.5, 1.2]:
        xw = np.array([math.sin(th) * 5, -10 + math.cos(th) * 5, 0.0])
        ok, uv = O64.camera_project(cam, xw)
        assert ok
        assert abs((uv[0] - cam.cx) - cam.fx * th) < 1e-9
    assert abs(O64.fisheye_theta_max(np.zeros(4)) - math.pi / 2) < 1e-12


def test_fisheye_theta_max_first_critical_point(O64):
    # d theta_d / d theta = 1 + 3 k1 theta^2 = 0  at theta = sqrt(-1/(3 k1))
    k1 = np.float32(-0.2)
    tm = O64.fisheye_theta_max(np.array([k1, 0, 0, 0], np.float32))
    assert abs(tm - math.sqrt(-1 / (3 * float(k1)))) < 1e-9


@pytest.mark.parametrize("model,k", [(0, (0, 0, 0, 0)), (1, (0.03, -0.02, 0.01, -0.004)),
                                     (1, (-0.05, 0.05, -0.05, 0.05))])
def test_camera_ray_round_trip(O64, model, k):
    cam = _cam(model, k)
    rng = np.random.default_rng(3)
    for _ in range(30):
        px, py = int(rng.integers(0, cam.width)), int(rng.integers(0, cam.height))
        ok, o, d = O64.camera_ray(cam, px, py)
        if not ok:
            continue
        assert abs(np.linalg.norm(d) - 1) < 1e-12
        ok2, uv = O64.camera_project(cam, o + 7.0 * d)
        assert ok2
        assert abs(uv[0] - (px + 0.5)) < 1e-8 and abs(uv[1] - (py + 0.5)) < 1e-8


# ------------------------------------------------------ unscented transform
@pytest.mark.parametrize("a,b,k", [(1.0, 2.0, 0.0), (0.5, 2.0, 1.0), (1.3, 0.0, 0.5)])
def test_ut_exact_for_affine_maps(O64, a, b, k):
    rng = np.random.default_rng(7)
    A = rng.normal(size=(2, 3))
    c = rng.normal(size=2)
    mu = rng.normal(size=3)
    R, s = O64.activate(rng.normal(-1, .3, (1, 3)).astype(np.float32),
                        rng.normal(size=(1, 4)).astype(np.float32))
    R, s = R[0], s[0]
    ok, m, cov = O64.unscented(mu, R, s, lambda x, i: (True, A @ x + c),
                               opts=O64.opts(ut_alpha=a, ut_beta=b, ut_kappa=k))
    Sig = R @ np.diag(s ** 2) @ R.T
    C = A @ Sig @ A.T
    assert ok
    assert np.allclose(m, A @ mu + c, atol=1e-12)
    assert np.allclose(cov, [C[0, 0], C[0, 1], C[1, 1]], atol=1e-12)


def test_ut_exact_for_planar_gaussian_facing_pinhole(O64):
    """All sigma points at one depth: perspective is affine there, so the UT
    returns the projected mean and (f/z)^2 times the in-plane covariance."""
    cam = _cam(0)
    sc = syn.tiny_scene(n=1)
    # camera at (0,-10,0) looking +y; place the Gaussian 12 m ahead, off-axis
    sc.means[0] = [1.5, 2.0, -0.7]
    # local axes: x, z in the image plane, local y (scale ~0) along the view axis
    sc.quats[0] = [1, 0, 0, 0]
    sc.log_scales[0] = [math.log(0.4), -80.0, math.log(0.25)]
    sc.opacity[0] = 0.9
    P, _ = O64.project_camera(sc, cam)
    z0 = 12.0
    u = cam.fx * 1.5 / z0 + cam.cx
    v = cam.fy * 0.7 / z0 + cam.cy     # camera y (down) = -world z
    assert P["valid"][0] == 1
    assert np.allclose(P["mean2d"][0], [u, v], atol=1e-10)
    f2 = (cam.fx / z0) ** 2
    assert np.allclose(P["cov2d"][0], [f2 * 0.4 ** 2, 0.0, f2 * 0.25 ** 2], atol=1e-10)


def _jacobian(O, cam, xw):
    h = 1e-6
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        J[:, k] = (np.array(O.camera_project(cam, xw + e)[1]) -
                   np.array(O.camera_project(cam, xw - e)[1])) / (2 * h)
    return J


def test_ut_converges_to_linearisation(O64):
    """UT covariance -> J Sigma J^T (EWA) as the Gaussian shrinks, with a
    relative error that falls like s^2 (log-log slope 2)."""
    cam = _cam(0)
    mu = np.array([2.0, -4.0, 1.0])
    R, _ = O64.activate(np.zeros((1, 3), np.float32), np.array([[.9, .2, .3, .1]], np.float32))
    J = _jacobian(O64, cam, mu)
    errs = []
    for sc_ in [0.4, 0.2, 0.1, 0.05]:
        s = np.array([sc_, 0.7 * sc_, 0.5 * sc_])
        ok, m, cov = O64.unscented(mu, R[0], s, lambda x, i: O64.camera_project(cam, x))
        Sig = R[0] @ np.diag(s ** 2) @ R[0].T
        E = J @ Sig @ J.T
        C = np.array([[cov[0], cov[1]], [cov[1], cov[2]]])
        errs.append(np.linalg.norm(C - E) / np.linalg.norm(E))
    slopes = np.diff(np.log(errs)) / np.diff(np.log([0.4, 0.2, 0.1, 0.05]))
    assert np.all(np.abs(slopes - 2.0) < 0.25), slopes


def test_ut_matches_monte_carlo_moments_lidar(O64):
    """App. F / Tab. 6: 7 sigma points give moments close to Monte Carlo.
    Spherical map of Eq. 3 sampled with 10^6 points in double."""
    rng = np.random.default_rng(11)
    mu = np.array([8.0, 3.0, 1.0])
    R, s = O64.activate(np.log(np.array([[0.6, 0.3, 0.2]], np.float32)),
                        np.array([[0.8, 0.1, -0.4, 0.3]], np.float32))
    R, s = R[0], s[0]

    def sph(x, i=0):
        r = np.linalg.norm(x)
        return True, np.array([math.degrees(math.atan2(x[1], x[0])),
                               math.degrees(math.asin(x[2] / r))])

    ok, m, cov = O64.unscented(mu, R, s, sph, wrap_first=True)
    X = mu + (rng.standard_normal((1_000_000, 3)) * s) @ R.T
    az = np.degrees(np.arctan2(X[:, 1], X[:, 0]))
    el = np.degrees(np.arcsin(X[:, 2] / np.linalg.norm(X, axis=1)))
    Y = np.stack([az, el], 1)
    mc_m = Y.mean(0)
    mc_c = np.cov(Y.T)
    assert np.abs(m - mc_m).max() < 0.02 * np.sqrt(np.diag(mc_c)).max()
    C = np.array([[cov[0], cov[1]], [cov[1], cov[2]]])
    assert np.linalg.norm(C - mc_c) / np.linalg.norm(mc_c) < 0.03


# ------------------------------------------------------------ LiDAR set-up
def test_elevation_tiling_uniform_table_gives_equal_tiles(O64):
    elev = np.linspace(-10, 10, 128).astype(np.float32)
    T, nth = O64.elevation_tiling(elev, 2048, 16, 32)
    tiles = np.array([O64.elev_tile(T, 16, e) for e in elev])
    counts = np.bincount(tiles, minlength=16)
    assert counts.min() >= 7 and counts.max() <= 9
    assert T[0] == np.float32(-10) and T[-1] == np.float32(10)
    assert nth == -(-counts.max() * 2048 // 32)


@pytest.mark.parametrize("nphi,M", [(8, 32), (16, 32), (16, 64), (32, 128), (64, 256)])
def test_elevation_tiling_bounds(O64, nphi, M):
    """Rays per tile <= M whenever N_theta divides the column count; the tile
    beam counts differ by no more than the beams of one histogram bin
    (Fig. 3 caption); boundaries are non-decreasing and span the table."""
    elev = syn.beam_table_128()
    ncols = 2048
    T, nth = O64.elevation_tiling(elev, ncols, nphi, M)
    assert np.all(np.diff(T) >= 0)
    assert T[0] == elev.min() and T[-1] >= elev.max()
    tiles = np.array([O64.elev_tile(T, nphi, e) for e in elev])
    counts = np.bincount(tiles, minlength=nphi)
    hist = np.histogram(elev, bins=400, range=(float(elev.min()), float(elev.max())))[0]
    assert counts.max() * ncols <= nth * M
    assert counts.max() - counts[counts > 0].min() <= 2 * hist.max()
    cols_per_tile = np.bincount((np.arange(ncols) * nth) // ncols)
    assert cols_per_tile.max() * counts.max() <= M + counts.max()


def test_paper_best_setting_gives_32_ray_tiles(O64):
    L = syn.street_lidar()
    T, nth = O64.elevation_tiling(L.elevations_deg, L.n_cols, 16, 32)
    tiles = np.array([O64.elev_tile(T, 16, e) for e in L.elevations_deg])
    counts = np.bincount(tiles, minlength=16)
    assert counts.max() == 8 and nth == 512     # 8 beams x 4 columns = 32 rays


def test_sat_counts_match_brute_force(O64):
    L = syn.street_lidar(n_cols=256)
    S = O64.lidar_setup(L)
    sat = S["sat"]
    A, E = sat.shape[0] - 1, sat.shape[1] - 1
    cell = np.diff(np.diff(sat, axis=0), axis=1)       # per-cell counts
    assert set(np.unique(cell)) <= {0, 1}
    rng = np.random.default_rng(2)
    for _ in range(200):
        x0, x1 = sorted(rng.integers(0, A, 2))
        y0, y1 = sorted(rng.integers(0, E, 2))
        assert O64.sat_count_wrap(L, int(x0), int(x1), int(y0), int(y1)) == \
            cell[x0:x1 + 1, y0:y1 + 1].sum()
    # seam: [A-3, A+2] wraps to [A-3, A-1] + [0, 2]
    assert O64.sat_count_wrap(L, A - 3, A + 2, 0, E - 1) == \
        cell[A - 3:, :].sum() + cell[:3, :].sum()
    # every ray's cell is occupied: 256 columns over 1600 cells, all beams
    assert cell.sum() == 256 * len(np.unique([O64.lib.or_elev_cell(
        S["T"].ctypes.data_as(__import__("ctypes").c_void_p), 16, 8,
        O64.real(e)) for e in L.elevations_deg]))


def test_lidar_axis_point_maps_to_origin(O64):
    L = syn.street_lidar(static=True)
    L.col_c2w[:] = np.array([1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0], np.float32)
    sc = syn.tiny_scene(n=2)
    sc.means[0] = [10, 0, 0]
    sc.means[1] = [5 * math.cos(0.7), 5 * math.sin(0.7), 5 * math.tan(math.radians(3.0))]
    sc.log_scales[:] = -9
    sc.opacity[:] = 0.9
    P, _ = O64.project_lidar(sc, L, O64.opts(cull=0))
    assert np.allclose(P["mean2d"][0], [0, 0], atol=1e-6)
    assert abs(P["mean2d"][1][0] - math.degrees(0.7)) < 1e-6
    assert abs(P["mean2d"][1][1] - 3.0) < 1e-6
    assert abs(P["depth"][0] - 10) < 1e-12


# ------------------------------------------------------------ compositing
def _one_gaussian_scene(mu, ls, sigma, rgb, q=(1, 0, 0, 0)):
    sc = syn.tiny_scene(n=1)
    sc.means[0] = mu
    sc.log_scales[0] = ls
    sc.quats[0] = q
    sc.opacity[0] = sigma
    sc.features[0] = rgb
    return sc


def test_single_gaussian_on_axis_closed_form(O64):
    cam = syn.tiny_camera()
    ok, o, d = O64.camera_ray(cam, 40, 21)
    mu = (o + 9.0 * d).astype(np.float32)
    for sigma in [0.3, 0.9, 1.0]:
        sc = _one_gaussian_scene(mu, [-1, -1.2, -0.8], sigma, [0.2, 0.5, 0.9])
        r = O64.render_camera(sc, cam, rays=[21 * 64 + 40])[0]
        a = min(float(np.float32(0.99)), float(np.float32(sigma)))
        assert np.allclose(r["out"], a * np.array([0.2, 0.5, 0.9], np.float32), atol=1e-9)
        assert abs(r["alpha"] - a) < 1e-9
        assert abs(r["depth"] - np.linalg.norm(mu - o)) < 1e-5


def test_two_gaussians_over_operator(O64):
    cam = syn.tiny_camera()
    ok, o, d = O64.camera_ray(cam, 30, 30)
    sc = syn.tiny_scene(n=2)
    sc.means[0] = o + 6 * d
    sc.means[1] = o + 12 * d
    sc.log_scales[:] = -1.0
    sc.quats[:] = [1, 0, 0, 0]
    sc.opacity[:] = [0.6, 0.7]
    sc.features[:] = [[1, 0, 0], [0, 0, 1]]
    r = O64.render_camera(sc, cam, rays=[30 * 64 + 30])[0]
    a1, a2 = float(np.float32(0.6)), float(np.float32(0.7))
    assert np.allclose(r["out"], [a1, 0, (1 - a1) * a2], atol=1e-6)
    assert abs(r["alpha"] - (a1 + (1 - a1) * a2)) < 1e-6


def test_flat_opaque_disk_returns_ray_plane_distance(O64):
    """A disk-like Gaussian (scales a, a, 1e-5; opacity 1): tau_max equals
    the ray-plane distance (mu - o).n / (d.n) for every ray that hits it."""
    cam = syn.tiny_camera()
    n = np.array([0.3, -0.9, 0.2])
    n /= np.linalg.norm(n)
    # rotation whose third column is n
    z = n
    x = np.cross([0, 0, 1.0], z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    Rm = np.stack([x, y, z], 1)
    w = math.sqrt(1 + np.trace(Rm)) / 2
    q = [w, (Rm[2, 1] - Rm[1, 2]) / (4 * w), (Rm[0, 2] - Rm[2, 0]) / (4 * w),
         (Rm[1, 0] - Rm[0, 1]) / (4 * w)]
    mu = np.array([0.5, 4.0, 0.3], np.float32)
    sc = _one_gaussian_scene(mu, [math.log(3.0), math.log(3.0), math.log(1e-5)], 1.0,
                             [1, 1, 1], q)
    r = O64.render_camera(sc, cam)
    hit = r["n_contrib"] > 0
    assert hit.sum() > 500
    idx = np.nonzero(hit)[0]
    for i in idx[::17]:
        ok, o, d = O64.camera_ray(cam, i % 64, i // 64)
        nn = Rm[:, 2]
        t_plane = np.dot(mu.astype(np.float64) - o, nn) / np.dot(d, nn)
        assert abs(r["depth"][i] - t_plane) < 1e-5 * t_plane


# ------------------------------------------------ LiDAR closed forms (Sec. 3.2-3.3)
def _beam_dir(L, beam, col):
    """World direction and origin of LiDAR ray (beam, col), written out from
    the sensor model: column c at azimuth az0 + (c + 1/2) 360 / N_cols, beam b
    at its table elevation, u = (cos el cos az, cos el sin az, sin el) in the
    sensor frame, mapped by the column's pose."""
    az = math.radians(L.az0_deg + (col + 0.5) * 360.0 / L.n_cols)
    el = math.radians(float(L.elevations_deg[beam]))
    u = np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    P = np.asarray(L.col_c2w[col], np.float64).reshape(3, 4)
    return P[:, 3], P[:, :3] @ u


def _one_lidar_gaussian(mu, ls, sigma, feat, q=(1, 0, 0, 0)):
    sc = syn.street_scene(1, seed=0, kind="lidar")
    sc.means[0] = mu
    sc.log_scales[0] = ls
    sc.quats[0] = q
    sc.opacity[0] = sigma
    sc.features[0] = feat
    return sc


@pytest.mark.parametrize("beam,col", [(60, 100), (10, 7), (120, 250)])
def test_lidar_single_gaussian_on_a_beam_closed_form(O64, beam, col):
    """A small Gaussian centred on ray (beam, col) at distance r: the ray
    passes through its mean, so D = 0, alpha = min(0.99, sigma), range = r,
    intensity = alpha zeta_0, and the drop probability is the softmax of the
    accumulated (beta_hit, beta_drop) = alpha (b_hit, b_drop):
    1 / (1 + exp(alpha (b_hit - b_drop))).  The neighbouring columns pass
    half a column's angle or more beside it and see far less."""
    L = syn.street_lidar(n_cols=256)
    o, d = _beam_dir(L, beam, col)
    r = 9.0
    mu = (o + r * d).astype(np.float32)
    sigma, feat = 0.7, [0.42, 1.3, -0.6]          # b_hit != b_drop
    sc = _one_lidar_gaussian(mu, [math.log(0.01)] * 3, sigma, feat)
    ray = beam * L.n_cols + col
    out = O64.render_lidar(sc, L, rays=[ray, ray - 1, ray + 1])
    rg, it, dr = O64.lidar_decode(out)
    a = float(np.float32(sigma))
    f = np.asarray(feat, np.float32).astype(np.float64)
    assert abs(out["alpha"][0] - a) < 1e-6
    assert abs(rg[0] - np.linalg.norm(mu - o)) < 1e-6 * r
    assert abs(it[0] - a * f[0]) < 1e-6
    assert abs(dr[0] - 1.0 / (1.0 + math.exp(a * (f[1] - f[2])))) < 1e-6
    # swapping beta_hit and beta_drop would give the complementary probability
    assert abs(dr[0] - 0.5) > 0.1
    assert out["alpha"][1] < 0.01 * a and out["alpha"][2] < 0.01 * a


def test_lidar_flat_opaque_disk_returns_beam_plane_distance(O64):
    """A disk-like LiDAR Gaussian (scales a, a, 1e-5; opacity 1): every beam
    that hits it returns the distance along the beam to the disk's plane,
    ((mu - o) . n) / (d . n), with d the beam direction written out above."""
    L = syn.street_lidar(n_cols=512)
    n = np.array([-0.8, 0.3, 0.52])
    n /= np.linalg.norm(n)
    x = np.cross([0, 0, 1.0], n)
    x /= np.linalg.norm(x)
    y = np.cross(n, x)
    Rm = np.stack([x, y, n], 1)
    w = math.sqrt(1 + np.trace(Rm)) / 2
    q = [w, (Rm[2, 1] - Rm[1, 2]) / (4 * w), (Rm[0, 2] - Rm[2, 0]) / (4 * w),
         (Rm[1, 0] - Rm[0, 1]) / (4 * w)]
    o0 = np.asarray(L.col_c2w[0], np.float64).reshape(3, 4)[:, 3]
    mu = (o0 + np.array([6.0, 1.0, 0.5])).astype(np.float32)
    sc = _one_lidar_gaussian(mu, [math.log(1.5), math.log(1.5), math.log(1e-5)], 1.0,
                             [0.5, 0.0, 0.0], q)
    out = O64.render_lidar(sc, L)
    hit = np.nonzero(out["n_contrib"] > 0)[0]
    assert len(hit) > 200
    rg, _, _ = O64.lidar_decode(out)
    for i in hit[::7]:
        o, d = _beam_dir(L, i // L.n_cols, i % L.n_cols)
        t_plane = np.dot(mu.astype(np.float64) - o, n) / np.dot(d, n)
        assert abs(rg[i] - t_plane) < 1e-5 * t_plane, (i, rg[i], t_plane)


# ---------------------------------------------------- per-ray SH (Eq. 1, SH_i(d))
def test_sh_per_ray_degree1_closed_form(O64):
    """With the per-ray reading a Gaussian's colour along ray d is
    max(0, 0.5 + Y_0^0 c_0 + sqrt(3 / 4 pi) (-d_y c_1 + d_z c_2 - d_x c_3)):
    the textbook real SH of degree <= 1 at the ray's own direction."""
    cam = syn.tiny_camera()
    ok, o, d = O64.camera_ray(cam, 32, 32)
    coeffs = np.array([[0.4, -0.3, 0.2], [0.5, 0.1, -0.4], [-0.2, 0.3, 0.6],
                       [0.3, -0.5, 0.1]], np.float32)
    sc = _one_gaussian_scene((o + 8.0 * d).astype(np.float32), [-0.2, -0.2, -0.2], 0.6,
                             [0, 0, 0])
    sc = dataclasses.replace(sc, features=coeffs.reshape(1, 12), feature_kind=syn.FEATURES_SH,
                             sh_degree=1)
    opts = O64.opts(sh_per_ray=1)
    r = O64.render_camera(sc, cam, opts)
    one = np.nonzero(r["n_contrib"] == 1)[0]
    assert len(one) > 200
    c = coeffs.astype(np.float64)
    k0, k1 = 0.5 / math.sqrt(math.pi), math.sqrt(3.0 / (4.0 * math.pi))
    for i in one[::5]:
        _, _, dd = O64.camera_ray(cam, i % 64, i // 64)
        col = np.maximum(0.0, 0.5 + k0 * c[0] + k1 * (-dd[1] * c[1] + dd[2] * c[2] - dd[0] * c[3]))
        assert np.allclose(r["out"][i] / r["alpha"][i], col, rtol=1e-9, atol=1e-12), i
    # the per-Gaussian reading gives one colour for the whole footprint
    g = O64.render_camera(sc, cam)
    cols = g["out"][one] / g["alpha"][one][:, None]
    assert np.abs(cols - cols[0]).max() < 1e-9
    assert np.abs(r["out"][one] / r["alpha"][one][:, None] - cols).max() > 1e-3


def test_sh_per_ray_equals_per_gaussian_on_the_axis_and_at_degree0(O64):
    """On the ray through the mean the two directions coincide; with degree-0
    SH the colour does not depend on the direction at all."""
    cam = syn.tiny_camera()
    ok, o, d = O64.camera_ray(cam, 40, 21)
    rng = np.random.default_rng(3)
    sc = _one_gaussian_scene((o + 9.0 * d).astype(np.float32), [-0.5, -0.7, -0.6], 0.8,
                             [0, 0, 0])
    sc = dataclasses.replace(sc, features=rng.normal(0, 0.4, (1, 48)).astype(np.float32),
                             feature_kind=syn.FEATURES_SH, sh_degree=3)
    a = O64.render_camera(sc, cam, O64.opts(sh_per_ray=1), rays=[21 * 64 + 40])[0]
    b = O64.render_camera(sc, cam, rays=[21 * 64 + 40])[0]
    assert np.allclose(a["out"], b["out"], atol=1e-6)
    s0 = dataclasses.replace(syn.tiny_scene(n=300, seed=4), feature_kind=syn.FEATURES_SH,
                             sh_degree=0)
    x = O64.render_camera(s0, cam, O64.opts(sh_per_ray=1))
    y = O64.render_camera(s0, cam)
    assert np.array_equal(x["out"], y["out"])
    with pytest.raises(ValueError):
        O64.backward_camera(s0, cam, np.zeros((4096, 3), np.float32),
                            np.zeros(4096, np.float32), np.zeros(4096, np.float32),
                            O64.opts(sh_per_ray=1))


@pytest.mark.slow
def test_sh_readings_on_the_street_workload(O64):
    """How far the per-ray reading of Eq. 1 (SH at each ray's direction) is
    from the per-Gaussian one the renderer uses, on 2000 random pixels of
    the street fisheye view with 1M degree-3 Gaussians: the colour moves by
    a few thousandths on average and by up to a few hundredths, far beyond
    the 1e-4 parity tolerance, so the choice is a reading, not rounding."""
    sc = syn.street_scene(1_000_000, seed=0, kind="camera")
    fish, _ = syn.street_cameras()
    rng = np.random.default_rng(0)
    rays = np.unique(rng.choice(fish.width * fish.height, 2000, replace=False))
    a = O64.render_camera(sc, fish, rays=rays)
    b = O64.render_camera(sc, fish, O64.opts(sh_per_ray=1), rays=rays)
    d = np.abs(a["out"] - b["out"]).max(axis=1)
    assert np.array_equal(a["alpha"], b["alpha"])       # only the colour changes
    assert 1e-3 < d.mean() < 2e-2 and d.max() < 0.1, (d.mean(), d.max())


@pytest.mark.parametrize("bits", [64, 32])
def test_tiny_config_invariants(bits):
    from oracle import Oracle
    O = Oracle(bits)
    sc, cam = syn.tiny_scene(), syn.tiny_camera()
    r = O.render_camera(sc, cam)
    rb = O.render_camera(sc, cam, bruteforce=True)
    # tiled == brute force, bit for bit, in the same precision
    for k in ("out", "alpha", "depth", "t_final", "n_contrib"):
        assert np.array_equal(r[k], rb[k])
    # omega = sum alpha_i T_i = 1 - T_final (Eq. 1 telescopes)
    tol = 1e-12 if bits == 64 else 2e-6
    assert np.abs(r["alpha"] - (1 - r["t_final"])).max() < tol
    assert np.all(r["t_final"] > 0) and np.all(r["t_final"] <= 1)
    assert np.all(r["out"] >= 0) and r["n_contrib"].sum() > 0


def test_bin_sort_matches_lexsort(O64):
    sc, cam = syn.tiny_scene(), syn.tiny_camera()
    P, (ntx, nty) = O64.project_camera(sc, cam)
    ids, tiles, ranges = O64.bin_sort(P, ntx, nty, False)
    T, D, I = [], [], []
    for g in np.nonzero(P["valid"])[0]:
        x0, x1, y0, y1 = P["tiles"][g]
        for ty in range(y0, y1 + 1):
            for tx in range(x0, x1 + 1):
                T.append(ty * ntx + tx)
                D.append(P["depth"][g])
                I.append(g)
    order = np.lexsort((I, D, T))
    assert np.array_equal(ids, np.array(I)[order])
    assert np.array_equal(tiles, np.array(T)[order])
    for t in range(ntx * nty):
        sel = np.nonzero(tiles == t)[0]
        if len(sel):
            assert ranges[t, 0] == sel[0] and ranges[t, 1] == sel[-1] + 1


def _lidar_toy(n=512, seed=0):
    L = syn.street_lidar(n_cols=256)
    sc = syn.street_scene(n, seed=seed, kind="lidar", length=60.0)
    return sc, L


@pytest.mark.parametrize("bits", [64, 32])
def test_lidar_tiled_equals_bruteforce_and_culling_invariance(bits):
    from oracle import Oracle
    O = Oracle(bits)
    sc, L = _lidar_toy(1500)
    r = O.render_lidar(sc, L)
    rb = O.render_lidar(sc, L, bruteforce=True)
    rn = O.render_lidar(sc, L, O.opts(cull=0))
    for k in ("out", "alpha", "depth", "n_contrib"):
        assert np.array_equal(r[k], rb[k])
        assert np.array_equal(r[k], rn[k])
    assert r["n_contrib"].sum() > 1000
    # culling removed some Gaussians (it does work) without changing outputs
    P1, _ = O.project_lidar(sc, L)
    P0, _ = O.project_lidar(sc, L, O.opts(cull=0))
    assert P1["valid"].sum() < P0["valid"].sum()
    # rays that hit nothing: drop probability 1/2
    rng_, inten, drop = O.lidar_decode(r)
    miss = r["n_contrib"] == 0
    assert miss.any() and np.allclose(drop[miss], 0.5)


def test_lidar_tiling_invariance(O64):
    """Sec. 4.3: the (M, N_phi) choice changes speed, not the result."""
    sc, L0 = _lidar_toy(800, seed=3)
    ref = O64.render_lidar(sc, L0)
    for M in (32, 64, 128, 256):
        for nphi in (8, 16, 32, 64):
            L = syn.Lidar(L0.elevations_deg, L0.n_cols, L0.az0_deg, L0.col_c2w, M, nphi)
            r = O64.render_lidar(sc, L)
            for k in ("out", "alpha", "depth"):
                assert np.array_equal(r[k], ref[k]), (M, nphi, k)


def test_lidar_static_pose_iterations_irrelevant(O64):
    sc, _ = _lidar_toy(600, seed=4)
    L = syn.street_lidar(n_cols=256, static=True)
    a = O64.render_lidar(sc, L, O64.opts(pose_iters=0))
    b = O64.render_lidar(sc, L, O64.opts(pose_iters=2))
    assert np.array_equal(a["out"], b["out"]) and np.array_equal(a["depth"], b["depth"])


# ---------------------------------------------------------------- backward
def _fd_setup():
    """16 Gaussians in front of a 12x10 camera, one tile, cutoffs off."""
    rng = np.random.default_rng(9)
    n = 16
    cam = syn.tiny_camera()
    cam.width, cam.height, cam.cx, cam.cy = 12, 10, 6.0, 5.0
    cam.fx = cam.fy = 8.0
    sc = syn.tiny_scene(n=n)
    sc.means[:] = np.stack([rng.uniform(-3, 3, n), rng.uniform(-4, 2, n),
                            rng.uniform(-2.5, 2.5, n)], 1)
    sc.log_scales[:] = rng.normal(-0.3, 0.3, (n, 3))
    sc.opacity[:] = rng.uniform(0.2, 0.8, n)
    deg = 3
    sc.features = rng.normal(0, 0.3, (n, 3 * (deg + 1) ** 2)).astype(np.float32)
    sc.features[:, :3] += 1.0
    sc.feature_kind, sc.sh_degree = syn.FEATURES_SH, deg
    return sc, cam


def _loss_cam(O, sc, cam, opts, gr, ga, gd):
    r = O.render_camera(sc, cam, opts)
    return (r["out"] * gr).sum() + (r["alpha"] * ga).sum() + (r["depth"] * gd).sum()


def test_backward_camera_matches_central_differences(O64):
    sc, cam = _fd_setup()
    opts = O64.opts(cutoffs=0, predicate=0, tile=64)
    nr = cam.width * cam.height
    rng = np.random.default_rng(1)
    gr = rng.normal(size=(nr, 3)).astype(np.float32)
    ga = rng.normal(size=nr).astype(np.float32)
    gd = (0.05 * rng.normal(size=nr)).astype(np.float32)
    G = O64.backward_camera(sc, cam, gr, ga, gd, opts)
    # perturb float32 parameters in double through a float64 copy of the scene
    checked = 0
    for name, arr in (("means", sc.means), ("log_scales", sc.log_scales),
                      ("quats", sc.quats), ("opacity", sc.opacity),
                      ("features", sc.features)):
        flat = arr.reshape(-1)
        gflat = G[name].reshape(-1)
        for i in range(0, flat.size, max(1, flat.size // 24)):
            x0 = float(flat[i])
            h = 2.0 ** -14
            flat[i] = np.float32(x0 + h)
            hp = float(flat[i]) - x0
            lp = _loss_cam(O64, sc, cam, opts, gr, ga, gd)
            flat[i] = np.float32(x0 - h)
            hm = x0 - float(flat[i])
            lm = _loss_cam(O64, sc, cam, opts, gr, ga, gd)
            flat[i] = np.float32(x0)
            fd = (lp - lm) / (hp + hm)
            scale = max(1.0, np.abs(gflat).max())
            assert abs(fd - gflat[i]) < 2e-4 * scale + 2e-5 * abs(fd), (name, i, fd, gflat[i])
            checked += 1
    assert checked > 100


def test_backward_single_gaussian_opacity_closed_form(O64):
    """omega = sigma rho for one Gaussian: d omega / d sigma = rho."""
    cam = syn.tiny_camera()
    ok, o, d = O64.camera_ray(cam, 20, 20)
    mu = (o + 8 * d + np.array([0.05, 0, 0.03])).astype(np.float32)
    sc = _one_gaussian_scene(mu, [-1.0, -1.0, -1.0], 0.5, [0.3, 0.3, 0.3])
    nr = 64 * 64
    ga = np.zeros(nr, np.float32)
    ga[20 * 64 + 20] = 1.0
    G = O64.backward_camera(sc, cam, np.zeros((nr, 3), np.float32), ga,
                            np.zeros(nr, np.float32))
    r = O64.render_camera(sc, cam, rays=[20 * 64 + 20])[0]
    assert abs(G["opacity"][0] - r["alpha"] / 0.5) < 1e-12


def test_backward_lidar_matches_central_differences(O64):
    L = syn.street_lidar(n_cols=64, n_beams=64)
    L.n_elev_tiles = 1
    L.max_rays_per_tile = 64 * 64
    rng = np.random.default_rng(4)
    n = 12
    sc = syn.street_scene(n, seed=5, kind="lidar", length=20.0)
    # compact Gaussians 8-14 m from the sensor: where a ray is perpendicular
    # to a Gaussian (tau_max ~ 0, the one remaining discontinuity with the
    # cutoffs off) its response is ~exp(-200), so the loss is smooth
    ang = rng.uniform(-np.pi, np.pi, n)
    rad = rng.uniform(8, 14, n)
    sc.means[:] = np.stack([30 + rad * np.cos(ang), rad * np.sin(ang),
                            rng.uniform(0, 2.5, n)], 1)
    sc.log_scales[:] = rng.normal(-1.0, 0.2, (n, 3))
    sc.opacity[:] = rng.uniform(0.2, 0.8, n)
    opts = O64.opts(cutoffs=0, predicate=0, cull=0)
    nr = L.n_beams * L.n_cols
    g = [rng.normal(size=nr).astype(np.float32) * s for s in (0.02, 1.0, 1.0, 1.0)]
    G = O64.backward_lidar(sc, L, *g, opts=opts)

    def loss():
        r = O64.render_lidar(sc, L, opts)
        rg, it, dr = O64.lidar_decode(r)
        return (rg * g[0]).sum() + (it * g[1]).sum() + (dr * g[2]).sum() + (r["alpha"] * g[3]).sum()

    for name, arr in (("means", sc.means), ("log_scales", sc.log_scales),
                      ("quats", sc.quats), ("opacity", sc.opacity),
                      ("features", sc.features)):
        flat = arr.reshape(-1)
        gflat = G[name].reshape(-1)
        for i in range(0, flat.size, max(1, flat.size // 10)):
            x0 = float(flat[i])
            h = 2.0 ** -14
            flat[i] = np.float32(x0 + h)
            hp = float(flat[i]) - x0
            lp = loss()
            flat[i] = np.float32(x0 - h)
            hm = x0 - float(flat[i])
            lm = loss()
            flat[i] = np.float32(x0)
            fd = (lp - lm) / (hp + hm)
            scale = max(1.0, np.abs(gflat).max())
            assert abs(fd - gflat[i]) < 2e-4 * scale + 2e-5 * abs(fd), (name, i, fd, gflat[i])


# ---------------------------------------- FP64 central differences, 512 Gaussians
# The gradient check of the differentiable step at its stated size: the 512
# Gaussians nearest to the sensor among those the projection keeps (the
# nearest 512 of all lie mostly below the LiDAR's lowest beam or beside the
# camera), a 32x32 fisheye crop and an 8x64 LiDAR crop, every cutoff off so
# that the loss is smooth, and central differences with step 1e-6 on a
# float64 copy of the parameters.  The loss is the mean over the crop's rays
# of <g, outputs> with g ~ N(0, 1) per output.  Agreement: relative 1e-6 or
# absolute 1e-9.
FD_STEP, FD_REL, FD_ABS = 1e-6, 1e-6, 1e-9


def _as64(sc):
    return dataclasses.replace(sc, **{k: getattr(sc, k).astype(np.float64) for k in
                                      ("means", "log_scales", "quats", "opacity", "features")})


def _nearest_visible(full, origin, project, n=512, pre=20000):
    d = np.linalg.norm(full.means.astype(np.float64) - origin, axis=1)
    idx = np.argsort(d)[:pre]
    P = project(full.subset(idx))
    keep = idx[P["valid"] == 1][:n]
    assert len(keep) == n
    return _as64(full.subset(np.sort(keep)))


def _fd_check(loss, G, sc, n_top=8, n_random=60, seed=0):
    """Every parameter of the n_top Gaussians with the largest mean
    gradients, plus n_random random (Gaussian, parameter) picks."""
    rng = np.random.default_rng(seed)
    top = np.argsort(-np.abs(G["means"]).sum(1))[:n_top]
    picks = []
    names = ("means", "log_scales", "quats", "opacity", "features")
    for name in names:
        per = getattr(sc, name).reshape(sc.n, -1).shape[1]
        picks += [(name, g * per + k) for g in top for k in range(per)]
    for _ in range(n_random):
        name = names[rng.integers(0, len(names))]
        size = getattr(sc, name).size
        picks.append((name, int(rng.integers(0, size))))
    worst = 0.0
    for name, i in picks:
        flat = getattr(sc, name).reshape(-1)
        g = G[name].reshape(-1)[i]
        x0 = flat[i]
        flat[i] = x0 + FD_STEP
        lp = loss()
        flat[i] = x0 - FD_STEP
        lm = loss()
        flat[i] = x0
        fd = (lp - lm) / (2 * FD_STEP)
        err = abs(fd - g)
        assert err <= max(FD_REL * abs(g), FD_ABS), (name, i, fd, g, err)
        worst = max(worst, err / max(abs(g), 1e-300))
    nonzero = sum(1 for name, i in picks if G[name].reshape(-1)[i] != 0)
    return len(picks), nonzero


@pytest.mark.slow
def test_backward_fisheye_crop_512_gaussians_fp64_central_differences(O64):
    full = syn.street_scene(1_000_000, seed=0, kind="camera")
    fish, _ = syn.street_cameras()
    opts = O64.opts(cutoffs=0, predicate=0)
    o = np.asarray(fish.c2w, np.float64).reshape(3, 4)[:, 3]
    sc = _nearest_visible(full, o, lambda s: O64.project_camera(s, fish, opts)[0])
    # the tile-aligned 32x32 crop that the most of their boxes overlap
    P, _ = O64.project_camera(sc, fish, opts)
    r, v = P["rect"], P["valid"] == 1
    best = (-1, 0, 0)
    for cy in range(0, fish.height - 32 + 1, 16):
        for cx in range(0, fish.width - 32 + 1, 16):
            c = int((v & (r[:, 0] <= cx + 32) & (r[:, 1] >= cx) & (r[:, 2] <= cy + 32)
                     & (r[:, 3] >= cy)).sum())
            best = max(best, (c, cx, cy))
    _, cx, cy = best
    rays = np.array([(cy + j) * fish.width + cx + i for j in range(32) for i in range(32)])
    nr = fish.width * fish.height
    rng = np.random.default_rng(1)
    gr = np.zeros((nr, 3), np.float32)
    ga = np.zeros(nr, np.float32)
    gd = np.zeros(nr, np.float32)
    gr[rays] = rng.normal(size=(len(rays), 3)) / len(rays)
    ga[rays] = rng.normal(size=len(rays)) / len(rays)
    gd[rays] = rng.normal(size=len(rays)) / len(rays)
    G = O64.backward_camera(sc, fish, gr, ga, gd, opts, rays=rays)

    def loss():
        out = O64.render_camera(sc, fish, opts, rays=rays)
        return ((out["out"] * gr[rays]).sum() + (out["alpha"] * ga[rays]).sum()
                + (out["depth"] * gd[rays]).sum())

    n, nonzero = _fd_check(loss, G, sc)
    assert n > 500 and nonzero > 300


@pytest.mark.slow
def test_backward_lidar_crop_512_gaussians_fp64_central_differences(O64):
    full = syn.street_scene(2_000_000, seed=1, kind="lidar")
    L = syn.street_lidar()
    opts = O64.opts(cutoffs=0, predicate=0, cull=0)
    o = L.col_c2w[L.n_cols // 2].astype(np.float64).reshape(3, 4)[:, 3]
    sc = _nearest_visible(full, o, lambda s: O64.project_lidar(s, L, opts)[0])
    P, _ = O64.project_lidar(sc, L, opts)
    r, v = P["rect"], P["valid"] == 1
    az = L.az0_deg + (np.arange(L.n_cols) + 0.5) * 360.0 / L.n_cols
    el = L.elevations_deg
    best = (-1, 0, 0)
    for b0 in range(0, L.n_beams - 8 + 1, 4):
        for c0 in range(0, L.n_cols - 64 + 1, 32):
            c = int((v & (r[:, 0] <= az[c0 + 63]) & (r[:, 1] >= az[c0]) & (r[:, 2] <= el[b0 + 7])
                     & (r[:, 3] >= el[b0])).sum())
            best = max(best, (c, b0, c0))
    _, b0, c0 = best
    rays = np.array([(b0 + j) * L.n_cols + c0 + i for j in range(8) for i in range(64)])
    nr = L.n_beams * L.n_cols
    rng = np.random.default_rng(2)
    g = [np.zeros(nr, np.float32) for _ in range(4)]
    for k, sd in enumerate((0.02, 1.0, 1.0, 1.0)):     # range, intensity, drop, alpha
        g[k][rays] = sd * rng.normal(size=len(rays)) / len(rays)
    G = O64.backward_lidar(sc, L, *g, opts=opts, rays=rays)

    def loss():
        out = O64.render_lidar(sc, L, opts, rays=rays)
        rg, it, dr = O64.lidar_decode(out)
        return ((rg * g[0][rays]).sum() + (it * g[1][rays]).sum() + (dr * g[2][rays]).sum()
                + (out["alpha"] * g[3][rays]).sum())

    n, nonzero = _fd_check(loss, G, sc)
    assert n > 150 and nonzero > 100


# ------------------------------------------------------------ LiDAR SH^l
def _lidar_sh_scene(sc, deg, coeffs):
    """A copy of LiDAR scene `sc` with LIDAR_SH features [n, (deg+1)^2, 3]."""
    import dataclasses
    n = sc.n
    return dataclasses.replace(sc, features=np.asarray(coeffs, np.float32).reshape(n, -1),
                               feature_kind=syn.FEATURES_LIDAR_SH, sh_degree=deg)


def test_lidar_sh_degree0_is_raw_features_over_y00(O64):
    """Degree 0: zeta = Y_00 c_0 with Y_00 = 1 / (2 sqrt(pi)), so c_0 = f / Y_00
    renders what the raw feature kind renders with f."""
    L = syn.street_lidar(n_cols=96, n_beams=64)
    sc = syn.street_scene(3000, seed=2, kind="lidar", length=40.0)
    y00 = 1.0 / (2.0 * math.sqrt(math.pi))
    sh = _lidar_sh_scene(sc, 0, sc.features.astype(np.float64) / y00)
    a = O64.render_lidar(sc, L)
    b = O64.render_lidar(sh, L)
    f32 = sh.features.astype(np.float64) * y00 - sc.features.astype(np.float64)
    tol = 1e-9 + 4 * np.abs(f32).max()          # the float32 rounding of c_0
    assert np.abs(a["out"] - b["out"]).max() < tol
    assert np.array_equal(a["alpha"], b["alpha"]) and np.array_equal(a["depth"], b["depth"])


def test_lidar_sh_direction_from_the_mean_column_origin(O64):
    """One Gaussian on the ray of (beam, col) of a moving sensor, 3 m out:
    the ray through its centre composites alpha * zeta with zeta = sum_k
    Y_k(d) c_k, d the ray direction (= the direction from that column's
    origin to the mean), no colour offset and no clamp.  The sensor moves
    1.5 m over the sweep, so the mid-sweep origin would see the mean from
    another direction."""
    L = syn.street_lidar(n_cols=128, n_beams=64)
    beam, col = 40, 5
    o, d, _, _ = O64.lidar_ray(L, beam, col)
    sc = syn.tiny_scene(n=1)
    sc.means[0] = o + 3.0 * d
    sc.log_scales[0] = [-2.5, -2.6, -2.4]
    sc.quats[0] = [1, 0, 0, 0]
    sc.opacity[0] = 0.8
    sc.feature_kind = syn.FEATURES_LIDAR
    rng = np.random.default_rng(3)
    c = rng.normal(0.0, 1.0, (1, 16, 3))
    c[0, 0] = [0.1, -3.0, 2.0]           # zeta < 0 in the logits: nothing clamps
    sh = _lidar_sh_scene(sc, 3, c)
    r = O64.render_lidar(sh, L, O64.opts(cull=0), rays=[beam * L.n_cols + col])[0]
    mu = sh.means[0].astype(np.float64)
    P, _ = O64.project_lidar(sh, L, O64.opts(cull=0))
    assert P["pose_col"][0] == col
    dirv = mu - o
    dirv /= np.linalg.norm(dirv)
    Y = O64.sh_basis(dirv)
    zeta = Y @ sh.features[0].astype(np.float64).reshape(16, 3)
    a = float(np.float32(0.8))
    assert abs(r["alpha"] - a) < 1e-9
    assert np.allclose(r["out"], a * zeta, atol=1e-9), (r["out"], a * zeta)
    # the mid-sweep origin would give a visibly different zeta
    om = L.col_c2w[L.n_cols // 2][[3, 7, 11]].astype(np.float64)
    dm = (mu - om) / np.linalg.norm(mu - om)
    assert np.abs(O64.sh_basis(dm) @ sh.features[0].astype(np.float64).reshape(16, 3) - zeta).max() > 0.05


def test_backward_lidar_sh_matches_central_differences(O64):
    """As test_backward_lidar_matches_central_differences, with degree-2
    SH^l features: the feature gradients are Y_k(dir) times the channel
    gradients and the means get the direction term."""
    L = syn.street_lidar(n_cols=64, n_beams=64)
    L.n_elev_tiles = 1
    L.max_rays_per_tile = 64 * 64
    rng = np.random.default_rng(6)
    n = 10
    sc = syn.street_scene(n, seed=7, kind="lidar_sh", sh_degree=2, length=20.0)
    ang = rng.uniform(-np.pi, np.pi, n)
    rad = rng.uniform(8, 14, n)
    sc.means[:] = np.stack([30 + rad * np.cos(ang), rad * np.sin(ang),
                            rng.uniform(0, 2.5, n)], 1)
    sc.log_scales[:] = rng.normal(-1.0, 0.2, (n, 3))
    sc.opacity[:] = rng.uniform(0.2, 0.8, n)
    sc.features[:] = rng.normal(0.0, 0.8, sc.features.shape)
    opts = O64.opts(cutoffs=0, predicate=0, cull=0)
    nr = L.n_beams * L.n_cols
    g = [rng.normal(size=nr).astype(np.float32) * s for s in (0.02, 1.0, 1.0, 1.0)]
    G = O64.backward_lidar(sc, L, *g, opts=opts)

    def loss():
        r = O64.render_lidar(sc, L, opts)
        rg, it, dr = O64.lidar_decode(r)
        return (rg * g[0]).sum() + (it * g[1]).sum() + (dr * g[2]).sum() + (r["alpha"] * g[3]).sum()

    for name, arr in (("means", sc.means), ("features", sc.features)):
        flat = arr.reshape(-1)
        gflat = G[name].reshape(-1)
        for i in range(0, flat.size, max(1, flat.size // 12)):
            x0 = float(flat[i])
            h = 2.0 ** -14
            flat[i] = np.float32(x0 + h)
            hp = float(flat[i]) - x0
            lp = loss()
            flat[i] = np.float32(x0 - h)
            hm = x0 - float(flat[i])
            lm = loss()
            flat[i] = np.float32(x0)
            fd = (lp - lm) / (hp + hm)
            scale = max(1.0, np.abs(gflat).max())
            assert abs(fd - gflat[i]) < 2e-4 * scale + 2e-5 * abs(fd), (name, i, fd, gflat[i])


# ------------------------------------------------------------ dynamic actors
def _compose(A, B):
    """Row-major [R | t] poses: A o B."""
    A = np.asarray(A, np.float64).reshape(3, 4)
    B = np.asarray(B, np.float64).reshape(3, 4)
    R = A[:, :3] @ B[:, :3]
    t = A[:, :3] @ B[:, 3] + A[:, 3]
    return np.concatenate([R, t[:, None]], 1).reshape(12)


def _inverse(A):
    A = np.asarray(A, np.float64).reshape(3, 4)
    R = A[:, :3].T
    return np.concatenate([R, (-R @ A[:, 3])[:, None]], 1).reshape(12)


def test_actors_at_identity_render_the_static_scene(O64):
    sc = syn.with_actors(syn.street_scene(3000, seed=4, length=30.0), n_actors=5, frac=0.3)
    sc.actor_poses[:] = syn.actor_pose(0.0, 0.0, 0.0)
    static = dataclasses.replace(sc, actor_of=None, actor_poses=None)
    cam = dataclasses.replace(syn.street_cameras()[1], width=320, height=180, fx=170.0,
                              fy=170.0, cx=160.0, cy=90.0)
    a = O64.render_camera(sc, cam)
    b = O64.render_camera(static, cam)
    for k in ("out", "alpha", "depth"):
        assert np.array_equal(a[k], b[k]), k


def _one_actor_scene(seed=5, kind="camera"):
    sc = syn.street_scene(2500, seed=seed, kind=kind, length=25.0)
    sc.actor_of = np.zeros(sc.n, np.int32)
    # a quarter turn about z and an integer shift: exact in float32
    sc.actor_poses = syn.actor_pose(7.0, -3.0, math.pi / 2)[None].copy()
    sc.actor_poses[0, [0, 1, 4, 5]] = [0.0, -1.0, 1.0, 0.0]
    return sc


def test_actor_pose_equals_moving_the_camera_into_its_frame(O64):
    """Every Gaussian in one actor with pose T, seen by a camera at C, renders
    as the static scene (the actor's frame) seen from T^-1 C, SH colour
    included: the appearance turns with the actor."""
    sc = _one_actor_scene()
    T = sc.actor_poses[0]
    static = dataclasses.replace(sc, actor_of=None, actor_poses=None)
    cam = dataclasses.replace(syn.street_cameras()[0], width=320, height=214, fx=107.0,
                              fy=107.0, cx=160.0, cy=107.0)
    moved = dataclasses.replace(cam, c2w=_compose(_inverse(T), cam.c2w).astype(np.float32))
    assert np.array_equal(moved.c2w.astype(np.float64), _compose(_inverse(T), cam.c2w))
    a = O64.render_camera(sc, cam)
    b = O64.render_camera(static, moved)
    assert (a["alpha"] > 0).mean() > 0.05
    for k in ("out", "alpha", "depth"):
        assert np.abs(a[k] - b[k]).max() < 1e-9, k


def test_actor_pose_equals_moving_the_lidar_into_its_frame(O64):
    sc = _one_actor_scene(6, kind="lidar_sh")
    T = sc.actor_poses[0]
    static = dataclasses.replace(sc, actor_of=None, actor_poses=None)
    L = syn.street_lidar(n_cols=128, n_beams=64, start_xyz=(8.0, -1.0, 1.8))
    moved = dataclasses.replace(L, col_c2w=np.stack(
        [_compose(_inverse(T), p) for p in L.col_c2w]).astype(np.float32))
    a = O64.render_lidar(sc, L)
    b = O64.render_lidar(static, moved)
    assert (a["alpha"] > 0).mean() > 0.05
    for k in ("out", "alpha", "depth"):
        assert np.abs(a[k] - b[k]).max() < 1e-9, k


def test_backward_with_actors_matches_central_differences(O64):
    """Two actors with generic poses (rotation about a tilted axis): the
    gradients in each Gaussian's own frame, SH direction term included."""
    sc, cam = _fd_setup()
    sc.actor_of = np.array([-1, 0, 1, 0] * 4, np.int32)
    sc.actor_poses = np.stack([_compose(syn.actor_pose(0.3, -0.2, 0.4),
                                        [1, 0, 0, 0, 0, math.cos(0.3), -math.sin(0.3), 0.1,
                                         0, math.sin(0.3), math.cos(0.3), -0.2]),
                               syn.actor_pose(-0.4, 0.5, -0.7)]).astype(np.float32)
    opts = O64.opts(cutoffs=0, predicate=0, tile=64)
    nr = cam.width * cam.height
    rng = np.random.default_rng(3)
    gr = rng.normal(size=(nr, 3)).astype(np.float32)
    ga = rng.normal(size=nr).astype(np.float32)
    gd = (0.05 * rng.normal(size=nr)).astype(np.float32)
    G = O64.backward_camera(sc, cam, gr, ga, gd, opts)
    for name, arr in (("means", sc.means), ("log_scales", sc.log_scales),
                      ("quats", sc.quats), ("features", sc.features)):
        flat = arr.reshape(-1)
        gflat = G[name].reshape(-1)
        for i in range(0, flat.size, max(1, flat.size // 16)):
            x0 = float(flat[i])
            h = 2.0 ** -14
            flat[i] = np.float32(x0 + h)
            hp = float(flat[i]) - x0
            lp = _loss_cam(O64, sc, cam, opts, gr, ga, gd)
            flat[i] = np.float32(x0 - h)
            hm = x0 - float(flat[i])
            lm = _loss_cam(O64, sc, cam, opts, gr, ga, gd)
            flat[i] = np.float32(x0)
            fd = (lp - lm) / (hp + hm)
            scale = max(1.0, np.abs(gflat).max())
            assert abs(fd - gflat[i]) < 2e-4 * scale + 2e-5 * abs(fd), (name, i, fd, gflat[i])


# ------------------------------------------------------------ beam divergence
def _rot_wxyz(q):
    from scipy.spatial.transform import Rotation
    w, x, y, z = np.asarray(q, np.float64) / np.linalg.norm(q)
    return Rotation.from_quat([x, y, z, w]).as_matrix()


def test_beam_divergence_response_brute_force(O64):
    """Eq. 6 on single Gaussians near a moving LiDAR: for rays around the
    mean, alpha = sigma exp(-D^2/2) with D^2 the minimum over the ray of the
    Mahalanobis distance under Sigma + (delta r)^2 (I - d d^T), r and d from
    the origin of the column pose that sees the mean, found by brute force
    along the ray; the opacity is not rescaled (alpha = sigma on the ray
    through the mean)."""
    L = syn.street_lidar(n_cols=128, n_beams=64)
    delta = 0.02
    opts = O64.opts(cull=0, predicate=0, beam_divergence=delta)
    rng = np.random.default_rng(8)
    for trial in range(3):
        beam, col = int(rng.integers(10, 54)), int(rng.integers(0, 128))
        o, d, _, _ = O64.lidar_ray(L, beam, col)
        sc = syn.tiny_scene(n=1)
        sc.means[0] = o + rng.uniform(2.0, 5.0) * d
        sc.log_scales[0] = rng.normal(-2.5, 0.3, 3)
        sc.quats[0] = rng.normal(size=4)
        sc.opacity[0] = 0.7
        sc.feature_kind = syn.FEATURES_LIDAR
        P, _ = O64.project_lidar(sc, L, opts)
        oc = L.col_c2w[P["pose_col"][0]][[3, 7, 11]].astype(np.float64)
        mu = sc.means[0].astype(np.float64)
        R = _rot_wxyz(sc.quats[0])
        S = R @ np.diag(np.exp(2.0 * sc.log_scales[0].astype(np.float64))) @ R.T
        v = mu - oc
        r = np.linalg.norm(v)
        Sh = S + (delta * r) ** 2 * (np.eye(3) - np.outer(v, v) / r ** 2)
        Ai = np.linalg.inv(Sh)
        rays = [beam * L.n_cols + (col + dc) % L.n_cols for dc in (-1, 0, 1)] + \
               [(beam + db) * L.n_cols + col for db in (-1, 1)]
        res = O64.render_lidar(sc, L, opts, rays=rays)
        for ray, rr in zip(rays, res):
            ro, rd, _, _ = O64.lidar_ray(L, ray // L.n_cols, ray % L.n_cols)
            t = np.linspace(0.0, 8.0, 200001)
            x = ro[None, :] + t[:, None] * rd[None, :] - mu[None, :]
            d2 = np.einsum("ni,ij,nj->n", x, Ai, x)
            k = int(np.argmin(d2))
            tt = np.linspace(t[max(k - 1, 0)], t[min(k + 1, len(t) - 1)], 20001)
            x = ro[None, :] + tt[:, None] * rd[None, :] - mu[None, :]
            a = min(0.99, float(np.float32(0.7)) * math.exp(-0.5 * np.einsum(
                "ni,ij,nj->n", x, Ai, x).min()))
            assert abs(rr["alpha"] - a) < 1e-7, (trial, ray, rr["alpha"], a)
        assert abs(res[1]["alpha"] - float(np.float32(0.7))) < 1e-3   # the central ray


def test_backward_beam_divergence_matches_central_differences(O64):
    L = syn.street_lidar(n_cols=64, n_beams=64)
    L.n_elev_tiles = 1
    L.max_rays_per_tile = 64 * 64
    rng = np.random.default_rng(12)
    n = 10
    sc = syn.street_scene(n, seed=13, kind="lidar", length=20.0)
    ang = rng.uniform(-np.pi, np.pi, n)
    rad = rng.uniform(6, 10, n)
    sc.means[:] = np.stack([30 + rad * np.cos(ang), rad * np.sin(ang),
                            rng.uniform(0, 2.5, n)], 1)
    sc.log_scales[:] = rng.normal(-1.4, 0.2, (n, 3))
    sc.opacity[:] = rng.uniform(0.2, 0.8, n)
    opts = O64.opts(cutoffs=0, predicate=0, cull=0, beam_divergence=0.03)
    nr = L.n_beams * L.n_cols
    g = [rng.normal(size=nr).astype(np.float32) * s for s in (0.02, 1.0, 1.0, 1.0)]
    G = O64.backward_lidar(sc, L, *g, opts=opts)

    def loss():
        r = O64.render_lidar(sc, L, opts)
        rg, it, dr = O64.lidar_decode(r)
        return (rg * g[0]).sum() + (it * g[1]).sum() + (dr * g[2]).sum() + (r["alpha"] * g[3]).sum()

    base = O64.render_lidar(sc, L, O64.opts(cutoffs=0, predicate=0, cull=0))
    assert np.abs(O64.render_lidar(sc, L, opts)["alpha"] - base["alpha"]).max() > 1e-2
    for name, arr in (("means", sc.means), ("log_scales", sc.log_scales),
                      ("quats", sc.quats), ("opacity", sc.opacity)):
        flat = arr.reshape(-1)
        gflat = G[name].reshape(-1)
        for i in range(0, flat.size, max(1, flat.size // 10)):
            x0 = float(flat[i])
            h = 2.0 ** -14
            flat[i] = np.float32(x0 + h)
            hp = float(flat[i]) - x0
            lp = loss()
            flat[i] = np.float32(x0 - h)
            hm = x0 - float(flat[i])
            lm = loss()
            flat[i] = np.float32(x0)
            fd = (lp - lm) / (hp + hm)
            scale = max(1.0, np.abs(gflat).max())
            assert abs(fd - gflat[i]) < 2e-4 * scale + 2e-5 * abs(fd), (name, i, fd, gflat[i])


# ------------------------------------------------------------ rolling shutter
def test_rolling_shutter_with_equal_rows_is_the_global_shutter(O64):
    sc = syn.street_scene(3000, seed=14, length=30.0)
    cam = dataclasses.replace(syn.street_cameras()[1], width=200, height=120, fx=110.0,
                              fy=110.0, cx=100.0, cy=60.0)
    rs = dataclasses.replace(cam, row_c2w=np.tile(cam.c2w, (cam.height, 1)))
    a = O64.render_camera(sc, cam)
    b = O64.render_camera(sc, rs)
    for k in ("out", "alpha", "depth"):
        assert np.array_equal(a[k], b[k]), k


def test_rolling_shutter_ray_is_the_ray_of_its_rows_pose(O64):
    """A pixel of row y renders what a global-shutter camera with row y's
    pose renders there (brute force, no extent test; Gaussians at
    well-separated depths so that every order agrees)."""
    rng = np.random.default_rng(15)
    n = 40
    sc = syn.tiny_scene(n=n)
    sc.means[:] = np.stack([rng.uniform(4, 40, n), rng.uniform(-3, 3, n), rng.uniform(0.5, 3, n)], 1)
    sc.means[:, 0] = np.sort(sc.means[:, 0]) + np.arange(n) * 0.5
    sc.log_scales[:] = rng.normal(-0.7, 0.2, (n, 3))
    sc.opacity[:] = rng.uniform(0.2, 0.9, n)
    cam = dataclasses.replace(syn.street_cameras()[1], width=160, height=90, fx=90.0, fy=90.0,
                              cx=80.0, cy=45.0)
    rs = syn.rolling_shutter(cam, speed=20.0, readout_s=0.05, yaw_rate=0.5)
    opts = O64.opts(predicate=0)
    pix = [(int(x), int(y)) for x, y in zip(rng.integers(0, 160, 12), rng.integers(0, 90, 12))]
    got = O64.render_camera(sc, rs, opts, bruteforce=True, rays=[y * 160 + x for x, y in pix])
    for (x, y), r in zip(pix, got):
        glob = dataclasses.replace(cam, c2w=rs.row_c2w[y].copy())
        ref = O64.render_camera(sc, glob, opts, bruteforce=True, rays=[y * 160 + x])[0]
        assert np.allclose(r["out"], ref["out"], atol=1e-12) and abs(r["alpha"] - ref["alpha"]) < 1e-12
        assert abs(r["depth"] - ref["depth"]) < 1e-9
    # the rows differ: the first and the last row see the scene from 1 m apart
    assert np.linalg.norm(rs.row_c2w[0][[3, 7, 11]] - rs.row_c2w[-1][[3, 7, 11]]) > 0.9


def test_rolling_shutter_mean_row_is_a_fixed_point(O64):
    """With enough iterations the row chosen for a Gaussian's mean sees the
    mean in that row: the mean projected with the row's pose falls in
    [row, row + 1) (the iteration's fixed point)."""
    sc = syn.street_scene(4000, seed=16, length=40.0)
    cam = dataclasses.replace(syn.street_cameras()[1], width=320, height=180, fx=170.0,
                              fy=170.0, cx=160.0, cy=90.0)
    rs = syn.rolling_shutter(cam, speed=30.0, readout_s=0.05, yaw_rate=1.0)
    P, _ = O64.project_camera(sc, rs, O64.opts(pose_iters=8))
    checked = 0
    for g in np.nonzero(P["valid"] == 1)[0][:400]:
        row = int(P["pose_col"][g])
        ok, uv = O64.camera_project(dataclasses.replace(cam, c2w=rs.row_c2w[row]),
                                    sc.means[g].astype(np.float64))
        if not ok or not (0 <= uv[1] < cam.height) or P["cmargin"][g] < 1e-3:
            continue
        assert row <= uv[1] < row + 1, (g, row, uv)
        checked += 1
    assert checked > 200


def test_backward_rolling_shutter_matches_central_differences(O64):
    sc, cam = _fd_setup()
    rs = syn.rolling_shutter(cam, speed=40.0, readout_s=0.05, yaw_rate=2.0)
    opts = O64.opts(cutoffs=0, predicate=0, tile=64)
    nr = cam.width * cam.height
    rng = np.random.default_rng(17)
    gr = rng.normal(size=(nr, 3)).astype(np.float32)
    ga = rng.normal(size=nr).astype(np.float32)
    gd = (0.05 * rng.normal(size=nr)).astype(np.float32)
    G = O64.backward_camera(sc, rs, gr, ga, gd, opts)
    for name, arr in (("means", sc.means), ("log_scales", sc.log_scales),
                      ("quats", sc.quats), ("features", sc.features)):
        flat = arr.reshape(-1)
        gflat = G[name].reshape(-1)
        for i in range(0, flat.size, max(1, flat.size // 16)):
            x0 = float(flat[i])
            h = 2.0 ** -14
            flat[i] = np.float32(x0 + h)
            hp = float(flat[i]) - x0
            lp = _loss_cam(O64, sc, rs, opts, gr, ga, gd)
            flat[i] = np.float32(x0 - h)
            hm = x0 - float(flat[i])
            lm = _loss_cam(O64, sc, rs, opts, gr, ga, gd)
            flat[i] = np.float32(x0)
            fd = (lp - lm) / (hp + hm)
            scale = max(1.0, np.abs(gflat).max())
            assert abs(fd - gflat[i]) < 2e-4 * scale + 2e-5 * abs(fd), (name, i, fd, gflat[i])
