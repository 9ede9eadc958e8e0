"""ctypes wrapper around the plain-C oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py``.  The
product path (the ``paper_2510_12901_gb300`` package) never imports it.

Two builds of the same C source: ``Oracle(64)`` computes in double (reference
values for floating-point outputs), ``Oracle(32)`` in float (the precision the
CUDA kernels take their integer decisions in).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "oracle.c"), os.path.join(_HERE, "oracle.h")]
_lock = threading.Lock()


def lib_path(bits: int) -> str:
    return os.path.join(_HERE, f"liboracle{bits}.so")


def build(force: bool = False, openmp: bool = False) -> None:
    """Compile liboracle64.so and liboracle32.so with gcc (seconds)."""
    newest = max(os.path.getmtime(p) for p in _SRC)
    for bits in (64, 32):
        out = lib_path(bits)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
            continue
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
               "-fPIC", "-shared", "-Wall", "-o", out + ".tmp",
               os.path.join(_HERE, "oracle.c"), "-lm"]
        if bits == 32:
            cmd.insert(1, "-DORACLE_F32")
        subprocess.check_call(cmd)
        os.replace(out + ".tmp", out)


def _structs(real):
    class Scene(C.Structure):
        _fields_ = [("n", C.c_int64), ("means", C.c_void_p), ("log_scales", C.c_void_p),
                    ("quats", C.c_void_p), ("opacity", C.c_void_p),
                    ("features", C.c_void_p), ("feature_kind", C.c_int),
                    ("sh_degree", C.c_int), ("actor_of", C.c_void_p), ("n_actors", C.c_int),
                    ("actor_poses", C.c_void_p)]

    class Camera(C.Structure):
        _fields_ = [("model", C.c_int), ("width", C.c_int), ("height", C.c_int),
                    ("fx", C.c_float), ("fy", C.c_float), ("cx", C.c_float),
                    ("cy", C.c_float), ("k", C.c_float * 4), ("c2w", C.c_float * 12),
                    ("row_c2w", C.c_void_p)]

    class Lidar(C.Structure):
        _fields_ = [("n_beams", C.c_int), ("n_cols", C.c_int), ("az0_deg", C.c_float),
                    ("elev_deg", C.c_void_p), ("col_c2w", C.c_void_p),
                    ("n_elev_tiles", C.c_int), ("max_rays_per_tile", C.c_int),
                    ("cull_az", C.c_int), ("cull_el_per_tile", C.c_int)]

    class Opts(C.Structure):
        _fields_ = [("alpha_min", C.c_float), ("alpha_max", C.c_float),
                    ("t_min", C.c_float), ("near_dist", C.c_float),
                    ("ut_alpha", C.c_float), ("ut_beta", C.c_float),
                    ("ut_kappa", C.c_float), ("tile", C.c_int), ("pose_iters", C.c_int),
                    ("cull", C.c_int), ("predicate", C.c_int), ("cutoffs", C.c_int),
                    ("beam_divergence", C.c_float), ("sh_per_ray", C.c_int)]

    class Setup(C.Structure):
        _fields_ = [("n_tiles_x", C.c_int), ("n_tiles_y", C.c_int),
                    ("theta_max", C.c_double), ("T", C.POINTER(C.c_float)),
                    ("n_theta", C.c_int), ("sat", C.POINTER(C.c_int)),
                    ("sat_w", C.c_int), ("sat_h", C.c_int)]

    class Proj(C.Structure):
        _fields_ = [("valid", C.c_int), ("mean2d", real * 2), ("cov2d", real * 3),
                    ("rect", real * 4), ("tiles", C.c_int * 4), ("count", C.c_int),
                    ("depth", real), ("pose_col", C.c_int), ("vmargin", real), ("ut", C.c_int),
                    ("pmargin", real), ("cmargin", real), ("kdelta", real)]

    class Ray(C.Structure):
        _fields_ = [("out", real * 3), ("alpha", real), ("depth", real), ("zsum", real),
                    ("t_final", real), ("n_visited", C.c_int), ("n_evaluated", C.c_int),
                    ("n_contrib", C.c_int), ("m_rect", real), ("m_alpha", real),
                    ("m_tmin", real), ("m_tau", real), ("m_order", real), ("m_kpose", real)]

    return Scene, Camera, Lidar, Opts, Setup, Proj, Ray


POINT_MAP = None  # set per precision


class Oracle:
    """One precision of the oracle.  Arrays in, numpy arrays out."""

    _cache: dict = {}

    def __new__(cls, bits: int = 64):
        with _lock:
            if bits not in cls._cache:
                build()
                self = super().__new__(cls)
                self._init(bits)
                cls._cache[bits] = self
            return cls._cache[bits]

    def _init(self, bits):
        self.bits = bits
        self.real = C.c_double if bits == 64 else C.c_float
        self.np_real = np.float64 if bits == 64 else np.float32
        self.lib = C.CDLL(lib_path(bits))
        (self.Scene, self.Camera, self.Lidar, self.Opts, self.Setup, self.Proj,
         self.Ray) = _structs(self.real)
        self.PointMap = C.CFUNCTYPE(C.c_int, C.c_void_p, C.POINTER(self.real), C.c_int,
                                    C.POINTER(self.real))
        L = self.lib
        L.or_default_opts.restype = self.Opts
        L.or_fisheye_theta_max.restype = C.c_double
        L.or_bin_sort.restype = C.c_int64
        L.or_unscented.argtypes = [C.POINTER(self.Opts), C.c_void_p, C.c_void_p, C.c_void_p,
                                   self.PointMap, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]

    # ---------------------------------------------------------------- helpers
    @staticmethod
    def _p(a):
        return a.ctypes.data_as(C.c_void_p)

    def opts(self, **kw):
        o = self.lib.or_default_opts()
        for k, v in kw.items():
            if not hasattr(o, k):
                raise KeyError(k)
            setattr(o, k, v)
        return o

    def _param(self, a):
        """A parameter array in the build's precision.  float64 arrays go to
        the double build unrounded (central differences in double); any
        other array is first rounded to float32, the precision of the
        library's inputs."""
        a = np.asarray(a)
        if self.bits == 64 and a.dtype == np.float64:
            return np.ascontiguousarray(a)
        return np.ascontiguousarray(a, np.float32).astype(self.np_real)

    def scene(self, sc):
        arrs = [self._param(a) for a in
                (sc.means, sc.log_scales, sc.quats, sc.opacity, sc.features)]
        s = self.Scene(sc.n, *[self._p(a) for a in arrs], sc.feature_kind, sc.sh_degree)
        if getattr(sc, "actor_of", None) is not None:
            ao = np.ascontiguousarray(sc.actor_of, np.int32)
            ap = np.ascontiguousarray(sc.actor_poses, np.float32).reshape(-1, 12)
            s.actor_of, s.n_actors, s.actor_poses = self._p(ao), ap.shape[0], self._p(ap)
            arrs = arrs + [ao, ap]
        s._keep = arrs
        return s

    def camera(self, cam):
        c = self.Camera()
        c.model, c.width, c.height = cam.model, cam.width, cam.height
        c.fx, c.fy, c.cx, c.cy = cam.fx, cam.fy, cam.cx, cam.cy
        c.k[:] = [float(v) for v in np.asarray(cam.k, np.float32)]
        c.c2w[:] = [float(v) for v in np.asarray(cam.c2w, np.float32)]
        rows = getattr(cam, "row_c2w", None)
        if rows is not None:
            rows = np.ascontiguousarray(rows, np.float32).reshape(cam.height, 12)
            c.row_c2w = self._p(rows)
            c._keep = rows
        return c

    def lidar(self, L):
        el = np.ascontiguousarray(L.elevations_deg, np.float32)
        poses = np.ascontiguousarray(L.col_c2w, np.float32)
        s = self.Lidar(L.n_beams, L.n_cols, L.az0_deg, self._p(el), self._p(poses),
                       L.n_elev_tiles, L.max_rays_per_tile, L.cull_az, L.cull_el_per_tile)
        s._keep = (el, poses)
        return s

    def _as_np(self, carr, n):
        if n == 0:
            return np.zeros(0, dtype=np.ctypeslib.as_array(carr.__class__._type_ * 1)().dtype)
        return np.ctypeslib.as_array(carr, shape=(n,))

    # ---------------------------------------------------------------- steps
    def activate(self, log_scales, quats):
        ls = self._param(log_scales)
        q = self._param(quats)
        n = ls.shape[0]
        R = np.zeros((n, 9), self.np_real)
        s = np.zeros((n, 3), self.np_real)
        self.lib.or_activate(C.c_int64(n), self._p(ls), self._p(q), self._p(R), self._p(s))
        return R.reshape(n, 3, 3), s

    def sh_basis(self, d):
        d = np.ascontiguousarray(d, self.np_real)
        Y = np.zeros(16, self.np_real)
        self.lib.or_sh_basis(self._p(d), self._p(Y))
        return Y

    def sh_basis_grad(self, d):
        d = np.ascontiguousarray(d, self.np_real)
        dY = np.zeros((16, 3), self.np_real)
        self.lib.or_sh_basis_grad(self._p(d), self._p(dY))
        return dY

    def fisheye_theta_max(self, k):
        kk = (C.c_float * 4)(*[float(v) for v in k])
        return self.lib.or_fisheye_theta_max(kk)

    def camera_project(self, cam, xw, opts=None):
        c = self.camera(cam)
        o = opts or self.opts()
        tm = self.fisheye_theta_max(cam.k) if cam.model == 1 else 0.0
        x = np.ascontiguousarray(xw, self.np_real)
        uv = np.zeros(2, self.np_real)
        ok = self.lib.or_camera_project(C.byref(c), C.c_double(tm), C.byref(o),
                                        self._p(x), self._p(uv))
        return bool(ok), uv

    def camera_ray(self, cam, px, py):
        c = self.camera(cam)
        tm = self.fisheye_theta_max(cam.k) if cam.model == 1 else 0.0
        o = np.zeros(3)
        d = np.zeros(3)
        ok = self.lib.or_camera_ray(C.byref(c), C.c_double(tm), int(px), int(py), self._p(o),
                                   self._p(d))
        return bool(ok), o, d

    def unscented(self, mu, R, s, fn, opts=None, wrap_first=False):
        """UT of one Gaussian through a Python point map fn(x[3]) -> (ok, y[2])."""
        o = opts or self.opts()
        mu = np.ascontiguousarray(mu, self.np_real)
        R = np.ascontiguousarray(R, self.np_real).reshape(9)
        s = np.ascontiguousarray(s, self.np_real)

        def cb(ctx, x, idx, y):
            ok, yy = fn(np.array([x[0], x[1], x[2]]), idx)
            y[0], y[1] = float(yy[0]), float(yy[1])
            return int(ok)

        cfn = self.PointMap(cb)
        m = np.zeros(2, self.np_real)
        cv = np.zeros(3, self.np_real)
        ok = self.lib.or_unscented(C.byref(o), self._p(mu), self._p(R), self._p(s), cfn,
                                   None, int(wrap_first), self._p(m), self._p(cv))
        return bool(ok), m, cv

    def elevation_tiling(self, elev, n_cols, n_phi, M):
        el = np.ascontiguousarray(elev, np.float32)
        T = np.zeros(n_phi + 1, np.float32)
        nth = C.c_int()
        self.lib.or_elevation_tiling(self._p(el), len(el), n_cols, n_phi, M, self._p(T),
                                     C.byref(nth))
        return T, nth.value

    def elev_tile(self, T, n_phi, el):
        T = np.ascontiguousarray(T, np.float32)
        return self.lib.or_elev_tile(self._p(T), n_phi, self.real(el))

    def lidar_setup(self, L):
        lid = self.lidar(L)
        S = self.Setup()
        self.lib.or_lidar_setup(C.byref(lid), C.byref(S))
        nphi = L.n_elev_tiles
        T = np.array(S.T[:nphi + 1], np.float32)
        sat = np.ctypeslib.as_array(S.sat, shape=(S.sat_w * S.sat_h,)).copy().reshape(
            S.sat_w, S.sat_h)
        out = dict(T=T, n_theta=S.n_theta, sat=sat)
        self.lib.or_setup_free(C.byref(S))
        return out

    def sat_count_wrap(self, L, x0, x1, y0, y1):
        lid = self.lidar(L)
        S = self.Setup()
        self.lib.or_lidar_setup(C.byref(lid), C.byref(S))
        r = self.lib.or_sat_count_wrap(C.byref(S), L.cull_az, x0, x1, y0, y1)
        self.lib.or_setup_free(C.byref(S))
        return r

    def lidar_ray(self, L, beam, col):
        lid = self.lidar(L)
        o = np.zeros(3)
        d = np.zeros(3)
        az = C.c_double()
        el = C.c_double()
        self.lib.or_lidar_ray(C.byref(lid), beam, col, self._p(o), self._p(d), C.byref(az),
                              C.byref(el))
        return o, d, az.value, el.value

    def project_camera(self, sc, cam, opts=None):
        o = opts or self.opts()
        s = self.scene(sc)
        c = self.camera(cam)
        S = self.Setup()
        self.lib.or_camera_setup(C.byref(c), C.byref(o), C.byref(S))
        P = (self.Proj * max(sc.n, 1))()
        self.lib.or_project_camera(C.byref(s), C.byref(c), C.byref(S), C.byref(o), P)
        return np.ctypeslib.as_array(P)[:sc.n].copy(), (S.n_tiles_x, S.n_tiles_y)

    def project_lidar(self, sc, L, opts=None):
        o = opts or self.opts()
        s = self.scene(sc)
        lid = self.lidar(L)
        S = self.Setup()
        self.lib.or_lidar_setup(C.byref(lid), C.byref(S))
        P = (self.Proj * max(sc.n, 1))()
        self.lib.or_project_lidar(C.byref(s), C.byref(lid), C.byref(S), C.byref(o), P)
        nt = (S.n_theta, L.n_elev_tiles)
        self.lib.or_setup_free(C.byref(S))
        return np.ctypeslib.as_array(P)[:sc.n].copy(), nt

    def bin_sort(self, proj, ntx, nty, wrap):
        P = np.ascontiguousarray(proj)
        n = P.shape[0]
        K = self.lib.or_bin_sort(C.c_int64(n), self._p(P), ntx, nty, int(wrap), None, None,
                                 C.c_int64(0), None)
        ids = np.zeros(max(K, 1), np.uint32)
        tiles = np.zeros(max(K, 1), np.uint32)
        ranges = np.zeros(ntx * nty * 2, np.uint32)
        self.lib.or_bin_sort(C.c_int64(n), self._p(P), ntx, nty, int(wrap), self._p(ids),
                             self._p(tiles), C.c_int64(K), self._p(ranges))
        return ids[:K], tiles[:K], ranges.reshape(-1, 2)

    def _rays_arg(self, rays):
        if rays is None:
            return None, -1, None
        r = np.ascontiguousarray(rays, np.int64)
        return self._p(r), len(r), r

    def render_camera(self, sc, cam, opts=None, bruteforce=False, rays=None):
        o = opts or self.opts()
        s = self.scene(sc)
        c = self.camera(cam)
        rp, nr, keep = self._rays_arg(rays)
        n = cam.width * cam.height if nr < 0 else nr
        out = (self.Ray * max(n, 1))()
        self.lib.or_render_camera(C.byref(s), C.byref(c), C.byref(o), int(bruteforce), rp,
                                  C.c_int64(nr), out)
        return np.ctypeslib.as_array(out)[:n].copy()

    def render_lidar(self, sc, L, opts=None, bruteforce=False, rays=None):
        o = opts or self.opts()
        s = self.scene(sc)
        lid = self.lidar(L)
        rp, nr, keep = self._rays_arg(rays)
        n = L.n_beams * L.n_cols if nr < 0 else nr
        out = (self.Ray * max(n, 1))()
        self.lib.or_render_lidar(C.byref(s), C.byref(lid), C.byref(o), int(bruteforce), rp,
                                 C.c_int64(nr), out)
        return np.ctypeslib.as_array(out)[:n].copy()

    def lidar_decode(self, rays):
        """(range, intensity, drop probability) from raw ray records
        (or_lidar_decode, Sec. 3.2), as float64 arrays."""
        R = np.ascontiguousarray(rays)
        n = R.shape[0]
        out = [np.zeros(max(n, 1), self.np_real) for _ in range(3)]
        self.lib.or_lidar_decode_n(C.c_int64(n), self._p(R), *[self._p(a) for a in out])
        return tuple(a[:n].astype(np.float64) for a in out)

    def _grads(self, sc):
        F = sc.features.shape[1]
        return dict(means=np.zeros((sc.n, 3), self.np_real),
                    log_scales=np.zeros((sc.n, 3), self.np_real),
                    quats=np.zeros((sc.n, 4), self.np_real),
                    opacity=np.zeros(sc.n, self.np_real),
                    features=np.zeros((sc.n, F), self.np_real))

    def backward_camera(self, sc, cam, g_rgb, g_alpha, g_depth, opts=None, rays=None):
        o = opts or self.opts()
        s = self.scene(sc)
        c = self.camera(cam)
        ga = [np.ascontiguousarray(a, np.float32) for a in (g_rgb, g_alpha, g_depth)]
        G = self._grads(sc)
        rp, nr, keep = self._rays_arg(rays)
        r = self.lib.or_backward_camera(C.byref(s), C.byref(c), C.byref(o), rp, C.c_int64(nr),
                                        *[self._p(a) for a in ga],
                                        *[self._p(G[k]) for k in
                                          ("means", "log_scales", "quats", "opacity",
                                           "features")])
        if r != 0:
            raise ValueError("or_backward_camera refused the options")
        return G

    def backward_lidar(self, sc, L, g_range, g_int, g_drop, g_alpha, opts=None, rays=None):
        o = opts or self.opts()
        s = self.scene(sc)
        lid = self.lidar(L)
        ga = [np.ascontiguousarray(a, np.float32) for a in (g_range, g_int, g_drop, g_alpha)]
        G = self._grads(sc)
        rp, nr, keep = self._rays_arg(rays)
        r = self.lib.or_backward_lidar(C.byref(s), C.byref(lid), C.byref(o), rp, C.c_int64(nr),
                                       *[self._p(a) for a in ga],
                                       *[self._p(G[k]) for k in
                                         ("means", "log_scales", "quats", "opacity",
                                          "features")])
        if r != 0:
            raise ValueError("or_backward_lidar refused the options")
        return G
