"""Thin ctypes binding of libsimgut (include/simgut.h).

The ``sg_*`` functions mirror the C entry points one for one and only
marshal arguments.  The small classes below (``Scene``, ``Camera``, ``Lidar``,
``Frame``) own handles and use PyTorch for device memory and the current
CUDA stream; every stage of the render runs in the library's CUDA kernels.

There is no fallback: if ``libsimgut.so`` is missing or was built for another
machine, importing the library raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsimgut.so")

SG_OK = 0
STATUS = {0: "SG_OK", -1: "SG_ERR_INVALID", -2: "SG_ERR_OOM", -3: "SG_ERR_CUDA",
          -4: "SG_ERR_OVERFLOW", -5: "SG_ERR_TIMEOUT", -6: "SG_ERR_BUSY"}
FEATURES_RGB, FEATURES_SH, FEATURES_LIDAR, FEATURES_LIDAR_SH = 0, 1, 2, 3
CAMERA_PINHOLE, CAMERA_FISHEYE = 0, 1
(FIELD_RECT, FIELD_TILES, FIELD_DEPTH, FIELD_COUNT, FIELD_PAIR_IDS, FIELD_PAIR_TILES,
 FIELD_RANGES, FIELD_RAY_STATE, FIELD_N_CONTRIB, FIELD_MEAN2D, FIELD_COV2D) = range(11)


class SimgutError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class sg_gaussians_desc(C.Structure):
    _fields_ = [("n", C.c_int64), ("d_means", C.c_void_p), ("d_log_scales", C.c_void_p),
                ("d_quats", C.c_void_p), ("d_opacity", C.c_void_p),
                ("d_features", C.c_void_p), ("feature_kind", C.c_int), ("sh_degree", C.c_int)]


class sg_render_opts(C.Structure):
    _fields_ = [("alpha_min", C.c_float), ("alpha_max", C.c_float), ("t_min", C.c_float),
                ("near_dist", C.c_float), ("ut_alpha", C.c_float), ("ut_beta", C.c_float),
                ("ut_kappa", C.c_float), ("pose_iters", C.c_int), ("cull", C.c_int),
                ("beam_divergence", C.c_float)]


class sg_grads(C.Structure):
    _fields_ = [("d_g_means", C.c_void_p), ("d_g_log_scales", C.c_void_p),
                ("d_g_quats", C.c_void_p), ("d_g_opacity", C.c_void_p),
                ("d_g_features", C.c_void_p)]


class sg_camera_view(C.Structure):
    _fields_ = [("camera", C.c_void_p), ("c2w", C.c_float * 12), ("frame", C.c_void_p),
                ("rgb", C.c_void_p), ("alpha", C.c_void_p), ("depth", C.c_void_p),
                ("stream", C.c_void_p), ("row_c2w", C.c_void_p)]


class sg_server_config(C.Structure):
    _fields_ = [("n_slots", C.c_int), ("memory_budget", C.c_size_t),
                ("queue_capacity", C.c_int), ("use_graphs", C.c_int),
                ("fifo_priority", C.c_int), ("max_batch", C.c_int)]


class sg_request(C.Structure):
    _fields_ = [("kind", C.c_int), ("scene", C.c_void_p), ("camera", C.c_void_p),
                ("lidar", C.c_void_p), ("c2w", C.c_float * 12), ("d_col_c2w", C.c_void_p),
                ("d_out", C.c_void_p * 4), ("opts", sg_render_opts)]


class sg_server_report(C.Structure):
    _fields_ = [("completed", C.c_int64), ("failed", C.c_int64), ("rays", C.c_int64),
                ("peak_in_flight", C.c_int64), ("queued", C.c_int64),
                ("graph_replays", C.c_int64), ("graph_captures", C.c_int64),
                ("overflow_rerenders", C.c_int64), ("batches", C.c_int64),
                ("batched_requests", C.c_int64), ("latency_mean_ms", C.c_double),
                ("latency_p50_ms", C.c_double),
                ("latency_p99_ms", C.c_double), ("latency_max_ms", C.c_double),
                ("span_s", C.c_double), ("mrays_per_s", C.c_double)]


REQ_CAMERA, REQ_LIDAR = 0, 1
(LOOKBACK_NONE, LOOKBACK_COMPACT, LOOKBACK_DEPTH_SORT, LOOKBACK_OFFSETS,
 LOOKBACK_TILE_SORT) = range(5)
_H = C.c_void_p
_P = C.c_void_p
_SIGNATURES = {
    "sg_version": (C.c_int, []),
    "sg_cuda_arch": (C.c_int, []),
    "sg_last_error": (C.c_char_p, []),
    "sg_launch_count": (C.c_int64, []),
    "sg_create_scene": (C.c_int, [C.POINTER(sg_gaussians_desc), _P, C.POINTER(_H)]),
    "sg_update_scene": (C.c_int, [_H, C.POINTER(sg_gaussians_desc), _P]),
    "sg_destroy_scene": (None, [_H]),
    "sg_scene_size": (C.c_int64, [_H]),
    "sg_create_camera": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_float, C.c_float, C.c_float,
                                   C.c_float, C.POINTER(C.c_float), C.POINTER(_H)]),
    "sg_destroy_camera": (None, [_H]),
    "sg_create_lidar": (C.c_int, [C.POINTER(C.c_float), C.c_int, C.c_int, C.c_float, C.c_int,
                                  C.c_int, C.c_int, C.c_int, C.POINTER(_H)]),
    "sg_destroy_lidar": (None, [_H]),
    "sg_lidar_tiling": (C.c_int, [_H, C.POINTER(C.c_float), C.POINTER(C.c_int)]),
    "sg_default_opts": (sg_render_opts, []),
    "sg_frame_create": (C.c_int, [C.POINTER(_H)]),
    "sg_frame_destroy": (None, [_H]),
    "sg_scene_set_actors": (C.c_int, [_H, _P, C.c_int, _P]),
    "sg_scene_set_actor_poses": (C.c_int, [_H, C.POINTER(C.c_float), _P]),
    "sg_frame_set_capacity": (C.c_int, [_H, C.c_int64]),
    "sg_frame_dropped_pairs": (C.c_int, [_H, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "sg_render_camera": (C.c_int, [_H, _H, C.POINTER(C.c_float), C.POINTER(sg_render_opts), _H,
                                   _P, _P, _P, _P]),
    "sg_render_lidar": (C.c_int, [_H, _H, _P, C.POINTER(sg_render_opts), _H, _P, _P, _P, _P,
                                  _P]),
    "sg_render_camera_rs": (C.c_int, [_H, _H, _P, C.POINTER(sg_render_opts), _H, _P, _P, _P,
                                      _P]),
    "sg_render_cameras": (C.c_int, [_H, C.c_int, C.POINTER(sg_camera_view),
                                    C.POINTER(sg_render_opts), C.c_int]),
    "sg_render_camera_host": (C.c_int, [_H, _H, C.POINTER(C.c_float),
                                        C.POINTER(sg_render_opts), _H, _P, _P, _P, _P]),
    "sg_render_lidar_host": (C.c_int, [_H, _H, _P, C.POINTER(sg_render_opts), _H, _P, _P, _P,
                                       _P, _P]),
    "sg_render_camera_static": (C.c_int, [_H, _H, C.POINTER(C.c_float),
                                          C.POINTER(sg_render_opts), _P, _P, _P, _P]),
    "sg_backward_camera": (C.c_int, [_H, _H, _P, _P, _P, C.POINTER(sg_grads), _P]),
    "sg_backward_lidar": (C.c_int, [_H, _H, _P, _P, _P, _P, C.POINTER(sg_grads), _P]),
    "sg_frame_field": (C.c_int, [_H, C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_int64)]),
    "sg_frame_stats": (C.c_int, [_H, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                 C.POINTER(C.c_int64)]),
    "sg_default_server_config": (sg_server_config, []),
    "sg_server_create": (C.c_int, [C.POINTER(sg_server_config), C.POINTER(_H)]),
    "sg_server_submit": (C.c_int, [_H, C.POINTER(sg_request), C.POINTER(C.c_uint64)]),
    "sg_server_wait": (C.c_int, [_H, C.c_uint64, C.c_double, C.POINTER(C.c_double)]),
    "sg_server_drain": (C.c_int, [_H, C.c_double]),
    "sg_server_stats": (C.c_int, [_H, C.POINTER(sg_server_report)]),
    "sg_server_reset_stats": (C.c_int, [_H]),
    "sg_server_destroy": (None, [_H]),
    "sg_frame_set_timing": (C.c_int, [_H, C.c_int]),
    "sg_frame_timing": (C.c_int, [_H, C.POINTER(C.c_float)]),
    "sg_frame_marks": (C.c_int, [_H, _H, C.POINTER(C.c_float)]),
    "sg_frame_sync_outputs": (C.c_int, [_H]),
    "sg_frame_status": (C.c_int, [_H, _P]),
    "sg_frame_set_backward_state": (C.c_int, [_H, C.c_int]),
    "sg_alloc_count": (C.c_int64, []),
    "sg_workspace_bytes": (C.c_int, [_H, C.c_int, C.c_int64, C.POINTER(C.c_size_t)]),
    "sg_frame_workspace_bytes": (C.c_int, [_H, C.POINTER(C.c_size_t)]),
    "sg_debug_lookback": (C.c_int, [C.c_uint32, C.c_int, C.c_int64]),
    "sg_debug_bulk_wait": (C.c_int, [C.c_int]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libsimgut.so; raises if it is absent (run __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIGNATURES)


def _check(status):
    if status != SG_OK:
        raise SimgutError(status, load().sg_last_error().decode())


# ------------------------------------------------------------ C entry points
def sg_version():
    return load().sg_version()


def sg_cuda_arch():
    return load().sg_cuda_arch()


def sg_last_error():
    return load().sg_last_error().decode()


def sg_launch_count():
    return load().sg_launch_count()


def sg_default_opts(**kw):
    o = load().sg_default_opts()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def sg_create_scene(desc, stream=0):
    h = _H()
    _check(load().sg_create_scene(C.byref(desc), _P(stream), C.byref(h)))
    return h


def sg_update_scene(scene, desc, stream=0):
    _check(load().sg_update_scene(scene, C.byref(desc), _P(stream)))


def sg_destroy_scene(scene):
    load().sg_destroy_scene(scene)


def sg_create_camera(model, width, height, fx, fy, cx, cy, k):
    h = _H()
    kk = (C.c_float * 4)(*[float(v) for v in k])
    _check(load().sg_create_camera(model, width, height, fx, fy, cx, cy, kk, C.byref(h)))
    return h


def sg_destroy_camera(cam):
    load().sg_destroy_camera(cam)


def sg_create_lidar(elev_deg, n_cols, az0_deg, max_rays_per_tile, n_elev_tiles, cull_az,
                    cull_el_per_tile):
    h = _H()
    el = np.ascontiguousarray(elev_deg, np.float32)
    _check(load().sg_create_lidar(el.ctypes.data_as(C.POINTER(C.c_float)), len(el), n_cols,
                                  az0_deg, max_rays_per_tile, n_elev_tiles, cull_az,
                                  cull_el_per_tile, C.byref(h)))
    return h


def sg_destroy_lidar(lid):
    load().sg_destroy_lidar(lid)


def sg_lidar_tiling(lid, n_elev_tiles):
    T = (C.c_float * (n_elev_tiles + 1))()
    nth = C.c_int()
    _check(load().sg_lidar_tiling(lid, T, C.byref(nth)))
    return np.array(T[:], np.float32), nth.value


def sg_frame_create():
    h = _H()
    _check(load().sg_frame_create(C.byref(h)))
    return h


def sg_frame_destroy(fr):
    load().sg_frame_destroy(fr)


def _pose12(c2w):
    a = np.ascontiguousarray(c2w, np.float32).reshape(12)
    return (C.c_float * 12)(*[float(v) for v in a])


def sg_render_camera(scene, cam, c2w, opts, frame, d_rgb, d_alpha, d_depth, stream=0):
    _check(load().sg_render_camera(scene, cam, _pose12(c2w), C.byref(opts), frame, _P(d_rgb),
                                   _P(d_alpha), _P(d_depth), _P(stream)))


def sg_render_lidar(scene, lid, d_col_c2w, opts, frame, d_range, d_int, d_drop, d_alpha,
                    stream=0):
    _check(load().sg_render_lidar(scene, lid, _P(d_col_c2w), C.byref(opts), frame,
                                  _P(d_range), _P(d_int), _P(d_drop), _P(d_alpha), _P(stream)))


def sg_render_camera_rs(scene, cam, d_row_c2w, opts, frame, d_rgb, d_alpha, d_depth, stream=0):
    _check(load().sg_render_camera_rs(scene, cam, _P(d_row_c2w), C.byref(opts), frame,
                                      _P(d_rgb), _P(d_alpha), _P(d_depth), _P(stream)))


def sg_camera_views(views):
    """An array of sg_camera_view from (camera, c2w, frame, rgb, alpha, depth,
    stream[, row_c2w]) tuples (handles and raw pointers; None or 0 for no
    output; row_c2w: device pointer of per-row poses, rolling shutter)."""
    arr = (sg_camera_view * len(views))()
    for v, t in zip(arr, views):
        cam, c2w, frame, rgb, alpha, depth, stream = t[:7]
        v.camera = cam
        v.c2w[:] = list(_pose12(c2w))
        v.frame = frame
        v.rgb, v.alpha, v.depth = rgb or None, alpha or None, depth or None
        v.stream = stream or None
        v.row_c2w = (t[7] if len(t) > 7 else None) or None
    return arr


def sg_render_cameras(scene, views, opts, host_outputs=0):
    """views: the array from sg_camera_views."""
    _check(load().sg_render_cameras(scene, len(views), views, C.byref(opts), int(host_outputs)))


def sg_render_camera_host(scene, cam, c2w, opts, frame, h_rgb, h_alpha, h_depth, stream=0):
    _check(load().sg_render_camera_host(scene, cam, _pose12(c2w), C.byref(opts), frame,
                                        _P(h_rgb), _P(h_alpha), _P(h_depth), _P(stream)))


def sg_render_lidar_host(scene, lid, h_col_c2w, opts, frame, h_range, h_int, h_drop, h_alpha,
                         stream=0):
    _check(load().sg_render_lidar_host(scene, lid, _P(h_col_c2w), C.byref(opts), frame,
                                       _P(h_range), _P(h_int), _P(h_drop), _P(h_alpha),
                                       _P(stream)))


def sg_render_camera_static(scene, cam, c2w, opts, d_rgb, d_alpha, d_depth, stream=0):
    _check(load().sg_render_camera_static(scene, cam, _pose12(c2w), C.byref(opts), _P(d_rgb),
                                          _P(d_alpha), _P(d_depth), _P(stream)))


def sg_backward_camera(scene, frame, d_g_rgb, d_g_alpha, d_g_depth, grads, stream=0):
    _check(load().sg_backward_camera(scene, frame, _P(d_g_rgb), _P(d_g_alpha), _P(d_g_depth),
                                     C.byref(grads), _P(stream)))


def sg_backward_lidar(scene, frame, d_g_range, d_g_int, d_g_drop, d_g_alpha, grads, stream=0):
    _check(load().sg_backward_lidar(scene, frame, _P(d_g_range), _P(d_g_int), _P(d_g_drop),
                                    _P(d_g_alpha), C.byref(grads), _P(stream)))


def sg_frame_field(frame, field):
    p = C.c_void_p()
    n = C.c_int64()
    _check(load().sg_frame_field(frame, field, C.byref(p), C.byref(n)))
    return p.value, n.value


def sg_frame_stats(frame):
    a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
    _check(load().sg_frame_stats(frame, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def sg_default_server_config(**kw):
    c = load().sg_default_server_config()
    for k, v in kw.items():
        if not hasattr(c, k):
            raise KeyError(k)
        setattr(c, k, v)
    return c


def sg_server_create(cfg):
    h = _H()
    _check(load().sg_server_create(C.byref(cfg), C.byref(h)))
    return h


def sg_server_submit(server, req):
    t = C.c_uint64()
    _check(load().sg_server_submit(server, C.byref(req), C.byref(t)))
    return t.value


def sg_server_wait(server, ticket, timeout_s=60.0):
    lat = C.c_double()
    _check(load().sg_server_wait(server, C.c_uint64(ticket), timeout_s, C.byref(lat)))
    return lat.value


def sg_server_drain(server, timeout_s=600.0):
    _check(load().sg_server_drain(server, timeout_s))


def sg_server_stats(server):
    st = sg_server_report()
    _check(load().sg_server_stats(server, C.byref(st)))
    return {k: getattr(st, k) for k, _ in st._fields_}


def sg_server_reset_stats(server):
    _check(load().sg_server_reset_stats(server))


def sg_server_destroy(server):
    load().sg_server_destroy(server)


def sg_frame_set_timing(frame, on):
    _check(load().sg_frame_set_timing(frame, int(on)))


def sg_frame_timing(frame):
    ms = (C.c_float * 4)()
    _check(load().sg_frame_timing(frame, ms))
    return list(ms)


def sg_frame_sync_outputs(frame):
    _check(load().sg_frame_sync_outputs(frame))


def sg_frame_set_backward_state(frame, keep):
    _check(load().sg_frame_set_backward_state(frame, int(bool(keep))))


def sg_frame_status(frame, stream=0):
    _check(load().sg_frame_status(frame, stream))


def sg_alloc_count():
    return load().sg_alloc_count()


def sg_workspace_bytes(scene, sensor_kind, n_rays):
    b = C.c_size_t()
    _check(load().sg_workspace_bytes(scene, sensor_kind, n_rays, C.byref(b)))
    return b.value


def sg_frame_workspace_bytes(frame):
    b = C.c_size_t()
    _check(load().sg_frame_workspace_bytes(frame, C.byref(b)))
    return b.value


def sg_debug_lookback(max_spins=0, hold_site=LOOKBACK_NONE, hold_tile=-1):
    _check(load().sg_debug_lookback(max_spins, hold_site, hold_tile))


def sg_debug_bulk_wait(give_up):
    _check(load().sg_debug_bulk_wait(1 if give_up else 0))


def sg_frame_marks(frame, ref):
    ms = (C.c_float * 5)()
    _check(load().sg_frame_marks(frame, ref, ms))
    return list(ms)


def sg_frame_set_capacity(frame, max_pairs):
    _check(load().sg_frame_set_capacity(frame, int(max_pairs)))


def sg_frame_dropped_pairs(frame):
    """(dropped, kept) pairs of the last capacity-mode render on `frame`."""
    d, k = C.c_int64(), C.c_int64()
    _check(load().sg_frame_dropped_pairs(frame, C.byref(d), C.byref(k)))
    return d.value, k.value


# ------------------------------------------------------------ torch helpers
def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Scene:
    """A Gaussian scene resident on the device (library-owned copy)."""

    def __init__(self, src, stream=None):
        torch = _torch()
        arrs = [src.means, src.log_scales, src.quats, src.opacity, src.features]
        self._dev = [a if isinstance(a, torch.Tensor) else torch.from_numpy(
            np.ascontiguousarray(a, np.float32)) for a in arrs]
        self._dev = [t.to("cuda", torch.float32).contiguous() for t in self._dev]
        self.n = int(self._dev[0].shape[0])
        self.feature_kind = int(src.feature_kind)
        self.sh_degree = int(getattr(src, "sh_degree", 0))
        self.F = int(self._dev[4].shape[1]) if self.n else 3
        desc = self._desc()
        self.handle = sg_create_scene(desc, _stream_ptr(stream))
        torch.cuda.current_stream().synchronize()
        self._dev = None   # the library holds its own copy
        self.n_actors = 0
        if getattr(src, "actor_of", None) is not None:
            poses = np.asarray(src.actor_poses, np.float32).reshape(-1, 12)
            self.set_actors(src.actor_of, poses.shape[0], stream)
            self.set_actor_poses(poses, stream)

    def set_actors(self, actor_of, n_actors, stream=None):
        """actor_of: [n] actor index per Gaussian (-1 static); None with
        n_actors = 0 makes every Gaussian static."""
        torch = _torch()
        a = None
        if actor_of is not None:
            a = torch.as_tensor(np.ascontiguousarray(actor_of, np.int32)).to("cuda")
            torch.cuda.current_stream().synchronize()
        _check(load().sg_scene_set_actors(self.handle, a.data_ptr() if a is not None else None,
                                          int(n_actors), _P(_stream_ptr(stream))))
        self.n_actors = int(n_actors)

    def set_actor_poses(self, poses, stream=None):
        p = np.ascontiguousarray(poses, np.float32).reshape(-1)
        _check(load().sg_scene_set_actor_poses(
            self.handle, p.ctypes.data_as(C.POINTER(C.c_float)), _P(_stream_ptr(stream))))

    def _desc(self, tensors=None):
        t = tensors or self._dev
        return sg_gaussians_desc(self.n, *[x.data_ptr() for x in t], self.feature_kind,
                                 self.sh_degree)

    def update(self, means, log_scales, quats, opacity, features, stream=None):
        ts = [means, log_scales, quats, opacity, features]
        sg_update_scene(self.handle, self._desc(ts), _stream_ptr(stream))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            sg_destroy_scene(h)
            self.handle = None


class Camera:
    def __init__(self, cam):
        self.model, self.width, self.height = cam.model, cam.width, cam.height
        self.handle = sg_create_camera(cam.model, cam.width, cam.height, cam.fx, cam.fy,
                                       cam.cx, cam.cy, np.asarray(cam.k, np.float32))

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            sg_destroy_camera(h)
            self.handle = None


class Lidar:
    def __init__(self, L):
        self.n_beams, self.n_cols, self.n_elev_tiles = L.n_beams, L.n_cols, L.n_elev_tiles
        self.handle = sg_create_lidar(L.elevations_deg, L.n_cols, L.az0_deg,
                                      L.max_rays_per_tile, L.n_elev_tiles, L.cull_az,
                                      L.cull_el_per_tile)

    def tiling(self):
        return sg_lidar_tiling(self.handle, self.n_elev_tiles)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            sg_destroy_lidar(h)
            self.handle = None


class Frame:
    def __init__(self):
        self.handle = sg_frame_create()

    def field(self, field, dtype, width=1):
        """Copy an intermediate buffer of the last render into a torch tensor."""
        torch = _torch()
        ptr, n = sg_frame_field(self.handle, field)
        itemsize = np.dtype(dtype).itemsize * width
        out = torch.empty(n * itemsize, dtype=torch.uint8, device="cuda")
        if n:
            cudart = _cudart()
            torch.cuda.current_stream().synchronize()
            r = cudart.cudaMemcpy(C.c_void_p(out.data_ptr()), C.c_void_p(ptr),
                                  C.c_size_t(n * itemsize), 3)
            if r != 0:
                raise RuntimeError(f"cudaMemcpy failed ({r})")
        return out.cpu().numpy().view(dtype).reshape((n, width) if width > 1 else (n,))

    def stats(self):
        return sg_frame_stats(self.handle)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h:
            sg_frame_destroy(h)
            self.handle = None


_cudart_lib = None


def _cudart():
    global _cudart_lib
    if _cudart_lib is None:
        load()
        _cudart_lib = C.CDLL("libcudart.so.13")
        _cudart_lib.cudaMemcpy.restype = C.c_int
        _cudart_lib.cudaMemcpy.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t, C.c_int]
    return _cudart_lib


def render_camera(scene: Scene, cam: Camera, c2w, opts=None, frame: Frame | None = None,
                  stream=None):
    """Render RGB [H,W,3], alpha [H,W], depth [H,W] as CUDA tensors."""
    torch = _torch()
    opts = opts or sg_default_opts()
    frame = frame or Frame()
    rgb = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    alpha = torch.empty((cam.height, cam.width), dtype=torch.float32, device="cuda")
    depth = torch.empty((cam.height, cam.width), dtype=torch.float32, device="cuda")
    sg_render_camera(scene.handle, cam.handle, c2w, opts, frame.handle, rgb.data_ptr(),
                     alpha.data_ptr(), depth.data_ptr(), _stream_ptr(stream))
    return dict(rgb=rgb, alpha=alpha, depth=depth, frame=frame)


def render_camera_rs(scene: Scene, cam: Camera, row_c2w, opts=None, frame: Frame | None = None,
                     stream=None):
    """Rolling-shutter render: row_c2w [H, 12] per-row poses.  The returned
    dict keeps the device copy of the poses alive (the backward reads them)."""
    torch = _torch()
    opts = opts or sg_default_opts()
    frame = frame or Frame()
    poses = row_c2w if isinstance(row_c2w, torch.Tensor) else torch.from_numpy(
        np.ascontiguousarray(row_c2w, np.float32))
    poses = poses.to("cuda", torch.float32).contiguous()
    rgb = torch.empty((cam.height, cam.width, 3), dtype=torch.float32, device="cuda")
    alpha = torch.empty((cam.height, cam.width), dtype=torch.float32, device="cuda")
    depth = torch.empty((cam.height, cam.width), dtype=torch.float32, device="cuda")
    sg_render_camera_rs(scene.handle, cam.handle, poses.data_ptr(), opts, frame.handle,
                        rgb.data_ptr(), alpha.data_ptr(), depth.data_ptr(), _stream_ptr(stream))
    return dict(rgb=rgb, alpha=alpha, depth=depth, frame=frame, poses=poses)


def render_lidar(scene: Scene, lid: Lidar, col_c2w, opts=None, frame: Frame | None = None,
                 stream=None):
    """Render range, intensity, drop probability and alpha, each [beams, cols]."""
    torch = _torch()
    opts = opts or sg_default_opts()
    frame = frame or Frame()
    poses = col_c2w if isinstance(col_c2w, torch.Tensor) else torch.from_numpy(
        np.ascontiguousarray(col_c2w, np.float32))
    poses = poses.to("cuda", torch.float32).contiguous()
    shape = (lid.n_beams, lid.n_cols)
    out = {k: torch.empty(shape, dtype=torch.float32, device="cuda")
           for k in ("range", "intensity", "drop", "alpha")}
    sg_render_lidar(scene.handle, lid.handle, poses.data_ptr(), opts, frame.handle,
                    out["range"].data_ptr(), out["intensity"].data_ptr(),
                    out["drop"].data_ptr(), out["alpha"].data_ptr(), _stream_ptr(stream))
    out["frame"] = frame
    out["poses"] = poses
    return out
