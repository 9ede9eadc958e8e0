"""Python side of the request server (sg_server_* in the C-ABI) and a
Poisson load driver for the serving measurement.

The server itself -- admission, worker streams, latency accounting -- is
C++ inside libsimgut; this module marshals requests and schedules arrivals.
"""
from __future__ import annotations

import ctypes as C
import threading
import time

import numpy as np

from . import simgut as sg


class Server:
    def __init__(self, n_slots=4, memory_budget=0, queue_capacity=4096, use_graphs=True,
                 fifo_priority=True, max_batch=4):
        cfg = sg.sg_default_server_config(n_slots=n_slots, memory_budget=memory_budget,
                                          queue_capacity=queue_capacity,
                                          use_graphs=int(bool(use_graphs)),
                                          fifo_priority=int(bool(fifo_priority)),
                                          max_batch=int(max_batch))
        self.handle = sg.sg_server_create(cfg)

    @staticmethod
    def camera_request(scene, cam, c2w, outs, opts=None):
        r = sg.sg_request()
        r.kind = sg.REQ_CAMERA
        r.scene = scene.handle
        r.camera = cam.handle
        r.c2w[:] = [float(v) for v in np.asarray(c2w, np.float32).reshape(12)]
        for i, t in enumerate(outs[:3]):
            r.d_out[i] = t.data_ptr() if t is not None else None
        r.opts = opts or sg.sg_default_opts()
        return r

    @staticmethod
    def lidar_request(scene, lid, d_poses, outs, opts=None):
        r = sg.sg_request()
        r.kind = sg.REQ_LIDAR
        r.scene = scene.handle
        r.lidar = lid.handle
        r.d_col_c2w = d_poses.data_ptr()
        for i, t in enumerate(outs[:4]):
            r.d_out[i] = t.data_ptr() if t is not None else None
        r.opts = opts or sg.sg_default_opts()
        return r

    def submit(self, req):
        return sg.sg_server_submit(self.handle, req)

    def wait(self, ticket, timeout_s=60.0):
        return sg.sg_server_wait(self.handle, ticket, timeout_s)

    def drain(self, timeout_s=600.0):
        sg.sg_server_drain(self.handle, timeout_s)

    def stats(self):
        return sg.sg_server_stats(self.handle)

    def reset_stats(self):
        sg.sg_server_reset_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            sg.sg_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()


def poisson_arrivals(n, rate_per_s, seed):
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, n))


def run_open_loop(server, requests, arrivals, timeout_s=600.0):
    """Submit requests[i] at time arrivals[i] (seconds from now) from a
    dedicated thread, wait for all, return the server's statistics."""
    server.reset_stats()
    tickets = [None] * len(requests)
    errors = []

    def feeder():
        t0 = time.perf_counter()
        for i, (req, t) in enumerate(zip(requests, arrivals)):
            dt = t0 + t - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            while True:
                try:
                    tickets[i] = server.submit(req)
                    break
                except sg.SimgutError as e:     # queue full: retry shortly
                    if e.status != -6:
                        errors.append(e)
                        return
                    time.sleep(0.0005)

    th = threading.Thread(target=feeder)
    th.start()
    th.join()
    for t in tickets:
        if t is not None:
            server.wait(t, timeout_s)
    if errors:
        raise errors[0]
    return server.stats()


def run_one_per_launch(requests, render_fn):
    """The baseline: one request at a time through the plain render call,
    each synchronised before the next.  Returns (requests/s, Mrays/s,
    latencies in ms)."""
    import torch
    lat = []
    rays = 0
    t0 = time.perf_counter()
    for req in requests:
        t = time.perf_counter()
        rays += render_fn(req)
        torch.cuda.synchronize()
        lat.append((time.perf_counter() - t) * 1e3)
    span = time.perf_counter() - t0
    return len(requests) / span, rays / span / 1e6, np.array(lat)


def run_one_per_launch_open_loop(requests, arrivals, render_fn):
    """The same baseline under the server's arrival process: one host thread
    renders the requests one at a time in arrival order (each waits for the
    one before it), latency from arrival to completion.  Returns (Mrays/s
    over the span, latencies in ms)."""
    import torch
    lat = []
    rays = 0
    t0 = time.perf_counter()
    for req, t in zip(requests, arrivals):
        dt = t0 + t - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        rays += render_fn(req)
        torch.cuda.synchronize()
        lat.append((time.perf_counter() - (t0 + t)) * 1e3)
    span = time.perf_counter() - (t0 + arrivals[0])
    return rays / span / 1e6, np.array(lat)


# ---------------------------------------------------------------- workload
class ServingWorkload:
    """Resident scenes, sensors and a seeded request stream.

    Scenes: for each size, 2/3 of the Gaussians form a camera scene (degree-3
    SH) and 1/3 a LiDAR scene, from the street generator with their own
    seeds.  Requests: 25% each of pinhole 1920x1080, fisheye 1280x960,
    LiDAR 64x1024 and LiDAR 128x2048, scene chosen uniformly, random pose
    along the street."""

    KINDS = ("pinhole", "fisheye", "lidar64", "lidar128")

    def __init__(self, sizes=(500_000, 1_500_000, 3_000_000), n_requests=400, seed=3,
                 ring=12, pinhole=(1920, 1080), fisheye=(1280, 960)):
        import torch
        from . import synthetic as syn
        self.scenes = []
        for i, n in enumerate(sizes):
            nc = (2 * n) // 3
            cam = syn.street_scene(nc, seed=100 + i, kind="camera")
            lid = syn.street_scene(n - nc, seed=200 + i, kind="lidar")
            self.scenes.append((sg.Scene(cam), sg.Scene(lid)))
        fish0, pin0 = syn.street_cameras()
        pin = syn.Camera(pin0.model, pinhole[0], pinhole[1], 1000.0, 1000.0,
                         pinhole[0] / 2, pinhole[1] / 2, pin0.k, pin0.c2w)
        fish = syn.Camera(fish0.model, fisheye[0], fisheye[1], 430.0, 430.0, fisheye[0] / 2,
                          fisheye[1] / 2, fish0.k, fish0.c2w)
        self.cams = {"pinhole": (pin, sg.Camera(pin)), "fisheye": (fish, sg.Camera(fish))}
        l64 = syn.street_lidar(n_beams=64, n_cols=1024)
        l128 = syn.street_lidar()
        self.lidars = {"lidar64": (l64, sg.Lidar(l64)), "lidar128": (l128, sg.Lidar(l128))}
        rng = np.random.default_rng(seed)
        self.kinds = rng.integers(0, 4, n_requests)
        self.scene_of = rng.integers(0, len(sizes), n_requests)
        self.poses = []
        for k in self.kinds:
            name = self.KINDS[k]
            if name in self.cams:
                self.poses.append(syn.random_street_pose_camera(rng, self.cams[name][0]).c2w)
            else:
                L = syn.random_street_pose_lidar(rng, self.lidars[name][0])
                self.poses.append(torch.from_numpy(L.col_c2w).cuda())
        # output rings, one per request kind
        self.outs = {}
        for name, (c, _) in self.cams.items():
            self.outs[name] = [[torch.empty((c.height, c.width, 3), device="cuda"),
                                torch.empty((c.height, c.width), device="cuda"),
                                torch.empty((c.height, c.width), device="cuda")]
                               for _ in range(ring)]
        for name, (L, _) in self.lidars.items():
            self.outs[name] = [[torch.empty((L.n_beams, L.n_cols), device="cuda")
                                for _ in range(4)] for _ in range(ring)]
        self.ring = ring

    def rays(self, i):
        name = self.KINDS[self.kinds[i]]
        if name in self.cams:
            c = self.cams[name][0]
            return c.width * c.height
        L = self.lidars[name][0]
        return L.n_beams * L.n_cols

    def request(self, i, outs=None):
        name = self.KINDS[self.kinds[i]]
        cs, ls = self.scenes[self.scene_of[i]]
        o = outs if outs is not None else self.outs[name][i % self.ring]
        if name in self.cams:
            return Server.camera_request(cs, self.cams[name][1], self.poses[i], o)
        return Server.lidar_request(ls, self.lidars[name][1], self.poses[i], o)

    def render_plain(self, i, frame, stream, outs=None):
        """Render request i through the plain (one call, one request) API."""
        name = self.KINDS[self.kinds[i]]
        cs, ls = self.scenes[self.scene_of[i]]
        o = outs if outs is not None else self.outs[name][i % self.ring]
        opts = sg.sg_default_opts()
        if name in self.cams:
            sg.sg_render_camera(cs.handle, self.cams[name][1].handle, self.poses[i], opts,
                                frame.handle, *[t.data_ptr() for t in o], stream)
        else:
            sg.sg_render_lidar(ls.handle, self.lidars[name][1].handle, self.poses[i].data_ptr(),
                               opts, frame.handle, *[t.data_ptr() for t in o], stream)
        return self.rays(i)


def measure_serving(n_requests=300, loads=(0.5, 0.8, 1.0, 1.2, 2.0), n_slots=4, seed=3,
                    memory_budget=0, **kw):
    """One-request-per-launch capacity, then open-loop Poisson arrivals at
    each load (a multiple of that capacity): Mrays/s and p50/p99 latency."""
    import torch
    W = ServingWorkload(n_requests=n_requests, seed=seed, **kw)
    frame = sg.Frame()
    sg.sg_frame_set_backward_state(frame.handle, 0)   # forward renders only, as the server's
    stream = torch.cuda.current_stream().cuda_stream
    for i in range(min(8, n_requests)):                 # warm the frame up
        W.render_plain(i, frame, stream)
    torch.cuda.synchronize()
    rps, mrays, lat = run_one_per_launch(range(n_requests),
                                         lambda i: W.render_plain(i, frame, stream))
    base = {"requests_per_s": rps, "mrays_per_s": mrays,
            "latency_p50_ms": float(np.percentile(lat, 50)),
            "latency_p99_ms": float(np.percentile(lat, 99)),
            "latency_note": "closed loop: each request's render alone, no queueing"}
    # the baseline under the same Poisson arrivals as the server (queueing
    # included), at the loads where it can keep up or nearly so
    base_open = []
    for load in [l for l in loads if l <= 1.0]:
        arr = poisson_arrivals(n_requests, load * rps, seed + int(load * 100))
        m, lo = run_one_per_launch_open_loop(range(n_requests), arr,
                                             lambda i: W.render_plain(i, frame, stream))
        base_open.append({"load": load, "mrays_per_s": m,
                          "latency_p50_ms": float(np.percentile(lo, 50)),
                          "latency_p99_ms": float(np.percentile(lo, 99))})
    reqs = [W.request(i) for i in range(n_requests)]

    def sweep(max_batch, load_list):
        srv = Server(n_slots=n_slots, memory_budget=memory_budget, max_batch=max_batch)
        # warm up: two bursts of the whole stream and one pass at the highest
        # load, so that every slot has grown its workspace and captured the
        # graphs of the combinations (and batch sizes) it serves
        for _ in range(2):
            warm = [srv.submit(r) for r in reqs]
            for t in warm:
                srv.wait(t)
        run_open_loop(srv, reqs, poisson_arrivals(n_requests, max(load_list) * rps, seed + 999))
        res = []
        for load in load_list:
            arr = poisson_arrivals(n_requests, load * rps, seed + int(load * 100))
            st = run_open_loop(srv, reqs, arr)
            res.append({"load": load, "offered_requests_per_s": load * rps,
                        "mrays_per_s": st["mrays_per_s"], "latency_p50_ms": st["latency_p50_ms"],
                        "latency_p99_ms": st["latency_p99_ms"], "completed": st["completed"],
                        "peak_in_flight": st["peak_in_flight"],
                        "graph_replays": st["graph_replays"],
                        "graph_captures": st["graph_captures"],
                        "overflow_rerenders": st["overflow_rerenders"],
                        "batches": st["batches"], "batched_requests": st["batched_requests"]})
        srv.close()
        return res

    out = sweep(4, loads)
    # the same server without batching
    single = sweep(1, loads)
    return {"one_request_per_launch": base, "one_request_per_launch_open_loop": base_open,
            "server": out, "server_no_batching": single,
            "n_slots": n_slots,
            "requests_per_load": n_requests,
            "mix": "25% each pinhole 1920x1080, fisheye 1280x960, LiDAR 64x1024, LiDAR 128x2048; "
                   "scenes of 0.5M/1.5M/3M Gaussians (2/3 camera, 1/3 LiDAR)"}
