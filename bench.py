#!/usr/bin/env python3
"""Throughput benchmark of the forward render (rendered Mrays/s).

Workload (one step): the synthetic street camera scene -- 1M Gaussians with
degree-3 SH colour -- rendered into one 1920x1280 OpenCV-fisheye view and one
1920x1080 pinhole view (RGB, alpha, depth): 4,531,200 rays per step.  The
scene is resident in HBM before timing starts; each step re-runs projection,
depth sort, binning, tile sort and compositing for both views.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One JSON line on rank 0.  N > 1 runs one process per GPU (torchrun), each
rendering the same workload (replicas, weak scaling): value = all ranks'
rays / max-over-ranks time.  --impl reference times the CPU oracle (the
plain C implementation written from the paper) on a bounded sample of the
same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rendered Mrays/s per GB300 (camera px + LiDAR rays); p50/p99 latency in serving loop"
WORKLOAD = ("street camera scene: 1M Gaussians (degree-3 SH), one 1920x1280 OpenCV-fisheye "
            "view + one 1920x1080 pinhole view per step, forward RGB+alpha+depth")
N_GAUSS = 1_000_000
# algorithmic FP32 work per evaluated (ray, Gaussian) pair: closest approach
# of the ray to the Gaussian in its own frame (M d: 15, moment cross product
# 9, two squared norms 10, dot product 5, two divisions 2), response and
# alpha (exp, product, clamp: 3), compositing (transmittance 2, weight 1,
# colour 6, depth 2, opacity 1): 56 flops
FLOP_PER_PAIR = 56
FP32_LANES = 128          # FP32 lanes per SM (Blackwell SM: 4 partitions x 32)


def sm_count():
    """Multiprocessors of the current device (cudaDevAttrMultiProcessorCount)."""
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serving-requests", type=int, default=300)
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the LiDAR sweep and differentiable-step measurements")
    ap.add_argument("--stream-sets", type=int, default=1, choices=[1, 2],
                    help="stream (and output) sets the steps alternate between: 2 lets a step's "
                         "front stages start while the previous step's compositing runs")
    ap.add_argument("--only", choices=["lidar", "serving"], default=None,
                    help="run one extra workload alone (for profiling) and print its line")

    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ------------------------------------------------------------------ ranks
def max_over_ranks(x, world, device):
    """The largest value of x over all ranks (the slowest rank's time)."""
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms_max):
    """Whole-job throughput (Munits/s): every rank processes units_per_rank
    in parallel, the job takes as long as the slowest rank."""
    return world * units_per_rank / (ms_max * 1e-3) / 1e6


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL,
                stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            if self.uuid and parts[1] != self.uuid:
                continue
            rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        smax = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i] == "Active"})
        load = [s for s in sm if smax and s > 0.5 * max(smax)] or sm
        return {"sm_mhz": float(np.median(load)) if load else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(rows)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def forward_frame(sg):
    """A frame for forward renders only: no per-ray state for a backward."""
    f = sg.Frame()
    sg.sg_frame_set_backward_state(f.handle, 0)
    return f


# ------------------------------------------------------------------ ours
def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_2510_12901_gb300 import _build
    _build.build()
    from paper_2510_12901_gb300 import simgut as sg
    from paper_2510_12901_gb300 import synthetic as syn

    if args.only == "lidar":
        return lidar_workload(torch, sg, syn, args.steps, args.warmup)
    if args.only == "serving":
        from paper_2510_12901_gb300 import serve
        return serve.measure_serving(n_requests=args.serving_requests)
    sc = syn.street_scene(N_GAUSS, seed=0, kind="camera")
    fish, pin = syn.street_cameras()
    S = sg.Scene(sc)
    cams = [(sg.Camera(fish), fish), (sg.Camera(pin), pin)]
    rays_per_step = sum(c.width * c.height for _, c in cams)
    nset = args.stream_sets
    out_sets = []
    for _ in range(nset):
        out_sets.append([[torch.empty((c.height, c.width, 3), device="cuda"),
                          torch.empty((c.height, c.width), device="cuda"),
                          torch.empty((c.height, c.width), device="cuda")] for _, c in cams])
    outs = out_sets[0]
    opts = sg.sg_default_opts()
    # two frame sets, alternated, so that the stage events of step i can be
    # read once step i+1 has passed its own mid-render synchronisation
    frames = [[forward_frame(sg) for _ in cams] for _ in range(2)]
    for fs in frames:
        for f in fs:
            sg.sg_frame_set_timing(f.handle, 1)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    # the two views of a step are one sg_render_cameras call, each view on
    # its own stream (a camera rig rendered per frame)
    # with two sets, step i uses stream set i % 2 (and output set i % 2), so
    # that step i+1's front stages can run while step i's compositing does
    vsets = [[torch.cuda.Stream() for _ in cams] for _ in range(nset)]
    vstreams = vsets[0]
    views = [sg.sg_camera_views([(ch.handle, c.c2w, f.handle, o[0].data_ptr(), o[1].data_ptr(),
                                  o[2].data_ptr(), vs.cuda_stream)
                                 for (ch, c), o, f, vs in zip(cams, out_sets[k % nset], fs,
                                                              vsets[k % nset])])
             for k, fs in enumerate(frames)]

    def fork():          # the view streams start after the work queued on `stream`
        ev = torch.cuda.Event()
        ev.record(stream)
        for vset in vsets:
            for vs in vset:
                vs.wait_event(ev)

    def join():          # `stream` continues once every view stream is done
        for vset in vsets:
            for vs in vset:
                ev = torch.cuda.Event()
                ev.record(vs)
                stream.wait_event(ev)

    def step(i):
        sg.sg_render_cameras(S.handle, views[i % 2], opts, 0)

    stage_ms = []
    render_union = []    # per step: time during which a view's compositing ran

    def harvest(i):
        fs = frames[i % 2]
        for f in fs:
            stage_ms.append(sg.sg_frame_timing(f.handle))
        iv = sorted(tuple(sg.sg_frame_marks(f.handle, fs[0].handle)[3:5]) for f in fs)
        tot, cur = 0.0, None
        for a, b in iv:
            if cur is None or a > cur[1]:
                tot += 0.0 if cur is None else cur[1] - cur[0]
                cur = [a, b]
            else:
                cur[1] = max(cur[1], b)
        render_union.append(tot + cur[1] - cur[0])

    fork()
    for i in range(args.warmup):
        step(i)
    join()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        uuid = None
    clk = ClockSampler(uuid)
    clk.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    l0 = sg.sg_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    t0 = time.perf_counter()
    e0.record(stream)
    fork()
    for i in range(args.steps):
        step(i)
        if i > 0:
            harvest(i - 1)
    join()
    e1.record(stream)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    harvest(args.steps - 1)
    launches = sg.sg_launch_count() - l0
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    dev_ms = e0.elapsed_time(e1) / args.steps
    wall_ms = (t1 - t0) * 1e3 / args.steps
    ms = max_over_ranks(dev_ms, world, "cuda")
    value = job_rate(rays_per_step, world, ms)

    # per-stage averages over the timed steps (ms per render)
    st = np.array(stage_ms)            # [2*steps, 4]: project, depth sort, bin+sort, render
    per_view = st.reshape(-1, len(cams), 4).mean(axis=0)
    stages = {"project": per_view[:, 0].tolist(), "depth_sort_offsets": per_view[:, 1].tolist(),
              "bin_tile_sort_ranges": per_view[:, 2].tolist(), "render": per_view[:, 3].tolist(),
              "views": ["fisheye", "pinhole"],
              "note": "events on each view's stream; the views overlap, so a view's stage "
                      "may include time the GPU spent on the other view"}

    # per-stage rooflines from a short sequential run (one view at a time on
    # `stream`, so that each stage's events time that stage alone)
    seq = []
    for i in range(12):
        for (ch, c), o, f in zip(cams, outs, frames[0]):
            sg.sg_render_camera(S.handle, ch.handle, c.c2w, opts, f.handle, o[0].data_ptr(),
                                o[1].data_ptr(), o[2].data_ptr(), sp)
            if i >= 2:
                seq.append(sg.sg_frame_timing(f.handle))
    torch.cuda.synchronize()
    seq_view = np.array(seq).reshape(-1, len(cams), 4).mean(axis=0)
    pairs = [sg.sg_frame_stats(f.handle)[0] for f in frames[0]]
    stage_roof = stage_rooflines(seq_view, pairs, N_GAUSS)

    # end-to-end through the C-ABI with host (pinned) output buffers, two
    # sets of buffers and frames: each step's copies are queued with it
    # (host_outputs = 2) and the host reads step i - 1's results once step i
    # is queued, as a pipelined caller does; the synchronous call (each step
    # waits for its own copies) is timed too
    e2e_steps = max(3, min(args.steps, 40))
    hsets = []
    for _ in range(2):
        host = []
        for _, c in cams:
            n = c.width * c.height
            host.append([torch.empty(3 * n, dtype=torch.float32).pin_memory(),
                         torch.empty(n, dtype=torch.float32).pin_memory(),
                         torch.empty(n, dtype=torch.float32).pin_memory()])
        ef = [forward_frame(sg) for _ in cams]
        hsets.append((host, ef, sg.sg_camera_views(
            [(ch.handle, c.c2w, f.handle, h[0].data_ptr(), h[1].data_ptr(), h[2].data_ptr(),
              vs.cuda_stream) for (ch, c), h, f, vs in zip(cams, host, ef, vstreams)])))

    def e2e_run(steps, mode):
        for i in range(steps):
            sg.sg_render_cameras(S.handle, hsets[i % 2][2], opts, mode)
            if mode == 2 and i > 0:
                for f in hsets[(i - 1) % 2][1]:
                    sg.sg_frame_sync_outputs(f.handle)   # step i - 1's results are in host memory
        for f in hsets[(steps - 1) % 2][1]:
            sg.sg_frame_sync_outputs(f.handle)
        torch.cuda.synchronize()

    e2e_out = {}
    for mode in (1, 2):
        e2e_run(2, mode)
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        e2e_run(e2e_steps, mode)
        e2e_out[mode] = max_over_ranks((time.perf_counter() - t0) * 1e3 / e2e_steps, world,
                                       "cuda")
    e2e_ms = e2e_out[2]
    d2h = sum(4 * 5 * c.width * c.height for _, c in cams)
    e2e = {"value": job_rate(rays_per_step, world, e2e_ms), "unit": "Mrays/s",
           "h2d_bytes_per_step": 2 * 12 * 4, "d2h_bytes_per_step": d2h,
           "ms_per_step": e2e_ms, "steps": e2e_steps,
           "path": "sg_render_cameras with host outputs (pinned buffers, two sets; the views on "
                   "two streams; each step's copies queued with it, step i - 1's results waited "
                   "for once step i is queued; every copy inside the timed region)",
           "synchronous": {"value": job_rate(rays_per_step, world, e2e_out[1]),
                           "ms_per_step": e2e_out[1],
                           "path": "the same call with host_outputs = 1: each step returns once "
                                   "its own copies are done"}}

    result = None
    if rank == 0:
        roof = roofline(per_view, float(np.mean(render_union)), seq_view, clocks)
        result = {
            "metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "gaussians": N_GAUSS,
                       "rays_per_step": rays_per_step, "parallelism": "replicas",
                       "views": "one sg_render_cameras call per step, each view on its own stream",
                       "stream_sets": nset,
                       "pair_counts": "exact (the host waits for each view's pair count)",
                       "frames": "forward only (sg_frame_set_backward_state 0: no per-ray "
                                 "state for a backward is written)",
                       "l2": "inputs larger than L2 (236 MB of scene planes read per view)",
                       "wall_ms_per_step": wall_ms},
            "roofline": roof, "e2e": e2e, "gpu_launches": int(launches),
            "launches_per_step": launches / args.steps,
            "clocks": clocks, "stages_ms": stages, "stage_rooflines": stage_roof,
        }
        if world == 1 and not args.no_cpu_baseline:
            result["cpu_baseline"] = cpu_baseline(sc, [c for _, c in cams], budget_s=20.0)
            result["cpu_baseline_all_cores"] = cpu_baseline_all_cores([c for _, c in cams])
    if rank == 0 and not args.no_extra:
        del S, frames, ef
        result["lidar"] = lidar_workload(torch, sg, syn, min(args.steps, 100), 5)
        result["lidar"]["sh_features"] = lidar_workload(torch, sg, syn, min(args.steps, 100), 5,
                                                        kind="lidar_sh")
        result["lidar"]["beam_divergence"] = lidar_workload(torch, sg, syn, min(args.steps, 100),
                                                            5, beam=0.003)
        result["train_step"] = train_step_workload(torch, sg, syn, min(args.steps, 30), 3)
        result["actors"] = actors_workload(torch, sg, syn, min(args.steps, 100), 5)
        result["rolling_shutter"] = rolling_shutter_workload(torch, sg, syn, min(args.steps, 100), 5)
    if not args.no_serving:
        from paper_2510_12901_gb300 import serve
        srv = serve.measure_serving(n_requests=args.serving_requests)
        if rank == 0:
            result["serving"] = srv
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return result


def _work(view):
    try:
        work = json.load(open(os.path.join(ROOT, "tests", "golden", "bench_work.json")))
        return work["views"][view]["evaluated_pairs"]
    except (OSError, KeyError, ValueError):
        return None


def lidar_workload(torch, sg, syn, steps, warmup, kind="lidar", beam=0.0):
    """The LiDAR sweep configuration: 2M LiDAR Gaussians, 128 beams x 2048
    columns, per-column poses over a 0.1 s sweep; range, intensity, drop and
    alpha per ray.  CUDA events over `steps` sweeps, inputs resident.
    kind='lidar_sh': the same scene with degree-3 SH^l features."""
    sc = syn.street_scene(2_000_000, seed=0, kind=kind)
    L = syn.street_lidar()
    S, Ld = sg.Scene(sc), sg.Lidar(L)
    poses = torch.from_numpy(np.ascontiguousarray(L.col_c2w, np.float32)).cuda()
    outs = [torch.empty((L.n_beams, L.n_cols), device="cuda") for _ in range(4)]
    frames = [forward_frame(sg), forward_frame(sg)]
    for f in frames:
        sg.sg_frame_set_timing(f.handle, 1)
    opts = sg.sg_default_opts(beam_divergence=beam)
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream

    def sweep(i):
        sg.sg_render_lidar(S.handle, Ld.handle, poses.data_ptr(), opts, frames[i % 2].handle,
                           *[o.data_ptr() for o in outs], sp)

    for i in range(warmup):
        sweep(i)
    torch.cuda.synchronize()
    stage = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(steps):
        sweep(i)
        if i > 0:
            stage.append(sg.sg_frame_timing(frames[(i - 1) % 2].handle))
    e1.record(stream)
    torch.cuda.synchronize()
    stage.append(sg.sg_frame_timing(frames[(steps - 1) % 2].handle))
    ms = e0.elapsed_time(e1) / steps
    st = np.array(stage).mean(axis=0)
    rays = L.n_beams * L.n_cols
    feats = ("intensity, ray-drop logits" if kind == "lidar" else
             "degree-3 SH^l of intensity and ray-drop logits, 48 floats")
    if beam > 0:
        feats += f"; beam divergence {beam * 1e3:g} mrad (Eq. 6 smoothing)"
    out = {"workload": f"street LiDAR scene: 2M Gaussians ({feats}), 128-beam "
                       "x 2048-column sweep, per-column poses over 0.1 s; range + intensity + drop",
           "value": rays / (ms * 1e-3) / 1e6, "unit": "Mrays/s", "ms_per_sweep": ms,
           "steps": steps, "stages_ms": {"project": st[0], "depth_sort_offsets": st[1],
                                         "bin_tile_sort_ranges": st[2], "render": st[3]}}
    pairs = _work("lidar")
    if pairs and kind == "lidar" and beam == 0:
        pk = peaks()
        peak = sm_count() * FP32_LANES * 2 * float(pk.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
        ach = pairs * FLOP_PER_PAIR / (st[3] * 1e-3) / 1e12
        out["roofline"] = {"kernel": "k_render_lidar_fwd", "bound": "alu", "achieved": ach,
                           "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                           "evaluated_pairs": pairs}
    return out


def actors_workload(torch, sg, syn, steps, warmup):
    """The street camera step with dynamic actors: 10% of the 1M Gaussians
    belong to 16 car-sized actors placed by their poses before projection.
    One sg_render_cameras call per step, the two views on two streams."""
    sc = syn.with_actors(syn.street_scene(N_GAUSS, seed=0, kind="camera"), n_actors=16,
                         frac=0.1)
    S = sg.Scene(sc)
    cams = [(sg.Camera(c), c) for c in syn.street_cameras()]
    outs = [[torch.empty((c.height, c.width, 3), device="cuda"),
             torch.empty((c.height, c.width), device="cuda"),
             torch.empty((c.height, c.width), device="cuda")] for _, c in cams]
    frames = [forward_frame(sg) for _ in cams]
    vs = [torch.cuda.Stream() for _ in cams]
    views = sg.sg_camera_views([(ch.handle, c.c2w, f.handle, o[0].data_ptr(), o[1].data_ptr(),
                                 o[2].data_ptr(), v.cuda_stream)
                                for (ch, c), o, f, v in zip(cams, outs, frames, vs)])
    opts = sg.sg_default_opts()
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        sg.sg_render_cameras(S.handle, views, opts, 0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ev = torch.cuda.Event()
    ev.record(stream)
    for v in vs:
        v.wait_event(ev)
    for _ in range(steps):
        sg.sg_render_cameras(S.handle, views, opts, 0)
    for v in vs:
        e = torch.cuda.Event()
        e.record(v)
        stream.wait_event(e)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    rays = sum(c.width * c.height for _, c in cams)
    return {"workload": "street camera scene with 16 car-sized actors holding 10% of the 1M "
                        "Gaussians; fisheye 1920x1280 + pinhole 1920x1080 per step",
            "value": rays / (ms * 1e-3) / 1e6, "unit": "Mrays/s", "ms_per_step": ms,
            "steps": steps}


def rolling_shutter_workload(torch, sg, syn, steps, warmup):
    """The street camera step with rolling shutters: both views read out
    top to bottom in 30 ms while the vehicle drives at 15 m/s and turns at
    0.1 rad/s, every pixel row with its own pose (one sg_render_cameras call,
    the views on two streams)."""
    sc = syn.street_scene(N_GAUSS, seed=0, kind="camera")
    S = sg.Scene(sc)
    cams = [(sg.Camera(c), syn.rolling_shutter(c)) for c in syn.street_cameras()]
    rows = [torch.from_numpy(np.ascontiguousarray(c.row_c2w, np.float32)).cuda() for _, c in cams]
    outs = [[torch.empty((c.height, c.width, 3), device="cuda"),
             torch.empty((c.height, c.width), device="cuda"),
             torch.empty((c.height, c.width), device="cuda")] for _, c in cams]
    frames = [forward_frame(sg) for _ in cams]
    opts = sg.sg_default_opts()
    stream = torch.cuda.current_stream()
    vs = [torch.cuda.Stream() for _ in cams]
    views = sg.sg_camera_views([(ch.handle, c.c2w, f.handle, o[0].data_ptr(), o[1].data_ptr(),
                                 o[2].data_ptr(), v.cuda_stream, r.data_ptr())
                                for (ch, c), r, o, f, v in zip(cams, rows, outs, frames, vs)])

    def step():
        sg.sg_render_cameras(S.handle, views, opts, 0)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ev = torch.cuda.Event()
    ev.record(stream)
    for v in vs:
        v.wait_event(ev)
    for _ in range(steps):
        step()
    for v in vs:
        e = torch.cuda.Event()
        e.record(v)
        stream.wait_event(e)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    rays = sum(c.width * c.height for _, c in cams)
    return {"workload": "street camera scene, 1M Gaussians; fisheye 1920x1280 + pinhole "
                        "1920x1080 with rolling shutters (30 ms readout, 15 m/s, 0.1 rad/s), "
                        "one sg_render_cameras call per step, the views on two streams",
            "value": rays / (ms * 1e-3) / 1e6, "unit": "Mrays/s", "ms_per_step": ms,
            "steps": steps}


def train_step_workload(torch, sg, syn, steps, warmup):
    """The differentiable step: the 1M-Gaussian camera scene into the
    1920x1280 fisheye view and the 2M-Gaussian LiDAR scene into the 128x2048
    sweep, L1 RGB + L1 range loss against seeded noisy targets, then the
    hand-written backward to every Gaussian parameter, through the
    torch.autograd.Function wrappers (parameters copied into the resident
    scenes each step, as a training loop does)."""
    from paper_2510_12901_gb300 import autograd as ag
    csc = syn.street_scene(1_000_000, seed=0, kind="camera")
    lsc = syn.street_scene(2_000_000, seed=0, kind="lidar")
    fish, _ = syn.street_cameras()
    L = syn.street_lidar()
    cS, lS, C, Ld = sg.Scene(csc), sg.Scene(lsc), sg.Camera(fish), sg.Lidar(L)
    poses = torch.from_numpy(np.ascontiguousarray(L.col_c2w, np.float32)).cuda()

    def params(sc):
        return {k: torch.from_numpy(np.ascontiguousarray(getattr(sc, a), np.float32)).cuda()
                .requires_grad_(True)
                for k, a in (("means", "means"), ("log_scales", "log_scales"),
                             ("quats", "quats"), ("opacity", "opacity"),
                             ("features", "features"))}

    cp, lp = params(csc), params(lsc)
    t_rgb = torch.from_numpy(syn.noisy_targets((fish.height, fish.width, 3), seed=4)).cuda()
    t_rng = torch.from_numpy(syn.noisy_targets((L.n_beams, L.n_cols), seed=5, lo=0.0,
                                               hi=80.0)).cuda()
    cf, lf = sg.Frame(), sg.Frame()

    def step():
        rgb, _, _ = ag.render_camera(cp, cS, C, fish.c2w, frame=cf)
        rng, _, _, _ = ag.render_lidar(lp, lS, Ld, poses, frame=lf)
        loss = (rgb - t_rgb).abs().mean() + (rng - t_rng).abs().mean()
        for d in (cp, lp):
            for t in d.values():
                t.grad = None
        loss.backward()
        return loss

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    rays = fish.width * fish.height + L.n_beams * L.n_cols
    return {"workload": "differentiable step: 1M-Gaussian camera scene into the 1920x1280 "
                        "fisheye + 2M-Gaussian LiDAR scene into the 128x2048 sweep, L1 RGB + L1 "
                        "range loss, backward to all Gaussian parameters",
            "ms_per_step": ms, "steps": steps, "rays_per_step": rays,
            "value": rays / (ms * 1e-3) / 1e6, "unit": "Mrays/s (forward + backward)"}


def stage_rooflines(seq_view, pairs, n_gauss):
    """Per stage and view, from a sequential run: HBM stages against the
    measured copy bandwidth with their algorithmic bytes (projection 336 B
    per Gaussian: 236 read, 100 written; depth sort 64 B per Gaussian: four
    passes reading and writing an 8-byte key-value pair; binning and tile
    sort 36 B per pair: written once, then read and written by the sort),
    the compositing against the FP32 peak (as the headline roofline)."""
    pk = peaks()
    hbm = float(pk.get("hbm_gbs", 6699.8))
    views = ("fisheye", "pinhole")
    out = {"peak_hbm_gbs": hbm, "views": list(views), "ms": seq_view.tolist()}
    rows = []
    for v, (tp, td, tb, tr) in enumerate(seq_view):
        r = {"project_gbs": 336 * n_gauss / (tp * 1e-3) / 1e9,
             "depth_sort_gbs": 64 * n_gauss / (td * 1e-3) / 1e9,
             "bin_tile_sort_gbs": 36 * pairs[v] / (tb * 1e-3) / 1e9, "pairs": int(pairs[v])}
        r.update({k.replace("_gbs", "_frac"): r[k] / hbm for k in list(r) if k.endswith("_gbs")})
        rows.append(r)
    out["per_view"] = rows
    out["note"] = ("stage times from 10 sequential steps on one stream (the headline step overlaps "
                   "the views); the sort stages are latency-bound, not HBM-bound (profiles/)")
    return out


def roofline(per_view, union_ms, seq_view, clocks):
    """Dominant kernel: the compositing kernel (largest stage share).  ALU
    bound: algorithmic FP32 flops = oracle-counted evaluated pairs x 56.
    Achieved = both views' flops over the time, per timed step, during which
    the compositing of at least one view ran (the two views' render stages
    placed on one time line from their CUDA events); per view, each render
    stage alone from the sequential run."""
    work_path = os.path.join(ROOT, "tests", "golden", "bench_work.json")
    pk = peaks()
    sm_max = float(pk.get("sm_max_mhz", 2070.0))
    sms = sm_count()
    peak_tflops = sms * FP32_LANES * 2 * sm_max * 1e6 / 1e12
    render_ms = per_view[:, 3]
    out = {"kernel": "k_render_camera_fwd", "bound": "alu", "peak": peak_tflops,
           "unit": "TFLOP/s",
           "peak_source": f"derived: {sms} SMs (queried from the device) x {FP32_LANES} FP32 "
                          f"lanes x 2 flop/FMA x "
                          f"{sm_max:.0f} MHz (max SM clock, MEASURED_PEAKS.json)",
           "traffic": None}
    try:
        work = json.load(open(work_path))
        pairs = [work["views"][v]["evaluated_pairs"] for v in ("fisheye", "pinhole")]
        flops = [p * FLOP_PER_PAIR for p in pairs]
        seq_ms = seq_view[:, 3]
        ach = [f / (t * 1e-3) / 1e12 for f, t in zip(flops, seq_ms)]
        tot = sum(flops) / (union_ms * 1e-3) / 1e12
        out.update(achieved=tot, frac=tot / peak_tflops, per_view_achieved_alone=ach,
                   per_view_frac_alone=[a / peak_tflops for a in ach],
                   evaluated_pairs=pairs, flop_per_pair=FLOP_PER_PAIR,
                   render_union_ms=union_ms, launch_ms_alone=seq_ms.tolist(),
                   launch_ms_overlapped=render_ms.tolist(),
                   timing_note="achieved: both views' flops over the union of their render "
                               "stages in the timed steps (CUDA events on each view's stream, "
                               "on one time line); per view alone: the sequential run")
    except (OSError, KeyError, ValueError):
        out.update(achieved=None, frac=None, note="tests/golden/bench_work.json missing")
    try:
        tr = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
        if tr.get("source_sha256") == kernel_source_hash():
            out["traffic"] = tr.get("k_render_camera_fwd")
            out["traffic_note"] = ("dram bytes per launch, mean of the fisheye and pinhole launches "
                                   "(ncu), profiles/")
            out["traffic_per_view"] = tr.get("per_view")
        else:
            out["traffic"] = None
            out["traffic_note"] = "kernel changed since the ncu capture in profiles/"
    except (OSError, ValueError):
        out["traffic"] = None
    return out


KERNEL_SOURCES = ("render_fwd.cu", "pairs.cuh", "render.cuh")


def kernel_source_hash(read=None):
    """sha256 over the compositing kernel's sources (its files, and the
    record layout from internal.h), to tell whether the ncu counters in
    profiles/ were taken on the kernel as it stands.  `read(name)` returns a
    file's bytes (default: the working tree)."""
    import hashlib
    if read is None:
        def read(name):
            with open(os.path.join(ROOT, "paper_2510_12901_gb300", "csrc", name), "rb") as fh:
                return fh.read()
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(read(f))
    inc = read("internal.h")
    a = inc.index(b"struct __align__(16) GRec")
    h.update(inc[a:inc.index(b"};", a)])
    return h.hexdigest()


# ------------------------------------------------------------------ oracle
def _oracle_sample_time(O, sc, cam, n_rays, seed):
    rng = np.random.default_rng(seed)
    rays = rng.choice(cam.width * cam.height, n_rays, replace=False)
    t = time.perf_counter()
    O.render_camera(sc, cam, rays=rays)
    return time.perf_counter() - t


_PW = {}


def _pool_init(n_gauss):
    from oracle import Oracle
    from paper_2510_12901_gb300 import synthetic as syn
    _PW["O"] = Oracle(64)
    _PW["sc"] = syn.street_scene(n_gauss, seed=0, kind="camera")
    _PW["cams"] = list(syn.street_cameras())


def _pool_task(args):
    view, n_rays, seed = args
    return _oracle_sample_time(_PW["O"], _PW["sc"], _PW["cams"][view], n_rays, seed)


def cpu_baseline_all_cores(cams, procs=None):
    """The same oracle on every host core: one process per core, each with
    its own copy of the scene, renders a share of the view's rays (so each
    repeats the projection and sort, as the oracle does per call).  Per view,
    two share sizes give the wall time's fixed and per-ray parts, and the
    full view is extrapolated to rays / cores rays per process."""
    import multiprocessing as mp
    P = procs or os.cpu_count() or 1
    total, used = 0.0, 0.0
    with mp.get_context("spawn").Pool(P, initializer=_pool_init, initargs=(N_GAUSS,)) as pool:
        pool.map(_pool_task, [(0, 10, 7 + i) for i in range(P)])     # warm every worker
        for v, cam in enumerate(cams):
            s1, s2 = 2000, 12000
            w1 = max(pool.map(_pool_task, [(v, s1, 300 + 31 * v + i) for i in range(P)]))
            w2 = max(pool.map(_pool_task, [(v, s2, 400 + 31 * v + i) for i in range(P)]))
            used += (w1 + w2) * P
            per_ray = max(w2 - w1, 0.0) / (s2 - s1)
            fixed = max(w1 - per_ray * s1, 0.0)
            total += fixed + per_ray * math.ceil(cam.width * cam.height / P)
    rays = sum(c.width * c.height for c in cams)
    return {"value": rays / total / 1e6, "unit": "Mrays/s", "cores": P, "kind": "oracle",
            "sample": f"per view, {P} processes each render 2000 and 12000 random rays "
                      f"(each process projects and sorts all {N_GAUSS} Gaussians); the "
                      f"full view is extrapolated to its rays split over {P} processes "
                      f"({used:.0f} s of CPU work); extrapolated seconds per step {total:.1f}"}


def cpu_baseline(sc, cams, budget_s=20.0):
    """The oracle as it stands (single-threaded C, double precision) on a
    bounded sample: per view, the full projection and sort of the scene plus
    the compositing of S random rays, at two sample sizes; the full-view time
    is the linear extrapolation (fixed cost + per-ray cost x rays)."""
    from oracle import Oracle
    O = Oracle(64)
    total = 0.0
    used = 0.0
    for i, cam in enumerate(cams):
        s1, s2 = 4000, 160000
        t1 = _oracle_sample_time(O, sc, cam, s1, 100 + i)
        t2 = _oracle_sample_time(O, sc, cam, s2, 200 + i)
        used += t1 + t2
        per_ray = max(t2 - t1, 0.0) / (s2 - s1)
        fixed = max(t1 - per_ray * s1, 0.0)
        total += fixed + per_ray * cam.width * cam.height
    rays = sum(c.width * c.height for c in cams)
    return {"value": rays / total / 1e6, "unit": "Mrays/s", "cores": 1, "kind": "oracle",
            "sample": f"per view: projection + sort of all {N_GAUSS} Gaussians and compositing "
                      f"of 4000 and 160000 random rays, extrapolated linearly to the full view "
                      f"({used:.1f} s of CPU work); extrapolated seconds per step {total:.1f}"}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return None
    from oracle import Oracle
    from paper_2510_12901_gb300 import synthetic as syn
    O = Oracle(64)
    sc = syn.street_scene(N_GAUSS, seed=0, kind="camera")
    cams = list(syn.street_cameras())
    n_rays = 2000          # per view per step: a bounded sample of the step
    for i in range(args.warmup):
        for c in cams:
            _oracle_sample_time(O, sc, c, 200, i)
    t = 0.0
    for i in range(args.steps):
        for j, c in enumerate(cams):
            t += _oracle_sample_time(O, sc, c, n_rays, 1000 * i + j)
    ms = t * 1e3 / args.steps
    value = 2 * n_rays / (ms * 1e-3) / 1e6
    sample = (f"each step: per view, projection + sort of all {N_GAUSS} Gaussians and "
              f"compositing of {n_rays} random rays (2 views)")
    return {"metric": METRIC, "value": value, "unit": "Mrays/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "gaussians": N_GAUSS,
                       "rays_per_step": 2 * n_rays, "parallelism": "none (CPU)"},
            "cpu_baseline": {"value": value, "unit": "Mrays/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "Mrays/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
