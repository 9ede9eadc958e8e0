"""Write tests/golden/bench_work.json: the algorithmic work of the benchmark
workloads as counted by the oracle (double precision), used as the numerator
of the compositing kernels' rooflines in bench.py.

For every ray of both views of the street camera workload (1M Gaussians,
1920x1280 fisheye + 1920x1080 pinhole) and of the LiDAR sweep workload (2M
LiDAR Gaussians, 128 beams x 2048 columns, per-column poses): the list
entries visited before the ray terminated, the entries that passed the
per-ray extent test and had their response evaluated, and the entries
composited.  Calls only oracle/.

    python tests/golden/make_bench_work.py [--procs 8]
"""
import argparse
import json
import multiprocessing as mp
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


_SCENES = {}


def _scene(kind):
    from paper_2510_12901_gb300 import synthetic as syn
    if kind not in _SCENES:
        _SCENES[kind] = (syn.street_scene(1_000_000, seed=0, kind="camera") if kind == "camera"
                         else syn.street_scene(2_000_000, seed=0, kind="lidar"))
    return _SCENES[kind]


def _chunk(args):
    view, lo, hi = args
    from oracle import Oracle
    from paper_2510_12901_gb300 import synthetic as syn
    if view == "lidar":
        r = Oracle(64).render_lidar(_scene("lidar"), syn.street_lidar(), rays=np.arange(lo, hi))
    else:
        cam = dict(zip(("fisheye", "pinhole"), syn.street_cameras()))[view]
        r = Oracle(64).render_camera(_scene("camera"), cam, rays=np.arange(lo, hi))
    return view, int(r["n_visited"].sum()), int(r["n_evaluated"].sum()), int(r["n_contrib"].sum())


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 4)
    ap.add_argument("--chunk", type=int, default=61440)
    a = ap.parse_args()
    from paper_2510_12901_gb300 import synthetic as syn
    cams = dict(zip(("fisheye", "pinhole"), syn.street_cameras()))
    L = syn.street_lidar()
    rays = {v: c.width * c.height for v, c in cams.items()}
    rays["lidar"] = L.n_beams * L.n_cols
    jobs = []
    for v, n in rays.items():
        jobs += [(v, lo, min(n, lo + a.chunk)) for lo in range(0, n, a.chunk)]
    tot = {v: [0, 0, 0] for v in rays}
    with mp.get_context("spawn").Pool(a.procs) as pool:
        for v, vis, ev, co in pool.imap_unordered(_chunk, jobs):
            t = tot[v]
            t[0] += vis
            t[1] += ev
            t[2] += co
    out = {"workload": "street camera scene, 1M Gaussians, seed 0; street_cameras() seed 1; "
                       "LiDAR: street LiDAR scene, 2M Gaussians, seed 0; street_lidar()",
           "counted_by": "oracle (double precision), every ray",
           "views": {v: {"rays": rays[v], "visited_entries": t[0],
                         "evaluated_pairs": t[1], "composited": t[2]}
                     for v, t in tot.items()}}
    with open(os.path.join(HERE, "bench_work.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
