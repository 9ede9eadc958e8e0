"""The multi-rank path of bench.py on CPU: two gloo ranks (processes) with
different step times agree on the slowest rank's time, and the whole-job
rate counts every rank's units over that time (replicas, weak scaling)."""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    my_ms = [3.0, 5.0][rank]
    ms = bench.max_over_ranks(my_ms, world, "cpu")
    q.put((rank, ms, bench.job_rate(4_531_200, world, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
    assert all(p.exitcode == 0 for p in ps)
    out = sorted(q.get(timeout=5) for _ in range(2))
    for rank, ms, rate in out:
        assert ms == 5.0                                   # the slower rank's time
        assert rate == pytest.approx(2 * 4_531_200 / 5e-3 / 1e6)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1, "cpu") == 2.5
    assert bench.job_rate(1_000_000, 1, 1.0) == pytest.approx(1000.0)
