"""Host side of the serving measurement, without a GPU: the Poisson arrival
process and the open-loop driver that submits requests to the server at
their arrival times (retrying while the server's queue is full), checked
against a stand-in server that records what it is given."""
import threading
import time

import numpy as np
import pytest

from paper_2510_12901_gb300 import serve
from paper_2510_12901_gb300 import simgut as sg

BUSY = -6


def test_poisson_arrivals_have_the_requested_rate_and_are_reproducible():
    a = serve.poisson_arrivals(20000, 2000.0, seed=5)
    assert np.all(np.diff(a) > 0) and a[0] > 0
    gaps = np.diff(np.r_[0.0, a])
    assert abs(gaps.mean() * 2000.0 - 1.0) < 0.03          # mean gap 1 / rate
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05      # exponential: CV 1
    assert np.array_equal(a, serve.poisson_arrivals(20000, 2000.0, seed=5))
    assert not np.array_equal(a, serve.poisson_arrivals(20000, 2000.0, seed=6))


class FakeServer:
    """Accepts a request unless `busy` says to refuse it; remembers when each
    request came in and which tickets were waited for."""

    def __init__(self, busy_first=0, fail_at=None):
        self.lock = threading.Lock()
        self.busy_left = busy_first
        self.fail_at = fail_at
        self.submitted, self.waited, self.t_submit = [], [], []
        self.resets = 0

    def reset_stats(self):
        self.resets += 1

    def submit(self, req):
        with self.lock:
            if self.busy_left > 0:
                self.busy_left -= 1
                raise sg.SimgutError(BUSY, "queue full")
            if self.fail_at is not None and req == self.fail_at:
                raise sg.SimgutError(-1, "refused")
            self.submitted.append(req)
            self.t_submit.append(time.perf_counter())
            return 1000 + req

    def wait(self, ticket, timeout_s):
        self.waited.append(ticket)

    def stats(self):
        return {"completed": len(self.waited)}


def test_open_loop_submits_in_arrival_order_at_the_arrival_times():
    reqs = list(range(12))
    arrivals = np.linspace(0.002, 0.024, 12)
    srv = FakeServer()
    t0 = time.perf_counter()
    st = serve.run_open_loop(srv, reqs, arrivals)
    assert srv.resets == 1
    assert srv.submitted == reqs
    assert srv.waited == [1000 + r for r in reqs]
    assert st == {"completed": 12}
    # no request goes in before its arrival time
    late = np.array(srv.t_submit) - t0 - arrivals
    assert late.min() > -1e-3


def test_open_loop_retries_while_the_queue_is_full():
    srv = FakeServer(busy_first=5)
    serve.run_open_loop(srv, [0, 1, 2], np.array([0.0, 0.001, 0.002]))
    assert srv.submitted == [0, 1, 2] and srv.busy_left == 0


def test_open_loop_stops_at_a_refusal_and_raises_it():
    srv = FakeServer(fail_at=2)
    with pytest.raises(sg.SimgutError) as e:
        serve.run_open_loop(srv, [0, 1, 2, 3], np.array([0.0, 0.001, 0.002, 0.003]))
    assert e.value.status == -1
    # the requests before the refused one were submitted and waited for
    assert srv.submitted == [0, 1] and srv.waited == [1000, 1001]
