"""The request-stream driver (serve.run_stream) on CPU, against a stand-in
server with the same calls as serve.Server (submit, step, completed, poll):
requests are submitted no earlier than their arrival times, results come back
in request order whatever the completion order, latency is counted from
arrival, and a stream that cannot finish raises TimeoutError."""
import time

import pytest

from paper_2407_20026_gb300.serve import run_stream


class StandInServer:
    """Finishes the queued request with the fewest remaining steps first, one
    step of work per call (so completion order differs from arrival order)."""

    def __init__(self, steps, stall=False):
        self.t0 = time.perf_counter()
        self.steps = steps
        self.stall = stall
        self.next_ticket = 1
        self.queue = {}  # ticket -> [remaining steps, request id]
        self.done = []
        self.results = {}
        self.submitted_at = {}

    def submit(self, mesh, w=1.0):
        t = self.next_ticket
        self.next_ticket += 1
        self.submitted_at[mesh["id"]] = time.perf_counter() - self.t0
        self.queue[t] = [self.steps[mesh["id"]], mesh["id"]]
        return t

    def step(self):
        time.sleep(0.001)
        if self.queue and not self.stall:
            t = min(self.queue, key=lambda k: (self.queue[k][0], k))
            self.queue[t][0] -= 1
            if self.queue[t][0] == 0:
                self.results[t] = self.queue.pop(t)[1]
                self.done.append(t)
        return len(self.queue), 0

    def completed(self):
        out, self.done = self.done, []
        return out

    def poll(self, ticket):
        if ticket not in self.results:
            return None
        return {"id": self.results.pop(ticket), "stats": {"status": 0}, "latency_ms": 1.0}


def _requests(arrivals):
    return [{"mesh": {"id": i}, "t_arrive": t} for i, t in enumerate(arrivals)]


def test_results_in_request_order_and_arrivals_respected():
    arrivals = [0.03, 0.0, 0.06, 0.0, 0.02, 0.09]
    steps = [5, 1, 2, 8, 1, 3]
    srv = StandInServer(steps)
    results, elapsed = run_stream(srv, _requests(arrivals), time_limit_s=10.0)
    assert [r["id"] for r in results] == list(range(len(arrivals)))
    for i, t in enumerate(arrivals):
        # the stand-in's clock started before the driver's, so this is a lower bound
        assert srv.submitted_at[i] >= t
        assert 0.0 <= results[i]["latency_arrival_ms"] <= 1000.0 * elapsed
    assert elapsed >= max(arrivals)


def test_idle_gap_waits_for_the_next_arrival():
    srv = StandInServer([1, 1])
    results, elapsed = run_stream(srv, _requests([0.0, 0.15]), time_limit_s=10.0)
    assert srv.submitted_at[1] >= 0.15
    assert results[1]["latency_arrival_ms"] < 100.0  # served soon after it arrived
    assert elapsed >= 0.15


def test_stream_that_cannot_finish_times_out():
    srv = StandInServer([3, 3], stall=True)
    with pytest.raises(TimeoutError):
        run_stream(srv, _requests([0.0, 0.0]), time_limit_s=0.2)


def test_stream_window_separates_the_drain():
    """bench.stream_window: a server that keeps up completes, between the
    arrivals' 10th and 90th percentiles, as many requests per second as
    arrive; one that falls behind completes fewer, leaves a backlog at the
    last arrival and drains after it."""
    import numpy as np
    import bench
    t = np.arange(1000) * 0.01            # 100 requests/s for 10 s
    keep = bench.stream_window(t, np.full(1000, 50.0))      # 50 ms each
    assert keep["offered_steady_per_s"] == pytest.approx(100.0, rel=1e-9)
    assert keep["achieved_steady_per_s"] == pytest.approx(100.0, rel=0.01)
    assert keep["backlog_at_last_arrival"] == 5             # the last 50 ms of arrivals
    assert keep["drain_s"] == pytest.approx(0.05)
    # a server of 80 requests/s: request k completes at (k + 1) / 80 s
    done = (np.arange(1000) + 1) / 80.0
    slow = bench.stream_window(t, 1e3 * (done - t))
    assert slow["achieved_steady_per_s"] == pytest.approx(80.0, rel=0.01)
    assert slow["backlog_at_last_arrival"] == 1000 - int(t[-1] * 80.0)
    assert slow["drain_s"] == pytest.approx(done[-1] - t[-1])
