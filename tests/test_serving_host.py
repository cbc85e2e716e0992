"""Host logic of the serving loop with a fake solver (no GPU): admission under the
memory budget, reuse of resident handles, LRU eviction, concurrency and latency
accounting."""
import threading
import time

import numpy as np

from paper_2304_04876_b300 import serving as S


class FakeInfo:
    def __init__(self, iters):
        self.iters, self.true_relres, self.converged = iters, 1e-9, 1


class FakeHandle:
    live = 0
    peak = 0
    lock = threading.Lock()

    def __init__(self, key, nbytes):
        self.key, self.nbytes, self.closed = key, nbytes, False
        with FakeHandle.lock:
            FakeHandle.live += nbytes
            FakeHandle.peak = max(FakeHandle.peak, FakeHandle.live)

    def stats(self):
        return {"device_bytes": self.nbytes}

    def close(self):
        if not self.closed:
            self.closed = True
            with FakeHandle.lock:
                FakeHandle.live -= self.nbytes


def _run(budget, workers, requests, sizes, solve_time=0.01):
    FakeHandle.live = FakeHandle.peak = 0
    active = {"now": 0, "max": 0}
    lk = threading.Lock()

    def solve(handle, b, stream, keep_x):
        with lk:
            active["now"] += 1
            active["max"] = max(active["max"], active["now"])
        time.sleep(solve_time)
        with lk:
            active["now"] -= 1
        return FakeInfo(int(b[0])), (b * 2 if keep_x else None)

    srv = S.Server(lambda key, stream: FakeHandle(key, sizes[key]), lambda key: sizes[key], budget,
                   workers=workers, keep_x=True, solve_fn=solve, stream_factory=lambda: None)
    res = srv.run(requests)
    return srv, res, active


def test_every_request_served_and_results_match_inputs():
    sizes = {"a": 10, "b": 20, "c": 30}
    reqs = [S.Request(0.002 * i, i, "abc"[i % 3], np.full(4, float(i))) for i in range(30)]
    srv, res, active = _run(budget=100, workers=4, requests=reqs, sizes=sizes)
    assert [r.rid for r in res] == list(range(30))
    assert all(np.array_equal(r.x, np.full(4, 2.0 * r.rid)) for r in res)
    assert all(r.iters == r.rid for r in res)
    assert srv.setups == 3 and srv.evictions == 0           # resident handles reused
    assert active["max"] > 1                                 # solves overlapped
    assert all(r.latency >= 0 and r.finish >= r.start >= r.arrival - 1e-9 for r in res)
    summ = S.summarize(res)
    assert summ["requests"] == 30 and summ["p99_ms"] >= summ["p50_ms"]


def test_budget_forces_eviction_and_is_never_exceeded():
    sizes = {f"k{i}": 40 for i in range(6)}
    reqs = [S.Request(0.001 * i, i, f"k{i % 6}", np.ones(2)) for i in range(24)]
    srv, res, active = _run(budget=100, workers=4, requests=reqs, sizes=sizes)
    assert len(res) == 24
    assert FakeHandle.peak <= 100
    assert srv.evictions > 0


def test_handle_never_shared_by_concurrent_requests():
    sizes = {"only": 10}
    inuse = {"n": 0, "max": 0}
    lk = threading.Lock()

    def solve(handle, b, stream, keep_x):
        with lk:
            inuse["n"] += 1
            inuse["max"] = max(inuse["max"], inuse["n"])
        time.sleep(0.005)
        with lk:
            inuse["n"] -= 1
        return FakeInfo(1), None

    srv = S.Server(lambda k, s: FakeHandle(k, 10), lambda k: 10, 100, workers=4, solve_fn=solve,
                   stream_factory=lambda: None)
    res = srv.run([S.Request(0.0, i, "only", np.ones(1)) for i in range(12)])
    assert len(res) == 12 and inuse["max"] == 1


def test_poisson_arrivals_rate():
    t = S.poisson_arrivals(100.0, 20000, seed=0)
    assert abs(len(t) / t[-1] - 100.0) < 3.0
    assert np.all(np.diff(t) > 0)


def test_same_new_problem_requested_twice_is_set_up_once():
    sizes = {"x": 10}
    made = []

    def make(k, s):
        made.append(k)
        time.sleep(0.02)
        return FakeHandle(k, 10)

    srv = S.Server(make, lambda k: 10, 100, workers=4, solve_fn=lambda h, b, st, kx: (FakeInfo(1), None),
                   stream_factory=lambda: None)
    res = srv.run([S.Request(0.0, i, "x", np.ones(1)) for i in range(6)])
    assert len(res) == 6 and made == ["x"]


def test_worker_errors_are_raised():
    import pytest

    def bad_make(k, s):
        raise RuntimeError("setup failed")

    srv = S.Server(bad_make, lambda k: 1, 10, workers=2, solve_fn=lambda *a: None, stream_factory=lambda: None)
    with pytest.raises(RuntimeError):
        srv.run([S.Request(0.0, 0, "a", np.ones(1))])


def test_plan_slots_admits_by_budget_then_adds_copies():
    """Every problem gets one slot while the budget allows (in order; one that does
    not fit is left out), then second copies round-robin while they fit."""
    probs = [("a", 1, 40), ("b", 3, 30), ("c", 1, 50), ("d", 1, 10)]
    plan = S.plan_slots(probs, budget_bytes=100, max_copies=2)
    assert plan[:3] == [("a", 1), ("b", 3), ("d", 1)]          # c (50) does not fit after a, b
    assert plan[3:] == [("d", 1)]                               # 80 used: only d's copy (10) fits
    assert S.plan_slots(probs, budget_bytes=0) == []
    big = S.plan_slots(probs, budget_bytes=10 ** 6, max_copies=3)
    assert [k for k, _ in big].count("a") == 3 and len(big) == 12
