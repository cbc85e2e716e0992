"""Continuous serving of GDSW-preconditioned solves on one GPU.

Requests arrive over time (each names a problem and brings a right-hand side).
The server admits them while others are on the GPU:

* a problem's handle (factors, Phi, A0^-1) is set up on first use and stays
  resident for later requests on the same problem, so repeated systems skip the
  setup (Sec. V-A1: the numeric phase is reused across right-hand sides);
* admission is bounded by a device-memory budget: a new handle is set up only
  when its estimated size fits; idle resident handles are evicted least
  recently used first; otherwise the request waits for memory to free up;
* up to `workers` solves run at once, each on its own CUDA stream, so the
  kernels of concurrent requests overlap on the device; a handle serves one
  request at a time (its Krylov workspace is per handle).

All computation goes through the C ABI (gdsw.Handle); this module only
schedules.  Latency = completion time - arrival time.

`BatchServer` below goes further (continuous batching): the resident problems
are solve slots of batched handles, and the iterations of all running requests
are shared launches, with requests joining and leaving between iterations.
"""
from __future__ import annotations

import heapq
import threading
import time
from collections import OrderedDict
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Optional

import numpy as np


@dataclass(order=True)
class Request:
    arrival: float                              # seconds after the start of the run
    rid: int
    key: str = field(compare=False)             # problem identity (resident handle cache key)
    b: np.ndarray = field(compare=False, repr=False)


@dataclass
class Result:
    rid: int
    key: str
    arrival: float
    start: float
    finish: float
    setup_s: float
    iters: int
    true_relres: float
    converged: bool
    x: Optional[np.ndarray] = None

    @property
    def latency(self) -> float:
        return self.finish - self.arrival


class _Resident:
    def __init__(self, handle, nbytes: int):
        self.handle = handle
        self.nbytes = nbytes
        self.busy = False


class Server:
    """Continuous admission, resident handles under a memory budget, concurrent streams.

    make_handle(key, stream) -> gdsw.Handle sets a problem up; estimate_bytes(key)
    predicts its device footprint before setup (the handle's own count replaces it
    afterwards).
    """

    def __init__(self, make_handle: Callable, estimate_bytes: Callable[[str], int], budget_bytes: int,
                 workers: int = 4, keep_x: bool = False, solve_fn: Optional[Callable] = None,
                 stream_factory: Optional[Callable] = None):
        self.solve_fn = solve_fn or _gpu_solve
        self.stream_factory = stream_factory or _cuda_stream
        self.make_handle = make_handle
        self.estimate_bytes = estimate_bytes
        self.budget = budget_bytes
        self.workers = workers
        self.keep_x = keep_x
        self._lock = threading.Condition()
        self._resident: "OrderedDict[str, _Resident]" = OrderedDict()
        self._reserved = 0             # bytes of handles being set up
        self._setting_up = set()       # keys whose handle is being set up
        self.evictions = 0
        self.setups = 0

    # ---- memory accounting -------------------------------------------------
    def _used(self) -> int:
        return self._reserved + sum(r.nbytes for r in self._resident.values())

    def _acquire(self, key: str, stream):
        """Return (resident entry, setup seconds); blocks until the handle is free
        or there is room to set it up."""
        with self._lock:
            while True:
                ent = self._resident.get(key)
                if ent is not None:
                    if not ent.busy:
                        ent.busy = True
                        self._resident.move_to_end(key)
                        return ent, 0.0
                    self._lock.wait(0.01)
                    continue
                if key in self._setting_up:          # another worker is setting it up
                    self._lock.wait(0.01)
                    continue
                need = self.estimate_bytes(key)
                # evict idle handles, least recently used first, until the new one fits
                for k in list(self._resident.keys()):
                    if self._used() + need <= self.budget:
                        break
                    e = self._resident[k]
                    if not e.busy:
                        e.handle.close()
                        del self._resident[k]
                        self.evictions += 1
                if self._used() + need <= self.budget or (not self._resident and self._reserved == 0):
                    self._reserved += need
                    self._setting_up.add(key)
                    break
                self._lock.wait(0.01)
        t0 = time.perf_counter()
        try:
            h = self.make_handle(key, stream)
        except BaseException:
            with self._lock:
                self._reserved -= need
                self._setting_up.discard(key)
                self._lock.notify_all()
            raise
        with self._lock:
            self._reserved -= need
        setup_s = time.perf_counter() - t0
        nbytes = int(h.stats()["device_bytes"])
        ent = _Resident(h, nbytes)
        ent.busy = True
        with self._lock:
            self._resident[key] = ent
            self._setting_up.discard(key)
            self.setups += 1
            self._lock.notify_all()
        return ent, setup_s

    def _release(self, ent: _Resident):
        with self._lock:
            ent.busy = False
            self._lock.notify_all()

    # ---- the run -------------------------------------------------------------
    def run(self, requests: List[Request]) -> List[Result]:
        pending = list(requests)
        heapq.heapify(pending)
        results: List[Result] = []
        queue: List[Request] = []
        qlock = threading.Condition()
        done_arrivals = threading.Event()
        t_start = time.perf_counter()

        def arrivals():
            while pending:
                req = heapq.heappop(pending)
                delay = req.arrival - (time.perf_counter() - t_start)
                if delay > 0:
                    time.sleep(delay)
                with qlock:
                    queue.append(req)
                    qlock.notify()
            done_arrivals.set()
            with qlock:
                qlock.notify_all()

        errors: List[BaseException] = []

        def worker():
            try:
                serve()
            except BaseException as e:          # reported after the run
                errors.append(e)
                done_arrivals.set()

        def serve():
            stream = self.stream_factory()
            while True:
                with qlock:
                    while not queue and not done_arrivals.is_set():
                        qlock.wait(0.05)
                    if not queue:
                        return
                    req = queue.pop(0)          # first come, first served
                t_begin = time.perf_counter() - t_start
                ent, setup_s = self._acquire(req.key, stream)
                try:
                    info, xh = self.solve_fn(ent.handle, req.b, stream, self.keep_x)
                finally:
                    self._release(ent)
                t_end = time.perf_counter() - t_start
                with qlock:
                    results.append(Result(req.rid, req.key, req.arrival, t_begin, t_end, setup_s, info.iters,
                                          info.true_relres, bool(info.converged), xh))

        threads = [threading.Thread(target=arrivals)] + [threading.Thread(target=worker)
                                                         for _ in range(self.workers)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        if errors:
            raise errors[0]
        results.sort(key=lambda r: r.rid)
        return results

    def close(self):
        with self._lock:
            for e in self._resident.values():
                e.handle.close()
            self._resident.clear()


# ---------------------------------------------------------------------------
# Continuous batching: solve slots of batched handles, shared launches
# ---------------------------------------------------------------------------

@dataclass
class Slot:
    pool: int                 # index of the batched handle (problems of one kind share one)
    member: int               # member of that handle
    key: str                  # problem it holds (resident factors, Phi, A0^-1)
    n: int


def plan_slots(problems: List[tuple], budget_bytes: int, max_copies: int = 2) -> List[tuple]:
    """Which problems become resident solve slots, and how many slots each gets.

    problems: [(key, kind, nbytes)] in order of preference (e.g. expected demand);
    kind groups problems that can share a batched handle (same unknowns per node).
    First every problem gets one slot while the budget allows (problems that do not
    fit are not admitted), then further copies round-robin up to `max_copies`, so
    concurrent requests for one problem need not wait for each other.
    Returns [(key, kind)] with one entry per slot."""
    used = 0
    slots = []
    admitted = []
    for key, kind, nb in problems:
        if used + nb <= budget_bytes:
            used += nb
            slots.append((key, kind))
            admitted.append((key, kind, nb))
    for _copy in range(1, max_copies):
        for key, kind, nb in admitted:
            if used + nb <= budget_bytes:
                used += nb
                slots.append((key, kind))
    return slots


class BatchServer:
    """Continuous batching of GDSW-PCG solves on one GPU.

    The resident problems are the members (solve slots) of a few batched handles,
    one per kind of problem (the unknowns per node must agree within a handle).
    Every round, each handle with running members enqueues `iterations` PCG
    iterations as shared launches (one SpMV and one launch per apply phase cover
    all its running members; stopped and idle members only check a flag), the
    handles' rounds run concurrently on their own streams, and between rounds the
    host retires members that have converged and starts queued requests on free
    slots.  A request therefore joins the running ones between iterations instead
    of waiting for them, and its result does not depend on which others run with
    it (members share no arithmetic).  Latency = completion time - arrival time.
    """

    def __init__(self, pools, slots: List[Slot], iterations: int = 4, keep_x: bool = False,
                 stream_factory: Optional[Callable] = None):
        self.pools = pools                      # gdsw.Handle (batched) per pool
        self.slots = slots
        self.iterations = iterations
        self.keep_x = keep_x
        self.stream_factory = stream_factory or _cuda_stream
        self.rounds = 0
        self.rejected = 0

    def run(self, requests: List[Request]) -> List[Result]:
        import torch
        streams = [self.stream_factory() for _ in self.pools]
        free: Dict[str, List[int]] = {}
        for i, sl in enumerate(self.slots):
            free.setdefault(sl.key, []).append(i)
        for v in free.values():
            v.reverse()                           # pop() hands out the lowest slot first
        pending = sorted(requests, key=lambda r: (r.arrival, r.rid))
        queue: List[Request] = []
        active: Dict[int, tuple] = {}           # slot -> (request, admitted at, device b)
        results: List[Result] = []
        t0 = time.perf_counter()
        pi = 0
        while pi < len(pending) or queue or active:
            now = time.perf_counter() - t0
            while pi < len(pending) and pending[pi].arrival <= now:
                req = pending[pi]
                pi += 1
                if req.key in free:
                    queue.append(req)
                else:                           # problem not admitted (memory budget)
                    self.rejected += 1
                    results.append(Result(req.rid, req.key, req.arrival, now, now, 0.0, 0, float("nan"), False))
            # first come, first served per problem; a request whose problem has no
            # free slot does not hold back requests for other problems
            waiting = []
            for req in queue:
                ids = free[req.key]
                if not ids:
                    waiting.append(req)
                    continue
                sid = ids.pop()
                sl = self.slots[sid]
                st = streams[sl.pool]
                with torch.cuda.stream(st):
                    bd = torch.from_numpy(np.ascontiguousarray(req.b, dtype=np.float64)).to("cuda", non_blocking=False)
                self.pools[sl.pool].batch_start(sl.member, bd, stream=st)
                active[sid] = (req, time.perf_counter() - t0, bd)
            queue = waiting
            if not active:
                if pi < len(pending):
                    delay = pending[pi].arrival - (time.perf_counter() - t0)
                    if delay > 0:
                        time.sleep(delay)
                continue
            busy = sorted({self.slots[sid].pool for sid in active})
            for p in busy:
                self.pools[p].batch_iterate(self.iterations, stream=streams[p])
            self.rounds += 1
            for p in busy:
                done, _iters, _rel = self.pools[p].batch_status(stream=streams[p])
                for sid in [s for s in active if self.slots[s].pool == p]:
                    sl = self.slots[sid]
                    if not done[sl.member]:
                        continue
                    x = torch.empty(sl.n, dtype=torch.float64, device="cuda") if self.keep_x else None
                    info, cont = self.pools[p].batch_finish(sl.member, x, stream=streams[p])
                    if cont:
                        continue
                    req, t_adm, _bd = active.pop(sid)
                    free[sl.key].append(sid)
                    t_end = time.perf_counter() - t0
                    results.append(Result(req.rid, req.key, req.arrival, t_adm, t_end, 0.0, info.iters,
                                          info.true_relres, bool(info.converged),
                                          x.cpu().numpy() if x is not None else None))
        results.sort(key=lambda r: r.rid)
        return results


def build_pools(problems: Dict[str, tuple], slot_plan: List[tuple], stream=None, **options):
    """Batched handles for a slot plan: problems[key] = (A, part, Z or None);
    slot_plan = [(key, kind)] (plan_slots).  Returns (pools, slots)."""
    from . import gdsw
    kinds: Dict[object, List[str]] = {}
    for key, kind in slot_plan:
        kinds.setdefault(kind, []).append(key)
    pools, slots = [], []
    for kind, keys in kinds.items():
        if len(keys) == 1:                      # a batched handle has two members at least
            keys = keys + keys
        members = [problems[k] for k in keys]
        h = gdsw.Handle.batch(members, stream=stream, **options)
        for m, k in enumerate(keys):
            slots.append(Slot(len(pools), m, k, int(members[m][0].n)))
        pools.append(h)
    return pools, slots


def _cuda_stream():
    import torch
    return torch.cuda.Stream()


def _gpu_solve(handle, b_host, stream, keep_x):
    """Copy b in, solve on the worker's stream, optionally copy x out."""
    import torch
    with torch.cuda.stream(stream):
        b = torch.tensor(b_host, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        info = handle.solve(b, x, stream=stream, raise_on_nonconvergence=False)
        xh = x.cpu().numpy() if keep_x else None
    stream.synchronize()
    return info, xh


def summarize(results: List[Result]) -> Dict[str, float]:
    lat = np.array([r.latency for r in results])
    span = max(r.finish for r in results) - min(r.arrival for r in results)
    return {"requests": len(results), "solves_per_s": len(results) / span if span > 0 else float("nan"),
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "mean_ms": 1e3 * float(lat.mean()), "all_converged": all(r.converged for r in results),
            "max_true_relres": max(r.true_relres for r in results)}


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate."""
    gaps = np.random.default_rng(seed).exponential(1.0 / rate, count)
    return np.cumsum(gaps)
