"""Benchmark: GDSW-preconditioned PCG to a 1e-8 relative residual on one B300.

Workload (default): 3D Poisson, 7-point, 128^3 unknowns, 8x8x8 = 512 subdomains of
16^3 nodes, overlap 1, GDSW coarse space (constants, n0 = 2863), IC(0) from 3
synchronous fixed-point sweeps, FP64 PCG.  A step is one full solve (setup
excluded, reported separately) of a seeded uniform right-hand side resident in
HBM.  The per-iteration working set (~0.9 GB) is far larger than the 126 MB L2,
so no explicit flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--variant NAME] [--impl reference]
    python bench.py --profile {solve,apply} [--profile-count C]   (untimed, for ncu)

One JSON line is printed by rank 0.  Under torchrun every rank solves its own
replica (independent problems, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

# the CPU oracle legs spread their local solves over processes (one BLAS thread
# each); set before numpy loads its BLAS
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2304_04876_b300 import problems as P  # noqa: E402
from paper_2304_04876_b300 import replicas as R  # noqa: E402

VARIANTS = {
    "fp64_levelsched": dict(local_solver="ic0", trsv="levelsched", precision="fp64"),
    "fp64_jacobi": dict(local_solver="ic0", trsv="jacobi", precision="fp64"),
    "fp32_levelsched": dict(local_solver="ic0", trsv="levelsched", precision="fp32"),
    "fp32_jacobi": dict(local_solver="ic0", trsv="jacobi", precision="fp32"),
    "fp16_levelsched": dict(local_solver="ic0", trsv="levelsched", precision="fp16"),
    "fp64_levelsched_rgdsw": dict(local_solver="ic0", trsv="levelsched", precision="fp64", coarse="rgdsw"),
    "fp32_levelsched_rgdsw": dict(local_solver="ic0", trsv="levelsched", precision="fp32", coarse="rgdsw"),
    "fp32_levelsched_ic1": dict(local_solver="ic0", trsv="levelsched", precision="fp32", fill_level=1),
    "fp32_levelsched_ic2": dict(local_solver="ic0", trsv="levelsched", precision="fp32", fill_level=2),
    "fp32_exact": dict(local_solver="exact", precision="fp32"),
    "fp16_exact": dict(local_solver="exact", precision="fp16"),
    "fp64_exact": dict(local_solver="exact", precision="fp64"),
}
DEFAULT_VARIANT = "fp32_levelsched"
METRIC = "PCG solves/s to 1e-8 relative residual (time-to-residual = 1/value)"
WORKLOAD = "poisson7_128^3_512sub16^3_gdsw_ic0"

# the other fixed workloads (python bench.py --config N); config 2 is the default line
CONFIGS = {
    1: dict(workload="poisson7_16^3_8sub8^3_gdsw_exact", metric=METRIC, make=lambda: P.config_problem(1),
            variants={"fp64_exact": dict(local_solver="exact", precision="fp64"),
                      "fp32_exact": dict(local_solver="exact", precision="fp32")},
            default="fp64_exact", Z=False),
    2: dict(workload=WORKLOAD, metric=METRIC, make=lambda: P.config_problem(2), variants=VARIANTS,
            default=DEFAULT_VARIANT, Z=False),
    3: dict(workload="elasticity_q1_48^3_64sub12^3_gdsw_rbm_ilu0_gmres30",
            metric="GMRES(30) solves/s to 1e-8 relative residual (time-to-residual = 1/value)",
            make=lambda: P.config_problem(3),
            variants={"fp64_levelsched": dict(local_solver="ilu0", krylov="gmres", restart=30),
                      "fp32_levelsched": dict(local_solver="ilu0", krylov="gmres", restart=30, precision="fp32"),
                      "fp64_jacobi": dict(local_solver="ilu0", krylov="gmres", restart=30, trsv="jacobi"),
                      "fp32_jacobi": dict(local_solver="ilu0", krylov="gmres", restart=30, trsv="jacobi",
                                          precision="fp32"),
                      "fp16_levelsched": dict(local_solver="ilu0", krylov="gmres", restart=30, precision="fp16"),
                      "fp32_levelsched_rgdsw": dict(local_solver="ilu0", krylov="gmres", restart=30,
                                                    precision="fp32", coarse="rgdsw"),
                      "fp32_levelsched_ilu1": dict(local_solver="ilu0", krylov="gmres", restart=30,
                                                   precision="fp32", fill_level=1),
                      "fp32_exact": dict(local_solver="exact", krylov="gmres", restart=30, precision="fp32")},
            default="fp32_levelsched", Z=True),
}

def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# ---------------------------------------------------------------------------
# algorithmic bytes (each array touched once per launch)
# ---------------------------------------------------------------------------

def apply_bytes(st: dict, vbytes: int, fbytes: int = None) -> dict:
    """Algorithmic bytes of the four apply phases: `vbytes` per value of Phi, the
    local vectors and inverses, `fbytes` per stored factor value (default vbytes)."""
    fbytes = vbytes if fbytes is None else fbytes
    n, sum_m, n0, nblk = st["n"], st["sum_omega"], st["n0"], st["n_blocks"]
    tri = 0
    for nnz, lev in ((st["nnz_L"], st["n_levels_L"]), (st["nnz_U"], st["n_levels_U"])):
        off = nnz - sum_m
        tri += off * (fbytes + 2) + sum_m * (fbytes + 2) + lev * 16
    if st["dense_local"]:
        # dense inverses are read once; multifrontal panels once per sweep
        tri = (st["dense_local"] * fbytes * 2 if st.get("mf_supernodes") else st["dense_local"] * vbytes)
    local = sum_m * (8 + 4) + tri + sum_m * vbytes + st["n_sub"] * 8
    phit = st["nnz_phi"] * vbytes + n * (8 + 4) + (nblk + 1) * 12 if n0 else 0
    coarse = st.get("a0_entries", n0 * n0) * 8 + n0 * 8 * 3 if n0 else 0
    combine = (sum_m * 4 + (n + 1) * 4 + sum_m * vbytes + n * 4 + st["nnz_phi"] * vbytes
               + n * 8 + nblk * 16)
    if n0 and st.get("phi_beside_local"):
        # Phi y formed on the coarse stream (Phi read, u written) and added by the
        # scatter-add (u read)
        coarse += st["nnz_phi"] * vbytes + n * vbytes
        combine += n * vbytes - st["nnz_phi"] * vbytes
    return {"local": local, "phiT": phit, "coarse": coarse, "combine": combine}


def spmv_bytes(st: dict) -> int:
    return st["nnz"] * 12 + (st["n"] + 1) * 4 + st["n"] * 16


def iteration_work(st: dict, vb: int, fb: int, flexible: bool) -> dict:
    """Algorithmic bytes and FP64 FMAs per launch of each kernel of a PCG iteration
    (the apply in its PCG form, dots fused into the scatter-add); FP32 or FP16
    preconditioners do their own arithmetic in FP32, which is not counted."""
    n, nnz = st["n"], st["nnz"]
    ab = apply_bytes(st, vb, fb)
    dots = 2 if flexible else 1
    fp64_pre = vb == 8
    tri = st["nnz_L"] + st["nnz_U"] - 2 * st["sum_omega"]
    return {
        "spmv": {"bytes": spmv_bytes(st), "fma64": nnz + n},
        "update": {"bytes": 24 * n, "fma64": 2 * n},
        "xupdate": {"bytes": 24 * n, "fma64": n},
        "local": {"bytes": ab["local"], "fma64": tri if fp64_pre and not st["dense_local"] else 0},
        "phiT": {"bytes": ab["phiT"], "fma64": st["nnz_phi"] if fp64_pre else 0},
        "coarse": {"bytes": ab["coarse"], "fma64": st.get("a0_entries", st["n0"] ** 2)
                   + (st["nnz_phi"] if fp64_pre and st.get("phi_beside_local") else 0)},
        "combine": {"bytes": ab["combine"] + 8 * dots * n,
                    "fma64": dots * n + (st["nnz_phi"] if fp64_pre and not st.get("phi_beside_local") else 0)},
        "pupdate": {"bytes": 24 * n, "fma64": n},
    }


def rooflines(kernel_ms: dict, work: dict, hbm: float, src: str, fp64_rate: float | None) -> dict:
    """Per kernel: algorithmic GB/s against the measured HBM peak and, where the
    kernel works in FP64, FMA/s against the measured FP64 FMA rate; `bound` is the
    resource with the larger fraction (max(bytes / BW, FMAs / FP64 rate))."""
    out = {}
    for k, ms in kernel_ms.items():
        if k not in work or ms <= 0:
            continue
        w = work[k]
        gbs = w["bytes"] / (ms * 1e-3) / 1e9
        e = {"us": 1e3 * ms, "algorithmic_bytes": int(w["bytes"]), "gbs": gbs, "hbm_frac": gbs / hbm,
             "hbm_peak_source": src}
        if fp64_rate and w["fma64"]:
            rate = w["fma64"] / (ms * 1e-3)
            e.update(fma64=int(w["fma64"]), fma64_per_s=rate, fp64_frac=rate / fp64_rate)
        e["bound"] = "fp64" if e.get("fp64_frac", 0.0) > e["hbm_frac"] else "hbm"
        out[k] = e
    return out


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        # the timed region starts once sampling has (the tool takes a moment to start)
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 3.0 and os.path.getsize(self.path) == 0 and self.proc.poll() is None:
            time.sleep(0.01)

    def stop(self) -> dict:
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
            if len(parts) >= 9:
                rows.append(parts)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        loaded = [s for s in sm if s > 0.5 * max(sm)] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


# ---------------------------------------------------------------------------
# CPU oracle baseline (rank 0, N = 1): bounded sample, single thread
# ---------------------------------------------------------------------------

def golden_iters(cfg: int, variant: str) -> int | None:
    path = os.path.join(ROOT, "tests", "golden", "oracle_pcg.json")
    if not os.path.exists(path):
        return None
    g = json.load(open(path))
    trsv = "jacobi" if "jacobi" in variant else "levelsched"
    key = {1: f"poisson_16_s8/exact/levelsched/seed0", 2: f"poisson_128_s16/ic0/{trsv}/seed0",
           3: f"elasticity_48_se12/ilu0/{trsv}/gmres30/body_force"}.get(cfg)
    e = g.get(key)
    return None if e is None else int(e["iters"])


def oracle_for_variant(prob, cfg: int, variant: str):
    from oracle import gdsw_oracle as O
    local = {1: O.EXACT, 2: O.IC0, 3: O.ILU0}.get(cfg, O.IC0)
    trsv = O.JACOBI if "jacobi" in variant else O.LEVELSCHED
    Z = prob.Z if cfg == 3 else None
    return O.GDSW(prob.A, prob.part, Z, local=local, trsv=trsv)


class OracleCores:
    """The oracle's preconditioner apply spread over the host cores: worker processes,
    forked after the oracle is built (so they share its factors) and before any CUDA
    call, each run the oracle's own `local_solve` for a slice of the subdomains into a
    shared buffer; the parent then sums the local terms in ascending subdomain order
    and adds the coarse term exactly as `GDSW.apply` does, so the result is the
    oracle's, value for value.  SpMV is the oracle's own (one core)."""

    def __init__(self, M, workers: int):
        import multiprocessing as mp
        from multiprocessing import shared_memory
        self.M = M
        sizes = [len(d) for d in M.omega]
        self.offs = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self._shm = [shared_memory.SharedMemory(create=True, size=max(8, 8 * M.n)),
                     shared_memory.SharedMemory(create=True, size=max(8, 8 * int(self.offs[-1])))]
        self.r = np.ndarray((M.n,), np.float64, buffer=self._shm[0].buf)
        self.zl = np.ndarray((int(self.offs[-1]),), np.float64, buffer=self._shm[1].buf)
        ns = len(M.omega)
        self.workers = max(1, min(workers, ns))
        # contiguous slices of subdomains, about equal in unknowns
        cuts = np.searchsorted(self.offs, np.linspace(0, self.offs[-1], self.workers + 1))
        cuts[0], cuts[-1] = 0, ns
        self.slices = [(int(a), int(b)) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]
        global _ORACLE_CORES
        _ORACLE_CORES = self
        self.pool = mp.get_context("fork").Pool(self.workers) if self.workers > 1 else None

    def apply(self, r):
        M = self.M
        self.r[:] = r
        if self.pool is None:
            _oracle_local_slice((0, len(M.omega)))
        else:
            self.pool.map(_oracle_local_slice, self.slices)
        z = np.zeros(M.n)
        for s, dofs in enumerate(M.omega):
            z[dofs] += self.zl[self.offs[s]:self.offs[s + 1]]
        if M.n0:
            import scipy.linalg as sla
            c = M.coarse.Phi.T @ r
            y = sla.cho_solve(M.A0fac, c)
            z += M.coarse.Phi @ y
        return z

    def close(self):
        if self.pool is not None:
            self.pool.terminate()
            self.pool.join()
        for m in self._shm:
            m.close()
            m.unlink()


_ORACLE_CORES = None


def _oracle_local_slice(bounds):
    oc = _ORACLE_CORES
    for s in range(bounds[0], bounds[1]):
        oc.zl[oc.offs[s]:oc.offs[s + 1]] = oc.M.local_solve(s, oc.r[oc.M.omega[s]])


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_iteration(M, apply, r, p):
    """One oracle Krylov iteration: SpMV, step, residual update, M^-1 apply, new direction."""
    q = M.spmv(p)
    alpha = (r @ p) / (p @ q)
    r = r - alpha * q
    z = apply(r)
    beta = (r @ z) / (r @ r + 1.0)
    return r, z + beta * p


def oracle_iteration_time(M, apply, b, n_iter: int) -> float:
    """Median time of one oracle Krylov iteration."""
    r = b.copy()
    p = apply(r)
    times = []
    for _ in range(n_iter):
        t1 = time.perf_counter()
        r, p = oracle_iteration(M, apply, r, p)
        times.append(time.perf_counter() - t1)
    return statistics.median(times)


def oracle_sample(prob, cfg: int, variant: str, iters_for_metric: int, n_iter: int = 3) -> dict:
    """The oracle on the full workload after its setup, its local solves on all host
    cores: solves/s = 1 / (seconds per Krylov iteration * iterations of a solve).
    Must run before the process makes its first CUDA call (the pool is forked)."""
    t0 = time.perf_counter()
    M = oracle_for_variant(prob, cfg, variant)
    setup_s = time.perf_counter() - t0
    oc = OracleCores(M, host_cores())
    try:
        t_it = oracle_iteration_time(M, oc.apply, prob.b, n_iter)
    finally:
        oc.close()
    return {"value": 1.0 / (t_it * iters_for_metric), "unit": "solves/s", "cores": oc.workers, "kind": "oracle",
            "cpu": cpu_model(), "host_cores": host_cores(),
            "sample": f"{n_iter} oracle Krylov iterations (SpMV + M^-1 apply + updates) on the full workload, "
                      f"local solves in {oc.workers} processes; median {t_it:.3f} s/iteration x "
                      f"{iters_for_metric} iterations per solve; oracle setup {setup_s:.1f} s not counted",
            "seconds_per_iteration": t_it, "oracle_setup_s": setup_s}


# ---------------------------------------------------------------------------
# reference arm: the oracle as it stands on the host cores
# ---------------------------------------------------------------------------

def run_reference(args, rank: int):
    if rank != 0:
        return
    cfg = args.config if args.config in CONFIGS else 2
    C = CONFIGS[cfg]
    variant = args.variant or C["default"]
    prob = C["make"]()
    iters = golden_iters(cfg, variant) or 40
    M = oracle_for_variant(prob, cfg, variant)
    oc = OracleCores(M, host_cores())
    state = {"r": prob.b.copy(), "p": oc.apply(prob.b)}

    def step():
        # one bounded sample of the workload: one oracle Krylov iteration
        state["r"], state["p"] = oracle_iteration(M, oc.apply, state["r"], state["p"])

    try:
        for _ in range(args.warmup):
            step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
        el = time.perf_counter() - t0
    finally:
        oc.close()
    t_it = el / args.steps
    value = 1.0 / (t_it * iters)
    line = {"impl": "reference", "metric": C["metric"], "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_it,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": C["workload"], "variant": variant, "n": prob.A.n},
            "step": f"one oracle Krylov iteration (SpMV + M^-1 apply + updates) on the full workload; "
                    f"value = solves/s = 1/(s per step x {iters} iterations of a solve)",
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": oc.workers, "kind": "oracle",
                             "cpu": cpu_model(), "host_cores": host_cores(),
                             "sample": f"each step = one oracle Krylov iteration on the full workload, local "
                                       f"solves in {oc.workers} processes; solves/s = 1/(s per iteration x "
                                       f"{iters} iterations)"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def timed_solves(h, bs, x, steps, warmup, stream, barrier, solve=None):
    import torch
    solve = solve or (lambda b, xx: h.solve(b, xx))
    for k in range(warmup):
        x.zero_()
        solve(bs[k % len(bs)], x)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    e0.record(stream)
    for k in range(steps):
        x.zero_()
        infos.append(solve(bs[k % len(bs)], x))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    return e0.elapsed_time(e1) / 1e3, infos


def kernel_measurements(h, st, vb, stream, v0, workload=None, variant=None, fb=None, flexible=False,
                        fp64_rate=None, krylov="pcg"):
    """Per-phase apply times (CUDA events on the launching stream), the apply as
    the solver runs it (branches overlapped) and the SpMV."""
    import torch
    rr = v0.clone()
    zz = torch.empty_like(rr)
    reps = 20
    for _ in range(3):
        h.apply_timed(rr, zz)
    phases = np.zeros(4)
    for _ in range(reps):
        phases += np.array(h.apply_timed(rr, zz))
    phases /= reps
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    for _ in range(reps):
        h.apply(rr, zz)
    eb.record(stream)
    torch.cuda.synchronize()
    overlapped = ea.elapsed_time(eb) / reps
    for _ in range(3):
        h.spmv(rr, zz)
    ea.record(stream)
    for _ in range(reps):
        h.spmv(rr, zz)
    eb.record(stream)
    torch.cuda.synchronize()
    spmv_ms = ea.elapsed_time(eb) / reps
    hbm, src = peaks()
    names = ["local", "phiT", "coarse", "combine"]
    phase_ms = dict(zip(names, phases.tolist()))
    ab = apply_bytes(st, vb, fb)
    # every kernel of a PCG iteration, timed one by one (CUDA events on the
    # launching stream); the dominant kernel is the slowest of them all
    work = iteration_work(st, vb, fb if fb is not None else vb, flexible)
    if st.get("n_problems", 1) == 1:
        acc = {}
        for _ in range(3):
            h.pcg_iteration_timed(v0)
        for _ in range(reps):
            for k, v in h.pcg_iteration_timed(v0).items():
                acc[k] = acc.get(k, 0.0) + v / reps
        kernel_ms = acc
        if krylov != "pcg":
            # GMRES has its own vector kernels; keep the SpMV and the apply's phases
            kernel_ms = {k: v for k, v in acc.items() if k not in ("update", "pupdate", "xupdate")}
    else:
        kernel_ms = {**phase_ms, "spmv": spmv_ms}
    per_kernel = rooflines(kernel_ms, work, hbm, src, fp64_rate)
    for k in per_kernel:
        per_kernel[k]["traffic"] = profiled_traffic(k, workload, variant)
    dom = max(per_kernel, key=lambda k: per_kernel[k]["us"])
    achieved = per_kernel[dom]["gbs"]
    dom_entry = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                 "frac": achieved / hbm, "traffic": profiled_traffic(dom, workload, variant),
                 "peak_source": src, "algorithmic_bytes_per_launch": per_kernel[dom]["algorithmic_bytes"],
                 "launch_us": per_kernel[dom]["us"]}
    if "fp64_frac" in per_kernel[dom]:
        dom_entry["fp64"] = {"fma_per_launch": per_kernel[dom]["fma64"],
                             "achieved_fma_per_s": per_kernel[dom]["fma64_per_s"], "peak_fma_per_s": fp64_rate,
                             "frac": per_kernel[dom]["fp64_frac"], "peak_source": "measured live "
                             "(gdsw_measure_fma_rate)"}
    return {
        "apply_ms": float(phases.sum()), "apply_phase_ms": phase_ms,
        "apply_gbs": sum(ab.values()) / (phases.sum() * 1e-3) / 1e9,
        "apply_overlapped_ms": overlapped,
        "apply_overlapped_gbs": sum(ab.values()) / (overlapped * 1e-3) / 1e9,
        "spmv_ms": spmv_ms, "spmv_gbs": spmv_bytes(st) / (spmv_ms * 1e-3) / 1e9,
        "iteration_kernel_us": {k: 1e3 * v for k, v in kernel_ms.items()},
        "rooflines": per_kernel,
        "roofline": dom_entry,
    }


KERNEL_SOURCE = {"local": "apply.cu", "phiT": "apply.cu", "coarse": "apply.cu", "combine": "apply.cu",
                 "update": "krylov.cu", "pupdate": "krylov.cu", "xupdate": "krylov.cu",
                 "spmv": "krylov.cu"}


def source_digest(name):
    """First 16 hex digits of the SHA-256 of a kernel source file."""
    import hashlib
    path = os.path.join(ROOT, "paper_2304_04876_b300", "csrc", name)
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def profiled_traffic(phase, workload, variant):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
    phase's kernel, from the ncu summary table in profiles/traffic.md, or None when
    no capture exists for it or the kernel's source has changed since."""
    path = os.path.join(ROOT, "profiles", "traffic.md")
    if not os.path.exists(path) or phase not in KERNEL_SOURCE:
        return None
    want = source_digest(KERNEL_SOURCE[phase])
    for line in open(path):
        cells = [c.strip() for c in line.strip().strip("|").split("|")]
        if len(cells) >= 5 and cells[0] == phase and cells[1] == workload and cells[2] == variant:
            try:
                return int(cells[3]) if cells[4] == want else None
            except ValueError:
                return None
    return None


def launches_per_solve(iters, krylov="pcg"):
    # prologue (SpMV, residual, 5 apply kernels) + 8 per PCG iteration + true residual
    return sum(9 + 8 * it for it in iters) if krylov == "pcg" else None


def run_single(args, world, rank, dist, barrier, cpu_baseline=None):
    import torch
    from paper_2304_04876_b300 import gdsw
    cfg = args.config
    C = CONFIGS[cfg]
    variant = args.variant or C["default"]
    opts = C["variants"][variant]
    prob = C["make"]()
    Z = prob.Z if C["Z"] else None
    t0 = time.perf_counter()
    h = gdsw.Handle(prob.A, prob.part, Z, **opts)
    setup_s = time.perf_counter() - t0
    st = h.stats()
    n = prob.A.n
    if cfg == 3:
        bs = [torch.tensor(prob.b, dtype=torch.float64, device="cuda")]
    else:
        bs = [torch.tensor(P.rhs_uniform(n, R.rhs_seed(rank, k)), dtype=torch.float64, device="cuda")
              for k in range(5)]
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    el, infos = timed_solves(h, bs, x, args.steps, args.warmup, stream, barrier)
    clk = clocks.stop()
    el = R.max_over_ranks(el, dist, "cuda")
    iters = [i.iters for i in infos]
    # end to end through the C ABI with host (page-locked) buffers: b in, x out,
    # from the zero initial guess
    bh = bs[0].cpu().pin_memory()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    h.solve_host(bh, xh, zero_guess=True)
    barrier()
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(args.steps):
        h.solve_host(bh, xh, zero_guess=True)
    e2e_el = R.max_over_ranks(time.perf_counter() - te, dist, "cuda")
    vb = 4 if opts.get("precision") in ("fp32", "fp16") else 8
    fb = 2 if opts.get("precision") == "fp16" else vb
    fp64_rate = gdsw.measure_fma_rate("fp64")
    km = kernel_measurements(h, st, vb, stream, bs[0], C["workload"], variant, fb, flexible=vb < 8,
                             fp64_rate=fp64_rate, krylov=opts.get("krylov", "pcg"))
    line = {
        "metric": C["metric"], "value": R.job_rate(args.steps, el, world), "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if vb == 4 else "f64", "data": "synthetic",
        "config": {"workload": C["workload"], "variant": variant, "n": n, "nnz": st["nnz"],
                   "subdomains": st["n_sub"], "n0": st["n0"], "overlap": 1, "tol": 1e-8,
                   "local_shape": [int(st["local_stages"]), int(st["local_threads"])],
                   "l2": "per-iteration working set larger than the 126 MB L2; no flush" if n > 1e6 else
                         "small workload: L2-resident, launch-latency bound",
                   "parallelism": f"replicas{world}"},
        "time_to_residual_ms": 1e3 * el / args.steps, "iters": iters,
        "true_relres_max": max(i.true_relres for i in infos),
        "setup_s": setup_s, "setup_phase_s": st["setup_phase_seconds"],
        **{k: v for k, v in km.items() if k != "roofline"},
        "roofline": km["roofline"],
        "e2e": {"value": R.job_rate(args.steps, e2e_el, world), "unit": "solves/s", "h2d_bytes_per_step": 8 * n,
                "d2h_bytes_per_step": 8 * n},
        "gpu_launches": launches_per_solve(iters, opts.get("krylov", "pcg")),
        "clocks": clk,
        "fp64_fma_per_s": fp64_rate,
    }
    if not args.no_variants and rank == 0:
        var = {}
        for name, vo in C["variants"].items():
            if name == variant:
                continue
            hv = gdsw.Handle(prob.A, prob.part, Z, **vo)
            el_v, inf = timed_solves(hv, bs, x, 3, 2, stream, lambda: None)
            var[name] = {"ms_per_solve": 1e3 * el_v / 3, "iters": [i.iters for i in inf],
                         "true_relres_max": max(i.true_relres for i in inf)}
            hv.close()
        line["variants"] = var
    if cpu_baseline is not None:
        line["cpu_baseline"] = cpu_baseline
    h.close()
    return line


def run_batch(args, world, rank, dist, barrier):
    """Config 4: 256 independent heterogeneous diffusion problems in one batched handle;
    a step is one batched PCG solve of all of them (FP32 local solves, FP64 outer)."""
    import torch
    from paper_2304_04876_b300 import gdsw
    count = args.batch_count
    mem = P.diffusion_batch(count, seed=rank)
    opts = dict(local_solver="ic0", trsv="levelsched", precision="fp32")
    t0 = time.perf_counter()
    h = gdsw.Handle.batch([(m.A, m.part, None) for m in mem], **opts)
    setup_s = time.perf_counter() - t0
    st = h.stats()
    n = st["n"]
    b = torch.tensor(np.concatenate([m.b for m in mem]), dtype=torch.float64, device="cuda")
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    el, infos = timed_solves(h, [b], x, args.steps, args.warmup, stream, barrier,
                             solve=lambda bb, xx: h.solve_batch(bb, xx))
    clk = clocks.stop()
    el = R.max_over_ranks(el, dist, "cuda")
    iters = [i.iters for i in infos[-1]]
    relres = max(i.true_relres for inf in infos for i in inf)
    # one problem at a time with its own handle (same options), on a sample
    sample = list(range(0, count, max(1, count // 8)))[:8]
    t_one = 0.0
    for i in sample:
        m = mem[i]
        h1 = gdsw.Handle(m.A, m.part, None, **opts)
        b1 = torch.tensor(m.b, dtype=torch.float64, device="cuda")
        x1 = torch.zeros_like(b1)
        e1, _ = timed_solves(h1, [b1], x1, 2, 1, stream, lambda: None)
        t_one += e1 / 2
        h1.close()
    seq_per_problem = t_one / len(sample)
    # end to end with host buffers (b in, x out, zero initial guess)
    bh = b.cpu().pin_memory()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    h.solve_host(bh, xh, zero_guess=True)
    te = time.perf_counter()
    for _ in range(args.steps):
        h.solve_host(bh, xh, zero_guess=True)
    e2e_el = R.max_over_ranks(time.perf_counter() - te, dist, "cuda")
    km = kernel_measurements(h, st, 4, stream, b, f"batch_{count}_diffusion7_edge16-64_sub8-16_k1e-2..1e2",
                             "fp32_levelsched")
    line = {
        "metric": "batched PCG problems solved/s to 1e-8 (256 diffusion problems per step)",
        "value": R.job_rate(count * args.steps, el, world), "unit": "problems/s", "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"batch_{count}_diffusion7_edge16-64_sub8-16_k1e-2..1e2", "n": n,
                   "nnz": st["nnz"], "subdomains": st["n_sub"], "n0": st["n0"], "problems": count,
                   "local_shape": [int(st["local_stages"]), int(st["local_threads"])],
                   "parallelism": f"replicas{world}"},
        "iters_min_max": [min(iters), max(iters)], "true_relres_max": relres, "setup_s": setup_s,
        "one_at_a_time_ms_per_problem": 1e3 * seq_per_problem,
        "one_at_a_time_problems_per_s": 1.0 / seq_per_problem,
        **{k: v for k, v in km.items() if k != "roofline"},
        "roofline": km["roofline"],
        "e2e": {"value": R.job_rate(count * args.steps, e2e_el, world), "unit": "problems/s",
                "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n},
        "gpu_launches": None,
        "clocks": clk,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle on a bounded sample: the two smallest members, full PCG solves
        from oracle import gdsw_oracle as O
        small = sorted(range(count), key=lambda i: mem[i].A.n)[:2]
        t_cpu, n_cpu = 0.0, 0
        for i in small:
            m = mem[i]
            M = O.GDSW(m.A, m.part, None, local=O.IC0)
            tt = time.perf_counter()
            O.pcg(M.spmv, M.apply, m.b, tol=1e-8)
            t_cpu += time.perf_counter() - tt
            n_cpu += m.A.n
        per_unknown = t_cpu / n_cpu
        line["cpu_baseline"] = {"value": 1.0 / (per_unknown * n / count), "unit": "problems/s", "cores": 1,
                                "kind": "oracle",
                                "sample": f"full oracle PCG solves of the two smallest members ({n_cpu} unknowns), "
                                          f"scaled by unknowns to the batch's mean problem"}
    h.close()
    return line


def run_serving(args, world, rank, dist, barrier):
    """Config 5: Poisson-arrival stream of mixed Poisson / Q1 elasticity requests served
    with continuous batching (resident solve slots of batched handles chosen under a
    memory budget; the iterations of all running requests are shared launches, and
    requests join and leave between iterations); p50/p99 latency and solves/s per
    arrival rate, beside the plain FP64 one-at-a-time solve of the same stream."""
    import torch
    from paper_2304_04876_b300 import gdsw
    from paper_2304_04876_b300 import serving as S
    pool = P.serving_pool(args.pool, seed=rank, dofs_max=args.serving_max_dofs)
    byname = {p.name: p for p in pool}
    opts = dict(local_solver="ic0", trsv="levelsched", precision="fp32")
    zof = lambda pr: pr.Z if pr.part.dpn == 3 else None  # noqa: E731
    free, _total = torch.cuda.mem_get_info()
    budget = int(args.serving_budget_gb * (1 << 30)) if args.serving_budget_gb else int(0.6 * free)
    est = [(p.name, p.part.dpn, gdsw.bytes_required(p.A, p.part, zof(p), **opts)[0]) for p in pool]
    plan = S.plan_slots(est, budget, max_copies=args.serving_copies)
    problems = {p.name: (p.A, p.part, zof(p)) for p in pool}
    t0 = time.perf_counter()
    pools, slots = S.build_pools(problems, plan, **opts)
    warm_s = time.perf_counter() - t0
    # every result is read back to the host, as a client would receive it
    srv = S.BatchServer(pools, slots, iterations=args.serving_iters, keep_x=True)
    # warm-up: every slot once
    srv.run([S.Request(0.0, i, sl.key, P.rhs_uniform(sl.n, 7)) for i, sl in enumerate(slots)])
    admitted = sorted({sl.key for sl in slots})

    def stream(lam, count):
        rng = np.random.default_rng(int(lam) + 17 * rank)
        arr = S.poisson_arrivals(lam, count, seed=int(lam))
        reqs = []
        for i, t in enumerate(arr):
            pr = byname[admitted[int(rng.integers(len(admitted)))]]
            reqs.append(S.Request(float(t), i, pr.name, P.rhs_uniform(pr.A.n, 1000 + i)))
        return reqs

    rates = {}
    for lam in args.rates:
        res = srv.run(stream(lam, args.requests))
        rates[str(lam)] = S.summarize(res)
    top = rates[str(max(args.rates))]
    # the plain FP64 one-problem-at-a-time solve of the same (saturated) stream:
    # one resident FP64 handle per problem, one solve at a time on one stream
    plain_opts = dict(local_solver="ic0", trsv="levelsched", precision="fp64")
    plain = S.Server(lambda key, st: gdsw.Handle(byname[key].A, byname[key].part, zof(byname[key]), stream=st,
                                                 **plain_opts),
                     lambda key: 0, budget_bytes=1 << 62, workers=1, keep_x=True)
    plain.run([S.Request(0.0, i, k, P.rhs_uniform(byname[k].A.n, 7)) for i, k in enumerate(admitted)])
    plain_top = S.summarize(plain.run(stream(max(args.rates), args.requests)))
    plain.close()
    sizes = sorted(p.A.n for p in pool)
    line = {
        "metric": "served solves/s (saturated) with p50/p99 latency, mixed Poisson / Q1 elasticity, "
                  "continuous batching",
        "value": world * top["solves_per_s"], "unit": "solves/s", "n_gpus": world, "steps": args.requests,
        "warmup": len(slots), "ms_per_step": 1e3 / top["solves_per_s"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"serving_pool{len(pool)}_poisson+elasticity_32^3-"
                               f"{round(args.serving_max_dofs ** (1 / 3))}^3", "pool_unknowns": sizes,
                   "slots": len(slots), "admitted_problems": len(admitted), "budget_bytes": budget,
                   "iterations_per_round": args.serving_iters, "rates_req_per_s": args.rates,
                   "requests_per_rate": args.requests, "parallelism": f"replicas{world}"},
        "rates": rates, "p50_ms": top["p50_ms"], "p99_ms": top["p99_ms"],
        "plain_fp64_one_at_a_time": plain_top,
        "served_over_plain": top["solves_per_s"] / plain_top["solves_per_s"],
        "warm_setup_s": warm_s, "rounds": srv.rounds, "rejected": srv.rejected,
        "e2e": {"value": world * top["solves_per_s"], "unit": "solves/s",
                "h2d_bytes_per_step": int(np.mean([8 * n for n in sizes])),
                "d2h_bytes_per_step": int(np.mean([8 * n for n in sizes]))},
        "gpu_launches": None, "roofline": None,
    }
    for h in pools:
        h.close()
    return line


def config_summaries(args, world, rank, dist, barrier) -> dict:
    """Bounded runs of the other workloads for the default line (configs 1, 3, 4, 5),
    each reduced to its headline numbers; the full lines come from --config N."""
    import copy
    out = {}
    keep = ("metric", "value", "unit", "ms_per_step", "iters", "iters_min_max", "true_relres_max", "setup_s",
            "one_at_a_time_problems_per_s", "p50_ms", "p99_ms", "plain_fp64_one_at_a_time", "served_over_plain",
            "rates", "slots", "roofline", "apply_phase_ms", "spmv_ms", "variants")
    for cfg, extra in ((1, dict(steps=40, warmup=20)), (3, dict(steps=3, warmup=3)),
                       (4, dict(steps=2, warmup=3)),
                       # (config 5 bounded: 10 problems of at most 96^3 unknowns, two rates)
                       (5, dict(requests=40, rates=[30.0, 1000.0], pool=10, serving_max_dofs=96 ** 3))):
        a = copy.copy(args)
        a.config, a.variant, a.no_cpu_baseline = cfg, None, True
        for k, v in extra.items():
            setattr(a, k, v)
        a.no_variants = True
        t0 = time.perf_counter()
        try:
            if cfg == 4:
                line = run_batch(a, world, rank, dist, barrier)
            elif cfg == 5:
                line = run_serving(a, world, rank, dist, barrier)
            else:
                line = run_single(a, world, rank, dist, barrier)
        except Exception as e:                      # reported, not fatal to the headline
            out[str(cfg)] = {"error": f"{type(e).__name__}: {e}"}
            continue
        d = {k: line[k] for k in keep if k in line}
        d["workload"] = line["config"]["workload"]
        d["steps"] = line.get("steps")
        if isinstance(d.get("roofline"), dict):
            r = d["roofline"]
            d["roofline"] = {k: r.get(k) for k in ("kernel", "achieved", "peak", "frac", "launch_us")}
        if "iters" in d and isinstance(d["iters"], list):
            d["iters"] = [min(d["iters"]), max(d["iters"])]
        d["wall_s"] = time.perf_counter() - t0
        out[str(cfg)] = d
    return out


def run_profile(args):
    """Untimed work for profiler captures (ncu): set up the config's variant, then run
    `--profile-count` solves (`--profile solve`) or preconditioner applies
    (`--profile apply`) on the first right-hand side, and print nothing but a summary.
    No number from such a run is a bench value."""
    import torch
    from paper_2304_04876_b300 import gdsw
    C = CONFIGS[args.config]
    variant = args.variant or C["default"]
    prob = C["make"]()
    h = gdsw.Handle(prob.A, prob.part, prob.Z if C["Z"] else None, **C["variants"][variant])
    b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    for _ in range(args.profile_count):
        if args.profile == "solve":
            x.zero_()
            h.solve(b, x)
        else:
            h.apply(b, x)
    torch.cuda.synchronize()
    st = h.stats()
    print(f"profile run: config {args.config} variant {variant}, {args.profile_count} {args.profile} calls, "
          f"n {st['n']}, subdomains {st['n_sub']}", flush=True)
    h.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2, choices=[1, 2, 3, 4, 5])
    ap.add_argument("--variant", default=None)
    ap.add_argument("--batch-count", type=int, default=256)
    ap.add_argument("--pool", type=int, default=16, help="serving: distinct problems")
    ap.add_argument("--serving-copies", type=int, default=2, help="serving: most slots per problem")
    ap.add_argument("--serving-iters", type=int, default=4, help="serving: PCG iterations per round")
    ap.add_argument("--serving-max-dofs", type=int, default=160 ** 3, help="serving: largest problem (unknowns)")
    ap.add_argument("--requests", type=int, default=60, help="serving: requests per rate")
    ap.add_argument("--rates", type=float, nargs="+", default=[10, 30, 100, 300, 1000])
    ap.add_argument("--workers", type=int, default=4)
    ap.add_argument("--serving-budget-gb", type=float, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="default line without the bounded runs of configs 1, 3, 4, 5")
    ap.add_argument("--profile", default=None, choices=["solve", "apply"],
                    help="untimed solves or applies for profiler captures (configs 1-3)")
    ap.add_argument("--profile-count", type=int, default=1)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.config in CONFIGS and args.variant is not None and args.variant not in CONFIGS[args.config]["variants"]:
        ap.error(f"variant must be one of {sorted(CONFIGS[args.config]['variants'])}")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    # the oracle's CPU baseline first: its worker processes are forked, which must
    # happen before this process makes any CUDA call
    cpu_baseline = None
    if (rank == 0 and world == 1 and not args.no_cpu_baseline and args.profile is None
            and args.config in (1, 2, 3)):
        C = CONFIGS[args.config]
        variant = args.variant or C["default"]
        cpu_baseline = oracle_sample(C["make"](), args.config, variant, golden_iters(args.config, variant) or 73)

    import torch
    from paper_2304_04876_b300 import build, gdsw
    if rank == 0 and not os.path.exists(gdsw.LIB_PATH):
        build.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    else:
        torch.cuda.set_device(0)

    def barrier():
        if dist is not None:
            dist.barrier()

    if args.profile is not None:
        if args.config not in (1, 2, 3):
            ap.error("--profile runs configs 1-3")
        run_profile(args)
        return
    if args.config == 4:
        line = run_batch(args, world, rank, dist, barrier)
    elif args.config == 5:
        line = run_serving(args, world, rank, dist, barrier)
    else:
        line = run_single(args, world, rank, dist, barrier, cpu_baseline)
        if args.config == 2 and not args.no_configs and world == 1:
            line["configs"] = config_summaries(args, world, rank, dist, barrier)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
