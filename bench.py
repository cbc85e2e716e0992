"""Benchmark: GDSW-preconditioned PCG to a 1e-8 relative residual on one B300.

Workload (default): 3D Poisson, 7-point, 128^3 unknowns, 8x8x8 = 512 subdomains of
16^3 nodes, overlap 1, GDSW coarse space (constants, n0 = 2863), IC(0) from 3
synchronous fixed-point sweeps, FP64 PCG.  A step is one full solve (setup
excluded, reported separately) of a seeded uniform right-hand side resident in
HBM.  The per-iteration working set (~0.9 GB) is far larger than the 126 MB L2,
so no explicit flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--variant NAME] [--impl reference]

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
import threading
import time

# the CPU oracle legs run single-threaded; set before numpy loads its BLAS
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2304_04876_b300 import problems as P  # noqa: E402

VARIANTS = {
    "fp64_levelsched": dict(local_solver="ic0", trsv="levelsched", precision="fp64"),
    "fp64_jacobi": dict(local_solver="ic0", trsv="jacobi", precision="fp64"),
    "fp32_levelsched": dict(local_solver="ic0", trsv="levelsched", precision="fp32"),
    "fp32_jacobi": dict(local_solver="ic0", trsv="jacobi", precision="fp32"),
}
DEFAULT_VARIANT = "fp64_levelsched"
METRIC = "PCG solves/s to 1e-8 relative residual (time-to-residual = 1/value)"
WORKLOAD = "poisson7_128^3_512sub16^3_gdsw_ic0"


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


# ---------------------------------------------------------------------------
# algorithmic bytes (each array touched once per launch)
# ---------------------------------------------------------------------------

def apply_bytes(st: dict, vbytes: int) -> dict:
    """Algorithmic bytes of the four apply phases for value size `vbytes`."""
    n, sum_m, n0, nblk = st["n"], st["sum_omega"], st["n0"], st["n_blocks"]
    tri = 0
    for nnz, lev in ((st["nnz_L"], st["n_levels_L"]), (st["nnz_U"], st["n_levels_U"])):
        off = nnz - sum_m
        tri += off * (vbytes + 2) + sum_m * (vbytes + 2) + lev * 16
    if st["dense_local"]:
        tri = st["dense_local"] * vbytes
    local = sum_m * (8 + 4) + tri + sum_m * vbytes + st["n_sub"] * 8
    phit = st["nnz_phi"] * vbytes + n * (8 + 4) + (nblk + 1) * 12 if n0 else 0
    coarse = n0 * n0 * 8 + n0 * 8 * 3 if n0 else 0
    combine = (sum_m * 4 + (n + 1) * 4 + sum_m * vbytes + n * 4 + st["nnz_phi"] * vbytes
               + n * 8 + nblk * 16)
    return {"local": local, "phiT": phit, "coarse": coarse, "combine": combine}


def spmv_bytes(st: dict) -> int:
    return st["nnz"] * 12 + (st["n"] + 1) * 4 + st["n"] * 16


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
        outdir = os.path.join(ROOT, "gpurun_out") if os.path.isdir(os.path.join(ROOT, "gpurun_out")) else None
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv", dir=outdir)
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

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

def golden_iters(variant: str) -> int | None:
    path = os.path.join(ROOT, "tests", "golden", "oracle_pcg.json")
    if not os.path.exists(path):
        return None
    g = json.load(open(path))
    trsv = "jacobi" if "jacobi" in variant else "levelsched"
    e = g.get(f"poisson_128_s16/ic0/{trsv}/seed0")
    return None if e is None else int(e["iters"])


def oracle_sample(prob, variant: str, iters_for_metric: int, n_iter: int = 2) -> dict:
    """Time the oracle's PCG iteration (SpMV + M^-1 apply + vector updates) on the full
    workload after its setup; solves/s = 1 / (t_iteration * iterations of a solve)."""
    from oracle import gdsw_oracle as O
    trsv = O.JACOBI if "jacobi" in variant else O.LEVELSCHED
    if True:
        t0 = time.perf_counter()
        M = O.GDSW(prob.A, prob.part, prob.Z, local=O.IC0, trsv=trsv)
        setup_s = time.perf_counter() - t0
        b = prob.b
        r = b.copy()
        p = M.apply(r)
        times = []
        for _ in range(n_iter):
            t1 = time.perf_counter()
            q = M.spmv(p)
            alpha = (r @ p) / (p @ q)
            r = r - alpha * q
            z = M.apply(r)
            beta = (r @ z) / (r @ r + 1.0)
            p = z + beta * p
            times.append(time.perf_counter() - t1)
    t_it = statistics.median(times)
    return {"value": 1.0 / (t_it * iters_for_metric), "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"{n_iter} oracle PCG iterations (SpMV + M^-1 apply + updates) on the full workload, "
                      f"median {t_it:.3f} s/iteration x {iters_for_metric} iterations per solve; "
                      f"oracle setup {setup_s:.1f} s not counted",
            "seconds_per_iteration": t_it, "oracle_setup_s": setup_s}


# ---------------------------------------------------------------------------
# reference arm: the oracle as it stands on the host cores
# ---------------------------------------------------------------------------

def run_reference(args, rank: int):
    if rank != 0:
        return
    prob = P.config_problem(2, seed=0)
    variant = args.variant
    iters = golden_iters(variant) or 40
    from oracle import gdsw_oracle as O
    trsv = O.JACOBI if "jacobi" in variant else O.LEVELSCHED
    if True:
        M = O.GDSW(prob.A, prob.part, prob.Z, local=O.IC0, trsv=trsv)

        def step():
            # one bounded sample: one PCG iteration of the oracle on the full workload
            q = M.spmv(prob.b)
            z = M.apply(prob.b - 1e-3 * q)
            return float(z[0])

        for _ in range(args.warmup):
            step()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            step()
        el = time.perf_counter() - t0
    t_it = el / args.steps
    value = 1.0 / (t_it * iters)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_it * iters,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "variant": variant, "n": prob.A.n,
                                            "subdomains": 512},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"each step = one oracle PCG iteration (SpMV + apply) on the full "
                                       f"workload; solves/s = 1/(s per iteration x {iters} iterations)"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--variant", default=DEFAULT_VARIANT, choices=sorted(VARIANTS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

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
    dev = torch.cuda.current_device()

    def barrier():
        if dist is not None:
            dist.barrier()

    prob = P.config_problem(2, seed=0)
    opts = VARIANTS[args.variant]
    t0 = time.perf_counter()
    h = gdsw.Handle(prob.A, prob.part, None, **opts)
    setup_s = time.perf_counter() - t0
    st = h.stats()
    n = prob.A.n
    bs = [torch.tensor(P.rhs_uniform(n, (rank * 5 + k) % 997), dtype=torch.float64, device="cuda")
          for k in range(5)]
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    infos = []
    for k in range(args.warmup):
        x.zero_()
        h.solve(bs[k % 5], x)
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(args.steps):
        x.zero_()
        infos.append(h.solve(bs[k % 5], x))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    el = e0.elapsed_time(e1) / 1e3
    if dist is not None:
        t = torch.tensor([el], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        el = float(t.item())
    iters = [i.iters for i in infos]
    relres = max(i.true_relres for i in infos)
    value = world * args.steps / el
    launches = sum(9 + 8 * it for it in iters)

    # end to end through the C ABI with host (page-locked) buffers
    bh = torch.tensor(P.rhs_uniform(n, rank * 5), dtype=torch.float64).pin_memory()
    xh = torch.zeros(n, dtype=torch.float64).pin_memory()
    h.solve_host(bh, xh)
    barrier()
    torch.cuda.synchronize()
    te = time.perf_counter()
    for k in range(args.steps):
        xh.zero_()
        h.solve_host(bh, xh)
    torch.cuda.synchronize()
    e2e_el = time.perf_counter() - te
    if dist is not None:
        t = torch.tensor([e2e_el], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_el = float(t.item())

    # per-phase apply times and SpMV (CUDA events on the launching stream)
    vb = 4 if opts["precision"] == "fp32" else 8
    rr = bs[0].clone()
    zz = torch.empty_like(rr)
    phases = np.zeros(4)
    reps = 20
    for _ in range(3):
        h.apply_timed(rr, zz)
    for _ in range(reps):
        phases += np.array(h.apply_timed(rr, zz))
    phases /= reps
    ab = apply_bytes(st, vb)
    # the apply as the solver runs it (branches overlapped), CUDA events
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    for _ in range(reps):
        h.apply(rr, zz)
    eb.record(stream)
    torch.cuda.synchronize()
    apply_overlapped_ms = ea.elapsed_time(eb) / reps
    es, ee = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(3):
        h.spmv(rr, zz)
    es.record(stream)
    for _ in range(reps):
        h.spmv(rr, zz)
    ee.record(stream)
    torch.cuda.synchronize()
    spmv_ms = es.elapsed_time(ee) / reps
    hbm, src = peaks()
    names = ["local", "phiT", "coarse", "combine"]
    phase_ms = dict(zip(names, phases.tolist()))
    dom = max(names, key=lambda k: phase_ms[k])
    achieved = ab[dom] / (phase_ms[dom] * 1e-3) / 1e9
    apply_ms = float(phases.sum())
    apply_gbs = sum(ab.values()) / (apply_ms * 1e-3) / 1e9

    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if vb == 4 else "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "variant": args.variant, "n": n, "nnz": st["nnz"],
                   "subdomains": st["n_sub"], "n0": st["n0"], "overlap": 1, "tol": 1e-8,
                   "l2": "per-iteration working set ~0.9 GB >> 126 MB L2; no flush",
                   "parallelism": f"replicas{world}"},
        "time_to_residual_ms": 1e3 * el / args.steps, "iters": iters, "true_relres_max": relres,
        "setup_s": setup_s, "setup_phase_s": st["setup_phase_seconds"],
        "apply_ms": apply_ms, "apply_phase_ms": phase_ms, "apply_gbs": apply_gbs,
        "apply_overlapped_ms": apply_overlapped_ms,
        "apply_overlapped_gbs": sum(ab.values()) / (apply_overlapped_ms * 1e-3) / 1e9,
        "apply_frac_of_measured_hbm": apply_gbs / hbm,
        "spmv_ms": spmv_ms, "spmv_gbs": spmv_bytes(st) / (spmv_ms * 1e-3) / 1e9,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": None, "peak_source": src,
                     "algorithmic_bytes_per_launch": ab[dom]},
        "e2e": {"value": world * args.steps / e2e_el, "unit": "solves/s", "h2d_bytes_per_step": 2 * 8 * n,
                "d2h_bytes_per_step": 8 * n},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if not args.no_variants and rank == 0:
        var = {}
        for name, vo in VARIANTS.items():
            if name == args.variant:
                continue
            hv = gdsw.Handle(prob.A, prob.part, None, **vo)
            for k in range(2):
                x.zero_()
                hv.solve(bs[0], x)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            inf = []
            for k in range(3):
                x.zero_()
                inf.append(hv.solve(bs[k], x))
            torch.cuda.synchronize()
            var[name] = {"ms_per_solve": 1e3 * (time.perf_counter() - t1) / 3, "iters": [i.iters for i in inf],
                         "true_relres_max": max(i.true_relres for i in inf)}
            hv.close()
        line["variants"] = var
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        it_ref = golden_iters(args.variant) or int(np.median(iters))
        line["cpu_baseline"] = oracle_sample(prob, args.variant, it_ref)
    if rank == 0:
        print(json.dumps(line), flush=True)
    h.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
