"""Write tests/golden/oracle_pcg.json: PCG iteration counts and final residuals of the
CPU oracle (oracle/ only) on the fixed Poisson workloads, used by the full-size GPU
parity tests and by bench.py's CPU baseline so neither has to rerun the slow oracle
solve.  Run: python tests/golden/make_golden.py   (several minutes on 8 cores)."""
import json
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import gdsw_oracle as O  # noqa: E402
from paper_2304_04876_b300 import problems as P  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_pcg.json")


def main():
    res = {"_about": "oracle PCG (tol 1e-8, x0 = 0) on seeded uniform right-hand sides; "
                     "written by tests/golden/make_golden.py from oracle/ only"}
    for name, cfg, seeds, variants in [
        ("poisson_16_s8", 1, range(5), [("exact", "levelsched"), ("ic0", "levelsched"), ("ic0", "jacobi")]),
        ("poisson_128_s16", 2, [0], [("ic0", "levelsched"), ("ic0", "jacobi")]),
    ]:
        base = P.config_problem(cfg, 0)
        M = None
        for local, trsv in variants:
            t0 = time.time()
            if M is None or M.local != local:
                M = O.GDSW(base.A, base.part, base.Z, local=local, trsv=trsv)
            M.trsv = trsv
            for seed in seeds:
                b = P.rhs_uniform(base.A.n, seed)
                x, info = O.pcg(M.spmv, M.apply, b, tol=1e-8)
                key = f"{name}/{local}/{trsv}/seed{seed}"
                res[key] = {"iters": info.iters, "relres": info.relres, "converged": bool(info.converged)}
                print(key, res[key], f"{time.time() - t0:.1f}s", flush=True)
    # Q1 elasticity 48^3 elements, 4^3 subdomains, ILU(0) 3 sweeps, right-preconditioned GMRES(30)
    prob = P.config_problem(3)
    t0 = time.time()
    M = O.GDSW(prob.A, prob.part, prob.Z, local=O.ILU0)
    for trsv in ("levelsched", "jacobi"):
        M.trsv = trsv
        x, info = O.gmres(M.spmv, M.apply, prob.b, tol=1e-8, restart=30)
        key = f"elasticity_48_se12/ilu0/{trsv}/gmres30/body_force"
        res[key] = {"iters": info.iters, "relres": info.relres, "converged": bool(info.converged)}
        print(key, res[key], f"{time.time() - t0:.1f}s", flush=True)
    json.dump(res, open(OUT, "w"), indent=1, sort_keys=True)


if __name__ == "__main__":
    main()
