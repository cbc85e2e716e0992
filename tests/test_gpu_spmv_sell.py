"""The SpMV for long rows from the sliced ELL copy (slices of 8 rows, entries
column-major within a slice, 16-bit column offsets; four lanes per row, 4 or 8 of a
lane's entries in flight) against the CSR kernel with lanes per row, both forced instead of chosen by
timing: each within 1e-13 of the CSR product on elasticity (81 entries per interior
row, shorter rows on the boundary and a ragged last slice), and the Krylov solves
that use it (PCG with the fused (p, Ap), GMRES, a batched handle whose stopped
members' rows are skipped) reach the tolerance with the iteration counts of the CSR
kernel."""
import os

import numpy as np
import pytest

from paper_2304_04876_b300 import problems as P
from tests.gpu_util import gpu_handle, gpu_solve, gpu_spmv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2304_04876_b300 import build
    build.build()
    assert torch.cuda.is_available()


def _with_spmv(kind, make):
    old = os.environ.get("GDSW_SPMV")
    os.environ["GDSW_SPMV"] = kind
    try:
        return make()
    finally:
        if old is None:
            os.environ.pop("GDSW_SPMV")
        else:
            os.environ["GDSW_SPMV"] = old


@pytest.mark.parametrize("make", [lambda: P.elasticity_problem(6, 2), lambda: P.elasticity_problem(7, 3),
                                  lambda: P.elasticity_problem(5, 5)], ids=["elast6", "elast7_ragged", "elast5"])
def test_sell_matches_csr_product(make):
    prob = make()
    ref_fn = prob.A.to_scipy()
    for seed in range(2):
        x = np.random.default_rng(seed).uniform(-1, 1, prob.A.n)
        ref = ref_fn @ x
        for kind in ("sell", "sell8", "rows"):
            h = _with_spmv(kind, lambda: gpu_handle(prob, local_solver="ilu0"))
            y = gpu_spmv(h, x)
            assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max(), kind
            h.close()


@pytest.mark.parametrize("krylov", ["pcg", "gmres"])
def test_sell_in_krylov_solves(krylov):
    prob = P.elasticity_problem(8, 4)
    its = {}
    for kind in ("sell", "rows"):
        h = _with_spmv(kind, lambda: gpu_handle(prob, local_solver="ilu0", krylov=krylov))
        x, info = gpu_solve(h, prob.b)
        assert info.converged and info.true_relres <= 1e-8, kind
        its[kind] = info.iters
        h.close()
    assert abs(its["sell"] - its["rows"]) <= 1, its


def test_sell_in_a_batched_handle():
    import torch
    from paper_2304_04876_b300 import gdsw as G
    mem = [P.elasticity_problem(4, 2), P.elasticity_problem(6, 2), P.elasticity_problem(6, 3)]
    b = np.concatenate([m.b for m in mem])
    out = {}
    for kind in ("sell", "rows"):
        h = _with_spmv(kind, lambda: G.Handle.batch(
            [(m.A, m.part, None if m.Z is None or m.Z.shape[1] == 1 else m.Z) for m in mem],
            local_solver="ilu0"))
        bt = torch.tensor(b, dtype=torch.float64, device="cuda")
        xt = torch.zeros_like(bt)
        infos = h.solve_batch(bt, xt)
        torch.cuda.synchronize()
        assert all(i.converged and i.true_relres <= 1e-8 for i in infos), kind
        out[kind] = [i.iters for i in infos]
        h.close()
    assert all(abs(a - c) <= 1 for a, c in zip(out["sell"], out["rows"])), out
