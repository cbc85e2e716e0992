"""Eq. 1's prolongation Phi y formed on the coarse stream beside the local solves
(k_prolong, one value per block-row position that the scatter-add adds) against the
product formed inside the scatter-add, both forced: the applies agree to rounding
(FP64 1e-13, FP32 1e-6) and with the oracle, the Krylov solves take the same number of
iterations, a batched handle skips a stopped member's positions, the stats report
where the product was formed, and without the override the fixed rule decides."""
import os

import numpy as np
import pytest

from paper_2304_04876_b300 import problems as P
from tests.gpu_util import gpu_apply, gpu_handle, gpu_solve, oracle_for, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2304_04876_b300 import build
    build.build()
    assert torch.cuda.is_available()


def _with(flag, make):
    old = os.environ.get("GDSW_PROLONG")
    os.environ["GDSW_PROLONG"] = flag
    try:
        return make()
    finally:
        if old is None:
            os.environ.pop("GDSW_PROLONG")
        else:
            os.environ["GDSW_PROLONG"] = old


CASES = [
    ("poisson12_ic0", lambda: P.poisson_problem(12, 4), dict(local_solver="ic0"), dict(local="ic0")),
    ("ragged13_exact", lambda: P.poisson_problem(13, 4, seed=3), dict(local_solver="exact"), dict(local="exact")),
    ("elast6_ilu0", lambda: P.elasticity_problem(6, 2), dict(local_solver="ilu0"), dict(local="ilu0")),
    ("elast8_rgdsw", lambda: P.elasticity_problem(8, 4), dict(local_solver="ilu0", coarse="rgdsw"),
     dict(local="ilu0", coarse="rgdsw")),
]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
@pytest.mark.parametrize("name,make,hopts,oopts", CASES, ids=[c[0] for c in CASES])
def test_prolongation_beside_local_solves_matches(name, make, hopts, oopts, precision, tol):
    prob = make()
    h1 = _with("1", lambda: gpu_handle(prob, precision=precision, **hopts))
    h0 = _with("0", lambda: gpu_handle(prob, precision=precision, **hopts))
    assert h1.stats()["phi_beside_local"] == 1 and h0.stats()["phi_beside_local"] == 0
    M = oracle_for(prob, **oopts)
    for seed in range(2):
        r = np.random.default_rng(seed).uniform(-1, 1, prob.A.n)
        z1, z0 = gpu_apply(h1, r), gpu_apply(h0, r)
        assert relerr(z1, z0) <= tol, name
        assert relerr(z1, M.apply(r)) <= (1e-10 if precision == "fp64" else 2e-5), name
        assert np.array_equal(gpu_apply(h1, r), z1)
    h1.close()
    h0.close()


@pytest.mark.parametrize("krylov", ["pcg", "gmres"])
def test_prolongation_in_krylov_solves(krylov):
    prob = P.elasticity_problem(8, 4)
    its = {}
    for flag in ("1", "0"):
        h = _with(flag, lambda: gpu_handle(prob, local_solver="ilu0", krylov=krylov))
        x, info = gpu_solve(h, prob.b)
        assert info.converged and info.true_relres <= 1e-8
        its[flag] = info.iters
        h.close()
    assert abs(its["1"] - its["0"]) <= 1, its


def test_prolongation_in_a_batched_handle():
    import torch
    from paper_2304_04876_b300 import gdsw as G
    mem = P.diffusion_batch(4, seed=2, nmin=7, nmax=12, smin=3, smax=5)
    b = np.concatenate([m.b if i != 1 else np.zeros(m.A.n) for i, m in enumerate(mem)])
    offs = np.cumsum([0] + [m.A.n for m in mem])
    out = {}
    for flag in ("1", "0"):
        h = _with(flag, lambda: G.Handle.batch([(m.A, m.part, None) for m in mem], local_solver="ic0"))
        assert h.stats()["phi_beside_local"] == int(flag)
        bt = torch.tensor(b, dtype=torch.float64, device="cuda")
        xt = torch.zeros_like(bt)
        infos = h.solve_batch(bt, xt)
        torch.cuda.synchronize()
        assert all(i.converged for i in infos)
        assert infos[1].iters == 0 and not np.any(xt.cpu().numpy()[offs[1]:offs[2]])
        out[flag] = (xt.cpu().numpy(), [i.iters for i in infos])
        h.close()
    assert all(abs(a - c) <= 1 for a, c in zip(out["1"][1], out["0"][1]))
    assert relerr(out["1"][0], out["0"][0]) <= 1e-8


def test_prolongation_default_rule():
    """Without GDSW_PROLONG: beside the local solves for one problem with fewer
    subdomains than SMs and n >= 65,536, or with n >= 2^20; in the scatter-add for
    smaller problems and for a batch."""
    from paper_2304_04876_b300 import gdsw as G
    assert os.environ.get("GDSW_PROLONG") is None
    for make, want in ((lambda: P.poisson_problem(12, 4), 0),        # n = 1,728
                       (lambda: P.poisson_problem(48, 12), 1),       # 64 subdomains, n = 110,592
                       (lambda: P.poisson_problem(48, 6), 0),        # 512 subdomains, n = 110,592
                       (lambda: P.poisson_problem(102, 17), 1)):     # 216 subdomains, n = 1,061,208
        prob = make()
        h = gpu_handle(prob, local_solver="ic0", precision="fp32")
        assert h.stats()["phi_beside_local"] == want, prob.name
        h.close()
    # 16 subdomains, ~150 K unknowns: beside the local solves were it one problem
    mem = P.diffusion_batch(2, seed=2, nmin=40, nmax=44, smin=20, smax=22)
    h = G.Handle.batch([(m.A, m.part, None) for m in mem], local_solver="ic0")
    assert h.stats()["phi_beside_local"] == 0
    h.close()
