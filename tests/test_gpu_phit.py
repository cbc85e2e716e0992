"""Eq. 1's restriction Phi^T r (the coarse right-hand side) in its two forms, both
forced: a warp per column of a chunk, or eight columns at a time over the chunk's
rows with a transposing butterfly: the applies agree with each other to rounding and
with the oracle (FP64 1e-10, FP32 2e-5), each form repeats bit for bit, the Krylov
solves take the oracle's iteration count, and without the override the fixed rule
picks the wide form only where the chunks' Phi blocks average 48 columns or more."""
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
    old = os.environ.get("GDSW_PHIT")
    if flag is None:
        os.environ.pop("GDSW_PHIT", None)
    else:
        os.environ["GDSW_PHIT"] = flag
    try:
        return make()
    finally:
        if old is None:
            os.environ.pop("GDSW_PHIT", None)
        else:
            os.environ["GDSW_PHIT"] = old


CASES = [
    # interior blocks of 343 rows and up to 7 columns
    ("poisson24_s8_ic0", lambda: P.poisson_problem(24, 8), dict(local_solver="ic0"), dict(local="ic0")),
    # blocks of over 1024 rows: several CTA chunks per block
    ("poisson36_s12_ic0", lambda: P.poisson_problem(36, 12), dict(local_solver="ic0"), dict(local="ic0")),
    # rigid-body modes: 36 to 156 columns per block, a ragged last group of eight
    ("elast18_s6_ilu0", lambda: P.elasticity_problem(18, 6), dict(local_solver="ilu0"), dict(local="ilu0")),
    ("elast12_s6_rgdsw", lambda: P.elasticity_problem(12, 6), dict(local_solver="ilu0", coarse="rgdsw"),
     dict(local="ilu0", coarse="rgdsw")),
]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
@pytest.mark.parametrize("name,make,hopts,oopts", CASES, ids=[c[0] for c in CASES])
def test_phiT_forms_match(name, make, hopts, oopts, precision, tol):
    prob = make()
    hw = _with("wide", lambda: gpu_handle(prob, precision=precision, **hopts))
    hc = _with("cols", lambda: gpu_handle(prob, precision=precision, **hopts))
    assert hw.stats()["phiT_wide"] == 1 and hc.stats()["phiT_wide"] == 0
    M = oracle_for(prob, **oopts)
    for seed in range(2):
        r = np.random.default_rng(seed).uniform(-1, 1, prob.A.n)
        zw, zc = gpu_apply(hw, r), gpu_apply(hc, r)
        assert relerr(zw, zc) <= tol, name
        assert relerr(zw, M.apply(r)) <= (1e-10 if precision == "fp64" else 2e-5), name
        assert np.array_equal(gpu_apply(hw, r), zw)
    hw.close()
    hc.close()


def test_phiT_wide_in_gmres_matches_oracle():
    from oracle import gdsw_oracle as O
    prob = P.elasticity_problem(18, 6)
    h = _with("wide", lambda: gpu_handle(prob, local_solver="ilu0", krylov="gmres"))
    assert h.stats()["phiT_wide"] == 1
    M = oracle_for(prob, local="ilu0")
    x, info = gpu_solve(h, prob.b)
    _, io = O.gmres(M.spmv, M.apply, prob.b, tol=1e-8, restart=30)
    assert info.converged and info.true_relres <= 1e-8
    assert abs(info.iters - io.iters) <= 2, (info.iters, io.iters)
    h.close()


@pytest.mark.parametrize("make,want", [
    (lambda: P.poisson_problem(24, 8), 0),         # up to 7 columns per block
    (lambda: P.elasticity_problem(12, 6), 0),      # 36 columns per block
    (lambda: P.elasticity_problem(18, 6), 1),      # 57.8 columns per block on average
], ids=["poisson24_s8", "elast12_s6", "elast18_s6"])
def test_phiT_default_rule(make, want):
    prob = make()
    h = _with(None, lambda: gpu_handle(prob, local_solver="ilu0" if prob.Z.shape[1] > 1 else "ic0"))
    assert h.stats()["phiT_wide"] == want
    h.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-13), ("fp32", 1e-6)])
def test_prolongation_reads_y_by_map_or_slots(monkeypatch, precision, tol):
    """Phi y beside the local solves (forced) reads y through the block-column map with
    the column form and from the gathered slots with the wide form: the same values,
    so the applies agree with each other to rounding and with the oracle."""
    prob = P.elasticity_problem(18, 6)
    monkeypatch.setenv("GDSW_PROLONG", "1")
    hw = _with("wide", lambda: gpu_handle(prob, local_solver="ilu0", precision=precision))
    hc = _with("cols", lambda: gpu_handle(prob, local_solver="ilu0", precision=precision))
    for h, wide in ((hw, 1), (hc, 0)):
        st = h.stats()
        assert st["phi_beside_local"] == 1 and st["phiT_wide"] == wide
    M = oracle_for(prob, local="ilu0")
    r = np.random.default_rng(7).uniform(-1, 1, prob.A.n)
    zw, zc = gpu_apply(hw, r), gpu_apply(hc, r)
    assert relerr(zw, zc) <= tol
    assert relerr(zc, M.apply(r)) <= (1e-10 if precision == "fp64" else 2e-5)
    hw.close()
    hc.close()
