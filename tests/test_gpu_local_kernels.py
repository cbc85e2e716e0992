"""The level-scheduled local solve (Sec. V-B2 substitution with the IC(k)/ILU(k)
factors of Sec. V-B3) in each of its kernels, forced by shape instead of chosen by
timing: with a barrier per level, and without one (per-row ready flags).  Each is
checked against the oracle's apply (FP64 within 1e-10, FP32 within 2e-5), and the
two kernels against each other bitwise, since they update every row in the same
arithmetic order; the barrier-free kernel's bounded waits are made to run out on
purpose (one level record withheld) and must report GDSW_ERR_TIMEOUT."""
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


def handle_with_shape(prob, shape, **opts):
    old = os.environ.get("GDSW_LOCAL_SHAPE")
    os.environ["GDSW_LOCAL_SHAPE"] = shape
    try:
        return gpu_handle(prob, **opts)
    finally:
        if old is None:
            os.environ.pop("GDSW_LOCAL_SHAPE")
        else:
            os.environ["GDSW_LOCAL_SHAPE"] = old


def _diffusion():
    k = 10 ** np.random.default_rng(7).uniform(-2, 2, (10, 10, 10))
    A = P.diffusion7(k)
    cuts = P.uniform_cuts(10, 4)
    part = P.Partition(10, 10, 10, 1, [cuts, cuts, cuts])
    return P.Problem("diff10", A, part, np.ones((A.n, 1)), P.rhs_uniform(A.n, 1))


CASES = [
    ("poisson12_ic0", lambda: P.poisson_problem(12, 4), dict(local="ic0")),
    ("poisson12_ilu0", lambda: P.poisson_problem(12, 4), dict(local="ilu0")),
    ("ragged13_ic0", lambda: P.poisson_problem(13, 4, seed=3), dict(local="ic0")),
    ("diffusion10_ic0", _diffusion, dict(local="ic0")),
    ("poisson12_ic1", lambda: P.poisson_problem(12, 4), dict(local="ic0", fill_level=1)),
    ("ragged13_ilu1", lambda: P.poisson_problem(13, 4, seed=3), dict(local="ilu0", fill_level=1)),
    ("overlap2_ic0", lambda: P.poisson_problem(12, 4), dict(local="ic0", overlap=2)),
    ("tiny_subdomains_ilu0", lambda: P.poisson_problem(9, 3), dict(local="ilu0")),
    ("poisson20_ic0_large", lambda: P.poisson_problem(20, 10), dict(local="ic0")),
]
SHAPES = ["4,128", "2,64", "8,256", "16,512"]


@pytest.mark.parametrize("name,make,opts", CASES, ids=[c[0] for c in CASES])
def test_both_kernels_match_oracle_and_each_other(name, make, opts):
    prob = make()
    M = oracle_for(prob, **opts)
    hopts = {("local_solver" if k == "local" else k): v for k, v in opts.items()}
    rs = [np.random.default_rng(seed).uniform(-1, 1, prob.A.n) for seed in range(2)]
    refs = [M.apply(r) for r in rs]
    for shape in SHAPES:
        out = {}
        for sf in (0, 1):
            h = handle_with_shape(prob, f"{shape},{sf}", **hopts)
            st = h.stats()
            assert st["local_stages"] == int(shape.split(",")[0]), (name, shape, st["local_stages"])
            out[sf] = [gpu_apply(h, r) for r in rs]
            for z, ref in zip(out[sf], refs):
                assert relerr(z, ref) <= 1e-10, (name, shape, sf)
            h.close()
        for a, b in zip(out[0], out[1]):
            assert np.array_equal(a, b), (name, shape)


@pytest.mark.parametrize("precision,tol", [("fp32", 2e-5), ("fp16", 5e-3)])
def test_reduced_precision_both_kernels(precision, tol):
    prob = P.poisson_problem(16, 8)
    M = oracle_for(prob, local="ic0")
    r = np.random.default_rng(3).uniform(-1, 1, prob.A.n)
    ref = M.apply(r)
    zs = []
    for sf in (0, 1):
        h = handle_with_shape(prob, f"8,128,{sf}", local_solver="ic0", precision=precision)
        z = gpu_apply(h, r)
        assert relerr(z, ref) <= tol, (precision, sf)
        zs.append(z)
        h.close()
    assert np.array_equal(zs[0], zs[1])


def test_barrier_free_kernel_is_deterministic_and_solves():
    prob = P.poisson_problem(16, 4)
    h = handle_with_shape(prob, "4,128,1", local_solver="ic0")
    r = np.random.default_rng(5).uniform(-1, 1, prob.A.n)
    z0 = gpu_apply(h, r)
    for _ in range(5):
        assert np.array_equal(gpu_apply(h, r), z0)
    from oracle import gdsw_oracle as O
    M = oracle_for(prob, local="ic0")
    x, info = gpu_solve(h, prob.b)
    _, io = O.pcg(M.spmv, M.apply, prob.b)
    assert info.converged and info.true_relres <= 1e-8
    assert abs(info.iters - io.iters) <= 1
    h.close()


def test_barrier_free_wait_that_runs_out_reports_timeout(monkeypatch):
    """GDSW_TEST_STALL=1 withholds one level record's copy: the consumers' wait for
    it, and then every wait for a row it would have made final, runs out after the
    budget (about 10 ms); the kernel records it, still meets its barriers, lets the
    copies it issued land and returns, and the host reports GDSW_ERR_TIMEOUT.  A
    handle without the stall then computes normally on the same context."""
    from paper_2304_04876_b300 import gdsw as G
    import torch
    prob = P.poisson_problem(12, 4)
    monkeypatch.setenv("GDSW_TEST_STALL", "1")
    h = handle_with_shape(prob, "4,128,1", local_solver="ic0", wait_budget_cycles=20_000_000)
    monkeypatch.delenv("GDSW_TEST_STALL")
    r = np.random.default_rng(0).uniform(-1, 1, prob.A.n)
    rt = torch.tensor(r, dtype=torch.float64, device="cuda")
    zt = torch.empty_like(rt)
    with pytest.raises(G.GdswError) as e:
        h.apply_timed(rt, zt)
    assert e.value.status == G.ERR_TIMEOUT
    h.close()
    M = oracle_for(prob, local="ic0")
    h2 = handle_with_shape(prob, "4,128,1", local_solver="ic0")
    assert relerr(gpu_apply(h2, r), M.apply(r)) <= 1e-10
    h2.close()


def test_spmv_kernels_match_csr_product_and_each_other():
    """The two tiled SpMV kernels (plain, and with the next tile's loads in flight),
    forced instead of chosen by timing: each within 1e-13 of the CSR product, and
    bitwise equal to each other (same sums in the same order)."""
    from paper_2304_04876_b300 import gdsw as G
    from tests.gpu_util import gpu_spmv
    for prob in (P.poisson_problem(40, 8), P.elasticity_problem(6, 2), P.poisson_problem(13, 4, seed=3)):
        x = np.random.default_rng(1).uniform(-1, 1, prob.A.n)
        ref = prob.A.to_scipy() @ x
        ys = []
        for kind in ("stream", "pipe"):
            old = os.environ.get("GDSW_SPMV")
            os.environ["GDSW_SPMV"] = kind
            try:
                h = gpu_handle(prob, local_solver="exact")
            finally:
                os.environ.pop("GDSW_SPMV") if old is None else os.environ.__setitem__("GDSW_SPMV", old)
            y = gpu_spmv(h, x)
            assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max(), kind
            ys.append(y)
            h.close()
        assert np.array_equal(ys[0], ys[1])


@pytest.mark.parametrize("sf", [0, 1])
def test_small_records_split_levels(sf, monkeypatch):
    """With 512-byte level records every wide level is split into several records
    (the consumers meet only after a level's last one) and many small levels share
    one copy: the solve equals the oracle's and, bit for bit, the one with the
    default records."""
    prob = P.poisson_problem(20, 10)
    M = oracle_for(prob, local="ic0")
    r = np.random.default_rng(2).uniform(-1, 1, prob.A.n)
    h = handle_with_shape(prob, f"16,128,{sf}", local_solver="ic0")
    z_default = gpu_apply(h, r)
    h.close()
    monkeypatch.setenv("GDSW_REC_CAP", "512")
    h = handle_with_shape(prob, f"16,128,{sf}", local_solver="ic0")
    z_small = gpu_apply(h, r)
    x, info = gpu_solve(h, prob.b)
    h.close()
    assert relerr(z_small, M.apply(r)) <= 1e-10
    assert np.array_equal(z_small, z_default)
    assert info.converged and info.true_relres <= 1e-8
