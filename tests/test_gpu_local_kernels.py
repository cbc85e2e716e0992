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
    """The SpMV kernels for short rows (tiled, tiled with the next tile's loads in
    flight, a thread per row), forced instead of chosen by timing: each within
    1e-13 of the CSR product, and bitwise equal to each other (same sums in the
    same order)."""
    from paper_2304_04876_b300 import gdsw as G
    from tests.gpu_util import gpu_spmv
    for prob in (P.poisson_problem(40, 8), P.elasticity_problem(6, 2), P.poisson_problem(13, 4, seed=3)):
        x = np.random.default_rng(1).uniform(-1, 1, prob.A.n)
        ref = prob.A.to_scipy() @ x
        ys = []
        for kind in ("stream", "pipe", "thread"):
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
        assert np.array_equal(ys[0], ys[1]) and np.array_equal(ys[0], ys[2])


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


def _handle_env(prob, env, **opts):
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return gpu_handle(prob, **opts)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v


JAC_CASES = [
    ("poisson16_ic0", lambda: P.poisson_problem(16, 8), dict(local="ic0")),
    ("ragged13_ilu0", lambda: P.poisson_problem(13, 4, seed=3), dict(local="ilu0")),
    ("elast6_ilu0", lambda: P.elasticity_problem(6, 2), dict(local="ilu0")),
    ("poisson12_ic1", lambda: P.poisson_problem(12, 4), dict(local="ic0", fill_level=1)),
    ("sweeps3", lambda: P.poisson_problem(12, 4), dict(local="ic0", sweeps_trsv=3)),
]


@pytest.mark.parametrize("precision,mode", [("fp64", 0), ("fp32", 0), ("fp32", 1), ("fp16", 2), ("fp16", 1)])
@pytest.mark.parametrize("name,make,opts", JAC_CASES, ids=[c[0] for c in JAC_CASES])
def test_resident_jacobi_matches_oracle_and_unpipelined(name, make, opts, precision, mode):
    """Jacobi sweeps (Sec. V-B3) on factor blocks resident in shared memory, the
    next block's copy overlapping the sweeps (mode 2) or one block at a time
    (mode 1): within 1e-10 of the oracle in FP64 (2e-5 FP32, 5e-3 FP16 storage), and
    in FP32/FP64 bitwise equal to the unpipelined Jacobi kernel, which forms every
    sum in the same order."""
    prob = make()
    M = oracle_for(prob, trsv="jacobi", **opts)
    hopts = {("local_solver" if k == "local" else k): v for k, v in opts.items()}
    hopts.update(trsv="jacobi", precision=precision)
    env = {"GDSW_JACOBI_MODE": str(mode)} if mode else {}
    h = _handle_env(prob, env, **hopts)
    assert h.stats()["local_kernel"] == 5, name
    ref_h = _handle_env(prob, {"GDSW_JACOBI_RESIDENT": "0"}, **hopts)
    assert ref_h.stats()["local_kernel"] == 2
    tol = {"fp64": 1e-10, "fp32": 2e-5, "fp16": 5e-3}[precision]
    for seed in range(2):
        r = np.random.default_rng(seed).uniform(-1, 1, prob.A.n)
        z = gpu_apply(h, r)
        assert relerr(z, M.apply(r)) <= tol, (name, precision, mode)
        if precision != "fp16":
            assert np.array_equal(z, gpu_apply(ref_h, r)), (name, precision, mode)
    h.close()
    ref_h.close()


def test_resident_jacobi_pcg_and_batched_members():
    """PCG with the resident-block Jacobi solve converges with the oracle's count
    (+-1); in a batched handle each member's solution equals its own solve alone."""
    from oracle import gdsw_oracle as O
    from paper_2304_04876_b300 import gdsw as G
    prob = P.poisson_problem(16, 8)
    M = oracle_for(prob, local="ic0", trsv="jacobi")
    h = gpu_handle(prob, local_solver="ic0", trsv="jacobi")
    assert h.stats()["local_kernel"] == 5
    x, info = gpu_solve(h, prob.b)
    _, io = O.pcg(M.spmv, M.apply, prob.b)
    assert info.converged and info.true_relres <= 1e-8 and abs(info.iters - io.iters) <= 1
    h.close()
    import torch
    probs = [P.poisson_problem(12, 4), P.poisson_problem(16, 8, seed=4)]
    hb = G.Handle.batch([(p.A, p.part, None) for p in probs], local_solver="ic0", trsv="jacobi", precision="fp32")
    assert hb.stats()["local_kernel"] == 5
    b = torch.tensor(np.concatenate([p.b for p in probs]), dtype=torch.float64, device="cuda")
    xb = torch.zeros_like(b)
    infos = hb.solve_batch(b, xb)
    off = 0
    for p, inf in zip(probs, infos):
        h1 = gpu_handle(p, local_solver="ic0", trsv="jacobi", precision="fp32")
        x1, i1 = gpu_solve(h1, p.b)
        assert inf.converged and abs(inf.iters - i1.iters) <= 1
        assert relerr(xb[off:off + p.A.n].cpu().numpy(), x1) <= 1e-6
        off += p.A.n
        h1.close()
    hb.close()


def test_resident_jacobi_wait_that_runs_out_reports_timeout(monkeypatch):
    """GDSW_TEST_STALL=1 withholds the first factor block of CTA 0: its bounded wait
    runs out (about 10 ms), the kernel lets its other copy land and returns, the host
    reports GDSW_ERR_TIMEOUT, and the context stays usable."""
    from paper_2304_04876_b300 import gdsw as G
    import torch
    prob = P.poisson_problem(12, 4)
    monkeypatch.setenv("GDSW_TEST_STALL", "1")
    h = gpu_handle(prob, local_solver="ic0", trsv="jacobi", wait_budget_cycles=20_000_000)
    monkeypatch.delenv("GDSW_TEST_STALL")
    assert h.stats()["local_kernel"] == 5
    rt = torch.tensor(np.random.default_rng(0).uniform(-1, 1, prob.A.n), dtype=torch.float64, device="cuda")
    with pytest.raises(G.GdswError) as e:
        h.apply_timed(rt, torch.empty_like(rt))
    assert e.value.status == G.ERR_TIMEOUT
    h.close()
    h2 = gpu_handle(prob, local_solver="ic0", trsv="jacobi")
    M = oracle_for(prob, local="ic0", trsv="jacobi")
    r = rt.cpu().numpy()
    assert relerr(gpu_apply(h2, r), M.apply(r)) <= 1e-10
    h2.close()
