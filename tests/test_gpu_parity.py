"""CUDA path against the oracle on small problems: the preconditioner apply (Eq. 1)
element by element, SpMV, and the Krylov solves.  FP64 apply tolerance 1e-10
relative (2-norm); PCG/GMRES iteration counts within +-1; true residual <= 1e-8."""
import numpy as np
import pytest

from paper_2304_04876_b300 import problems as P
from tests.gpu_util import gpu_apply, gpu_handle, gpu_solve, gpu_spmv, oracle_for, relerr

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2304_04876_b300 import build
    build.build()
    assert torch.cuda.is_available()


def _ragged():
    # 13 nodes per axis with blocks of 4: three full blocks and a last block of one node
    return P.poisson_problem(13, 4, seed=3)


def _diffusion():
    k = 10 ** np.random.default_rng(7).uniform(-2, 2, (10, 10, 10))
    A = P.diffusion7(k)
    cuts = P.uniform_cuts(10, 4)
    part = P.Partition(10, 10, 10, 1, [cuts, cuts, cuts])
    return P.Problem("diff10", A, part, np.ones((A.n, 1)), P.rhs_uniform(A.n, 1))


APPLY_CASES = [
    ("cfg1_exact", lambda: P.config_problem(1), dict(local="exact")),
    ("poisson12_ic0_ls", lambda: P.poisson_problem(12, 4), dict(local="ic0", trsv="levelsched")),
    ("poisson12_ic0_jac", lambda: P.poisson_problem(12, 4), dict(local="ic0", trsv="jacobi")),
    ("poisson12_ilu0_ls", lambda: P.poisson_problem(12, 4), dict(local="ilu0", trsv="levelsched")),
    ("poisson12_ilu0_jac", lambda: P.poisson_problem(12, 4), dict(local="ilu0", trsv="jacobi")),
    ("ragged13_ic0", _ragged, dict(local="ic0")),
    ("ragged13_exact", _ragged, dict(local="exact")),
    ("diffusion10_ic0", _diffusion, dict(local="ic0")),
    ("elast4_exact", lambda: P.elasticity_problem(4, 2), dict(local="exact")),
    ("elast6_ilu0", lambda: P.elasticity_problem(6, 2), dict(local="ilu0")),
    ("elast6_ilu0_jac", lambda: P.elasticity_problem(6, 2), dict(local="ilu0", trsv="jacobi")),
    ("one_level", lambda: P.poisson_problem(12, 4), dict(local="ic0", coarse="none")),
    ("single_subdomain", lambda: P.poisson_problem(6, 6), dict(local="exact")),
    ("overlap2", lambda: P.poisson_problem(12, 4), dict(local="ic0", overlap=2)),
    ("sweeps7", lambda: P.poisson_problem(12, 4), dict(local="ic0", trsv="jacobi", sweeps_factor=7, sweeps_trsv=2)),
    ("rgdsw_poisson12_exact", lambda: P.poisson_problem(12, 4), dict(local="exact", coarse="rgdsw")),
    ("rgdsw_ragged13_ic0", _ragged, dict(local="ic0", coarse="rgdsw")),
    ("rgdsw_diffusion10_ic0", _diffusion, dict(local="ic0", coarse="rgdsw")),
    ("rgdsw_elast6_ilu0", lambda: P.elasticity_problem(6, 2), dict(local="ilu0", coarse="rgdsw")),
    ("rgdsw_two_blocks", lambda: P.poisson_problem(8, 4), dict(local="exact", coarse="rgdsw")),
    ("poisson12_ic1", lambda: P.poisson_problem(12, 4), dict(local="ic0", fill_level=1)),
    ("poisson12_ic2_jac", lambda: P.poisson_problem(12, 4), dict(local="ic0", trsv="jacobi", fill_level=2)),
    ("ragged13_ilu1", _ragged, dict(local="ilu0", fill_level=1)),
    ("diffusion10_ic2", _diffusion, dict(local="ic0", fill_level=2)),
    ("elast6_ilu1", lambda: P.elasticity_problem(6, 2), dict(local="ilu0", fill_level=1)),
    ("overlap0_block_jacobi", lambda: P.poisson_problem(12, 4), dict(local="ic0", overlap=0)),
    ("tiny_subdomains", lambda: P.poisson_problem(9, 3), dict(local="ilu0")),
    ("elast_ragged7", lambda: P.elasticity_problem(7, 3), dict(local="ilu0")),
    ("elast_ragged7_rgdsw_exact", lambda: P.elasticity_problem(7, 3), dict(local="exact", coarse="rgdsw")),
]


@pytest.mark.parametrize("name,make,opts", APPLY_CASES, ids=[c[0] for c in APPLY_CASES])
def test_apply_matches_oracle(name, make, opts):
    prob = make()
    M = oracle_for(prob, **opts)
    h = gpu_handle(prob, **{("local_solver" if k == "local" else k): v for k, v in opts.items()})
    st = h.stats()
    assert st["n0"] == M.n0 and st["sum_omega"] == sum(len(o) for o in M.omega)
    if opts.get("local", "ic0") != "exact":
        # the factor pattern (fill included) is the oracle's, entry for entry in count
        assert st["nnz_L"] == sum(f[1].nnz for f in M.factors)
    for seed in range(3):
        r = np.random.default_rng(seed).uniform(-1, 1, prob.A.n)
        z = gpu_apply(h, r)
        assert relerr(z, M.apply(r)) <= TOL_FP64, name
    h.close()


@pytest.mark.parametrize("local,trsv", [("ic0", "levelsched"), ("ic0", "jacobi"), ("exact", "levelsched"),
                                        ("ilu0", "levelsched")])
def test_fp32_preconditioner_close_to_fp64(local, trsv):
    prob = P.poisson_problem(12, 4)
    M = oracle_for(prob, local=local, trsv=trsv)
    h = gpu_handle(prob, local_solver=local, trsv=trsv, precision="fp32")
    r = np.random.default_rng(0).uniform(-1, 1, prob.A.n)
    assert relerr(gpu_apply(h, r), M.apply(r)) <= 2e-5


def test_spmv_matches_csr_product():
    for prob in (P.poisson_problem(12, 4), P.elasticity_problem(4, 2)):
        h = gpu_handle(prob, local_solver="exact")
        x = np.random.default_rng(1).uniform(-1, 1, prob.A.n)
        y = gpu_spmv(h, x)
        ref = prob.A.to_scipy() @ x
        assert np.abs(y - ref).max() <= 1e-13 * np.abs(ref).max()


def test_apply_is_deterministic():
    prob = P.poisson_problem(12, 4)
    h = gpu_handle(prob, local_solver="ic0")
    r = np.random.default_rng(5).uniform(-1, 1, prob.A.n)
    z0 = gpu_apply(h, r)
    for _ in range(9):
        assert np.array_equal(gpu_apply(h, r), z0)


PCG_CASES = [
    ("cfg1_exact", lambda: P.config_problem(1), dict(local="exact")),
    ("poisson12_ic0", lambda: P.poisson_problem(12, 4), dict(local="ic0")),
    ("poisson12_ic0_jac", lambda: P.poisson_problem(12, 4), dict(local="ic0", trsv="jacobi")),
    ("ragged13_ilu0", _ragged, dict(local="ilu0")),
    ("diffusion10_ic0", _diffusion, dict(local="ic0")),
    ("elast6_exact", lambda: P.elasticity_problem(6, 2), dict(local="exact")),
    ("rgdsw_poisson12_ic0", lambda: P.poisson_problem(12, 4), dict(local="ic0", coarse="rgdsw")),
    ("rgdsw_elast6_exact", lambda: P.elasticity_problem(6, 2), dict(local="exact", coarse="rgdsw")),
    ("poisson12_ic1", lambda: P.poisson_problem(12, 4), dict(local="ic0", fill_level=1)),
    ("elast6_ilu2", lambda: P.elasticity_problem(6, 2), dict(local="ilu0", fill_level=2)),
]


@pytest.mark.parametrize("name,make,opts", PCG_CASES, ids=[c[0] for c in PCG_CASES])
def test_pcg_matches_oracle(name, make, opts):
    from oracle import gdsw_oracle as O
    prob = make()
    M = oracle_for(prob, **opts)
    xo, io = O.pcg(M.spmv, M.apply, prob.b, tol=1e-8)
    h = gpu_handle(prob, **{("local_solver" if k == "local" else k): v for k, v in opts.items()})
    x, info = gpu_solve(h, prob.b)
    assert info.converged and info.true_relres <= 1e-8
    assert abs(info.iters - io.iters) <= 1, (info.iters, io.iters)
    true = np.linalg.norm(prob.b - prob.A.to_scipy() @ x) / np.linalg.norm(prob.b)
    assert true <= 1e-8
    assert relerr(x, xo) <= 1e-6


def test_pcg_single_subdomain_one_iteration_and_zero_rhs():
    prob = P.poisson_problem(6, 6)
    h = gpu_handle(prob, local_solver="exact")
    x, info = gpu_solve(h, prob.b)
    assert info.iters == 1 and info.converged
    x, info = gpu_solve(h, np.zeros(prob.A.n))
    assert info.iters == 0 and not x.any()
    # warm start at the solution
    xs = np.linalg.solve(prob.A.to_scipy().toarray(), prob.b)
    x, info = gpu_solve(h, prob.b, x0=xs)
    assert info.iters == 0


def test_gmres_matches_oracle():
    from oracle import gdsw_oracle as O
    prob = P.elasticity_problem(6, 2)
    M = oracle_for(prob, local="ilu0")
    xo, io = O.gmres(M.spmv, M.apply, prob.b, tol=1e-8, restart=30)
    h = gpu_handle(prob, local_solver="ilu0", krylov="gmres", restart=30)
    x, info = gpu_solve(h, prob.b)
    assert info.converged and info.true_relres <= 1e-8
    assert abs(info.iters - io.iters) <= 1, (info.iters, io.iters)
    # a short restart forces restarts and still converges
    h2 = gpu_handle(prob, local_solver="ilu0", krylov="gmres", restart=5)
    xo2, io2 = O.gmres(M.spmv, M.apply, prob.b, tol=1e-8, restart=5)
    x2, info2 = gpu_solve(h2, prob.b)
    assert info2.converged and abs(info2.iters - io2.iters) <= 2


def test_gmres_exact_preconditioner_one_step_and_poisson():
    """One subdomain with the exact local solve makes A M^-1 = I: the first Arnoldi
    vector is already in the basis (the second Gram-Schmidt pass finds a zero
    remainder) and GMRES stops after one step.  GMRES on a Poisson problem with
    fill and FP32 factors matches the oracle's count."""
    from oracle import gdsw_oracle as O
    one = P.poisson_problem(6, 6)
    h = gpu_handle(one, local_solver="exact", krylov="gmres")
    x, info = gpu_solve(h, one.b)
    assert info.converged and info.iters == 1 and info.true_relres <= 1e-8
    prob = P.poisson_problem(12, 4)
    M = oracle_for(prob, local="ic0", fill_level=1)
    _, io = O.gmres(M.spmv, M.apply, prob.b, tol=1e-8, restart=30)
    h = gpu_handle(prob, local_solver="ic0", fill_level=1, krylov="gmres")
    x, info = gpu_solve(h, prob.b)
    assert info.converged and abs(info.iters - io.iters) <= 1 and info.true_relres <= 1e-8
    h32 = gpu_handle(prob, local_solver="ic0", fill_level=1, krylov="gmres", precision="fp32")
    _, info32 = gpu_solve(h32, prob.b)
    assert info32.converged and abs(info32.iters - io.iters) <= 1
    # the single-reduce orthogonalisation still converges to the true residual
    h1 = gpu_handle(prob, local_solver="ic0", fill_level=1, krylov="gmres", gmres_orth="single")
    _, info1 = gpu_solve(h1, prob.b)
    assert info1.converged and info1.true_relres <= 1e-8 and info1.iters >= io.iters - 1


def test_fp32_pcg_iteration_inflation_and_fp64_residual():
    prob = P.poisson_problem(16, 4)
    h64 = gpu_handle(prob, local_solver="ic0")
    h32 = gpu_handle(prob, local_solver="ic0", precision="fp32")
    _, i64 = gpu_solve(h64, prob.b)
    x32, i32 = gpu_solve(h32, prob.b)
    assert i32.converged and i32.true_relres <= 1e-8
    assert i32.iters <= i64.iters + 2


def test_solve_host_matches_device_solve():
    prob = P.poisson_problem(12, 4)
    h = gpu_handle(prob, local_solver="ic0")
    xd, infod = gpu_solve(h, prob.b)
    xh = np.zeros(prob.A.n)
    infoh = h.solve_host(np.ascontiguousarray(prob.b), xh)
    assert infoh.iters == infod.iters and np.array_equal(xh, xd)
    # from the zero initial guess: x_host is only written (its contents are ignored),
    # twice in a row with the same result
    for _ in range(2):
        xz = np.full(prob.A.n, 7.0)
        infoz = h.solve_host(np.ascontiguousarray(prob.b), xz, zero_guess=True)
        assert infoz.iters == infod.iters and np.array_equal(xz, xd)


def test_solve_host_zero_guess_on_a_batch():
    """The zero-guess host solve on a batched handle equals the batched device solve."""
    from paper_2304_04876_b300 import gdsw as G
    import torch
    mem = [P.poisson_problem(8, 4), P.poisson_problem(12, 4)]
    h = G.Handle.batch([(m.A, m.part, None) for m in mem], local_solver="ic0")
    b = np.concatenate([m.b for m in mem])
    bt = torch.tensor(b, device="cuda")
    xt = torch.zeros_like(bt)
    h.solve_batch(bt, xt)
    xz = np.full(b.size, -1.0)
    info = h.solve_host(np.ascontiguousarray(b), xz, zero_guess=True)
    assert info.converged and np.array_equal(xz, xt.cpu().numpy())


def test_host_made_faults():
    from paper_2304_04876_b300 import gdsw as G
    # indefinite local matrix: IC(0) sweep breaks down (negative diagonal)
    prob = P.poisson_problem(8, 4)
    A = prob.A.to_scipy().tolil()
    A[10, 10] = -6.0
    bad = P.CSR.from_scipy(A.tocsr())
    with pytest.raises(G.GdswError) as e:
        G.Handle(bad, prob.part, None, local_solver="ic0")
    assert e.value.status == G.ERR_BREAKDOWN
    # NaN in the right-hand side: reported as not converged, no hang
    h = gpu_handle(prob, local_solver="ic0")
    b = prob.b.copy()
    b[3] = np.nan
    x, info = gpu_solve(h, b, raise_on_nonconvergence=False)
    assert not info.converged


@pytest.mark.parametrize("make,opts", [
    (lambda: P.poisson_problem(12, 4), dict(local_solver="ic0")),
    (lambda: P.elasticity_problem(6, 2), dict(local_solver="ilu0", krylov="gmres", restart=30)),
    (lambda: P.poisson_problem(13, 4), dict(local_solver="ilu0", fill_level=1)),
], ids=["poisson12_ic0", "elast6_ilu0_gmres", "ragged13_ilu1"])
def test_fp16_factor_storage(make, opts):
    """Factors stored in FP16 and applied in FP32: the apply stays within FP16's
    rounding of the FP64 one and the FP64 Krylov solve still reaches 1e-8."""
    prob = make()
    local = opts["local_solver"]
    M = oracle_for(prob, local=local, fill_level=opts.get("fill_level", 0))
    h16 = gpu_handle(prob, precision="fp16", **opts)
    h64 = gpu_handle(prob, **opts)
    r = np.random.default_rng(0).uniform(-1, 1, prob.A.n)
    assert relerr(gpu_apply(h16, r), M.apply(r)) <= 5e-3
    _, i64 = gpu_solve(h64, prob.b)
    x, i16 = gpu_solve(h16, prob.b)
    assert i16.converged and i16.true_relres <= 1e-8
    assert i16.iters <= i64.iters + 5


def test_handles_with_different_shared_memory_needs_interleave():
    """Kernel launch limits are per kernel, not per handle: a handle created later with
    smaller needs must not break an earlier one with larger needs."""
    big = P.poisson_problem(20, 20)            # one subdomain of 8000 unknowns
    small = P.poisson_problem(8, 4)
    Mb = oracle_for(big, local="ic0")
    hb = gpu_handle(big, local_solver="ic0")
    hs = gpu_handle(small, local_solver="ic0")
    r = np.random.default_rng(1).uniform(-1, 1, big.A.n)
    assert relerr(gpu_apply(hb, r), Mb.apply(r)) <= 1e-10
    hs2 = gpu_handle(small, local_solver="ic0", precision="fp32")
    assert relerr(gpu_apply(hb, r), Mb.apply(r)) <= 1e-10
    for h in (hb, hs, hs2):
        h.close()


def _diffusion_k(seed):
    k = 10 ** np.random.default_rng(seed).uniform(-2, 2, (10, 10, 10))
    A = P.diffusion7(k)
    cuts = P.uniform_cuts(10, 4)
    part = P.Partition(10, 10, 10, 1, [cuts, cuts, cuts])
    return P.Problem("diff10", A, part, np.ones((A.n, 1)), P.rhs_uniform(A.n, 1))


@pytest.mark.parametrize("opts", [dict(local_solver="ic0"), dict(local_solver="exact", coarse="rgdsw"),
                                  dict(local_solver="ilu0", precision="fp32")])
def test_refactor_equals_fresh_setup(opts):
    """New values on the same pattern: the numeric phase alone gives what a fresh
    setup gives, bit for bit; a matrix that breaks the factorization leaves the
    handle as it was."""
    p1, p2 = _diffusion_k(7), _diffusion_k(8)
    assert np.array_equal(p1.A.colind, p2.A.colind) and np.array_equal(p1.A.rowptr, p2.A.rowptr)
    h = gpu_handle(p1, **opts)
    r = np.random.default_rng(3).uniform(-1, 1, p1.A.n)
    z1 = gpu_apply(h, r)
    h.refactor(p2.A.val)
    fresh = gpu_handle(p2, **opts)
    z2 = gpu_apply(h, r)
    assert np.array_equal(z2, gpu_apply(fresh, r))
    assert h.stats()["n0"] == fresh.stats()["n0"]
    if opts.get("precision", "fp64") == "fp64":
        local = {"local_solver": "local"}
        M = oracle_for(p2, **{local.get(k, k): v for k, v in opts.items()})
        assert relerr(z2, M.apply(r)) <= TOL_FP64
    x, info = gpu_solve(h, p2.b)
    assert info.converged and info.true_relres <= 1e-8
    # an indefinite matrix (negated) fails in the numeric phase; the handle keeps the p2 factors
    from paper_2304_04876_b300 import gdsw as G
    with pytest.raises(G.GdswError):
        h.refactor(-p2.A.val)
    assert np.array_equal(gpu_apply(h, r), z2)
    assert not np.array_equal(z1, z2)
    h.close()
    fresh.close()


@pytest.mark.parametrize("make,opts", [
    (lambda: P.config_problem(1), dict(local_solver="exact")),
    (lambda: P.poisson_problem(12, 4), dict(local_solver="ic0")),
    (lambda: P.poisson_problem(12, 4), dict(local_solver="ic0", precision="fp16", trsv="jacobi")),
    (lambda: P.elasticity_problem(6, 2), dict(local_solver="ilu0", krylov="gmres")),
    (lambda: P.elasticity_problem(6, 2), dict(local_solver="ilu0", coarse="rgdsw", precision="fp32")),
])
def test_bytes_required_bounds_the_handle(make, opts):
    """The host-only footprint estimate is an upper bound of what setup allocates,
    and a tight one (no null-space column is dropped for these problems except
    the elasticity edges, rank 5 of 6)."""
    from paper_2304_04876_b300 import gdsw as G
    prob = make()
    Z = None if prob.Z is None or prob.Z.shape[1] == 1 and np.all(prob.Z == 1) else prob.Z
    resident, scratch = G.bytes_required(prob.A, prob.part, Z, **opts)
    h = gpu_handle(prob, **opts)
    held = h.stats()["device_bytes"]
    h.close()
    assert held <= resident <= 1.15 * held + (1 << 20), (held, resident)
    assert scratch > 0


def test_bounded_wait_that_runs_out_reports_timeout(monkeypatch):
    """A local-solve wait that can never complete (GDSW_TEST_STALL=1 withholds one
    level record's copy, so its barrier is a flag that nothing sets) runs out after
    its budget (here about 10 ms): the kernel records it, lets the copies it did issue
    land and returns, and the host reports GDSW_ERR_TIMEOUT.  The context stays usable:
    a handle without the stall computes normally afterwards."""
    from paper_2304_04876_b300 import gdsw as G
    import torch
    prob = P.poisson_problem(12, 4)
    monkeypatch.setenv("GDSW_TEST_STALL", "1")
    h = gpu_handle(prob, local_solver="ic0", wait_budget_cycles=20_000_000)
    monkeypatch.delenv("GDSW_TEST_STALL")
    if h.stats()["local_stages"] == 0:
        pytest.skip("the pipelined local solve is not used for this problem")
    r = np.random.default_rng(0).uniform(-1, 1, prob.A.n)
    rt = torch.tensor(r, dtype=torch.float64, device="cuda")
    zt = torch.empty_like(rt)
    with pytest.raises(G.GdswError) as e:
        h.apply_timed(rt, zt)
    assert e.value.status == G.ERR_TIMEOUT
    h.close()
    M = oracle_for(prob, local="ic0")
    h2 = gpu_handle(prob, local_solver="ic0")
    assert relerr(gpu_apply(h2, r), M.apply(r)) <= TOL_FP64


def test_setup_from_device_csr():
    """A matrix given in device memory (gdsw_csr.mem = GDSW_MEM_DEVICE) sets up the same
    preconditioner as the same matrix in host memory: bitwise equal applies, equal
    footprint estimates and multifrontal plans, and a batch member given on the device."""
    import types
    import torch
    from paper_2304_04876_b300 import gdsw as G
    prob = P.elasticity_problem(6, 2)
    dA = types.SimpleNamespace(n=prob.A.n,
                               rowptr=torch.tensor(prob.A.rowptr, dtype=torch.int32, device="cuda"),
                               colind=torch.tensor(prob.A.colind, dtype=torch.int32, device="cuda"),
                               val=torch.tensor(prob.A.val, dtype=torch.float64, device="cuda"))
    r = np.random.default_rng(0).uniform(-1, 1, prob.A.n)
    for opts in (dict(local_solver="ilu0"), dict(local_solver="exact")):
        hh = G.Handle(prob.A, prob.part, prob.Z, **opts)
        hd = G.Handle(dA, prob.part, prob.Z, **opts)
        assert np.array_equal(gpu_apply(hh, r), gpu_apply(hd, r))
        assert G.bytes_required(prob.A, prob.part, prob.Z, **opts) == G.bytes_required(dA, prob.part, prob.Z, **opts)
        hh.close(); hd.close()
    ph = G.mf_plan(prob.A, prob.part, 3, local_solver="exact")
    pd = G.mf_plan(dA, prob.part, 3, local_solver="exact")
    assert all(np.array_equal(ph[k], pd[k]) for k in ph)
    small = P.elasticity_problem(4, 2)      # batch members share the unknowns per node
    bh = G.Handle.batch([(prob.A, prob.part, prob.Z), (small.A, small.part, small.Z)], local_solver="ic0")
    bd = G.Handle.batch([(dA, prob.part, prob.Z), (small.A, small.part, small.Z)], local_solver="ic0")
    rb = np.random.default_rng(1).uniform(-1, 1, prob.A.n + small.A.n)
    assert np.array_equal(gpu_apply(bh, rb), gpu_apply(bd, rb))
