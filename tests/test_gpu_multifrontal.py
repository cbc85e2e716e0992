"""The multifrontal exact local solver (nested dissection, supernodal fronts, partitioned
inverse of each diagonal block) against the oracle's exact local solves (Sec. V-B1:
exact Cholesky of every A_s).  The path is taken for subdomains above the dense-inverse
size; GDSW_EXACT_DENSE_MAX=0 forces it on the small cases here.  FP64 apply within
1e-10 relative; PCG iterations within +-1 of the oracle; true residual <= 1e-8."""
import numpy as np
import pytest

from paper_2304_04876_b300 import problems as P
from tests.gpu_util import gpu_apply, gpu_handle, gpu_solve, oracle_for, relerr

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2304_04876_b300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.fixture(autouse=True)
def _force_multifrontal(monkeypatch):
    monkeypatch.setenv("GDSW_EXACT_DENSE_MAX", "0")


def _diffusion():
    k = 10 ** np.random.default_rng(7).uniform(-2, 2, (10, 10, 10))
    A = P.diffusion7(k)
    cuts = P.uniform_cuts(10, 4)
    part = P.Partition(10, 10, 10, 1, [cuts, cuts, cuts])
    return P.Problem("diff10", A, part, np.ones((A.n, 1)), P.rhs_uniform(A.n, 1))


CASES = [
    ("cfg1", lambda: P.config_problem(1), {}, None),
    ("poisson12", lambda: P.poisson_problem(12, 4), {}, None),
    ("ragged13", lambda: P.poisson_problem(13, 4, seed=3), {}, None),
    ("single_subdomain", lambda: P.poisson_problem(6, 6), {}, None),
    ("diffusion10", _diffusion, {}, None),
    ("overlap2", lambda: P.poisson_problem(12, 4), dict(overlap=2), None),
    ("no_overlap", lambda: P.poisson_problem(12, 4), dict(overlap=0), None),
    ("rgdsw", lambda: P.poisson_problem(12, 4), dict(coarse="rgdsw"), None),
    ("elast4", lambda: P.elasticity_problem(4, 2), {}, None),
    ("elast_ragged7", lambda: P.elasticity_problem(7, 3), {}, None),
    ("leaf1", lambda: P.poisson_problem(12, 4), {}, "1"),
    ("leaf4_elast", lambda: P.elasticity_problem(6, 2), {}, "4"),
    ("leaf200_one_front", lambda: P.poisson_problem(12, 4), {}, "200"),
]


@pytest.mark.parametrize("name,make,opts,leaf", CASES, ids=[c[0] for c in CASES])
def test_apply_matches_oracle(name, make, opts, leaf, monkeypatch):
    if leaf is not None:
        monkeypatch.setenv("GDSW_MF_LEAF", leaf)
    prob = make()
    M = oracle_for(prob, local="exact", **opts)
    h = gpu_handle(prob, local_solver="exact", **opts)
    st = h.stats()
    dense = sum(len(o) ** 2 for o in M.omega)
    # the factor panels replace the dense inverses; a lone leaf front is a dense triangle
    assert 0 < st["dense_local"] <= dense
    for seed in range(3):
        r = np.random.default_rng(seed).uniform(-1, 1, prob.A.n)
        assert relerr(gpu_apply(h, r), M.apply(r)) <= TOL_FP64, name
    h.close()


def test_fp32_close_to_fp64_and_deterministic():
    prob = P.poisson_problem(12, 4)
    M = oracle_for(prob, local="exact")
    h = gpu_handle(prob, local_solver="exact", precision="fp32")
    r = np.random.default_rng(0).uniform(-1, 1, prob.A.n)
    z = gpu_apply(h, r)
    assert relerr(z, M.apply(r)) <= 2e-5
    for _ in range(5):
        assert np.array_equal(gpu_apply(h, r), z)


def test_local_solve_exact_without_overlap_or_coarse():
    """With no overlap and no coarse space M^-1 is block diagonal: on each block the
    apply is A_ss^-1 r_s, so A_ss z_s = r_s to rounding (a property that does not need
    the oracle)."""
    prob = P.poisson_problem(16, 8)
    h = gpu_handle(prob, local_solver="exact", overlap=0, coarse="none")
    r = np.random.default_rng(2).uniform(-1, 1, prob.A.n)
    z = gpu_apply(h, r)
    A = prob.A.to_scipy().tocsr()
    # blocks of the partition: nodes with the same (bx, by, bz)
    n = 16
    cuts = prob.part.cuts[0]
    blk = np.searchsorted(np.asarray(cuts), np.arange(n), side="left")
    idx = np.arange(prob.A.n)
    x, y, zc = idx % n, (idx // n) % n, idx // (n * n)
    nbk = len(cuts) + 1
    key = blk[x] + nbk * (blk[y] + nbk * blk[zc])
    for b in np.unique(key)[:4]:
        rows = np.where(key == b)[0]
        Ab = A[rows][:, rows]
        res = np.linalg.norm(Ab @ z[rows] - r[rows]) / np.linalg.norm(r[rows])
        assert res <= 1e-12, (b, res)


PCG_CASES = [
    ("poisson12", lambda: P.poisson_problem(12, 4), {}),
    ("elast6", lambda: P.elasticity_problem(6, 2), {}),
    ("rgdsw_elast6", lambda: P.elasticity_problem(6, 2), dict(coarse="rgdsw")),
]


@pytest.mark.parametrize("name,make,opts", PCG_CASES, ids=[c[0] for c in PCG_CASES])
def test_pcg_matches_oracle(name, make, opts):
    from oracle import gdsw_oracle as O
    prob = make()
    M = oracle_for(prob, local="exact", **opts)
    _, io = O.pcg(M.spmv, M.apply, prob.b, tol=1e-8)
    for prec in ("fp64", "fp32"):
        h = gpu_handle(prob, local_solver="exact", precision=prec, **opts)
        x, info = gpu_solve(h, prob.b)
        assert info.converged and info.true_relres <= 1e-8
        assert abs(info.iters - io.iters) <= 1, (prec, info.iters, io.iters)


def test_default_threshold_takes_the_multifrontal_path(monkeypatch):
    """Subdomains of 13^3 = 2197 unknowns are above the dense-inverse size, so the
    default options factor them by nested dissection; the apply still matches the
    oracle's exact solves."""
    monkeypatch.delenv("GDSW_EXACT_DENSE_MAX")
    prob = P.poisson_problem(24, 12)
    M = oracle_for(prob, local="exact")
    h = gpu_handle(prob, local_solver="exact")
    assert h.stats()["dense_local"] < sum(len(o) ** 2 for o in M.omega) // 4
    r = np.random.default_rng(4).uniform(-1, 1, prob.A.n)
    assert relerr(gpu_apply(h, r), M.apply(r)) <= TOL_FP64


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_bytes_required_bounds_the_handle(prec):
    """The host-only footprint estimate covers the multifrontal factor (panels, solve
    lists, update arena) and stays tight."""
    from paper_2304_04876_b300 import gdsw as G
    prob = P.elasticity_problem(6, 2)
    opts = dict(local_solver="exact", precision=prec)
    resident, scratch = G.bytes_required(prob.A, prob.part, prob.Z, **opts)
    h = gpu_handle(prob, **opts)
    held = h.stats()["device_bytes"]
    assert h.stats()["mf_supernodes"] > 0
    h.close()
    assert held <= resident <= 1.15 * held + (1 << 20), (held, resident)
    assert scratch > 0


def test_fp16_panels():
    """FP16 precision stores the exact factor panels in half precision (computed in
    FP32): the apply is the exact solve to about the panels' rounding, and PCG still
    reaches the FP64 true residual within a few more iterations than the oracle's."""
    from oracle import gdsw_oracle as O
    prob = P.poisson_problem(12, 4)
    M = oracle_for(prob, local="exact")
    h = gpu_handle(prob, local_solver="exact", precision="fp16")
    r = np.random.default_rng(0).uniform(-1, 1, prob.A.n)
    assert relerr(gpu_apply(h, r), M.apply(r)) <= 1e-2
    h32 = gpu_handle(prob, local_solver="exact", precision="fp32")
    assert h.stats()["device_bytes"] < h32.stats()["device_bytes"]
    _, io = O.pcg(M.spmv, M.apply, prob.b, tol=1e-8)
    _, info = gpu_solve(h, prob.b)
    assert info.converged and info.true_relres <= 1e-8 and io.iters - 1 <= info.iters <= io.iters + 3


def _diffusion_k(seed):
    k = 10 ** np.random.default_rng(seed).uniform(-2, 2, (10, 10, 10))
    A = P.diffusion7(k)
    cuts = P.uniform_cuts(10, 4)
    part = P.Partition(10, 10, 10, 1, [cuts, cuts, cuts])
    return P.Problem("diff10", A, part, np.ones((A.n, 1)), P.rhs_uniform(A.n, 1))


def test_refactor_equals_fresh_setup():
    """New values on the same pattern refactor the multifrontal panels; the result is
    a fresh setup's, bit for bit, and the oracle's to 1e-10; an indefinite matrix
    fails in the numeric phase and leaves the previous factors in place."""
    from paper_2304_04876_b300 import gdsw as G
    p1, p2 = _diffusion_k(7), _diffusion_k(8)
    h = gpu_handle(p1, local_solver="exact")
    assert h.stats()["mf_supernodes"] > 0
    r = np.random.default_rng(3).uniform(-1, 1, p1.A.n)
    z1 = gpu_apply(h, r)
    h.refactor(p2.A.val)
    z2 = gpu_apply(h, r)
    assert np.array_equal(z2, gpu_apply(gpu_handle(p2, local_solver="exact"), r))
    assert relerr(z2, oracle_for(p2, local="exact").apply(r)) <= TOL_FP64
    with pytest.raises(G.GdswError):
        h.refactor(-p2.A.val)
    assert np.array_equal(gpu_apply(h, r), z2) and not np.array_equal(z1, z2)


def test_batched_handle():
    """Independent problems in one batched handle: every member's exact local solves
    go through the multifrontal path and match that member's oracle."""
    from paper_2304_04876_b300 import gdsw as G
    mem = P.diffusion_batch(4, seed=5, nmin=7, nmax=12, smin=3, smax=6)
    h = G.Handle.batch([(m.A, m.part, None) for m in mem], local_solver="exact")
    assert h.stats()["mf_supernodes"] > 0
    offs = np.cumsum([0] + [m.A.n for m in mem])
    r = np.random.default_rng(1).uniform(-1, 1, offs[-1])
    z = gpu_apply(h, r)
    for i, m in enumerate(mem):
        zi = oracle_for(m, local="exact").apply(r[offs[i]:offs[i + 1]])
        assert relerr(z[offs[i]:offs[i + 1]], zi) <= TOL_FP64, i


def test_gmres_with_multifrontal_local_solves():
    """GMRES(30) with the exact multifrontal local solves (the elasticity setting of
    config 3 at small size) takes the oracle's GMRES iteration count, +-1."""
    from oracle import gdsw_oracle as O
    prob = P.elasticity_problem(6, 2)
    M = oracle_for(prob, local="exact")
    _, io = O.gmres(M.spmv, M.apply, prob.b, tol=1e-8, restart=30)
    h = gpu_handle(prob, local_solver="exact", krylov="gmres", restart=30, precision="fp32")
    assert h.stats()["mf_supernodes"] > 0
    _, info = gpu_solve(h, prob.b)
    assert info.converged and info.true_relres <= 1e-8
    assert abs(info.iters - io.iters) <= 1, (info.iters, io.iters)
