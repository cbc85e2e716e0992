"""Seeded random small problems against the oracle (Eq. 1 apply, FP64, 1e-10 relative):
non-cubic grids, different block sizes per axis (ragged last blocks), coefficient jumps
of four orders of magnitude, overlap 0-2, GDSW or reduced GDSW, and every local solver
(exact by dense inverse or multifrontal, IC(k)/ILU(k) level-scheduled or by Jacobi
sweeps).  Each case is drawn from its seed alone, so a failure names a reproducible
problem."""
import numpy as np
import pytest

from paper_2304_04876_b300 import problems as P
from tests.gpu_util import gpu_apply, gpu_handle, oracle_for, relerr

pytestmark = pytest.mark.gpu

SEEDS = list(range(40))


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2304_04876_b300 import build
    build.build()
    assert torch.cuda.is_available()


def _case(seed):
    rng = np.random.default_rng(1000 + seed)
    nx, ny, nz = (int(v) for v in rng.integers(5, 12, 3))
    cuts = []
    for n in (nx, ny, nz):
        s = int(rng.integers(2, 6))
        cuts.append(P.uniform_cuts(n, s))
    if not any(cuts):                       # at least two subdomains
        cuts[0] = P.uniform_cuts(nx, 3)
    k = 10 ** rng.uniform(-2, 2, (nz, ny, nx))
    A = P.diffusion7(k)
    part = P.Partition(nx, ny, nz, 1, cuts)
    prob = P.Problem(f"rand{seed}", A, part, np.ones((A.n, 1)), P.rhs_uniform(A.n, seed))
    local = ["exact", "exact_mf", "ic0", "ilu0"][seed % 4]
    opts = dict(overlap=int(rng.integers(0, 3)))
    # reduced GDSW needs a vertex in every component's closure: cuts on every axis
    if all(cuts) and rng.random() < 0.5:
        opts["coarse"] = "rgdsw"
    if local in ("ic0", "ilu0"):
        opts["fill_level"] = int(rng.integers(0, 2))
        if rng.random() < 0.3:
            opts["trsv"] = "jacobi"
    return prob, local, opts


@pytest.mark.parametrize("seed", SEEDS)
def test_random_problem_apply(seed, monkeypatch):
    prob, local, opts = _case(seed)
    if local == "exact_mf":
        monkeypatch.setenv("GDSW_EXACT_DENSE_MAX", "0")
        local = "exact"
    M = oracle_for(prob, local=local, **opts)
    h = gpu_handle(prob, local_solver=local, **opts)
    assert h.stats()["n0"] == M.n0
    for rs in range(2):
        r = np.random.default_rng(rs).uniform(-1, 1, prob.A.n)
        assert relerr(gpu_apply(h, r), M.apply(r)) <= 1e-10, (seed, local, opts)
    h.close()


@pytest.mark.parametrize("seed", SEEDS[:12])
def test_random_problem_pcg(seed, monkeypatch):
    """PCG on the same random problems: the oracle's iteration count +-1 and the FP64
    true residual."""
    from oracle import gdsw_oracle as O
    from tests.gpu_util import gpu_solve
    prob, local, opts = _case(seed)
    if local == "exact_mf":
        monkeypatch.setenv("GDSW_EXACT_DENSE_MAX", "0")
        local = "exact"
    M = oracle_for(prob, local=local, **opts)
    _, io = O.pcg(M.spmv, M.apply, prob.b, tol=1e-8)
    h = gpu_handle(prob, local_solver=local, **opts)
    x, info = gpu_solve(h, prob.b)
    assert info.converged and info.true_relres <= 1e-8
    assert abs(info.iters - io.iters) <= 1, (seed, info.iters, io.iters)
    h.close()


ELAST_SEEDS = list(range(8))


@pytest.mark.parametrize("seed", ELAST_SEEDS)
def test_random_elasticity_apply(seed, monkeypatch):
    """Q1 elasticity (three unknowns per node, rigid-body null space) with random element
    counts and block sizes, ragged last blocks included, every local solver."""
    rng = np.random.default_rng(2000 + seed)
    ne = int(rng.integers(4, 8))
    se = int(rng.integers(2, 4))
    prob = P.elasticity_problem(ne, se)
    local = ["exact", "exact_mf", "ilu0", "ic0"][seed % 4]
    opts = dict(overlap=int(rng.integers(0, 2)))
    if rng.random() < 0.5:
        opts["coarse"] = "rgdsw"
    if local in ("ic0", "ilu0"):
        opts["fill_level"] = int(rng.integers(0, 2))
    if local == "exact_mf":
        monkeypatch.setenv("GDSW_EXACT_DENSE_MAX", "0")
        local = "exact"
    M = oracle_for(prob, local=local, **opts)
    h = gpu_handle(prob, local_solver=local, **opts)
    assert h.stats()["n0"] == M.n0
    r = np.random.default_rng(seed).uniform(-1, 1, prob.A.n)
    assert relerr(gpu_apply(h, r), M.apply(r)) <= 1e-10, (seed, ne, se, local, opts)
    h.close()


@pytest.mark.parametrize("seed", SEEDS[12:20])
def test_random_problem_gmres(seed, monkeypatch):
    """GMRES on the random problems, with a random restart length: the oracle's GMRES
    iteration count within +-2 (short restarts amplify rounding differences between
    the device's CGS2 and the oracle's MGS) and the FP64 true residual."""
    from oracle import gdsw_oracle as O
    from tests.gpu_util import gpu_solve
    prob, local, opts = _case(seed)
    if local == "exact_mf":
        monkeypatch.setenv("GDSW_EXACT_DENSE_MAX", "0")
        local = "exact"
    restart = int(np.random.default_rng(3000 + seed).integers(5, 31))
    M = oracle_for(prob, local=local, **opts)
    _, io = O.gmres(M.spmv, M.apply, prob.b, tol=1e-8, restart=restart)
    h = gpu_handle(prob, local_solver=local, krylov="gmres", restart=restart, **opts)
    x, info = gpu_solve(h, prob.b)
    assert info.converged and info.true_relres <= 1e-8
    assert abs(info.iters - io.iters) <= 2, (seed, restart, info.iters, io.iters)
    h.close()


@pytest.mark.parametrize("seed", SEEDS[20:28])
def test_random_problem_fp32_preconditioner(seed, monkeypatch):
    """The FP32 preconditioner on the random problems: the apply within 2e-5 of the
    oracle's FP64 one (factors, Phi and the scatter rounded to FP32)."""
    prob, local, opts = _case(seed)
    if local == "exact_mf":
        monkeypatch.setenv("GDSW_EXACT_DENSE_MAX", "0")
        local = "exact"
    M = oracle_for(prob, local=local, **opts)
    h = gpu_handle(prob, local_solver=local, precision="fp32", **opts)
    r = np.random.default_rng(seed).uniform(-1, 1, prob.A.n)
    assert relerr(gpu_apply(h, r), M.apply(r)) <= 2e-5, (seed, local, opts)
    h.close()
