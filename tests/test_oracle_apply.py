"""Pins of the oracle's preconditioner apply (Eq. 1) by brute force on tiny grids,
symmetry / positive definiteness, and the special cases that reduce to textbook
operators."""
import numpy as np
import pytest

from oracle import gdsw_oracle as O
from paper_2304_04876_b300 import problems as P


def _brute_force_M(M: O.GDSW, Ad: np.ndarray) -> np.ndarray:
    """Dense M^-1 from its definition with numpy inverses of every block."""
    n = Ad.shape[0]
    Minv = np.zeros((n, n))
    for dofs in M.omega:
        Minv[np.ix_(dofs, dofs)] += np.linalg.inv(Ad[np.ix_(dofs, dofs)])
    if M.n0:
        Phi = M.coarse.Phi.toarray()
        Minv += Phi @ np.linalg.inv(Phi.T @ Ad @ Phi) @ Phi.T
    return Minv


CASES = [
    ("poisson8_s4", lambda: P.poisson_problem(8, 4)),
    ("poisson6_s2", lambda: P.poisson_problem(6, 2)),
    ("poisson7_s3", lambda: P.poisson_problem(7, 3)),        # ragged last block
    ("elasticity4_s2", lambda: P.elasticity_problem(4, 2)),
]


@pytest.mark.parametrize("name,make", CASES)
def test_apply_equals_brute_force_inverse(name, make):
    prob = make()
    M = O.GDSW(prob.A, prob.part, prob.Z, local=O.EXACT)
    Ad = prob.A.to_scipy().toarray()
    Mb = _brute_force_M(M, Ad)
    rng = np.random.default_rng(0)
    R = rng.standard_normal((prob.A.n, 4))
    Z = np.column_stack([M.apply(R[:, j]) for j in range(R.shape[1])])
    assert np.abs(Z - Mb @ R).max() <= 1e-12 * np.abs(Mb @ R).max()
    # M^-1 symmetric positive definite, so M^-1 A has real positive spectrum
    assert np.abs(Mb - Mb.T).max() <= 1e-12 * np.abs(Mb).max()
    assert np.linalg.eigvalsh(0.5 * (Mb + Mb.T)).min() > 0
    ev = np.linalg.eigvals(Mb @ Ad)
    assert np.abs(ev.imag).max() < 1e-8 and ev.real.min() > 0


def test_single_subdomain_is_exact_inverse():
    """n_p = 1: no interface, no coarse space, M^-1 = A^-1 and PCG converges in one step."""
    prob = P.poisson_problem(6, 6)
    M = O.GDSW(prob.A, prob.part, prob.Z, local=O.EXACT)
    assert M.n0 == 0 and len(M.omega) == 1
    Ad = prob.A.to_scipy().toarray()
    r = np.random.default_rng(0).standard_normal(prob.A.n)
    assert np.allclose(M.apply(r), np.linalg.solve(Ad, r), atol=1e-13)
    x, info = O.pcg(M.spmv, M.apply, prob.b, tol=1e-8)
    assert info.iters == 1 and info.converged


def test_one_level_is_additive_schwarz():
    prob = P.poisson_problem(8, 4)
    M = O.GDSW(prob.A, prob.part, prob.Z, local=O.EXACT, coarse=False)
    Ad = prob.A.to_scipy().toarray()
    r = np.random.default_rng(1).standard_normal(prob.A.n)
    ref = np.zeros(prob.A.n)
    for dofs in M.omega:
        ref[dofs] += np.linalg.solve(Ad[np.ix_(dofs, dofs)], r[dofs])
    assert np.allclose(M.apply(r), ref, atol=1e-13)


def test_iterations_flat_under_weak_scaling():
    """GDSW keeps PCG counts roughly flat as subdomains are added at fixed H/h (Sec. III);
    the one-level method does not."""
    its2, its1 = [], []
    for nb in (2, 3, 4):
        prob = P.poisson_problem(4 * nb, 4)
        M2 = O.GDSW(prob.A, prob.part, prob.Z, local=O.EXACT)
        M1 = O.GDSW(prob.A, prob.part, prob.Z, local=O.EXACT, coarse=False)
        its2.append(O.pcg(M2.spmv, M2.apply, prob.b)[1].iters)
        its1.append(O.pcg(M1.spmv, M1.apply, prob.b)[1].iters)
    # counts grow at most logarithmically with GDSW, faster without a coarse space
    assert its2[-1] <= 1.3 * its2[0]
    assert its1[-1] / its1[0] > its2[-1] / its2[0]
    assert its1[-1] > its2[-1]


def test_inexact_local_solvers_converge():
    """IC(0)/ILU(0) sweeps with level-scheduled or Jacobi triangular solves stay convergent and
    need at least as many iterations as exact local solves (Table IV ordering)."""
    prob = P.poisson_problem(12, 4)
    exact = O.GDSW(prob.A, prob.part, prob.Z, local=O.EXACT)
    it_exact = O.pcg(exact.spmv, exact.apply, prob.b)[1].iters
    for local in (O.IC0, O.ILU0):
        for trsv in (O.LEVELSCHED, O.JACOBI):
            M = O.GDSW(prob.A, prob.part, prob.Z, local=local, trsv=trsv)
            x, info = O.pcg(M.spmv, M.apply, prob.b)
            assert info.converged and info.relres <= 1e-8
            assert info.iters >= it_exact


def test_ic0_apply_matches_factor_definition():
    """The inexact local operator is D^-1/2 (L L^T)^-1 D^-1/2 with L from the sweeps."""
    prob = P.poisson_problem(8, 4)
    M = O.GDSW(prob.A, prob.part, prob.Z, local=O.IC0, sweeps_factor=3)
    _, Lm, Um, s = M.factors[2]
    L = Lm.toarray()
    r = np.random.default_rng(4).standard_normal(len(s))
    ref = s * np.linalg.solve(L.T, np.linalg.solve(L, s * r))
    assert np.allclose(M.local_solve(2, r), ref, atol=1e-13)


@pytest.mark.parametrize("name,make", [("poisson12_s4", lambda: P.poisson_problem(12, 4)),
                                       ("elasticity6_s2", lambda: P.elasticity_problem(6, 2))])
def test_rgdsw_apply_equals_brute_force_and_converges(name, make):
    prob = make()
    M = O.GDSW(prob.A, prob.part, prob.Z, local=O.EXACT, coarse_variant="rgdsw")
    Ad = prob.A.to_scipy().toarray()
    Mb = _brute_force_M(M, Ad)
    R = np.random.default_rng(0).standard_normal((prob.A.n, 2))
    Z = np.column_stack([M.apply(R[:, j]) for j in range(2)])
    assert np.abs(Z - Mb @ R).max() <= 1e-12 * np.abs(Mb @ R).max()
    assert np.linalg.eigvalsh(0.5 * (Mb + Mb.T)).min() > 0
    x, info = O.pcg(M.spmv, M.apply, prob.b)
    assert info.converged
    Mg = O.GDSW(prob.A, prob.part, prob.Z, local=O.EXACT)
    assert M.n0 < Mg.n0
