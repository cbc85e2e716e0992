"""Pins of the oracle's Krylov solvers against independent library implementations and
closed-form behaviour."""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import gdsw_oracle as O
from paper_2304_04876_b300 import problems as P


def test_pcg_matches_scipy_cg():
    A = P.poisson7(10).to_scipy()
    b = P.rhs_uniform(A.shape[0], 3)
    d = A.diagonal()
    count = [0]
    xs, info = spla.cg(A, b, rtol=1e-10, M=sp.diags(1 / d), callback=lambda xk: count.__setitem__(0, count[0] + 1))
    assert info == 0
    x, sinfo = O.pcg(lambda v: A @ v, lambda v: v / d, b, tol=1e-10)
    assert sinfo.converged and sinfo.relres <= 1e-10
    assert abs(sinfo.iters - count[0]) <= 1
    assert np.allclose(x, xs, atol=1e-8 * np.abs(xs).max())


def test_pcg_exact_preconditioner_one_step_and_zero_rhs():
    A = P.poisson7(5).to_scipy()
    Ad = A.toarray()
    b = P.rhs_uniform(A.shape[0], 1)
    x, info = O.pcg(lambda v: A @ v, lambda v: np.linalg.solve(Ad, v), b)
    assert info.iters == 1 and np.allclose(A @ x, b)
    x, info = O.pcg(lambda v: A @ v, lambda v: v, np.zeros(A.shape[0]))
    assert info.iters == 0 and not x.any()
    # warm start at the solution: zero iterations
    xs = np.linalg.solve(Ad, b)
    x, info = O.pcg(lambda v: A @ v, lambda v: v, b, x0=xs)
    assert info.iters == 0


def test_pcg_flexible_same_as_standard_for_fixed_spd_preconditioner():
    A = P.poisson7(8).to_scipy()
    b = P.rhs_uniform(A.shape[0], 2)
    d = A.diagonal()
    _, i1 = O.pcg(lambda v: A @ v, lambda v: v / d, b)
    _, i2 = O.pcg(lambda v: A @ v, lambda v: v / d, b, flexible=True)
    assert abs(i1.iters - i2.iters) <= 1


def test_gmres_matches_direct_solve_nonsymmetric():
    rng = np.random.default_rng(0)
    n = 60
    A = sp.csr_matrix(np.diag(4 + rng.uniform(0, 1, n)) + np.diag(rng.uniform(-1, 1, n - 1), 1)
                      + np.diag(rng.uniform(-1.5, 0, n - 1), -1))
    b = rng.standard_normal(n)
    d = A.diagonal()
    x, info = O.gmres(lambda v: A @ v, lambda v: v / d, b, restart=10, tol=1e-10)
    assert info.converged and info.relres <= 1e-10
    assert np.allclose(x, spla.spsolve(A.tocsc(), b), atol=1e-8)
    # full GMRES terminates in at most n steps; an exact preconditioner in one
    x, info = O.gmres(lambda v: A @ v, lambda v: v, b, restart=n, tol=1e-12)
    assert info.iters <= n
    Ad = A.toarray()
    x, info = O.gmres(lambda v: A @ v, lambda v: np.linalg.solve(Ad, v), b)
    assert info.iters == 1


def test_gmres_with_gdsw_agrees_with_pcg_solution():
    prob = P.poisson_problem(8, 4)
    M = O.GDSW(prob.A, prob.part, prob.Z, local=O.ILU0)
    x1, i1 = O.gmres(M.spmv, M.apply, prob.b)
    x2, i2 = O.pcg(M.spmv, M.apply, prob.b)
    assert i1.converged and i2.converged
    assert np.allclose(x1, x2, atol=1e-7 * np.abs(x2).max())
