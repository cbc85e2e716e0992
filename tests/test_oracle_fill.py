"""Pins of the oracle's level-of-fill factorisations IC(k)/ILU(k) (Sec. V-B, Table I's
ILU(k)/FastILU(k)): the level-k pattern against closed forms and against the pattern of
an exact LU from LAPACK, the fixed-point sweeps against the defining property of an
incomplete factorisation on that pattern, and the preconditioner's behaviour."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import gdsw_oracle as O
from paper_2304_04876_b300 import problems as P


def _csr_parts(M):
    M = sp.csr_matrix(M)
    M.sort_indices()
    return M.indptr.astype(np.int64), M.indices.astype(np.int64), M.data.astype(float)


def _pattern_set(ptr, col):
    return {(i, int(j)) for i in range(len(ptr) - 1) for j in col[ptr[i]:ptr[i + 1]]}


def test_no_fill_for_tridiagonal_and_full_band():
    m = 10
    T = sp.diags([-1.0, 4.0, -1.0], [-1, 0, 1], shape=(m, m))
    ptr, col, _ = _csr_parts(T)
    for k in (1, 2, 5):
        fp, fc, lev = O.level_fill_pattern(ptr, col, k)
        assert _pattern_set(fp, fc) == _pattern_set(ptr, col) and not lev.any()
    B = sp.diags([1.0, 1.0, 5.0, 1.0, 1.0], [-2, -1, 0, 1, 2], shape=(m, m))     # full band: no fill either
    ptr, col, _ = _csr_parts(B)
    fp, fc, _ = O.level_fill_pattern(ptr, col, 3)
    assert _pattern_set(fp, fc) == _pattern_set(ptr, col)


def test_five_point_level_one_closed_form():
    """2D 5-point stencil on an n x n grid, natural order: eliminating node (x, y) through
    its south neighbour creates (x+1, y-1), through its west neighbour (x-1, y+1), both
    at level 1; so ILU(1) adds exactly 2 (n-1)^2 entries at offsets -(n-1) and +(n-1)."""
    n = 6
    A = P.poisson7(n, n, 1).to_scipy()
    ptr, col, _ = _csr_parts(A)
    fp, fc, lev = O.level_fill_pattern(ptr, col, 1)
    fill = _pattern_set(fp, fc) - _pattern_set(ptr, col)
    expect = set()
    for y in range(n):
        for x in range(n):
            i = x + n * y
            if x < n - 1 and y > 0:
                expect.add((i, i - n + 1))
            if x > 0 and y < n - 1:
                expect.add((i, i + n - 1))
    assert len(expect) == 2 * (n - 1) ** 2
    assert fill == expect
    assert set(lev[lev > 0]) == {1}


def test_level_patterns_nested_and_symmetric():
    A = P.poisson7(4, 3, 3).to_scipy()
    ptr, col, _ = _csr_parts(A)
    prev = _pattern_set(ptr, col)
    for k in (1, 2, 3):
        fp, fc, _ = O.level_fill_pattern(ptr, col, k)
        cur = _pattern_set(fp, fc)
        assert prev <= cur
        assert cur == {(j, i) for i, j in cur}
        prev = cur


def test_large_level_is_the_exact_lu_pattern():
    """With k >= m nothing is dropped: the pattern is that of the exact LU factors, here
    taken from LAPACK's LU of a strongly diagonally dominant matrix with random values on
    the pattern (partial pivoting then keeps the natural order)."""
    A = P.poisson7(3, 3, 3).to_scipy().tolil()
    rng = np.random.default_rng(3)
    m = A.shape[0]
    for i, j in zip(*A.nonzero()):
        A[i, j] = 100.0 if i == j else rng.uniform(0.1, 1.0)
    A = A.tocsr()
    lu, piv = sla.lu_factor(A.toarray())
    assert np.array_equal(piv, np.arange(m))
    lu_pat = {(i, j) for i in range(m) for j in range(m) if i == j or abs(lu[i, j]) > 1e-300}
    ptr, col, _ = _csr_parts(A)
    fp, fc, _ = O.level_fill_pattern(ptr, col, m)
    assert _pattern_set(fp, fc) == lu_pat


@pytest.mark.parametrize("k", [1, 2])
def test_fill_sweeps_reach_the_incomplete_factor(k):
    """Enough synchronous sweeps on the level-k pattern give the incomplete factor:
    (L U)_ij = a_ij (ILU) and (L L^T)_ij = a_ij (IC) at every position of the pattern,
    fill positions included (where a_ij = 0)."""
    A = P.poisson7(4, 3, 3).to_scipy()
    m = A.shape[0]
    ptr, col, val = _csr_parts(A)
    fp, fc, _ = O.level_fill_pattern(ptr, col, k)
    fv = O.pad_to_pattern(ptr, col, val, fp, fc)
    pat = np.zeros((m, m), dtype=bool)
    for i in range(m):
        pat[i, fc[fp[i]:fp[i + 1]]] = True
    Ad = A.toarray()
    (qp, qc, qv), s = O.ilu0_sweeps(fp, fc, fv, 80)
    F = np.zeros((m, m))
    for i in range(m):
        F[i, qc[qp[i]:qp[i + 1]]] = qv[qp[i]:qp[i + 1]]
    L = np.diag(1 / s) @ (np.tril(F, -1) + np.eye(m)) @ np.diag(s)
    U = np.diag(1 / s) @ np.triu(F) @ np.diag(1 / s)
    assert np.abs((L @ U - Ad)[pat]).max() < 1e-11
    (lp, lc, lv), s = O.ic0_sweeps(fp, fc, fv, 80)
    Lc = np.zeros((m, m))
    for i in range(m):
        Lc[i, lc[lp[i]:lp[i + 1]]] = lv[lp[i]:lp[i + 1]]
    Lc = np.diag(1 / s) @ Lc
    assert np.abs((Lc @ Lc.T - Ad)[np.tril(pat)]).max() < 1e-11
    # and more fill is a better factor: the residual A - L U off the pattern shrinks
    (qp0, qc0, qv0), s0 = O.ilu0_sweeps(ptr, col, val, 80)
    F0 = np.zeros((m, m))
    for i in range(m):
        F0[i, qc0[qp0[i]:qp0[i + 1]]] = qv0[qp0[i]:qp0[i + 1]]
    L0 = np.diag(1 / s0) @ (np.tril(F0, -1) + np.eye(m)) @ np.diag(s0)
    U0 = np.diag(1 / s0) @ np.triu(F0) @ np.diag(1 / s0)
    assert np.linalg.norm(L @ U - Ad) < np.linalg.norm(L0 @ U0 - Ad)


def test_fill_in_the_preconditioner():
    """IC(1) needs no more PCG iterations than IC(0) (the paper's Table IV/V trend), and
    with a level above the subdomain size plus enough sweeps the local solve is exact, so
    one subdomain gives M^-1 = A^-1."""
    prob = P.poisson_problem(12, 4)
    its = []
    for k in (0, 1, 2):
        M = O.GDSW(prob.A, prob.part, None, local=O.IC0, fill_level=k)
        _, info = O.pcg(M.spmv, M.apply, prob.b, tol=1e-8)
        its.append(info.iters)
    assert its[2] <= its[1] <= its[0] and its[2] < its[0]
    one = P.poisson_problem(5, 5)
    M = O.GDSW(one.A, one.part, None, local=O.ILU0, fill_level=one.A.n, sweeps_factor=60)
    r = np.random.default_rng(0).uniform(-1, 1, one.A.n)
    x = np.linalg.solve(one.A.to_scipy().toarray(), r)
    assert np.linalg.norm(M.apply(r) - x) <= 1e-10 * np.linalg.norm(x)
