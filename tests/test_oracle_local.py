"""Pins of the oracle's local solvers: fixed-point IC(0)/ILU(0) sweeps and Jacobi
triangular sweeps (Sec. V-B3), against closed forms, textbook factorisations and
finite termination."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import gdsw_oracle as O
from paper_2304_04876_b300 import problems as P


def _csr_parts(M):
    M = sp.csr_matrix(M)
    M.sort_indices()
    return M.indptr.astype(np.int64), M.indices.astype(np.int64), M.data.astype(float)


def _dense_lower(lp, lc, lv, m):
    L = np.zeros((m, m))
    for i in range(m):
        L[i, lc[lp[i]:lp[i + 1]]] = lv[lp[i]:lp[i + 1]]
    return L


def test_ic0_sweep_closed_form_3x3():
    """Synchronous sweeps on tridiag(beta, 1, gamma): after one sweep l32 = gamma and
    l33 = sqrt(1 - gamma^2); after two l32 = gamma / sqrt(1 - beta^2); after three exact."""
    beta, gamma = 0.3, -0.4
    A = np.array([[1, beta, 0], [beta, 1, gamma], [0, gamma, 1.0]])
    ptr, col, val = _csr_parts(A)
    (lp, lc, lv), s = O.ic0_sweeps(ptr, col, val, 1)
    L1 = _dense_lower(lp, lc, lv, 3)
    assert np.allclose(s, 1.0)
    assert L1[2, 1] == pytest.approx(gamma) and L1[2, 2] == pytest.approx(np.sqrt(1 - gamma ** 2))
    assert L1[1, 1] == pytest.approx(np.sqrt(1 - beta ** 2))
    (lp, lc, lv), _ = O.ic0_sweeps(ptr, col, val, 2)
    L2 = _dense_lower(lp, lc, lv, 3)
    assert L2[2, 1] == pytest.approx(gamma / np.sqrt(1 - beta ** 2))
    assert L2[2, 2] == pytest.approx(np.sqrt(1 - gamma ** 2))
    (lp, lc, lv), _ = O.ic0_sweeps(ptr, col, val, 3)
    L3 = _dense_lower(lp, lc, lv, 3)
    assert np.allclose(L3, np.linalg.cholesky(A), atol=1e-15)


def test_ic0_of_tridiagonal_is_cholesky():
    """IC(0) of a tridiagonal SPD matrix has no dropped fill, so it is the Cholesky factor."""
    m = 30
    rng = np.random.default_rng(3)
    off = rng.uniform(-1, 1, m - 1)
    A = np.diag(np.abs(np.r_[off, 0]) + np.abs(np.r_[0, off]) + 0.5) + np.diag(off, 1) + np.diag(off, -1)
    ptr, col, val = _csr_parts(A)
    Lseq = O.ic0_sequential(ptr, col, val)
    assert np.allclose(Lseq, np.linalg.cholesky(A), atol=1e-13)
    (lp, lc, lv), s = O.ic0_sweeps(ptr, col, val, m)      # depth m -> exact
    L = np.diag(1 / s) @ _dense_lower(lp, lc, lv, m)
    assert np.allclose(L, np.linalg.cholesky(A), atol=1e-12)


@pytest.mark.parametrize("which", ["poisson", "diffusion"])
def test_ic0_sweeps_reach_textbook_ic0(which):
    """Enough sweeps reach the fixed point: the textbook IC(0), whose defining property is
    (L L^T)_ij = a_ij on the pattern of tril(A)."""
    if which == "poisson":
        A = P.poisson7(4, 3, 3).to_scipy()
    else:
        k = 10 ** np.random.default_rng(2).uniform(-2, 2, (3, 3, 4))
        A = P.diffusion7(k).to_scipy()
    m = A.shape[0]
    ptr, col, val = _csr_parts(A)
    Lseq = O.ic0_sequential(ptr, col, val)
    Ad = A.toarray()
    pat = (np.tril(Ad) != 0)
    assert np.abs((Lseq @ Lseq.T - Ad)[pat]).max() < 1e-12 * np.abs(Ad).max()
    (lp, lc, lv), s = O.ic0_sweeps(ptr, col, val, 60)
    L = np.diag(1 / s) @ _dense_lower(lp, lc, lv, m)
    assert np.allclose(L, Lseq, atol=1e-11 * np.abs(Lseq).max())
    # three sweeps are not yet the fixed point on this 3D pattern
    (lp, lc, lv), s = O.ic0_sweeps(ptr, col, val, 3)
    L3 = np.diag(1 / s) @ _dense_lower(lp, lc, lv, m)
    assert np.abs(L3 - Lseq).max() > 1e-8


def test_ilu0_sweeps_reach_textbook_ilu0():
    rng = np.random.default_rng(5)
    A = P.poisson7(3, 3, 2).to_scipy().tolil()
    # make it nonsymmetric in value, same symmetric pattern
    for i, j in zip(*A.nonzero()):
        if i != j:
            A[i, j] = A[i, j] * (1 + 0.3 * rng.uniform(-1, 1))
    A = A.tocsr()
    m = A.shape[0]
    ptr, col, val = _csr_parts(A)
    Lq, Uq = O.ilu0_sequential(ptr, col, val)
    Ad = A.toarray()
    pat = Ad != 0
    assert np.abs((Lq @ Uq - Ad)[pat]).max() < 1e-12
    (fp, fc, fv), s = O.ilu0_sweeps(ptr, col, val, 60)
    F = np.zeros((m, m))
    for i in range(m):
        F[i, fc[fp[i]:fp[i + 1]]] = fv[fp[i]:fp[i + 1]]
    L = np.tril(F, -1) + np.eye(m)
    U = np.triu(F)
    # undo the symmetric scaling: A = S^-1 L U S^-1
    Sinv = np.diag(1 / s)
    Ls = Sinv @ L @ np.diag(s)
    Us = np.diag(1 / s) @ U @ Sinv
    assert np.allclose(Ls, Lq, atol=1e-11)
    assert np.allclose(Us, Uq, atol=1e-11)


def test_ilu0_equals_ic0_on_spd():
    """On an SPD matrix the fixed points agree: L_ilu U_ilu = L_ic L_ic^T."""
    A = P.poisson7(3, 3, 3).to_scipy()
    m = A.shape[0]
    ptr, col, val = _csr_parts(A)
    (lp, lc, lv), s = O.ic0_sweeps(ptr, col, val, 40)
    Lc = _dense_lower(lp, lc, lv, m)
    (fp, fc, fv), _ = O.ilu0_sweeps(ptr, col, val, 40)
    F = np.zeros((m, m))
    for i in range(m):
        F[i, fc[fp[i]:fp[i + 1]]] = fv[fp[i]:fp[i + 1]]
    L = np.tril(F, -1) + np.eye(m)
    U = np.triu(F)
    assert np.allclose(L @ U, Lc @ Lc.T, atol=1e-12)


def test_breakdown_reported():
    A = np.array([[1.0, 2.0], [2.0, 1.0]])          # indefinite: pivot 1 - 4 < 0
    ptr, col, val = _csr_parts(A)
    with pytest.raises(O.Breakdown):
        O.ic0_sweeps(ptr, col, val, 2)
    with pytest.raises(O.Breakdown):
        O.ic0_sweeps(*_csr_parts(np.array([[-1.0, 0], [0, 1.0]])), 1)


def test_jacobi_trsv_finite_termination():
    """Jacobi sweeps on a triangular system are exact once sweeps >= depth - 1 (nilpotent
    iteration matrix), and not before; a 2x2 system is exact after one sweep."""
    m = 6
    rng = np.random.default_rng(0)
    L = np.diag(rng.uniform(1, 2, m)) + np.diag(rng.uniform(-1, 1, m - 1), -1)   # bidiagonal: depth m
    b = rng.standard_normal(m)
    Ls = sp.csr_matrix(L)
    exact = np.linalg.solve(L, b)
    assert np.allclose(O.trsv_jacobi(Ls, b, m - 1), exact, atol=1e-14)
    assert np.abs(O.trsv_jacobi(Ls, b, m - 2) - exact).max() > 1e-6
    assert np.allclose(O.trsv_substitution(Ls, b, True), exact, atol=1e-14)
    U = sp.csr_matrix(L.T)
    assert np.allclose(O.trsv_jacobi(U, b, m - 1), np.linalg.solve(L.T, b), atol=1e-14)
    assert np.allclose(O.trsv_substitution(U, b, False), np.linalg.solve(L.T, b), atol=1e-14)
    # closed form after one sweep on 2x2
    T = np.array([[2.0, 0], [3.0, 4.0]])
    y = O.trsv_jacobi(sp.csr_matrix(T), np.array([2.0, 1.0]), 1)
    assert np.allclose(y, [1.0, (1.0 - 3.0) / 4.0])


def test_local_exact_solve_matches_dense_inverse():
    prob = P.poisson_problem(8, 4)
    M = O.GDSW(prob.A, prob.part, prob.Z, local=O.EXACT)
    Ad = prob.A.to_scipy().toarray()
    r = np.random.default_rng(1).standard_normal(M.omega[3].size)
    z = M.local_solve(3, r)
    dofs = M.omega[3]
    assert np.allclose(z, np.linalg.inv(Ad[np.ix_(dofs, dofs)]) @ r, atol=1e-12)
    # banded path (m > 1500) of the exact solver
    prob = P.poisson_problem(14, 14)
    Mb = O.GDSW(prob.A, prob.part, prob.Z, local=O.EXACT)
    r = np.random.default_rng(2).standard_normal(prob.A.n)
    assert np.allclose(Mb.local_solve(0, r), np.linalg.solve(prob.A.to_scipy().toarray(), r), atol=1e-11)
