"""Pins of the oracle's coarse space: Eq. 2 and the null-space properties of Sec. III."""
import numpy as np
import scipy.sparse as sp

from oracle import gdsw_oracle as O
from paper_2304_04876_b300 import problems as P


def _interior_dofs(dec, dpn):
    return O.node_dofs(np.concatenate(dec.sub_interior_nodes), dpn)


def test_mgs_basis_closed_forms():
    rng = np.random.default_rng(1)
    X = rng.standard_normal((20, 3))
    Q = O.mgs_basis(np.column_stack([X[:, 0], X[:, 1], X[:, 0] + 2 * X[:, 1], X[:, 2]]))
    assert Q.shape == (20, 3)                              # dependent third column dropped
    assert np.allclose(Q.T @ Q, np.eye(3), atol=1e-14)
    # span(Q) == span(X): projection residual vanishes
    assert np.linalg.norm(X - Q @ (Q.T @ X)) < 1e-13
    # a single constant column on m nodes normalises to 1/sqrt(m)
    q = O.mgs_basis(np.ones((7, 1)))
    assert np.allclose(q, 1 / np.sqrt(7))
    # rigid-body modes: plane region -> 6, straight line -> 5, one point -> 3
    pts_plane = np.array([[0.5, y, z] for y in (0, .1, .2) for z in (0, .1)])
    pts_line = np.array([[0.5, 0.2, z] for z in (0, .1, .2, .3)])
    pts_pt = np.array([[0.3, 0.2, 0.1]])
    assert O.mgs_basis(P.rigid_body_modes(pts_plane)).shape[1] == 6
    assert O.mgs_basis(P.rigid_body_modes(pts_line)).shape[1] == 5
    assert O.mgs_basis(P.rigid_body_modes(pts_pt)).shape[1] == 3


def _setup(prob):
    dec = O.decompose(prob.part)
    cs = O.coarse_space(prob.A, prob.part, dec, prob.Z)
    return dec, cs


def test_extension_is_discrete_harmonic():
    """(A Phi)_I = A_II Phi_I + A_IGamma Phi_Gamma = 0 on every interior (Eq. 2)."""
    for prob in (P.poisson_problem(12, 4), P.elasticity_problem(6, 2)):
        dec, cs = _setup(prob)
        A = prob.A.to_scipy()
        AP = (A @ cs.Phi).toarray()
        I = _interior_dofs(dec, prob.part.dpn)
        assert np.abs(AP[I]).max() <= 1e-12 * np.abs(AP).max()


def test_partition_of_unity_constants():
    """With the constant null space, sum_i sqrt(|Gamma_i|) Phi_:,i = 1 on Gamma, and on the
    interior of a floating subdomain (zero row sums there) the extension reproduces 1."""
    prob = P.poisson_problem(12, 4)                # 3^3 blocks: block 13 is floating
    dec, cs = _setup(prob)
    w = np.zeros(cs.n0)
    for nodes, cc in zip(dec.comp_nodes, cs.comp_cols):
        w[cc] = np.sqrt(len(nodes))
    v = cs.Phi @ w
    G = np.nonzero(dec.node_gamma)[0]
    assert np.allclose(v[G], 1.0, atol=1e-14)
    A = prob.A.to_scipy()
    rowsum = np.asarray(A.sum(axis=1)).ravel()
    centre = dec.sub_interior_nodes[13]
    assert np.all(rowsum[centre] == 0)
    assert np.allclose(v[centre], 1.0, atol=1e-12)
    # a subdomain touching the Dirichlet boundary does not reproduce the constant
    corner = dec.sub_interior_nodes[0]
    assert np.abs(v[corner] - 1).max() > 1e-3


def test_rigid_body_modes_reproduced():
    """Q1 elasticity: on subdomains away from the clamp (A Z = 0 on their rows), Phi reproduces
    every rigid-body mode, rotations included."""
    prob = P.elasticity_problem(6, 2)
    dec, cs = _setup(prob)
    A = prob.A.to_scipy()
    Z = prob.Z
    # least-squares coefficients from the Gamma rows: Z_Gamma = Phi_Gamma C exactly
    G = O.node_dofs(np.nonzero(dec.node_gamma)[0], 3)
    PhiG = cs.Phi[G].toarray()
    C, *_ = np.linalg.lstsq(PhiG, Z[G], rcond=None)
    assert np.linalg.norm(PhiG @ C - Z[G]) < 1e-12 * np.linalg.norm(Z[G])
    PZ = cs.Phi @ C
    nx = prob.part.nx
    for s, inodes in enumerate(dec.sub_interior_nodes):
        I = O.node_dofs(inodes, 3)
        floating = np.abs(A[I] @ Z).max() < 1e-12
        err = np.abs(PZ[I] - Z[I]).max()
        if floating:
            assert err < 1e-10
        else:
            assert err > 1e-6


def test_coarse_matrix_spd_and_basis_invariance():
    """A0 = Phi^T A Phi is SPD, and Phi A0^-1 Phi^T is unchanged by Phi -> Phi T."""
    prob = P.poisson_problem(8, 4)
    dec, cs = _setup(prob)
    A = prob.A.to_scipy().toarray()
    A0 = cs.A0
    assert np.allclose(A0, A0.T, atol=1e-13 * np.abs(A0).max())
    assert np.linalg.eigvalsh(A0).min() > 0
    Phi = cs.Phi.toarray()
    T = np.random.default_rng(0).standard_normal((cs.n0, cs.n0)) + 3 * np.eye(cs.n0)
    C1 = Phi @ np.linalg.solve(Phi.T @ A @ Phi, Phi.T)
    P2 = Phi @ T
    C2 = P2 @ np.linalg.solve(P2.T @ A @ P2, P2.T)
    assert np.allclose(C1, C2, atol=1e-10 * np.abs(C1).max())
    assert np.allclose(A0, Phi.T @ A @ Phi, atol=1e-13 * np.abs(A0).max())


def test_edges_vertices_do_not_extend_for_7pt():
    """With a 7-point stencil the interior couples only to face nodes, so edge and vertex
    basis functions vanish on every interior."""
    prob = P.poisson_problem(12, 4)
    dec, cs = _setup(prob)
    I = _interior_dofs(dec, 1)
    PhiI = cs.Phi[I].tocsc()
    for t, cc in zip(dec.comp_type, cs.comp_cols):
        nz = PhiI[:, cc].nnz
        assert (nz > 0) == (t == 1)


def test_rgdsw_vertex_closure_and_sizes():
    """Reduced GDSW: one coarse function per vertex and null-space vector; every edge
    of a 3^3 decomposition has 2 vertices in its closure and every interior face 4,
    faces and edges touching the outer boundary fewer."""
    prob = P.poisson_problem(12, 4)
    dec = O.decompose(prob.part)
    clo = O.vertex_closure(dec, prob.part)
    counts = {1: [], 2: []}
    for c, vs in enumerate(clo):
        if dec.comp_type[c] in counts:
            counts[int(dec.comp_type[c])].append(len(vs))
    # 2 planes per axis: vertices 8; faces have 1, 2 or 4 vertices, edges 1 or 2
    assert int((dec.comp_type == 3).sum()) == 8
    assert set(counts[1]) <= {1, 2, 4} and 4 in counts[1]
    assert set(counts[2]) <= {1, 2} and 2 in counts[2]
    cs = O.coarse_space(prob.A, prob.part, dec, prob.Z, "rgdsw")
    assert cs.n0 == 8
    # closed form: the central face of the 3^3 split touches the 4 vertices of its plane
    for c, vs in enumerate(clo):
        if dec.comp_type[c] == 1 and len(vs) == 4:
            xs = set(int(k) for k in dec.comp_key[vs][:, :, 1].ravel())
            assert xs <= {0, 1}


def test_rgdsw_partition_of_unity_and_extension():
    prob = P.poisson_problem(12, 4)
    dec = O.decompose(prob.part)
    cs = O.coarse_space(prob.A, prob.part, dec, prob.Z, "rgdsw")
    G = np.nonzero(dec.node_gamma)[0]
    # weights: the norm of each vertex's unnormalised function (sum of its squared weights)
    clo = O.vertex_closure(dec, prob.part)
    verts = sorted(np.nonzero(dec.comp_type == 3)[0])
    wsq = {v: 0.0 for v in verts}
    for c, vs in enumerate(clo):
        for v in vs:
            wsq[v] += len(dec.comp_nodes[c]) / len(vs) ** 2
    w = np.array([np.sqrt(wsq[v]) for v in verts])
    u = cs.Phi @ w
    assert np.allclose(u[G], 1.0, atol=1e-13)
    A = prob.A.to_scipy()
    I = O.node_dofs(np.concatenate(dec.sub_interior_nodes), 1)
    AP = (A @ cs.Phi).toarray()
    assert np.abs(AP[I]).max() <= 1e-12 * np.abs(AP).max()
    assert np.allclose(u[dec.sub_interior_nodes[13]], 1.0, atol=1e-12)   # floating block


def test_rgdsw_rigid_body_modes():
    """Elasticity: six functions per vertex (rotations are independent on the support),
    and every rigid-body mode reproduced on subdomains away from the clamp."""
    prob = P.elasticity_problem(6, 2)
    dec = O.decompose(prob.part)
    cs = O.coarse_space(prob.A, prob.part, dec, prob.Z, "rgdsw")
    assert cs.n0 == 6 * int((dec.comp_type == 3).sum())
    A = prob.A.to_scipy()
    G = O.node_dofs(np.nonzero(dec.node_gamma)[0], 3)
    PhiG = cs.Phi[G].toarray()
    C, *_ = np.linalg.lstsq(PhiG, prob.Z[G], rcond=None)
    assert np.linalg.norm(PhiG @ C - prob.Z[G]) < 1e-11 * np.linalg.norm(prob.Z[G])
    PZ = cs.Phi @ C
    for inodes in dec.sub_interior_nodes:
        I = O.node_dofs(inodes, 3)
        if np.abs(A[I] @ prob.Z).max() < 1e-12:
            assert np.abs(PZ[I] - prob.Z[I]).max() < 1e-10
