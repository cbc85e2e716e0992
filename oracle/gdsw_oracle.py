"""Plain CPU FP64 oracle of the GDSW two-level overlapping Schwarz preconditioner.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its CPU-baseline and reference legs) may import this module.  It
shares no code with the CUDA library: it reads the same seeded inputs (CSR
matrix, structured partition, null space) and computes everything else
itself, slowly and in the order the paper states it.

Paper: Yamazaki, Heinlein, Rajamanickam, "An Experimental Study of Two-Level
Schwarz Domain Decomposition Preconditioners on GPUs" (arXiv 2304.04876).

What it computes (Sec. III, Eq. 1):

    M^-1 r = Phi A0^-1 Phi^T r + sum_s R_s^T A_s^-1 R_s r,   A0 = Phi^T A Phi,

with Phi the GDSW energy-minimising extension of Eq. 2 and A_s^-1 either an
exact Cholesky solve or an incomplete factorisation built by the fixed-point
sweeps of Sec. V-B3 and applied by exact substitution or Jacobi sweeps.

Readings taken where the paper is silent or garbled (each is listed in the
design notes):

* Gamma and its components: geometric, from separator node planes (Fig. 1).
  A component is a face, edge or vertex; components are disjoint, so the
  partition-of-unity scalings D_Gamma_i are identities.
* Overlap: algebraic, one layer at node level (Sec. VII "algebraic overlap of
  one"): Omega_s' = block s plus every node coupled to it through A.
* Phi_Gamma is n_Gamma x (n_c n_n) (the paper prints n_I); each block
  Phi_Gamma_i is the null space restricted to component i, orthonormalised by
  modified Gram-Schmidt, columns whose remaining norm falls below 1e-10 of
  their original norm dropped.
* A0 = Phi^T A Phi (the paper prints Phi A Phi^T).
* IC(0)/ILU(0) sweeps: symmetric unit-diagonal scaling, synchronous (Jacobi)
  updates from tril / triu of the scaled matrix; Jacobi triangular sweeps
  start from D^-1 b with damping 1.
* Scatter: contributions summed in ascending subdomain order, coarse term last.

parity unpinned: nothing; every function below is pinned by a test in
``tests/test_oracle_*.py`` (brute force, closed forms, invariants, special
cases, finite termination).
"""
from __future__ import annotations

import heapq
from dataclasses import dataclass
from typing import List, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

EXACT, IC0, ILU0 = "exact", "ic0", "ilu0"
LEVELSCHED, JACOBI = "levelsched", "jacobi"

DROP_TOL = 1e-10


class Breakdown(RuntimeError):
    """A non-positive (IC) or zero (ILU) pivot appeared during a factor sweep."""


# ----------------------------------------------------------------------------
# CSR helpers (plain index arithmetic, structural zeros kept)
# ----------------------------------------------------------------------------

def _csr(n, rowptr, colind, val):
    return sp.csr_matrix((np.asarray(val, dtype=np.float64), np.asarray(colind), np.asarray(rowptr)),
                         shape=(n, n))


def _row_of_entry(rowptr):
    return np.repeat(np.arange(len(rowptr) - 1), np.diff(rowptr))


def submatrix(rowptr, colind, val, n, rows, cols):
    """Rows ``rows`` and columns ``cols`` (sorted global indices) of a CSR matrix.

    Stored entries, explicit zeros included, are kept; the result is CSR with
    sorted columns (the local order is the order of ``rows``/``cols``).
    """
    cmap = -np.ones(n, dtype=np.int64)
    cmap[cols] = np.arange(len(cols))
    starts, ends = rowptr[rows], rowptr[rows + 1]
    lens = ends - starts
    ent = np.concatenate([np.arange(a, b) for a, b in zip(starts, ends)]) if len(rows) else np.zeros(0, np.int64)
    lrow = np.repeat(np.arange(len(rows)), lens)
    lcol = cmap[colind[ent]]
    keep = lcol >= 0
    lrow, lcol, lval = lrow[keep], lcol[keep], val[ent][keep]
    order = np.lexsort((lcol, lrow))
    lrow, lcol, lval = lrow[order], lcol[order], lval[order]
    ptr = np.zeros(len(rows) + 1, dtype=np.int64)
    np.add.at(ptr, lrow + 1, 1)
    ptr = np.cumsum(ptr)
    return ptr, lcol, lval


def _values_at(M: sp.csr_matrix, rows, cols):
    """M[rows[e], cols[e]] for each e (0 where M stores nothing)."""
    M = M.tocsr()
    M.sort_indices()
    out = np.zeros(len(rows))
    if M.nnz == 0 or len(rows) == 0:
        return out
    n = M.shape[1]
    mrow = _row_of_entry(M.indptr)
    mkey = mrow.astype(np.int64) * n + M.indices
    key = np.asarray(rows, dtype=np.int64) * n + np.asarray(cols)
    pos = np.searchsorted(mkey, key)
    pos = np.minimum(pos, len(mkey) - 1)
    hit = mkey[pos] == key
    out[hit] = M.data[pos[hit]]
    return out


# ----------------------------------------------------------------------------
# Sec. III: nonoverlapping decomposition, interface and its components (Fig. 1)
# ----------------------------------------------------------------------------

@dataclass
class Decomposition:
    n_sub: int
    node_sub: np.ndarray        # block of every node (plane nodes belong to the lower block)
    node_gamma: np.ndarray      # node lies on >= 1 separator plane
    node_comp: np.ndarray       # interface component of every node, -1 for interior nodes
    comp_type: np.ndarray       # 1 face, 2 edge, 3 vertex
    comp_nodes: List[np.ndarray]
    sub_interior_nodes: List[np.ndarray]
    sub_nodes: List[np.ndarray]
    comp_key: np.ndarray = None     # (ncomp, 3, 2): per axis (on_plane, plane or block index)


def decompose(part) -> Decomposition:
    """Blocks, interface Gamma and its components from the separator planes.

    A node belongs to block (bx, by, bz) where b_a counts the planes strictly
    below its coordinate on axis a; Gamma is the set of nodes on a plane
    (Sec. III, the interior/interface split of the 2x2 block form).  The
    component of a Gamma node is identified by, per axis, either the plane it
    lies on or the block it lies in; one plane gives a face, two an edge and
    three a vertex.  Components are numbered by their smallest node index.
    """
    dims = (part.nx, part.ny, part.nz)
    blk, onp = [], []
    for a in range(3):
        idx = np.arange(dims[a])
        c = np.asarray(sorted(part.cuts[a]), dtype=np.int64)
        blk.append(np.searchsorted(c, idx, side="left"))
        onp.append(np.isin(idx, c))
    nb = [len(part.cuts[a]) + 1 for a in range(3)]
    K, J, I = np.meshgrid(np.arange(dims[2]), np.arange(dims[1]), np.arange(dims[0]), indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    bx, by, bz = blk[0][I], blk[1][J], blk[2][K]
    px, py, pz = onp[0][I], onp[1][J], onp[2][K]
    node_sub = bx + nb[0] * (by + nb[1] * bz)
    gamma = px | py | pz
    # component key: per axis (2*index + on_plane)
    cx, cy, cz = 2 * bx + px, 2 * by + py, 2 * bz + pz
    key = cx + (2 * nb[0]) * (cy + (2 * nb[1]) * cz)
    node_comp = -np.ones(part.n_nodes, dtype=np.int64)
    gnodes = np.nonzero(gamma)[0]
    ukeys, first, inv = np.unique(key[gnodes], return_index=True, return_inverse=True)
    order = np.argsort(gnodes[first], kind="stable")          # by smallest node
    rank = np.empty_like(order)
    rank[order] = np.arange(len(order))
    node_comp[gnodes] = rank[inv]
    ntype = (px.astype(int) + py + pz)
    comp_type = np.zeros(len(order), dtype=np.int64)
    comp_type[node_comp[gnodes]] = ntype[gnodes]
    comp_nodes = [np.zeros(0, np.int64)] * len(order)
    if len(gnodes):
        srt = np.argsort(node_comp[gnodes], kind="stable")
        bounds = np.searchsorted(node_comp[gnodes][srt], np.arange(len(order) + 1))
        comp_nodes = [gnodes[srt[bounds[i]:bounds[i + 1]]] for i in range(len(order))]
    n_sub = nb[0] * nb[1] * nb[2]
    srt = np.argsort(node_sub, kind="stable")
    bounds = np.searchsorted(node_sub[srt], np.arange(n_sub + 1))
    sub_nodes = [srt[bounds[s]:bounds[s + 1]] for s in range(n_sub)]
    sub_interior = [nodes[~gamma[nodes]] for nodes in sub_nodes]
    comp_key = np.zeros((len(order), 3, 2), dtype=np.int64)
    if len(gnodes):
        first_node = np.array([nodes[0] for nodes in comp_nodes])
        for a, (bb, pp) in enumerate(((bx, px), (by, py), (bz, pz))):
            comp_key[:, a, 0] = pp[first_node]
            comp_key[:, a, 1] = bb[first_node]
    return Decomposition(n_sub, node_sub, gamma, node_comp, comp_type, comp_nodes,
                         sub_interior, sub_nodes, comp_key)


def vertex_closure(dec: Decomposition, part) -> List[np.ndarray]:
    """For every interface component, the vertex components in its closure.

    A vertex lies in the closure of component c when, on every axis, it sits on
    c's plane if c lies on a plane there, and on one of the two planes bounding
    c's block otherwise (block b is bounded by planes b-1 and b).
    """
    ncut = [len(part.cuts[a]) for a in range(3)]
    verts = np.nonzero(dec.comp_type == 3)[0]
    vkey = {tuple(dec.comp_key[v, :, 1]): v for v in verts}
    out = []
    for c in range(len(dec.comp_nodes)):
        if dec.comp_type[c] == 3:
            out.append(np.array([c]))
            continue
        choices = []
        for a in range(3):
            on, idx = dec.comp_key[c, a]
            choices.append([idx] if on else [q for q in (idx - 1, idx) if 0 <= q < ncut[a]])
        vs = sorted(vkey[(x, y, z)] for x in choices[0] for y in choices[1] for z in choices[2]
                    if (x, y, z) in vkey)
        out.append(np.array(vs, dtype=np.int64))
    return out


def node_dofs(nodes: np.ndarray, dpn: int) -> np.ndarray:
    """All unknowns of the given nodes, node-major."""
    return (dpn * np.asarray(nodes, dtype=np.int64)[:, None] + np.arange(dpn)).ravel()


def overlapping_subdomains(A, part, dec: Decomposition, delta: int = 1) -> List[np.ndarray]:
    """Omega_s' (Sec. III): block s grown by ``delta`` layers of algebraic overlap.

    One layer adds every node v with A[u, v] stored for some node u already in
    the set (all unknowns of a node move together).  Returns sorted node lists.
    """
    dpn = part.dpn
    rows = _row_of_entry(A.rowptr) // dpn
    cols = A.colind.astype(np.int64) // dpn
    nn = part.n_nodes
    G = sp.csr_matrix((np.ones(len(rows), dtype=np.int8), (rows, cols)), shape=(nn, nn))
    G.data[:] = 1
    S = sp.csr_matrix((np.ones(nn, dtype=np.int8), (dec.node_sub, np.arange(nn))),
                      shape=(dec.n_sub, nn))
    for _ in range(delta):
        S = (S + S @ G).tocsr()
        S.data[:] = 1
    S.sort_indices()
    return [S.indices[S.indptr[s]:S.indptr[s + 1]].astype(np.int64) for s in range(dec.n_sub)]


# ----------------------------------------------------------------------------
# Sec. III, step 3-4: null space on the components and the extension (Eq. 2)
# ----------------------------------------------------------------------------

def mgs_basis(Zc: np.ndarray) -> np.ndarray:
    """Orthonormal basis of span(Zc) by modified Gram-Schmidt in column order.

    A column whose norm after orthogonalisation is below DROP_TOL times its
    original norm is dropped (it adds nothing to the span).
    """
    Q = []
    for c in range(Zc.shape[1]):
        v = Zc[:, c].astype(np.float64).copy()
        n0 = np.linalg.norm(v)
        for q in Q:
            v -= (q @ v) * q
        nv = np.linalg.norm(v)
        if n0 == 0.0 or nv < DROP_TOL * n0:
            continue
        Q.append(v / nv)
    return np.stack(Q, axis=1) if Q else np.zeros((Zc.shape[0], 0))


def _spd_solve(M: sp.csr_matrix, B: np.ndarray) -> np.ndarray:
    """Exact solve with an SPD matrix: dense Cholesky when small, banded Cholesky
    (natural order, LAPACK pbtrf/pbtrs through scipy) otherwise."""
    n = M.shape[0]
    if n == 0:
        return np.zeros_like(B)
    if n <= 1500:
        c = sla.cho_factor(M.toarray(), lower=True)
        return sla.cho_solve(c, B)
    Mc = M.tocoo()
    u = int(np.max(np.abs(Mc.col - Mc.row)))
    ab = np.zeros((u + 1, n))
    up = Mc.col >= Mc.row
    ab[u + Mc.row[up] - Mc.col[up], Mc.col[up]] = Mc.data[up]
    cb = sla.cholesky_banded(ab, lower=False)
    return sla.cho_solve_banded((cb, False), B)


@dataclass
class Coarse:
    n0: int
    Phi: sp.csr_matrix           # n x n0
    A0: np.ndarray               # n0 x n0 (dense)
    comp_cols: List[np.ndarray]  # coarse columns of each component


def coarse_space(A, part, dec: Decomposition, Z: np.ndarray, variant: str = "gdsw") -> Coarse:
    """GDSW coarse basis (Eq. 2) and coarse matrix A0 = Phi^T A Phi.

    variant "gdsw": Phi_Gamma = [R_Gamma_1^T Phi_Gamma_1, ...] with Phi_Gamma_i an
    orthonormal basis of the null space restricted to component i (D_Gamma_i = I).
    variant "rgdsw" (reduced: coarse functions for vertices only, Sec. III): the
    function of vertex v and null-space vector z is z on v and z / N_c on every
    edge or face c whose closure holds N_c vertices, v among them (a partition of
    unity on Gamma); each vertex's functions are orthonormalised over their support.
    Phi_I = -A_II^-1 A_IGamma Phi_Gamma, solved exactly per interior block since
    A_II is block diagonal (Sec. III).
    """
    n = A.n
    dpn = part.dpn
    Asp = _csr(n, A.rowptr, A.colind, A.val)
    rows, cols, vals = [], [], []
    comp_cols = []
    n0 = 0
    if variant == "gdsw":
        supports = [(node_dofs(nodes, dpn), np.ones(len(nodes) * dpn)) for nodes in dec.comp_nodes]
    elif variant == "rgdsw":
        closure = vertex_closure(dec, part)
        owners = {v: [] for v in np.nonzero(dec.comp_type == 3)[0]}
        for c, vs in enumerate(closure):
            if len(vs) == 0:
                raise ValueError("rGDSW needs a vertex in the closure of every interface component")
            for v in vs:
                owners[v].append((c, 1.0 / len(vs)))
        supports = []
        for v in sorted(owners):
            dofs = np.concatenate([node_dofs(dec.comp_nodes[c], dpn) for c, _ in owners[v]])
            w = np.concatenate([np.full(len(dec.comp_nodes[c]) * dpn, wt) for c, wt in owners[v]])
            supports.append((dofs, w))
    else:
        raise ValueError(variant)
    for dofs, w in supports:
        Q = mgs_basis(w[:, None] * Z[dofs, :])
        k = Q.shape[1]
        cc = np.arange(n0, n0 + k)
        comp_cols.append(cc)
        n0 += k
        rows.append(np.repeat(dofs, k))
        cols.append(np.tile(cc, len(dofs)))
        vals.append(Q.ravel())
    if n0 == 0:
        return Coarse(0, sp.csr_matrix((n, 0)), np.zeros((0, 0)), comp_cols)
    PhiG = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n0))
    PhiG.sum_duplicates()
    irows, icols, ivals = [], [], []
    for inodes in dec.sub_interior_nodes:
        I = node_dofs(inodes, dpn)
        if len(I) == 0:
            continue
        B = (Asp[I, :] @ PhiG)                    # A_I,Gamma Phi_Gamma (Gamma rows only in PhiG)
        B = B.tocsc()
        nzc = np.nonzero(np.diff(B.indptr))[0]
        if len(nzc) == 0:
            continue
        Bd = B[:, nzc].toarray()
        AII = Asp[I, :][:, I]
        X = -_spd_solve(AII, Bd)
        irows.append(np.repeat(I, len(nzc)))
        icols.append(np.tile(nzc, len(I)))
        ivals.append(X.ravel())
    if irows:
        PhiI = sp.csr_matrix((np.concatenate(ivals), (np.concatenate(irows), np.concatenate(icols))),
                             shape=(n, n0))
        Phi = (PhiG + PhiI).tocsr()
    else:
        Phi = PhiG.tocsr()
    A0 = (Phi.T @ (Asp @ Phi)).toarray()
    return Coarse(n0, Phi, A0, comp_cols)


# ----------------------------------------------------------------------------
# Sec. V-B3: incomplete factors by fixed-point sweeps, triangular solves
# ----------------------------------------------------------------------------

def scaled(ptr, col, val):
    """D^-1/2 A D^-1/2 of a local CSR matrix and the scaling vector D^-1/2."""
    m = len(ptr) - 1
    row = _row_of_entry(ptr)
    d = np.zeros(m)
    dmask = row == col
    d[row[dmask]] = val[dmask]
    if np.any(d <= 0):
        raise Breakdown("non-positive diagonal")
    s = 1.0 / np.sqrt(d)
    return val * s[row] * s[col], s


def ic0_sweeps(ptr, col, val, sweeps: int):
    """IC(0) of the scaled local matrix by synchronous Chow-Patel sweeps.

    On the pattern of tril(A~): start from L = tril(A~); in each sweep every
    entry is recomputed from the previous sweep's values,
        s_ij = a~_ij - sum_{k<j} l_ik l_jk,
        l_ij = s_ij / l_jj (i > j),   l_jj = sqrt(s_jj).
    The sum is (Ls Ls^T)_ij with Ls the strict lower part.  Returns the lower
    CSR (ptr, col, L values) and the scaling D^-1/2.
    """
    m = len(ptr) - 1
    at, s = scaled(ptr, col, val)
    row = _row_of_entry(ptr)
    low = col <= row
    lrow, lcol, la = row[low], col[low], at[low]
    lptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(lptr, lrow + 1, 1)
    lptr = np.cumsum(lptr)
    L = la.copy()
    diag = lrow == lcol
    for _ in range(sweeps):
        strict = ~diag
        Ls = sp.csr_matrix((L[strict], (lrow[strict], lcol[strict])), shape=(m, m))
        P = _values_at((Ls @ Ls.T).tocsr(), lrow, lcol)
        S = la - P
        ljj = np.zeros(m)
        ljj[lrow[diag]] = L[diag]
        new = np.empty_like(L)
        if np.any(S[diag] <= 0):
            raise Breakdown("IC(0) sweep: non-positive pivot")
        new[diag] = np.sqrt(S[diag])
        new[strict] = S[strict] / ljj[lcol[strict]]
        L = new
    return (lptr, lcol, L), s


def ilu0_sweeps(ptr, col, val, sweeps: int):
    """ILU(0) of the scaled local matrix by synchronous Chow-Patel sweeps.

    On the pattern of A~, L unit lower and U upper: start from L = strict
    tril(A~) + I, U = triu(A~); each sweep recomputes, from the previous values,
        l_ij = (a~_ij - sum_{k<j} l_ik u_kj) / u_jj   (i > j),
        u_ij =  a~_ij - sum_{k<i} l_ik u_kj           (i <= j).
    Both sums equal (Ls U_strict)_ij.  Returns (ptr, col, values) holding the
    strict lower part of L and all of U in one array, and the scaling.
    """
    m = len(ptr) - 1
    at, s = scaled(ptr, col, val)
    row = _row_of_entry(ptr)
    F = at.copy()
    lower = col < row
    upper = ~lower
    ustrict = col > row
    diag = col == row
    for _ in range(sweeps):
        Ls = sp.csr_matrix((F[lower], (row[lower], col[lower])), shape=(m, m))
        Us = sp.csr_matrix((F[ustrict], (row[ustrict], col[ustrict])), shape=(m, m))
        P = _values_at((Ls @ Us).tocsr(), row, col)
        S = at - P
        ujj = np.zeros(m)
        ujj[row[diag]] = F[diag]
        if np.any(ujj == 0) or not np.all(np.isfinite(S)):
            raise Breakdown("ILU(0) sweep: zero pivot")
        new = np.empty_like(F)
        new[upper] = S[upper]
        new[lower] = S[lower] / ujj[col[lower]]
        F = new
    return (ptr, col, F), s


def level_fill_pattern(ptr, col, k: int):
    """Pattern of the level-of-fill incomplete factorisation ILU(k) (Sec. V-B:
    the KokkosKernels ILU(k) and the fixed-point FastILU(k) of Table I).

    Entries of A have level 0.  Eliminating row i with pivot p (in increasing
    column order, fill included) creates or lowers entry (i, j), j > p, to level
    lev(i, p) + lev(p, j) + 1, where lev(p, j) is the final level of row p; the
    pattern keeps every entry of level <= k.  Returns (ptr, col, level), rows
    sorted by column.
    """
    m = len(ptr) - 1
    upper = []                       # finished rows: [(j, level)] for j > row
    out_ptr = [0]
    out_col, out_lev = [], []
    for i in range(m):
        lev = {int(j): 0 for j in col[ptr[i]:ptr[i + 1]]}
        heap = [j for j in lev if j < i]
        heapq.heapify(heap)
        seen = set()
        while heap:
            p = heapq.heappop(heap)
            if p in seen:
                continue
            seen.add(p)
            lip = lev[p]
            for j, lpj in upper[p]:
                new = lip + lpj + 1
                if new > k:
                    continue
                if j not in lev:
                    lev[j] = new
                    if j < i:
                        heapq.heappush(heap, j)
                elif new < lev[j]:
                    lev[j] = new
        cols = sorted(lev)
        upper.append([(j, lev[j]) for j in cols if j > i])
        out_col.extend(cols)
        out_lev.extend(lev[j] for j in cols)
        out_ptr.append(len(out_col))
    return (np.asarray(out_ptr, dtype=np.int64), np.asarray(out_col, dtype=np.int64),
            np.asarray(out_lev, dtype=np.int64))


def pad_to_pattern(ptr, col, val, fptr, fcol):
    """Values of (ptr, col, val) on the larger pattern (fptr, fcol), zero on fill."""
    m = len(ptr) - 1
    out = np.zeros(len(fcol))
    for i in range(m):
        pos = {int(j): q for q, j in enumerate(fcol[fptr[i]:fptr[i + 1]], start=int(fptr[i]))}
        for e in range(ptr[i], ptr[i + 1]):
            out[pos[int(col[e])]] = val[e]
    return out


def ic0_sequential(ptr, col, val):
    """Textbook IC(0) (row-by-row, in place on the pattern of tril(A)); small cases.

    Used as the fixed point the sweeps must reach.  Unscaled input.
    """
    m = len(ptr) - 1
    rows = [dict() for _ in range(m)]
    for i in range(m):
        for e in range(ptr[i], ptr[i + 1]):
            if col[e] <= i:
                rows[i][int(col[e])] = float(val[e])
    for i in range(m):
        for j in sorted(rows[i]):
            s = rows[i][j]
            for k, lik in rows[i].items():
                if k < j and k in rows[j]:
                    s -= lik * rows[j][k]
            if j < i:
                rows[i][j] = s / rows[j][j]
            else:
                if s <= 0:
                    raise Breakdown("IC(0): non-positive pivot")
                rows[i][i] = np.sqrt(s)
    out = np.zeros((m, m))
    for i in range(m):
        for j, v in rows[i].items():
            out[i, j] = v
    return out


def ilu0_sequential(ptr, col, val):
    """Textbook ILU(0), IKJ order, on the pattern of A; returns dense (L unit, U)."""
    m = len(ptr) - 1
    a = [dict() for _ in range(m)]
    for i in range(m):
        for e in range(ptr[i], ptr[i + 1]):
            a[i][int(col[e])] = float(val[e])
    for i in range(1, m):
        for k in sorted(c for c in a[i] if c < i):
            a[i][k] /= a[k][k]
            for j, ukj in a[k].items():
                if j > k and j in a[i]:
                    a[i][j] -= a[i][k] * ukj
    Lm, Um = np.eye(m), np.zeros((m, m))
    for i in range(m):
        for j, v in a[i].items():
            if j < i:
                Lm[i, j] = v
            else:
                Um[i, j] = v
    return Lm, Um


def trsv_substitution(T: sp.csr_matrix, b: np.ndarray, lower: bool) -> np.ndarray:
    """Exact triangular solve (what a level-scheduled solve computes)."""
    return spla.spsolve_triangular(T.tocsr(), b, lower=lower)


def trsv_jacobi(T: sp.csr_matrix, b: np.ndarray, sweeps: int) -> np.ndarray:
    """Fixed number of Jacobi sweeps on T y = b (Sec. V-B3):
    y0 = D^-1 b,  y_{k+1} = D^-1 (b - (T - D) y_k), damping 1."""
    d = T.diagonal()
    off = T - sp.diags(d)
    y = b / d
    for _ in range(sweeps):
        y = (b - off @ y) / d
    return y


# ----------------------------------------------------------------------------
# Eq. 1: the preconditioner
# ----------------------------------------------------------------------------

class GDSW:
    """M^-1 = Phi A0^-1 Phi^T + sum_s R_s^T A_s^-1 R_s (Eq. 1).

    local: EXACT (Cholesky of A_s), IC0 or ILU0 (Chow-Patel sweeps);
    trsv: LEVELSCHED (exact substitution) or JACOBI (fixed sweeps).
    coarse=False gives the one-level additive Schwarz operator; coarse_variant
    "rgdsw" the reduced (vertex) coarse space.
    """

    def __init__(self, A, part, Z=None, local=EXACT, trsv=LEVELSCHED, sweeps_factor=3,
                 sweeps_trsv=5, overlap=1, coarse=True, coarse_variant="gdsw", fill_level=0):
        self.A = A
        self.fill_level = fill_level
        self.part = part
        self.n = A.n
        self.local, self.trsv = local, trsv
        self.sweeps_factor, self.sweeps_trsv = sweeps_factor, sweeps_trsv
        self.dec = decompose(part)
        self.omega_nodes = overlapping_subdomains(A, part, self.dec, overlap)
        self.omega = [node_dofs(nd, part.dpn) for nd in self.omega_nodes]
        if Z is None:
            Z = np.ones((A.n, 1))
        self.Asp = _csr(A.n, A.rowptr, A.colind, A.val)
        self.coarse = coarse_space(A, part, self.dec, Z, coarse_variant) if coarse else None
        if self.coarse is not None and self.coarse.n0:
            self.A0fac = sla.cho_factor(self.coarse.A0, lower=True)
        self.factors = [self._factor(dofs) for dofs in self.omega]

    @property
    def n0(self) -> int:
        return 0 if self.coarse is None else self.coarse.n0

    def local_matrix(self, dofs):
        return submatrix(self.A.rowptr, self.A.colind, self.A.val, self.n, dofs, dofs)

    def _factor(self, dofs):
        ptr, col, val = self.local_matrix(dofs)
        m = len(dofs)
        if self.local == EXACT:
            As = _csr(m, ptr, col, val)
            return ("exact", As)
        if self.fill_level > 0:
            # IC(k)/ILU(k): the same sweeps over the level-k pattern, zero on fill
            fptr, fcol, _ = level_fill_pattern(ptr, col, self.fill_level)
            val = pad_to_pattern(ptr, col, val, fptr, fcol)
            ptr, col = fptr, fcol
        if self.local == IC0:
            (lp, lc, lv), s = ic0_sweeps(ptr, col, val, self.sweeps_factor)
            Lm = _csr(m, lp, lc, lv)
            return ("ic0", Lm, Lm.T.tocsr(), s)
        (fp, fc, fv), s = ilu0_sweeps(ptr, col, val, self.sweeps_factor)
        row = _row_of_entry(fp)
        lo = fc < row
        Lm = sp.csr_matrix((np.concatenate([fv[lo], np.ones(m)]),
                            (np.concatenate([row[lo], np.arange(m)]),
                             np.concatenate([fc[lo], np.arange(m)]))), shape=(m, m))
        Um = sp.csr_matrix((fv[~lo], (row[~lo], fc[~lo])), shape=(m, m))
        return ("ilu0", Lm, Um, s)

    def local_solve(self, s: int, rs: np.ndarray) -> np.ndarray:
        """A_s^-1 r_s with the local solver of subdomain s."""
        f = self.factors[s]
        if f[0] == "exact":
            return _spd_solve(f[1], rs[:, None])[:, 0]
        _, Lm, Um, sc = f
        b = sc * rs
        if self.trsv == LEVELSCHED:
            y = trsv_substitution(Lm, b, lower=True)
            z = trsv_substitution(Um, y, lower=False)
        else:
            y = trsv_jacobi(Lm, b, self.sweeps_trsv)
            z = trsv_jacobi(Um, y, self.sweeps_trsv)
        return sc * z

    def apply(self, r: np.ndarray) -> np.ndarray:
        """z = M^-1 r (Eq. 1): local terms in ascending subdomain order, coarse last."""
        r = np.asarray(r, dtype=np.float64)
        z = np.zeros(self.n)
        for s, dofs in enumerate(self.omega):
            z[dofs] += self.local_solve(s, r[dofs])
        if self.n0:
            c = self.coarse.Phi.T @ r
            y = sla.cho_solve(self.A0fac, c)
            z += self.coarse.Phi @ y
        return z

    def spmv(self, x: np.ndarray) -> np.ndarray:
        return self.Asp @ x


# ----------------------------------------------------------------------------
# Krylov solvers (textbook recurrences)
# ----------------------------------------------------------------------------

@dataclass
class SolveInfo:
    iters: int
    relres: float            # true ||b - A x|| / ||b|| at exit
    converged: bool


def pcg(A_mv, M_apply, b, x0=None, tol=1e-8, maxit=2000, flexible=False):
    """Preconditioned conjugate gradients.

    x0 = 0 unless given; r = b - A x0; z = M r; p = z.  Each iteration:
    q = A p, alpha = (r,z)/(p,q), x += alpha p, r -= alpha q; stop when
    ||r|| <= tol ||b||; z = M r; beta = (r,z)/(r_old,z_old) (or the flexible
    (r, z - z_old)/(r_old, z_old)); p = z + beta p.  At a stop the true
    residual b - A x is recomputed and the iteration continues from it if it
    is not below tol.  The count is the number of products with A after the
    initial residual.
    """
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    if nb == 0.0:
        return np.zeros_like(b), SolveInfo(0, 0.0, True)
    r = b - A_mv(x)
    if np.linalg.norm(r) <= tol * nb:
        return x, SolveInfo(0, np.linalg.norm(r) / nb, True)
    z = M_apply(r)
    p = z.copy()
    rz = r @ z
    it = 0
    while it < maxit:
        q = A_mv(p)
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        if np.linalg.norm(r) <= tol * nb:
            r = b - A_mv(x)
            if np.linalg.norm(r) <= tol * nb:
                return x, SolveInfo(it, np.linalg.norm(r) / nb, True)
        z_old = z
        z = M_apply(r)
        rz_new = (r @ (z - z_old)) if flexible else (r @ z)
        beta = rz_new / rz
        rz = r @ z
        p = z + beta * p
    rtrue = b - A_mv(x)
    return x, SolveInfo(it, np.linalg.norm(rtrue) / nb, False)


def gmres(A_mv, M_apply, b, x0=None, tol=1e-8, restart=30, maxit=2000):
    """Right-preconditioned restarted GMRES(m) with modified Gram-Schmidt and
    Givens rotations; the monitored quantity is the unpreconditioned residual
    |g_{j+1}|, stop when <= tol ||b||; the true residual is recomputed at
    every restart and at exit.  The count is the number of Arnoldi steps."""
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    if nb == 0.0:
        return np.zeros_like(b), SolveInfo(0, 0.0, True)
    it = 0
    while True:
        r = b - A_mv(x)
        beta = np.linalg.norm(r)
        if beta <= tol * nb or it >= maxit:
            return x, SolveInfo(it, beta / nb, beta <= tol * nb)
        m = restart
        V = np.zeros((m + 1, len(b)))
        Zs = np.zeros((m, len(b)))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            Zs[j] = M_apply(V[j])
            w = A_mv(Zs[j])
            for i in range(j + 1):
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            it += 1
            j_done = j + 1
            if abs(g[j + 1]) <= tol * nb or it >= maxit:
                break
        y = sla.solve_triangular(H[:j_done, :j_done], g[:j_done])
        x = x + Zs[:j_done].T @ y
