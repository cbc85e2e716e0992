"""Seeded synthetic inputs for the GDSW-preconditioned Krylov solve.

This module only builds inputs: sparse matrices, right-hand sides, the
structured partition (separator planes) and null-space matrices.  It holds
none of the preconditioner's arithmetic, so both the CUDA path and the CPU
oracle can take their inputs from here.

The paper never specifies its elasticity problem (Sec. VII), so the problems
follow the readings recorded in the design notes:

* Poisson: 7-point stencil on an n^3 grid of interior nodes, Dirichlet values
  eliminated, diagonal 6 and off-diagonals -1 (h^2 dropped), x-fastest order.
* Diffusion: cell-centred 7-point finite volumes, face weight = harmonic mean
  2 ka kb / (ka + kb), Dirichlet boundary face weight 2 k_cell,
  k = 10^U(-2, 2) per cell.
* Elasticity: unit cube, trilinear Q1 hexahedra with 2x2x2 Gauss quadrature,
  E = 1, nu = 0.3, nodes on x = 0 clamped (eliminated), uniform body force
  (0, 0, -1), degrees of freedom interleaved per node.

Every matrix is returned as CSR with int32 row pointers / column indices and
float64 values, columns sorted within each row.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np
import scipy.sparse as sp


@dataclass
class CSR:
    """A square sparse matrix in CSR form (int32 indices, float64 values)."""

    n: int
    rowptr: np.ndarray
    colind: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_scipy(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.val, self.colind, self.rowptr), shape=(self.n, self.n))

    @staticmethod
    def from_scipy(m) -> "CSR":
        m = sp.csr_matrix(m)
        m.sort_indices()
        return CSR(m.shape[0], m.indptr.astype(np.int32), m.indices.astype(np.int32),
                   m.data.astype(np.float64))


@dataclass
class Partition:
    """Structured nonoverlapping decomposition of a node grid.

    Unknown ``d`` of node ``(i, j, k)`` has index ``d + dpn*(i + nx*(j + ny*k))``.
    ``cuts[a]`` lists, in ascending order, the separator node planes along axis
    ``a``; a plane belongs to the block below it, so block ``b`` along an axis
    spans ``(cuts[b-1], cuts[b]]``.
    """

    nx: int
    ny: int
    nz: int
    dpn: int
    cuts: List[List[int]] = field(default_factory=lambda: [[], [], []])

    @property
    def n_nodes(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n(self) -> int:
        return self.dpn * self.n_nodes

    @property
    def n_sub(self) -> int:
        return (len(self.cuts[0]) + 1) * (len(self.cuts[1]) + 1) * (len(self.cuts[2]) + 1)


@dataclass
class Problem:
    name: str
    A: CSR
    part: Partition
    Z: np.ndarray                 # n x nn null-space columns (column-major use)
    b: Optional[np.ndarray] = None
    coords: Optional[np.ndarray] = None


def uniform_cuts(n: int, s: int) -> List[int]:
    """Separator planes for blocks of ``s`` nodes: i = s-1, 2s-1, ... below n-1."""
    return [i for i in range(s - 1, n - 1, s)]


def rhs_uniform(n: int, seed: int) -> np.ndarray:
    """Right-hand side with entries uniform in [-1, 1) from ``seed`` (FP64)."""
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


def _sorted_csr(m) -> CSR:
    return CSR.from_scipy(m)


def poisson7(n: int, ny: Optional[int] = None, nz: Optional[int] = None) -> CSR:
    """7-point Laplacian on an nx*ny*nz grid of interior nodes (diag 6, off -1)."""
    nx = n
    ny = n if ny is None else ny
    nz = n if nz is None else nz

    def lap1(m):
        return sp.diags([-np.ones(m - 1), np.zeros(m), -np.ones(m - 1)], [-1, 0, 1])

    Ix, Iy, Iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    off = (sp.kron(Iz, sp.kron(Iy, lap1(nx))) + sp.kron(Iz, sp.kron(lap1(ny), Ix))
           + sp.kron(lap1(nz), sp.kron(Iy, Ix)))
    A = off + 6.0 * sp.identity(nx * ny * nz)
    return _sorted_csr(A.tocsr())


def diffusion7(kcell: np.ndarray) -> CSR:
    """Cell-centred 7-point diffusion with harmonic-mean face weights.

    ``kcell`` has shape (nz, ny, nx); cell (i, j, k) is unknown i + nx*(j + ny*k).
    A boundary face (Dirichlet) has weight 2*k_cell.
    """
    nz, ny, nx = kcell.shape
    k = kcell.reshape(-1)
    N = k.size
    idx = np.arange(N).reshape(nz, ny, nx)
    diag = np.zeros(N)
    rows, cols, vals = [], [], []
    for axis in (2, 1, 0):          # x, y, z neighbours
        a = np.moveaxis(idx, axis, 0)
        kk = np.moveaxis(kcell, axis, 0)
        lo, hi = a[:-1].reshape(-1), a[1:].reshape(-1)
        klo, khi = kk[:-1].reshape(-1), kk[1:].reshape(-1)
        w = 2.0 * klo * khi / (klo + khi)
        np.add.at(diag, lo, w)
        np.add.at(diag, hi, w)
        rows += [lo, hi]
        cols += [hi, lo]
        vals += [-w, -w]
        # the two boundary layers along this axis
        first, last = a[0].reshape(-1), a[-1].reshape(-1)
        np.add.at(diag, first, 2.0 * kk[0].reshape(-1))
        np.add.at(diag, last, 2.0 * kk[-1].reshape(-1))
    rows.append(np.arange(N))
    cols.append(np.arange(N))
    vals.append(diag)
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(N, N))
    return _sorted_csr(A)


def _q1_element_stiffness(h: float, E: float, nu: float) -> np.ndarray:
    """24x24 stiffness of a cube Q1 element of side h, 2x2x2 Gauss quadrature.

    Local node a = ax + 2*ay + 4*az with (ax, ay, az) in {0,1}^3; dof 3*a + d.
    """
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[0, 0] = D[1, 1] = D[2, 2] = lam + 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    g = 1.0 / np.sqrt(3.0)
    corners = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)], dtype=float)
    sgn = 2 * corners - 1                    # -1 / +1 per axis
    Ke = np.zeros((24, 24))
    detJ = (h / 2) ** 3
    for gp in np.array(np.meshgrid([-g, g], [-g, g], [-g, g], indexing="ij")).reshape(3, -1).T:
        # dN/dxi for the 8 shape functions N = prod (1 + s xi)/2
        f = (1 + sgn * gp) / 2                 # (8, 3)
        dN = np.empty((8, 3))
        dN[:, 0] = sgn[:, 0] / 2 * f[:, 1] * f[:, 2]
        dN[:, 1] = sgn[:, 1] / 2 * f[:, 0] * f[:, 2]
        dN[:, 2] = sgn[:, 2] / 2 * f[:, 0] * f[:, 1]
        dN *= 2.0 / h                           # d/dx = (2/h) d/dxi
        B = np.zeros((6, 24))
        for a in range(8):
            x, y, z = dN[a]
            c = 3 * a
            B[0, c] = x
            B[1, c + 1] = y
            B[2, c + 2] = z
            B[3, c] = y; B[3, c + 1] = x
            B[4, c + 1] = z; B[4, c + 2] = y
            B[5, c] = z; B[5, c + 2] = x
        Ke += B.T @ D @ B * detJ
    return Ke


def elasticity_q1(ne: int, E: float = 1.0, nu: float = 0.3,
                  force=(0.0, 0.0, -1.0)) -> Problem:
    """Q1 linear elasticity on the unit cube with ne^3 elements, clamped at x = 0.

    Free nodes are (i, j, k) with i = 1..ne (i = 0 is clamped) and j, k = 0..ne;
    they are numbered i' + nx*(j + ny*k) with i' = i - 1, nx = ne, ny = nz = ne+1.
    Every node pair sharing an element stores a full 3x3 block (explicit zeros
    kept), as finite-element assembly does.
    """
    h = 1.0 / ne
    Ke = _q1_element_stiffness(h, E, nu)
    nn1 = ne + 1
    # block stencil: blocks[node, offset(27), 3, 3] on the full (ne+1)^3 node grid
    nfull = nn1 ** 3
    blocks = np.zeros((nfull, 27, 3, 3))
    ex = np.arange(ne)
    EX, EY, EZ = np.meshgrid(ex, ex, ex, indexing="ij")
    EX, EY, EZ = EX.ravel(), EY.ravel(), EZ.ravel()
    corner = [(a & 1, (a >> 1) & 1, (a >> 2) & 1) for a in range(8)]
    for a in range(8):
        ua = (EX + corner[a][0]) + nn1 * ((EY + corner[a][1]) + nn1 * (EZ + corner[a][2]))
        for b in range(8):
            d = [corner[b][t] - corner[a][t] for t in range(3)]
            off = (d[0] + 1) + 3 * ((d[1] + 1) + 3 * (d[2] + 1))
            blocks[ua, off] += Ke[3 * a:3 * a + 3, 3 * b:3 * b + 3]
    # free-node numbering
    nx, ny, nz = ne, nn1, nn1
    nfree = nx * ny * nz
    fr = np.arange(nfree)
    fi, fj, fk = fr % nx + 1, (fr // nx) % ny, fr // (nx * ny)
    ufull = fi + nn1 * (fj + nn1 * fk)
    # neighbour offsets in (dz, dy, dx) order give ascending neighbour ids, so the
    # rows come out sorted: row (u, p) lists, per valid offset, the 3 dofs q of v
    offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    valid = np.empty((nfree, 27), dtype=bool)
    vid = np.empty((nfree, 27), dtype=np.int64)
    for t, (dx, dy, dz) in enumerate(offs):
        vi, vj, vk = fi + dx, fj + dy, fk + dz
        valid[:, t] = (vi >= 1) & (vi <= ne) & (vj >= 0) & (vj <= ne) & (vk >= 0) & (vk <= ne)
        vid[:, t] = (vi - 1) + nx * (vj + ny * vk)
    off_idx = np.array([(dx + 1) + 3 * ((dy + 1) + 3 * (dz + 1)) for dx, dy, dz in offs])
    blk = blocks[ufull][:, off_idx]                      # (nfree, 27, 3, 3) in offset order
    del blocks
    vals4 = np.transpose(blk, (0, 2, 1, 3))             # (u, p, offset, q)
    cols4 = 3 * vid[:, None, :, None] + np.arange(3)[None, None, None, :]
    mask4 = np.broadcast_to(valid[:, None, :, None], vals4.shape)
    vals = vals4[mask4]
    cols = np.broadcast_to(cols4, vals4.shape)[mask4]
    n = 3 * nfree
    per_row = np.repeat(3 * valid.sum(axis=1), 3)
    rowptr = np.concatenate([[0], np.cumsum(per_row)])
    A = CSR(n, rowptr.astype(np.int32), cols.astype(np.int32), vals.astype(np.float64))
    # consistent load of a uniform body force: h^3/8 per element corner
    load = np.zeros((nfull, 3))
    for a in range(8):
        ua = (EX + corner[a][0]) + nn1 * ((EY + corner[a][1]) + nn1 * (EZ + corner[a][2]))
        np.add.at(load, ua, np.asarray(force) * h ** 3 / 8.0)
    b = load[ufull].reshape(-1)
    coords = np.stack([fi * h, fj * h, fk * h], axis=1)
    Z = rigid_body_modes(coords)
    part = Partition(nx, ny, nz, 3, [[], [], []])
    return Problem(f"elasticity_q1_{ne}", A, part, Z, b, coords)


def rigid_body_modes(coords: np.ndarray) -> np.ndarray:
    """Three translations and three linearised rotations at the given node coordinates.

    Rotations: (0, -z, y), (z, 0, -x), (-y, x, 0); dofs interleaved per node.
    """
    m = coords.shape[0]
    x, y, z = coords[:, 0], coords[:, 1], coords[:, 2]
    Z = np.zeros((3 * m, 6))
    for d in range(3):
        Z[d::3, d] = 1.0
    Z[1::3, 3] = -z; Z[2::3, 3] = y
    Z[0::3, 4] = z; Z[2::3, 4] = -x
    Z[0::3, 5] = -y; Z[1::3, 5] = x
    return Z


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def poisson_problem(n: int, s: int, seed: int = 0) -> Problem:
    """Poisson 7-point on n^3 with cubic subdomains of s nodes per axis."""
    A = poisson7(n)
    cuts = uniform_cuts(n, s)
    part = Partition(n, n, n, 1, [list(cuts), list(cuts), list(cuts)])
    return Problem(f"poisson_{n}_s{s}", A, part, np.ones((A.n, 1)), rhs_uniform(A.n, seed))


def elasticity_problem(ne: int = 48, se: int = 12) -> Problem:
    """Q1 elasticity, ne^3 elements, subdomains of se^3 elements (planes every se nodes)."""
    prob = elasticity_q1(ne)
    full_planes = [i for i in range(se, ne, se)]          # node indices on the full grid
    cx = [i - 1 for i in full_planes]                      # x is shifted by the clamp
    prob.part.cuts = [cx, list(full_planes), list(full_planes)]
    return prob


def diffusion_batch(count: int = 256, seed: int = 0, nmin: int = 16, nmax: int = 64,
                    smin: int = 8, smax: int = 16) -> List[Problem]:
    """Independent heterogeneous diffusion problems with seeded sizes and coefficients."""
    rng = np.random.default_rng(seed)
    out = []
    for p in range(count):
        n = int(rng.integers(nmin, nmax + 1))
        s = int(rng.integers(smin, smax + 1))
        kcell = 10.0 ** rng.uniform(-2.0, 2.0, size=(n, n, n))
        A = diffusion7(kcell)
        cuts = uniform_cuts(n, s)
        part = Partition(n, n, n, 1, [list(cuts), list(cuts), list(cuts)])
        b = rng.uniform(-1.0, 1.0, A.n)
        out.append(Problem(f"diffusion_{p}_n{n}_s{s}", A, part, np.ones((A.n, 1)), b))
    return out


def serving_pool(count: int = 8, seed: int = 0, dofs_min: int = 32 ** 3, dofs_max: int = 160 ** 3,
                 poisson_sub: int = 16, elasticity_sub: int = 12) -> List[Problem]:
    """Half Poisson 7-point, half Q1 elasticity, total unknowns log-uniform in
    [dofs_min, dofs_max]: Poisson edge cbrt(N) with subdomains of poisson_sub nodes
    per axis, elasticity element edge cbrt(N/3) - 1 with subdomains of
    elasticity_sub elements per axis."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = float(np.exp(rng.uniform(np.log(dofs_min), np.log(dofs_max))))
        if i % 2 == 0:
            n = max(4, int(round(N ** (1.0 / 3.0))))
            prob = poisson_problem(n, min(poisson_sub, n), seed=seed * 1000 + i)
        else:
            ne = max(2, int(round((N / 3.0) ** (1.0 / 3.0) - 1)))
            prob = elasticity_problem(ne, min(elasticity_sub, ne))
        prob.name = f"{prob.name}_pool{i}"
        out.append(prob)
    return out


def config_problem(cfg: int, seed: int = 0) -> Problem:
    """The fixed workloads: 1 = Poisson 16^3 / 2^3 subdomains, 2 = Poisson 128^3 / 8^3,
    3 = Q1 elasticity 48^3 elements / 4^3 subdomains."""
    if cfg == 1:
        return poisson_problem(16, 8, seed)
    if cfg == 2:
        return poisson_problem(128, 16, seed)
    if cfg == 3:
        return elasticity_problem(48, 12)
    raise ValueError(cfg)
