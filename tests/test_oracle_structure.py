"""Pins of the oracle's decomposition (Sec. III, Fig. 1) and overlap (Sec. VII).

Expected sizes are closed forms worked out by hand in tests/golden/structure_counts.json.
"""
import json
import os

import numpy as np
import pytest

from oracle import gdsw_oracle as O
from paper_2304_04876_b300 import problems as P

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "structure_counts.json")))


def _check_counts(prob, g, dpn=1):
    dec = O.decompose(prob.part)
    omega = O.overlapping_subdomains(prob.A, prob.part, dec, 1)
    assert dec.n_sub == g["n_sub"]
    assert int(dec.node_gamma.sum()) == g["gamma_nodes"]
    types = np.bincount(dec.comp_type, minlength=4)
    assert (types[1], types[2], types[3]) == (g["faces"], g["edges"], g["vertices"])
    ni = [len(x) * dpn for x in dec.sub_interior_nodes]
    return dec, omega, ni


def test_counts_poisson_16():
    g = GOLD["poisson_16_s8"]
    prob = P.config_problem(1)
    dec, omega, ni = _check_counts(prob, g)
    assert (min(ni), max(ni)) == (g["interior_min"], g["interior_max"])
    assert sum(len(o) for o in omega) == g["sum_omega"]
    assert max(len(o) for o in omega) == g["max_omega"]
    cs = O.coarse_space(prob.A, prob.part, dec, prob.Z)
    assert cs.n0 == g["n0_constants"]


def test_counts_poisson_128():
    g = GOLD["poisson_128_s16"]
    prob = P.poisson_problem(128, 16)
    dec, omega, ni = _check_counts(prob, g)
    assert (min(ni), max(ni)) == (g["interior_min"], g["interior_max"])
    assert sum(len(o) for o in omega) == g["sum_omega"]
    assert max(len(o) for o in omega) == g["max_omega"]


def test_counts_elasticity_48():
    g = GOLD["elasticity_48_se12"]
    prob = P.elasticity_problem(48, 12)
    dec, omega, ni = _check_counts(prob, g, dpn=3)
    assert (min(ni), max(ni)) == (g["interior_min_dofs"], g["interior_max_dofs"])
    assert sum(3 * len(o) for o in omega) == g["sum_omega_dofs"]
    # ranks of the rigid-body modes per component type: 6 / 5 / 3
    n0 = 0
    for nodes, t in zip(dec.comp_nodes, dec.comp_type):
        k = O.mgs_basis(prob.Z[O.node_dofs(nodes, 3)]).shape[1]
        assert k == {1: 6, 2: 5, 3: 3}[int(t)]
        n0 += k
    assert n0 == g["n0_rbm"]


@pytest.mark.parametrize("n,s", [(9, 3), (10, 4), (7, 7), (12, 5)])
def test_partition_invariants(n, s):
    prob = P.poisson_problem(n, s)
    dec = O.decompose(prob.part)
    # components are disjoint and cover Gamma exactly
    allc = np.concatenate(dec.comp_nodes) if dec.comp_nodes else np.zeros(0, int)
    assert len(allc) == len(np.unique(allc)) == int(dec.node_gamma.sum())
    assert np.all(dec.node_gamma[allc])
    # interiors + Gamma partition all nodes
    alli = np.concatenate(dec.sub_interior_nodes)
    assert len(alli) + len(allc) == prob.part.n_nodes
    assert not np.any(dec.node_gamma[alli])
    # every component is a connected box: extent along each axis = number of distinct coordinates
    nx = prob.part.nx
    for nodes in dec.comp_nodes:
        I, J, K = nodes % nx, (nodes // nx) % nx, nodes // (nx * nx)
        ext = [(c.max() - c.min() + 1) for c in (I, J, K)]
        assert np.prod(ext) == len(nodes)


def test_interior_block_diagonal():
    """A_II is block diagonal over subdomain interiors (Sec. III), for 7- and 27-point couplings."""
    for prob in (P.poisson_problem(12, 4), P.elasticity_problem(6, 2)):
        dec = O.decompose(prob.part)
        dpn = prob.part.dpn
        sub_of_dof = np.repeat(np.where(dec.node_gamma, -1, dec.node_sub), dpn)
        rows = np.repeat(np.arange(prob.A.n), np.diff(prob.A.rowptr))
        a, b = sub_of_dof[rows], sub_of_dof[prob.A.colind]
        both = (a >= 0) & (b >= 0)
        assert np.all(a[both] == b[both])


def test_overlap_closed_forms():
    # 7-point: block plus one s^2 slab per neighbouring block face
    prob = P.poisson_problem(12, 4)
    dec = O.decompose(prob.part)
    om = O.overlapping_subdomains(prob.A, prob.part, dec, 1)
    for s, nodes in enumerate(om):
        bx, by, bz = s % 3, (s // 3) % 3, s // 9
        nbr = sum(1 for b in (bx, by, bz) for d in (-1, 1) if 0 <= b + d < 3)
        assert len(nodes) == 64 + 16 * nbr
        assert set(dec.sub_nodes[s]).issubset(set(nodes))
    # two layers of overlap on the 7-point graph: block plus slabs at distance <= 2
    om2 = O.overlapping_subdomains(prob.A, prob.part, dec, 2)
    centre = 13
    # |{v : L1 distance from the 4^3 box <= 2}| = 64 + 6*2*16 + 12*(1)*4 (edge-adjacent at distance 2)
    assert len(om2[centre]) == 64 + 6 * 2 * 16 + 12 * 4
    # 27-point (Q1): box grown by one node per side
    prob = P.elasticity_problem(6, 2)
    dec = O.decompose(prob.part)
    om = O.overlapping_subdomains(prob.A, prob.part, dec, 1)
    nx, ny = prob.part.nx, prob.part.ny
    for s, nodes in enumerate(om):
        blk = dec.sub_nodes[s]
        lo = [c(blk).min() for c in (lambda u: u % nx, lambda u: (u // nx) % ny, lambda u: u // (nx * ny))]
        hi = [c(blk).max() for c in (lambda u: u % nx, lambda u: (u // nx) % ny, lambda u: u // (nx * ny))]
        dims = (prob.part.nx, prob.part.ny, prob.part.nz)
        ext = [min(hi[a] + 1, dims[a] - 1) - max(lo[a] - 1, 0) + 1 for a in range(3)]
        assert len(nodes) == int(np.prod(ext))
