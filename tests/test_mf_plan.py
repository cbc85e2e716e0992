"""Host symbolic phase of the multifrontal exact local solver (gdsw_mf_plan_export), on
the CPU: the nested-dissection order, the supernode tree and the fronts S u B(S),
checked against the exact Cholesky factor of A_s (LAPACK, in that order) and against
the oracle's overlapping subdomain (Sec. III / VII overlap).  Every nonzero of the
factor must lie inside the planned fronts, which is what makes the device
factorisation exact."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import gdsw_oracle as O
from paper_2304_04876_b300 import gdsw as G
from paper_2304_04876_b300 import problems as P

CASES = [
    ("poisson12", lambda: P.poisson_problem(12, 4)),
    ("ragged13", lambda: P.poisson_problem(13, 4, seed=3)),
    ("one_subdomain", lambda: P.poisson_problem(7, 7)),
    ("elasticity6", lambda: P.elasticity_problem(6, 2)),
    ("elasticity_ragged7", lambda: P.elasticity_problem(7, 3)),
]


@pytest.fixture(scope="module")
def lib():
    from paper_2304_04876_b300 import build
    build.build()
    return G.load()


def _check_plan(prob, q, plan, omega):
    nd, sn_ptr, parent = plan["nd_dof"], plan["sn_ptr"], plan["parent"]
    b_ptr, b_pos = plan["b_ptr"], plan["b_pos"]
    m, nsn = len(nd), len(parent)
    # the ordering is a permutation of the oracle's overlapping subdomain
    assert m == len(omega) and set(nd.tolist()) == set(np.asarray(omega).tolist())
    assert sn_ptr[0] == 0 and sn_ptr[-1] == m and np.all(np.diff(sn_ptr) > 0)
    last = sn_ptr[1:] - 1
    B = [b_pos[b_ptr[s]:b_ptr[s + 1]] for s in range(nsn)]
    for s in range(nsn):
        # postorder; B(S) ascending, above S; a root has no B
        assert np.all(np.diff(B[s]) > 0) and (len(B[s]) == 0 or B[s][0] > last[s])
        if parent[s] < 0:
            assert len(B[s]) == 0
            continue
        p = parent[s]
        assert p > s
        front_p = set(range(sn_ptr[p], sn_ptr[p + 1])) | set(B[p].tolist())
        assert set(B[s].tolist()) <= front_p, s      # extend-add lands in the parent's front
    # the exact factor of A_s in this order stays inside the fronts
    As = prob.A.to_scipy()[nd][:, nd].toarray()
    L = sla.cholesky(As, lower=True)
    owner = np.searchsorted(sn_ptr, np.arange(m), side="right") - 1
    rows, cols = np.nonzero(np.tril(L, -1))
    for s in np.unique(owner[cols]):
        sel = owner[cols] == s
        allowed = np.zeros(m, bool)
        allowed[sn_ptr[s]:sn_ptr[s + 1]] = True
        allowed[B[s]] = True
        assert np.all(allowed[rows[sel]]), (q, s)
    # and the fronts are not grossly larger than the factor's pattern
    planned = sum((sn_ptr[s + 1] - sn_ptr[s]) * (sn_ptr[s + 1] - sn_ptr[s] + 1) // 2 +
                  (sn_ptr[s + 1] - sn_ptr[s]) * len(B[s]) for s in range(nsn))
    assert planned <= 3 * (len(rows) + m)


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_plan_fronts_hold_the_exact_factor(lib, name, make):
    prob = make()
    dec = O.decompose(prob.part)
    omegas = O.overlapping_subdomains(prob.A, prob.part, dec, 1)
    for q in sorted({0, len(omegas) // 2, len(omegas) - 1}):
        plan = G.mf_plan(prob.A, prob.part, q, local_solver="exact")
        _check_plan(prob, q, plan, O.node_dofs(omegas[q], prob.part.dpn))


def test_leaf_size_and_range_errors(lib, monkeypatch):
    """GDSW_MF_LEAF bounds the childless supernodes (whole nodes, so at most the leaf
    size); a subdomain index out of range is an invalid argument."""
    prob = P.poisson_problem(12, 4)
    monkeypatch.setenv("GDSW_MF_LEAF", "6")
    plan = G.mf_plan(prob.A, prob.part, 13, local_solver="exact")
    has_child = np.zeros(len(plan["parent"]), bool)
    has_child[plan["parent"][plan["parent"] >= 0]] = True
    sizes = np.diff(plan["sn_ptr"])
    assert sizes[~has_child].max() <= 6
    monkeypatch.setenv("GDSW_MF_LEAF", "1000")
    one = G.mf_plan(prob.A, prob.part, 13, local_solver="exact")
    assert len(one["parent"]) == 1 and len(one["b_pos"]) == 0      # a single dense front
    with pytest.raises(G.GdswError):
        G.mf_plan(prob.A, prob.part, 27, local_solver="exact")
