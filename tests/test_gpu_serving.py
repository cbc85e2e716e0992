"""The serving loop on the GPU: requests on a mix of Poisson and elasticity problems
arrive while others run, and every result equals the same request solved alone
(FP64 path: bitwise target, 1e-12 relative accepted)."""
import numpy as np
import pytest

from paper_2304_04876_b300 import problems as P
from paper_2304_04876_b300 import serving as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2304_04876_b300 import build
    build.build()
    assert torch.cuda.is_available()


def test_results_same_alone_and_in_the_mix():
    from paper_2304_04876_b300 import gdsw as G
    pool = {p.name: p for p in [P.poisson_problem(12, 4), P.poisson_problem(16, 8),
                                P.elasticity_problem(6, 2), P.elasticity_problem(8, 4)]}
    keys = sorted(pool)

    def make(key, stream):
        pr = pool[key]
        return G.Handle(pr.A, pr.part, pr.Z if pr.part.dpn == 3 else None, stream=stream, local_solver="ic0")

    rng = np.random.default_rng(0)
    arrivals = S.poisson_arrivals(200.0, 24, seed=1)
    reqs = []
    for i, t in enumerate(arrivals):
        k = keys[int(rng.integers(len(keys)))]
        reqs.append(S.Request(float(t), i, k, P.rhs_uniform(pool[k].A.n, 100 + i)))
    srv = S.Server(make, lambda k: 64 << 20, budget_bytes=1 << 34, workers=3, keep_x=True)
    res = srv.run(reqs)
    srv.close()
    assert len(res) == len(reqs) and all(r.converged and r.true_relres <= 1e-8 for r in res)
    # every request again, alone, on a fresh handle
    for r in res[:12]:
        h = make(r.key, None)
        import torch
        b = torch.tensor(reqs[r.rid].b, dtype=torch.float64, device="cuda")
        x = torch.zeros_like(b)
        info = h.solve(b, x)
        xa = x.cpu().numpy()
        assert info.iters == r.iters
        err = np.linalg.norm(xa - r.x) / np.linalg.norm(xa)
        assert err <= 1e-12, (r.key, err)
        h.close()
    summ = S.summarize(res)
    assert summ["p99_ms"] >= summ["p50_ms"] > 0


# ---- continuous batching: members of batched handles as solve slots ----------

def _oracle_iters(prob, b):
    from oracle import gdsw_oracle as O
    M = O.GDSW(prob.A, prob.part, prob.Z if prob.part.dpn == 3 else None, local=O.IC0)
    _, io = O.pcg(M.spmv, M.apply, b)
    return io.iters


def _drive(h, starts, ns, iters_per_round=1):
    """Run members of batched handle h: starts = {round: [(member, b)]} (members join
    at the start of that round); returns {member: (x, info)} as each finishes."""
    import torch
    out = {}
    running = set()
    rnd = 0
    last_start = max(starts)
    while rnd <= last_start or running:
        for m, b in starts.get(rnd, []):
            h.batch_start(m, torch.tensor(b, dtype=torch.float64, device="cuda"))
            running.add(m)
        if running:
            h.batch_iterate(iters_per_round)
            done, _, _ = h.batch_status()
            for m in sorted(running):
                if done[m]:
                    x = torch.empty(ns[m], dtype=torch.float64, device="cuda")
                    info, cont = h.batch_finish(m, x)
                    if not cont:
                        running.discard(m)
                        out[m] = (x.cpu().numpy(), info)
        rnd += 1
        assert rnd < 5000
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_member_joining_midsolve_matches_alone_bitwise(precision):
    """Three Poisson problems of different sizes in one batched handle: each solved
    alone, then all three with the second and third joining while the first is
    mid-solve.  Every member's solution and iteration count are the same bit for bit;
    the FP64 path needs the oracle's iteration count (+-1) and reaches 1e-8."""
    from paper_2304_04876_b300 import gdsw as G
    probs = [P.poisson_problem(12, 4), P.poisson_problem(16, 8), P.poisson_problem(10, 5, seed=2)]
    h = G.Handle.batch([(p.A, p.part, None) for p in probs], local_solver="ic0", precision=precision)
    ns = [p.A.n for p in probs]
    bs = [P.rhs_uniform(p.A.n, 40 + i) for i, p in enumerate(probs)]
    alone = {}
    for m in range(3):
        alone.update(_drive(h, {0: [(m, bs[m])]}, ns))
    mixed = _drive(h, {0: [(0, bs[0])], 3: [(1, bs[1])], 5: [(2, bs[2])]}, ns)
    for m in range(3):
        xa, ia = alone[m]
        xm, im = mixed[m]
        assert ia.converged and im.converged and ia.true_relres <= 1e-8
        assert ia.iters == im.iters
        assert np.array_equal(xa, xm), m
        if precision == "fp64":
            assert abs(ia.iters - _oracle_iters(probs[m], bs[m])) <= 1
            res = np.linalg.norm(probs[m].A.to_scipy() @ xa - bs[m]) / np.linalg.norm(bs[m])
            assert res <= 1e-8
    h.close()


def test_member_restart_and_zero_rhs():
    """A member started again while running begins afresh (same result as a clean
    start); a zero right-hand side finishes at once with x = 0."""
    from paper_2304_04876_b300 import gdsw as G
    probs = [P.poisson_problem(12, 4), P.poisson_problem(12, 4, seed=5)]
    h = G.Handle.batch([(p.A, p.part, None) for p in probs], local_solver="ic0")
    ns = [p.A.n for p in probs]
    b = P.rhs_uniform(ns[0], 7)
    ref = _drive(h, {0: [(0, b)]}, ns)[0]
    again = _drive(h, {0: [(0, 0.5 * b)], 2: [(0, b)]}, ns)[0]
    assert np.array_equal(ref[0], again[0]) and ref[1].iters == again[1].iters
    z = _drive(h, {0: [(1, np.zeros(ns[1]))]}, ns)[1]
    assert z[1].converged and z[1].iters == 0 and not np.any(z[0])
    h.close()


def test_batch_server_mixed_kinds_same_alone_and_in_the_mix():
    """BatchServer over a Poisson pool and an elasticity pool (two slots for one
    problem): requests arriving while others run give the same solution and iteration
    count, bit for bit, as the same request served alone."""
    pool = {p.name: p for p in [P.poisson_problem(12, 4), P.poisson_problem(16, 8),
                                P.elasticity_problem(6, 2), P.elasticity_problem(8, 4)]}
    keys = sorted(pool)
    problems = {k: (pool[k].A, pool[k].part, pool[k].Z if pool[k].part.dpn == 3 else None) for k in keys}
    plan = S.plan_slots([(k, pool[k].part.dpn, 1) for k in keys] + [(keys[0], pool[keys[0]].part.dpn, 1)],
                        budget_bytes=100, max_copies=1)
    pools, slots = S.build_pools(problems, plan, local_solver="ic0")
    assert len(pools) == 2 and len(slots) == 5
    rng = np.random.default_rng(0)
    arrivals = S.poisson_arrivals(400.0, 20, seed=3)
    reqs = []
    for i, t in enumerate(arrivals):
        k = keys[int(rng.integers(len(keys)))]
        reqs.append(S.Request(float(t), i, k, P.rhs_uniform(pool[k].A.n, 200 + i)))
    srv = S.BatchServer(pools, slots, iterations=2, keep_x=True)
    res = srv.run(reqs)
    assert len(res) == len(reqs) and all(r.converged and r.true_relres <= 1e-8 for r in res)
    for r in res[:10]:
        alone = S.BatchServer(pools, slots, iterations=3, keep_x=True).run(
            [S.Request(0.0, r.rid, r.key, reqs[r.rid].b)])[0]
        assert alone.iters == r.iters and np.array_equal(alone.x, r.x), r.key
    summ = S.summarize(res)
    assert summ["p99_ms"] >= summ["p50_ms"] > 0
    for h in pools:
        h.close()
