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
