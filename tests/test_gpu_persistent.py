"""PCG as one persistent cooperative kernel (Sec. II's PCG around Eq. 1, for small
problems with dense exact local solves; opt-in with GDSW_PERSISTENT=1): the
iteration count and solution agree with the graph-launched loop (the same steps,
reductions summed in another fixed order), the solve meets the tolerance, the result is deterministic, the iteration
limit is honoured, and a grid barrier that never completes is reported as a timeout
with the context still usable."""
import os

import numpy as np
import pytest

from oracle import gdsw_oracle as O
from paper_2304_04876_b300 import problems as P
from tests.gpu_util import gpu_handle, gpu_solve, oracle_for, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2304_04876_b300 import build
    build.build()
    assert torch.cuda.is_available()


def handle_env(prob, env, **opts):
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        return gpu_handle(prob, **opts)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k)
            else:
                os.environ[k] = v


CASES = [
    ("poisson16_s8", lambda: P.poisson_problem(16, 8)),
    ("poisson12_s4", lambda: P.poisson_problem(12, 4)),
    ("ragged11_s4", lambda: P.poisson_problem(11, 4, seed=3)),
    ("poisson9_s3", lambda: P.poisson_problem(9, 3)),
]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-6)])
@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_persistent_pcg_matches_graph_loop(name, make, precision, tol):
    prob = make()
    hp = handle_env(prob, {"GDSW_PERSISTENT": "1"}, local_solver="exact", precision=precision)
    assert hp.stats()["pcg_persistent_grid"] > 0, name
    hg = gpu_handle(prob, local_solver="exact", precision=precision)
    assert hg.stats()["pcg_persistent_grid"] == 0
    xp, ip = gpu_solve(hp, prob.b)
    xg, ig = gpu_solve(hg, prob.b)
    assert ip.converged and ip.true_relres <= 1e-8
    assert abs(ip.iters - ig.iters) <= 1
    assert relerr(xp, xg) <= tol
    if precision == "fp64":
        M = oracle_for(prob, local="exact")
        _, io = O.pcg(M.spmv, M.apply, prob.b)
        assert abs(ip.iters - io.iters) <= 1
    x2, i2 = gpu_solve(hp, prob.b)
    assert i2.iters == ip.iters and np.array_equal(x2, xp)
    hp.close()
    hg.close()


def test_persistent_pcg_stops_at_maxit():
    prob = P.poisson_problem(12, 4)
    h = handle_env(prob, {"GDSW_PERSISTENT": "1"}, local_solver="exact", maxit=3)
    assert h.stats()["pcg_persistent_grid"] > 0
    import torch
    from paper_2304_04876_b300 import gdsw as G
    b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(G.GdswError) as e:
        h.solve(b, x)
    assert e.value.status == G.ERR_NOT_CONVERGED
    h.close()


def test_persistent_grid_barrier_that_runs_out_reports_timeout():
    """GDSW_TEST_STALL=1: CTA 0 withholds its first barrier arrival, every CTA's
    bounded wait runs out (about 10 ms), the kernel returns, the host reports
    GDSW_ERR_TIMEOUT; a handle without the stall then solves on the same context."""
    import torch
    from paper_2304_04876_b300 import gdsw as G
    prob = P.poisson_problem(12, 4)
    h = handle_env(prob, {"GDSW_TEST_STALL": "1", "GDSW_PERSISTENT": "1"}, local_solver="exact",
                   wait_budget_cycles=20_000_000)
    assert h.stats()["pcg_persistent_grid"] > 0
    b = torch.tensor(prob.b, dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    with pytest.raises(G.GdswError) as e:
        h.solve(b, x)
    assert e.value.status == G.ERR_TIMEOUT
    h.close()
    h2 = gpu_handle(prob, local_solver="exact")
    _, info = gpu_solve(h2, prob.b)
    assert info.converged and info.true_relres <= 1e-8
    h2.close()
