"""The level-scheduled local solve from node programs (Sec. V-B2 substitution with the
ILU(0) and IC(0) factors of Sec. V-B3 on elasticity, three unknowns per node; 2, 4 or 8 lanes
per node sum the couplings of the node's three rows to other nodes at once, then one
lane solves the three rows in order; 256 or 512 threads): forced by shape, it stays within the FP32
tolerance of the oracle and of the record-streaming kernel, with pieces split inside
a level as well as whole, solves GMRES with the oracle's iteration count, is not
used outside its scope, and its bounded wait for a withheld piece reports a
timeout and leaves the context usable."""
import os

import numpy as np
import pytest

from paper_2304_04876_b300 import problems as P
from tests.gpu_util import gpu_apply, gpu_handle, gpu_solve, oracle_for, relerr

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
    ("elast4_ilu0", lambda: P.elasticity_problem(4, 2), dict(local="ilu0")),
    ("elast6_ilu0", lambda: P.elasticity_problem(6, 2), dict(local="ilu0")),
    ("elast_ragged7_ilu0", lambda: P.elasticity_problem(7, 3), dict(local="ilu0")),
    ("elast6_overlap2", lambda: P.elasticity_problem(6, 3), dict(local="ilu0", overlap=2)),
    ("elast8_rgdsw", lambda: P.elasticity_problem(8, 4), dict(local="ilu0", coarse="rgdsw")),
    ("elast6_ic0", lambda: P.elasticity_problem(6, 2), dict(local="ic0")),
]


@pytest.mark.parametrize("split", [False, True], ids=["whole_levels", "split_levels"])
@pytest.mark.parametrize("name,make,opts", CASES, ids=[c[0] for c in CASES])
def test_node_programs_match_oracle_and_record_kernel(name, make, opts, split):
    prob = make()
    M = oracle_for(prob, **opts)
    hopts = {("local_solver" if k == "local" else k): v for k, v in opts.items()}
    rs = [np.random.default_rng(seed).uniform(-1, 1, prob.A.n) for seed in range(2)]
    h0 = handle_env(prob, {"GDSW_LOCAL_SHAPE": "4,256,0"}, precision="fp32", **hopts)
    assert h0.stats()["local_kernel"] == 3
    base = [gpu_apply(h0, r) for r in rs]
    h0.close()
    env = {"GDSW_LOCAL_SHAPE": "3,512,3"}
    if split:
        env["GDSW_NODE_PIECE_BYTES"] = "1024"     # a few nodes per piece
    for stages, nt, lanes in ((2, 512, 4), (3, 512, 8), (4, 256, 2), (6, 256, 4), (2, 256, 8)):
        env["GDSW_LOCAL_SHAPE"] = f"{stages},{nt},3,{lanes}"
        h = handle_env(prob, env, precision="fp32", **hopts)
        st = h.stats()
        assert st["local_kernel"] == 7 and st["local_stages"] == stages, (name, stages, st["local_kernel"])
        assert st["local_threads"] == nt
        for r, z0 in zip(rs, base):
            z = gpu_apply(h, r)
            assert relerr(z, M.apply(r)) <= 2e-5, (name, stages)
            assert relerr(z, z0) <= 2e-5, (name, stages)
            # every launch forms the same sums in the same order
            assert np.array_equal(gpu_apply(h, r), z)
        h.close()


@pytest.mark.parametrize("opts", [dict(local_solver="ilu0", precision="fp64"),
                                  dict(local_solver="ilu0", precision="fp16"),
                                  dict(local_solver="ilu0", precision="fp32", trsv="jacobi")])
def test_node_programs_not_used_outside_their_scope(opts):
    # FP64 or FP16 storage, Jacobi sweeps: no node programs, the shape request
    # leaves another kernel in place
    prob = P.elasticity_problem(6, 2)
    h = handle_env(prob, {"GDSW_LOCAL_SHAPE": "3,512,3"}, **opts)
    assert h.stats()["local_kernel"] != 7
    h.close()


def test_node_programs_not_built_for_one_unknown_per_node():
    prob = P.poisson_problem(12, 4)
    h = handle_env(prob, {"GDSW_LOCAL_SHAPE": "3,512,3"}, local_solver="ic0", precision="fp32")
    assert h.stats()["local_kernel"] != 7
    h.close()


def test_node_programs_gmres_matches_oracle():
    from oracle import gdsw_oracle as O
    prob = P.elasticity_problem(8, 4)
    h = handle_env(prob, {"GDSW_LOCAL_SHAPE": "3,512,3"}, local_solver="ilu0", krylov="gmres",
                   precision="fp32")
    assert h.stats()["local_kernel"] == 7
    M = oracle_for(prob, local="ilu0")
    x, info = gpu_solve(h, prob.b)
    _, io = O.gmres(M.spmv, M.apply, prob.b, tol=1e-8, restart=30)
    assert info.converged and info.true_relres <= 1e-8
    assert abs(info.iters - io.iters) <= 2, (info.iters, io.iters)
    h.close()


def test_node_programs_pcg_ic0_matches_oracle():
    """IC(0) factors (Sec. V-B3) on elasticity through the node programs: PCG within
    one iteration of the oracle's count and to the tolerance on the true residual."""
    from oracle import gdsw_oracle as O
    prob = P.elasticity_problem(8, 4)
    h = handle_env(prob, {"GDSW_LOCAL_SHAPE": "3,256,3,4"}, local_solver="ic0", precision="fp32")
    assert h.stats()["local_kernel"] == 7
    M = oracle_for(prob, local="ic0")
    x, info = gpu_solve(h, prob.b)
    _, io = O.pcg(M.spmv, M.apply, prob.b)
    assert info.converged and info.true_relres <= 1e-8
    assert abs(info.iters - io.iters) <= 1, (info.iters, io.iters)
    h.close()


def test_node_programs_wait_that_runs_out_reports_timeout(monkeypatch):
    """GDSW_TEST_STALL=1 withholds the first piece of CTA 0: every thread's bounded
    wait for it runs out (about 10 ms), the issuing thread lets its other copies land, the
    kernel returns without writing z, the host reports GDSW_ERR_TIMEOUT, and a handle
    without the stall then computes normally on the same context."""
    from paper_2304_04876_b300 import gdsw as G
    import torch
    prob = P.elasticity_problem(6, 2)
    monkeypatch.setenv("GDSW_TEST_STALL", "1")
    h = handle_env(prob, {"GDSW_LOCAL_SHAPE": "3,512,3"}, local_solver="ilu0", precision="fp32",
                   wait_budget_cycles=20_000_000)
    monkeypatch.delenv("GDSW_TEST_STALL")
    assert h.stats()["local_kernel"] == 7
    r = np.random.default_rng(0).uniform(-1, 1, prob.A.n)
    rt = torch.tensor(r, dtype=torch.float64, device="cuda")
    with pytest.raises(G.GdswError) as e:
        h.apply_timed(rt, torch.empty_like(rt))
    assert e.value.status == G.ERR_TIMEOUT
    h.close()
    M = oracle_for(prob, local="ilu0")
    h2 = handle_env(prob, {"GDSW_LOCAL_SHAPE": "3,512,3"}, local_solver="ilu0", precision="fp32")
    assert relerr(gpu_apply(h2, r), M.apply(r)) <= 2e-5
    h2.close()


def test_node_programs_in_a_batched_handle():
    """A batched FP32 handle of elasticity members (three unknowns per node) takes the
    node programs; a member that has stopped is skipped (the per-subdomain gate), and
    every member converges with the iteration count of the record kernel (within one)
    and a solution within 1e-6."""
    import torch
    from paper_2304_04876_b300 import gdsw as G
    mem = [P.elasticity_problem(4, 2), P.elasticity_problem(6, 2), P.elasticity_problem(6, 3)]
    b = np.concatenate([m.b for m in mem])
    out = {}
    for shape, kernel in (("4,256,0", 3), ("3,256,3,4", 7)):
        old = os.environ.get("GDSW_LOCAL_SHAPE")
        os.environ["GDSW_LOCAL_SHAPE"] = shape
        try:
            h = G.Handle.batch([(m.A, m.part, None if m.Z is None or m.Z.shape[1] == 1 else m.Z) for m in mem],
                               local_solver="ilu0", precision="fp32")
        finally:
            if old is None:
                os.environ.pop("GDSW_LOCAL_SHAPE")
            else:
                os.environ["GDSW_LOCAL_SHAPE"] = old
        assert h.stats()["local_kernel"] == kernel, shape
        bt = torch.tensor(b, dtype=torch.float64, device="cuda")
        xt = torch.zeros_like(bt)
        infos = h.solve_batch(bt, xt)
        torch.cuda.synchronize()
        assert all(i.converged and i.true_relres <= 1e-8 for i in infos), shape
        out[shape] = (xt.cpu().numpy(), [i.iters for i in infos])
        h.close()
    (x0, it0), (x1, it1) = out["4,256,0"], out["3,256,3,4"]
    assert all(abs(a - c) <= 1 for a, c in zip(it0, it1)), (it0, it1)
    assert relerr(x1, x0) <= 1e-6

