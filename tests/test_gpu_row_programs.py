"""The level-scheduled local solve from row programs (Sec. V-B2 substitution with
the IC(0)/ILU(0) factors of Sec. V-B3; every thread copies its own rows several
steps ahead, one CTA barrier per level): forced by shape, it must compute the
same values as the record-streaming kernel bit for bit (the same FMAs in the same
order), stay within the FP32 tolerance of the oracle, give up on problems it does
not take (wider rows, FP64), solve PCG with the oracle's iteration count, and
work gated inside a batched handle.  The kernel has no spin-wait (its waits are
the hardware's wait for a thread's own copies and CTA barriers), so it has no
timeout path to test."""
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


def handle_with_shape(prob, shape, **opts):
    old = os.environ.get("GDSW_LOCAL_SHAPE")
    os.environ["GDSW_LOCAL_SHAPE"] = shape
    try:
        return gpu_handle(prob, **opts)
    finally:
        if old is None:
            os.environ.pop("GDSW_LOCAL_SHAPE")
        else:
            os.environ["GDSW_LOCAL_SHAPE"] = old


def _diffusion():
    k = 10 ** np.random.default_rng(7).uniform(-2, 2, (10, 10, 10))
    A = P.diffusion7(k)
    cuts = P.uniform_cuts(10, 4)
    part = P.Partition(10, 10, 10, 1, [cuts, cuts, cuts])
    return P.Problem("diff10", A, part, np.ones((A.n, 1)), P.rhs_uniform(A.n, 1))


CASES = [
    ("poisson12_ic0", lambda: P.poisson_problem(12, 4), dict(local="ic0")),
    ("poisson12_ilu0", lambda: P.poisson_problem(12, 4), dict(local="ilu0")),
    ("ragged13_ic0", lambda: P.poisson_problem(13, 4, seed=3), dict(local="ic0")),
    ("diffusion10_ic0", _diffusion, dict(local="ic0")),
    ("overlap2_ic0", lambda: P.poisson_problem(12, 4), dict(local="ic0", overlap=2)),
    ("tiny_subdomains_ilu0", lambda: P.poisson_problem(9, 3), dict(local="ilu0")),
    # levels of up to ~300 rows: several steps per level
    ("poisson24_wide_levels_ic0", lambda: P.poisson_problem(24, 12), dict(local="ic0")),
]


@pytest.mark.parametrize("name,make,opts", CASES, ids=[c[0] for c in CASES])
def test_row_programs_match_record_kernel_bitwise_and_oracle(name, make, opts):
    prob = make()
    M = oracle_for(prob, **opts)
    hopts = {("local_solver" if k == "local" else k): v for k, v in opts.items()}
    rs = [np.random.default_rng(seed).uniform(-1, 1, prob.A.n) for seed in range(2)]
    refs = [M.apply(r) for r in rs]
    h0 = handle_with_shape(prob, "4,128,0", precision="fp32", **hopts)
    assert h0.stats()["local_kernel"] == 3
    base = [gpu_apply(h0, r) for r in rs]
    h0.close()
    for depth in (4, 8, 12):
        h = handle_with_shape(prob, f"{depth},128,2", precision="fp32", **hopts)
        st = h.stats()
        assert st["local_kernel"] == 6 and st["local_stages"] == depth, (name, depth, st["local_kernel"])
        for r, ref, z0 in zip(rs, refs, base):
            z = gpu_apply(h, r)
            assert np.array_equal(z, z0), (name, depth)
            assert relerr(z, ref) <= 2e-5, (name, depth)
        h.close()


@pytest.mark.parametrize("opts", [dict(local_solver="ic0", fill_level=1, precision="fp32"),
                                  dict(local_solver="ic0", precision="fp64"),
                                  dict(local_solver="ic0", precision="fp16")])
def test_row_programs_not_used_outside_their_scope(opts):
    # rows wider than three entries (IC(1)), FP64 or FP16 storage: the shape
    # request falls back to the record kernel
    prob = P.poisson_problem(12, 4)
    h = handle_with_shape(prob, "8,128,2", **opts)
    assert h.stats()["local_kernel"] != 6
    h.close()


def test_row_programs_pcg_matches_oracle_and_is_deterministic():
    from oracle import gdsw_oracle as O
    prob = P.poisson_problem(16, 4)
    h = handle_with_shape(prob, "8,128,2", local_solver="ic0", precision="fp32")
    r = np.random.default_rng(5).uniform(-1, 1, prob.A.n)
    z0 = gpu_apply(h, r)
    for _ in range(5):
        assert np.array_equal(gpu_apply(h, r), z0)
    M = oracle_for(prob, local="ic0")
    x, info = gpu_solve(h, prob.b)
    _, io = O.pcg(M.spmv, M.apply, prob.b)
    assert info.converged and info.true_relres <= 1e-8
    assert abs(info.iters - io.iters) <= 1
    h.close()


def test_row_programs_in_a_batched_handle():
    import torch
    from paper_2304_04876_b300 import gdsw as G
    mem = P.diffusion_batch(4, seed=5, nmin=7, nmax=12, smin=3, smax=5)
    b = np.concatenate([m.b for m in mem])
    out = {}
    for shape in ("4,128,0", "8,128,2"):
        old = os.environ.get("GDSW_LOCAL_SHAPE")
        os.environ["GDSW_LOCAL_SHAPE"] = shape
        try:
            h = G.Handle.batch([(m.A, m.part, None) for m in mem], local_solver="ic0", precision="fp32")
        finally:
            if old is None:
                os.environ.pop("GDSW_LOCAL_SHAPE")
            else:
                os.environ["GDSW_LOCAL_SHAPE"] = old
        bt = torch.tensor(b, dtype=torch.float64, device="cuda")
        xt = torch.zeros_like(bt)
        infos = h.solve_batch(bt, xt)
        torch.cuda.synchronize()
        assert all(i.converged and i.true_relres <= 1e-8 for i in infos)
        out[shape] = (xt.cpu().numpy(), [i.iters for i in infos], h.stats()["local_kernel"])
        h.close()
    assert out["8,128,2"][2] == 6
    assert out["4,128,0"][1] == out["8,128,2"][1]
    assert np.array_equal(out["4,128,0"][0], out["8,128,2"][0])

