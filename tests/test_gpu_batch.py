"""Batched handle (independent problems in one block-diagonal system): the apply and
the batched PCG against the oracle of every member, and every member's result the
same alone and in the batch."""
import numpy as np
import pytest

from oracle import gdsw_oracle as O
from paper_2304_04876_b300 import problems as P
from tests.gpu_util import gpu_apply, gpu_handle, gpu_solve, oracle_for, relerr

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2304_04876_b300 import build
    build.build()
    assert torch.cuda.is_available()


def _members(count=5, seed=3):
    # seeded heterogeneous diffusion problems of different sizes and subdomain sizes
    return P.diffusion_batch(count, seed=seed, nmin=7, nmax=14, smin=3, smax=6)


def _batch_solve(h, b):
    import torch
    bt = torch.tensor(b, dtype=torch.float64, device="cuda")
    xt = torch.zeros_like(bt)
    infos = h.solve_batch(bt, xt)
    torch.cuda.synchronize()
    return xt.cpu().numpy(), infos


@pytest.mark.parametrize("local", ["ic0", "exact"])
def test_batch_apply_matches_members(local):
    from paper_2304_04876_b300 import gdsw as G
    mem = _members()
    h = G.Handle.batch([(m.A, m.part, None) for m in mem], local_solver=local)
    assert h.stats()["n_problems"] == len(mem)
    offs = np.cumsum([0] + [m.A.n for m in mem])
    r = np.random.default_rng(0).uniform(-1, 1, offs[-1])
    z = gpu_apply(h, r)
    for i, m in enumerate(mem):
        M = oracle_for(m, local=local)
        zi = M.apply(r[offs[i]:offs[i + 1]])
        assert relerr(z[offs[i]:offs[i + 1]], zi) <= 1e-10, i


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_pcg_matches_members_alone(precision):
    from paper_2304_04876_b300 import gdsw as G
    mem = _members()
    h = G.Handle.batch([(m.A, m.part, None) for m in mem], local_solver="ic0", precision=precision)
    b = np.concatenate([m.b for m in mem])
    offs = np.cumsum([0] + [m.A.n for m in mem])
    x, infos = _batch_solve(h, b)
    for i, m in enumerate(mem):
        xi = x[offs[i]:offs[i + 1]]
        assert infos[i].converged and infos[i].true_relres <= 1e-8
        true = np.linalg.norm(m.b - m.A.to_scipy() @ xi) / np.linalg.norm(m.b)
        assert true <= 1e-8
        # the same problem alone on the GPU
        ha = gpu_handle(m, local_solver="ic0", precision=precision)
        xa, ia = gpu_solve(ha, m.b)
        # FP64: same iterations, solutions equal to 1e-12 (reductions are tiled differently);
        # FP32 preconditioner: a flipped float rounding can move one iteration, so the
        # solutions agree to the solver tolerance
        if precision == "fp64":
            assert ia.iters == infos[i].iters
            assert relerr(xi, xa) <= 1e-12
        else:
            assert abs(ia.iters - infos[i].iters) <= 1
            assert relerr(xi, xa) <= 1e-6
        if precision == "fp64":
            M = oracle_for(m, local="ic0")
            _, io = O.pcg(M.spmv, M.apply, m.b, tol=1e-8)
            assert abs(infos[i].iters - io.iters) <= 1


def test_batch_with_zero_rhs_member_and_elasticity_null_space():
    from paper_2304_04876_b300 import gdsw as G
    mem = [P.elasticity_problem(4, 2), P.elasticity_problem(6, 2)]
    h = G.Handle.batch([(m.A, m.part, m.Z) for m in mem], local_solver="ic0")
    b = np.concatenate([np.zeros(mem[0].A.n), mem[1].b])
    x, infos = _batch_solve(h, b)
    assert infos[0].iters == 0 and not x[:mem[0].A.n].any()
    assert infos[1].converged and infos[1].true_relres <= 1e-8
    M = oracle_for(mem[1], local="ic0")
    _, io = O.pcg(M.spmv, M.apply, mem[1].b, tol=1e-8)
    assert abs(infos[1].iters - io.iters) <= 1
