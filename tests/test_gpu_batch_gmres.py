"""Batched GMRES (Sec. II's restarted GMRES with the GDSW preconditioner of Eq. 1,
every member of a batched handle iterating in the same launches): each member's
iteration count agrees with the same problem solved alone (the same steps, its dots
summed over its own tiles instead of the whole-vector reduction) and with the
oracle's GMRES, each member meets the tolerance on its true residual, restarts and
the single-reduce form work, a zero right-hand side finishes at once, and the
rigid-body null space of elasticity members is carried per member."""
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


def _batch_solve(h, b):
    import torch
    bt = torch.tensor(b, dtype=torch.float64, device="cuda")
    xt = torch.zeros_like(bt)
    infos = h.solve_batch(bt, xt)
    torch.cuda.synchronize()
    return xt.cpu().numpy(), infos


def _zof(m):
    return None if m.Z is None or m.Z.shape[1] == 1 and np.all(m.Z == 1) else m.Z


@pytest.mark.parametrize("precision,restart", [("fp64", 30), ("fp64", 5), ("fp32", 12)])
def test_batched_gmres_matches_members_alone(precision, restart):
    from paper_2304_04876_b300 import gdsw as G
    mem = P.diffusion_batch(5, seed=11, nmin=7, nmax=13, smin=3, smax=6)
    opts = dict(local_solver="ilu0", krylov="gmres", restart=restart, precision=precision)
    h = G.Handle.batch([(m.A, m.part, None) for m in mem], **opts)
    b = np.concatenate([m.b for m in mem])
    offs = np.cumsum([0] + [m.A.n for m in mem])
    x, infos = _batch_solve(h, b)
    for i, m in enumerate(mem):
        xi = x[offs[i]:offs[i + 1]]
        assert infos[i].converged and infos[i].true_relres <= 1e-8, i
        true = np.linalg.norm(m.b - m.A.to_scipy() @ xi) / np.linalg.norm(m.b)
        assert true <= 1e-8
        ha = gpu_handle(m, **opts)
        xa, ia = gpu_solve(ha, m.b)
        assert abs(ia.iters - infos[i].iters) <= 1, (i, ia.iters, infos[i].iters)
        assert relerr(xi, xa) <= (1e-7 if precision == "fp64" else 1e-5)
        ha.close()
        if precision == "fp64":
            M = oracle_for(m, local="ilu0")
            _, io = O.gmres(M.spmv, M.apply, m.b, tol=1e-8, restart=restart)
            assert abs(infos[i].iters - io.iters) <= 2, (i, infos[i].iters, io.iters)
    h.close()


def test_batched_gmres_single_reduce_and_zero_rhs():
    from paper_2304_04876_b300 import gdsw as G
    mem = P.diffusion_batch(4, seed=3, nmin=7, nmax=11, smin=3, smax=5)
    h = G.Handle.batch([(m.A, m.part, None) for m in mem], local_solver="ilu0", krylov="gmres",
                       gmres_orth="single")
    b = np.concatenate([m.b if i != 2 else np.zeros(m.A.n) for i, m in enumerate(mem)])
    offs = np.cumsum([0] + [m.A.n for m in mem])
    x, infos = _batch_solve(h, b)
    for i, m in enumerate(mem):
        assert infos[i].converged, i
        if i == 2:
            assert infos[i].iters == 0 and not np.any(x[offs[i]:offs[i + 1]])
        else:
            assert infos[i].true_relres <= 1e-8
    h.close()


def test_batched_gmres_elasticity_members_with_null_space():
    from paper_2304_04876_b300 import gdsw as G
    mem = [P.elasticity_problem(4, 2), P.elasticity_problem(6, 2), P.elasticity_problem(6, 3)]
    opts = dict(local_solver="ilu0", krylov="gmres", restart=30)
    h = G.Handle.batch([(m.A, m.part, _zof(m)) for m in mem], **opts)
    b = np.concatenate([m.b for m in mem])
    x, infos = _batch_solve(h, b)
    for i, m in enumerate(mem):
        assert infos[i].converged and infos[i].true_relres <= 1e-8, i
        M = oracle_for(m, local="ilu0")
        _, io = O.gmres(M.spmv, M.apply, m.b, tol=1e-8, restart=30)
        assert abs(infos[i].iters - io.iters) <= 2, (i, infos[i].iters, io.iters)
    h.close()
