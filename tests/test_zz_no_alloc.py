"""gdsw_spmv_dot_noalloc, the entry point for callers that cannot allocate device memory
(for instance programs whose own pool allocator owns all of it), checked against the
regular entry point gdsw_spmv and a dot product of its output.

It runs last in the suite (file name) and also passes on its own in a fresh process."""
import numpy as np
import pytest

from paper_2304_04876_b300 import problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    from paper_2304_04876_b300 import build
    build.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("make", [lambda: P.poisson_problem(12, 4), lambda: P.elasticity_problem(4, 2)],
                         ids=["poisson12", "elasticity4"])
def test_noalloc_spmv_dot_matches_regular_entry_point(make):
    import torch
    from paper_2304_04876_b300 import gdsw as G
    prob = make()
    A = prob.A
    h = G.Handle(A, prob.part, None, local_solver="exact")
    dev = "cuda"
    rowptr = torch.tensor(A.rowptr, dtype=torch.int32, device=dev)
    colind = torch.tensor(A.colind, dtype=torch.int32, device=dev)
    val = torch.tensor(A.val, dtype=torch.float64, device=dev)
    for call in range(2):                      # two calls in a row share the static scratch
        x = torch.tensor(np.random.default_rng(call).uniform(-1, 1, A.n), dtype=torch.float64, device=dev)
        y_ref = torch.empty_like(x)
        h.spmv(x, y_ref)
        y = torch.full_like(x, np.nan)
        dot = torch.zeros(1, dtype=torch.float64, device=dev)
        G.spmv_dot_noalloc(rowptr, colind, val, x, y, dot, A.nnz)
        torch.cuda.synchronize()
        yr = y_ref.cpu().numpy()
        assert np.abs(y.cpu().numpy() - yr).max() <= 1e-13 * np.abs(yr).max()
        ref_dot = float(x.cpu().numpy() @ yr)
        assert abs(dot.item() - ref_dot) <= 1e-12 * abs(ref_dot)
    h.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    from paper_2304_04876_b300 import gdsw as G
    lib = G.load()
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    ti = torch.zeros(4, dtype=torch.int32, device="cuda")
    # 7 entries per row -> 32 rows per block -> at most 65536*32 rows; the check happens before any launch
    n = 65536 * 32 + 1
    st = lib.gdsw_spmv_dot_noalloc(n, 7 * n, ti.data_ptr(), ti.data_ptr(), t.data_ptr(), t.data_ptr(),
                                   t.data_ptr(), t.data_ptr(), None)
    assert st == G.ERR_UNSUPPORTED
    assert b"static scratch" in lib.gdsw_last_error()
