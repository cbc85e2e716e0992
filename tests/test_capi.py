"""Host-side checks of the C ABI: the library loads, exports every entry point the
header declares, and rejects malformed input in the symbolic phase (before any
device work, so these run without a GPU)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2304_04876_b300 import build as B
from paper_2304_04876_b300 import gdsw as G
from paper_2304_04876_b300 import problems as P

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "gdsw.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return G.load()


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"GDSW_API\s+[\w\s\*]+?\b(gdsw_\w+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 11
    for name in names:
        assert hasattr(lib, name), name
        assert name in G.SIGNATURES, f"binding lacks {name}"


def test_default_options_and_status_strings(lib):
    o = G.default_options()
    assert (o.local_solver, o.trsv, o.sweeps_factor, o.sweeps_trsv, o.overlap) == (1, 0, 3, 5, 1)
    assert (o.precision, o.krylov, o.restart, o.maxit, o.coarse, o.flexible) == (0, 0, 30, 2000, 0, -1)
    assert o.fill_level == 0 and o.autotune == 1 and o.gmres_orth == 0
    assert o.tol == 1e-8 and o.wait_budget_cycles == 0
    for s in range(8):
        assert lib.gdsw_status_string(s)
    assert lib.gdsw_status_string(99) == b"unknown status"
    assert lib.gdsw_destroy(None) == G.OK


def _expect(status, A, part, **opts):
    with pytest.raises(G.GdswError) as e:
        G.Handle(A, part, None, stream=False, **opts)
    assert e.value.status == status
    return str(e.value)


def test_rejects_malformed_input_on_host(lib):
    prob = P.poisson_problem(8, 4)
    A, part = prob.A, prob.part
    # partition size mismatch
    bad = P.Partition(8, 8, 7, 1, part.cuts)
    assert "unknowns" in _expect(G.ERR_INVALID_ARG, A, bad)
    # cut outside the grid / not ascending
    _expect(G.ERR_INVALID_ARG, A, P.Partition(8, 8, 8, 1, [[7], [3], [3]]))
    _expect(G.ERR_INVALID_ARG, A, P.Partition(8, 8, 8, 1, [[3, 2], [3], [3]]))
    # unsorted columns
    ci = A.colind.copy()
    ci[0], ci[1] = ci[1], ci[0]
    _expect(G.ERR_INVALID_ARG, P.CSR(A.n, A.rowptr, ci, A.val), part)
    # a row without diagonal
    Ad = A.to_scipy().tolil()
    Ad[5, 5] = 0
    Ad = Ad.tocsr()
    Ad.eliminate_zeros()
    _expect(G.ERR_INVALID_ARG, P.CSR.from_scipy(Ad), part)
    # structurally nonsymmetric pattern
    Ad = A.to_scipy().tolil()
    Ad[0, 9] = -0.5
    _expect(G.ERR_INVALID_ARG, P.CSR.from_scipy(Ad.tocsr()), part)
    # partition that does not split the graph: a coupling across a block boundary
    # that skips the separator plane
    Ad = A.to_scipy().tolil()
    Ad[0, 5] = -0.1
    Ad[5, 0] = -0.1
    assert "split" in _expect(G.ERR_INVALID_ARG, P.CSR.from_scipy(Ad.tocsr()), part)
    # invalid options
    _expect(G.ERR_INVALID_ARG, A, part, local_solver=7)
    _expect(G.ERR_INVALID_ARG, A, part, tol=0.0)
    _expect(G.ERR_INVALID_ARG, A, part, local_solver="exact", fill_level=1)
    _expect(G.ERR_INVALID_ARG, A, part, fill_level=-1)


def test_structs_match_header(lib):
    """Field order and sizes of the binding's structs follow the header."""
    text = open(HEADER).read()
    body = text[text.index("typedef struct {\n  int32_t local_solver"):]
    body = body[:body.index("} gdsw_options;")]
    fields = re.findall(r"(?:int32_t|int64_t|double)\s+(\w+);", body)
    assert fields == [f for f, _ in G.Options._fields_]
    assert C.sizeof(G.Options) == 14 * 4 + 8 + 8
    assert C.sizeof(G.CSRStruct) == 40          # n, three pointers, mem (padded)
    assert C.sizeof(G.Stats) == 24 * 8 + 9 * 8 + 4 * 8   # ... setup times, local_kernel, persistent grid, Phi y, Phi^T r


def test_batch_rejects_bad_members_on_host(lib):
    a = P.poisson_problem(6, 3)
    e = P.elasticity_problem(2, 1)
    with pytest.raises(G.GdswError) as ex:      # different unknowns per node
        G.Handle.batch([(a.A, a.part, None), (e.A, e.part, None)], stream=False)
    assert ex.value.status == G.ERR_INVALID_ARG
    with pytest.raises(G.GdswError) as ex:      # batched GMRES: CGS2 or single-reduce only
        G.Handle.batch([(a.A, a.part, None)], stream=False, krylov="gmres", gmres_orth="dcgs2")
    assert ex.value.status == G.ERR_UNSUPPORTED


def test_refactor_rejects_null_arguments(lib):
    v = np.zeros(4)
    assert lib.gdsw_refactor(None, v.ctypes.data, None) == G.ERR_INVALID_ARG


def test_bytes_required_from_the_symbolic_phase(lib):
    """The footprint estimate needs no device: it grows with the problem, counts the
    matrix and Krylov vectors at least, and follows the storage precision."""
    small, big = P.poisson_problem(12, 4), P.poisson_problem(24, 4)
    r_s, s_s = G.bytes_required(small.A, small.part)
    r_b, _ = G.bytes_required(big.A, big.part)
    assert 0 < r_s < r_b and s_s > 0
    A = small.A
    assert r_s >= 12 * len(A.colind) + 6 * 8 * A.n
    r32, _ = G.bytes_required(small.A, small.part, precision="fp32")
    r16, _ = G.bytes_required(small.A, small.part, precision="fp16")
    assert r16 < r32 < r_s
    # no coarse space: less than with one
    r1, _ = G.bytes_required(small.A, small.part, coarse="none")
    assert r1 < r_s
    # rGDSW keeps one function per vertex: a smaller A0 than GDSW
    e = P.elasticity_problem(6, 2)
    rg, _ = G.bytes_required(e.A, e.part, e.Z, local_solver="ilu0")
    rr, _ = G.bytes_required(e.A, e.part, e.Z, local_solver="ilu0", coarse="rgdsw")
    assert rr < rg
    # level-1 fill widens the local factors
    rf, _ = G.bytes_required(small.A, small.part, fill_level=1)
    assert rf > r_s
    # GMRES(30) adds 61 basis vectors of n doubles
    rgm, _ = G.bytes_required(e.A, e.part, e.Z, local_solver="ilu0", krylov="gmres")
    assert rgm - rg >= 61 * 8 * e.A.n
    with pytest.raises(G.GdswError):
        G.bytes_required(small.A, P.Partition(12, 12, 11, 1, small.part.cuts))


def test_csr_memory_kind_is_checked(lib):
    """gdsw_csr.mem must be GDSW_MEM_HOST or GDSW_MEM_DEVICE; any other value is an
    invalid argument (checked before any device call)."""
    import ctypes as C
    from paper_2304_04876_b300 import problems as P
    prob = P.poisson_problem(6, 3)
    csr, ps, zp, nn, keep = G._marshal(prob.A, prob.part, None)
    csr.mem = 7
    o = G.make_options()
    res, scr = C.c_int64(), C.c_int64()
    st = lib.gdsw_bytes_required(C.byref(csr), C.byref(ps), zp, nn, C.byref(o), C.byref(res), C.byref(scr))
    assert st == 1 and b"mem" in lib.gdsw_last_error()
    csr.mem = G.MEM_HOST
    st = lib.gdsw_bytes_required(C.byref(csr), C.byref(ps), zp, nn, C.byref(o), C.byref(res), C.byref(scr))
    assert st == 0 and res.value > 0
