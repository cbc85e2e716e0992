"""Thin Python binding of libgdsw (include/gdsw.h): argument marshalling only.

Every step of setup, apply and solve runs in the CUDA library; this module
converts numpy arrays and torch tensors to the pointers and structs of the C
ABI and turns status codes into exceptions.  There is no fallback: if the
library is missing or fails to load, ``load()`` raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libgdsw.so")

OK, ERR_INVALID_ARG, ERR_OUT_OF_MEMORY, ERR_BREAKDOWN, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_CUDA, \
    ERR_UNSUPPORTED = range(8)
LOCAL = {"exact": 0, "ic0": 1, "ilu0": 2}
TRSV = {"levelsched": 0, "jacobi": 1}
PRECISION = {"fp64": 0, "fp32": 1, "fp16": 2}
KRYLOV = {"pcg": 0, "gmres": 1}
COARSE = {"gdsw": 0, "none": 1, "rgdsw": 2}
GMRES_ORTH = {"cgs2": 0, "single": 1, "dcgs2": 2}


class CSRStruct(C.Structure):
    _fields_ = [("n", C.c_int32), ("rowptr", C.c_void_p), ("colind", C.c_void_p), ("val", C.c_void_p),
                ("mem", C.c_int32)]


MEM_HOST, MEM_DEVICE = 0, 1


def _csr_struct(A):
    """CSRStruct for A (problems.CSR with numpy arrays, or any object with n and CUDA
    tensors rowptr/colind (int32) and val (float64)) and the buffers it borrows."""
    if getattr(A.rowptr, "is_cuda", False):
        rp, ci, va = A.rowptr, A.colind, A.val
        assert rp.dtype == ci.dtype and str(rp.dtype) == "torch.int32" and str(va.dtype) == "torch.float64"
        assert rp.is_contiguous() and ci.is_contiguous() and va.is_contiguous()
        return CSRStruct(int(A.n), rp.data_ptr(), ci.data_ptr(), va.data_ptr(), MEM_DEVICE), [rp, ci, va]
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(A.colind, dtype=np.int32)
    va = np.ascontiguousarray(A.val, dtype=np.float64)
    return CSRStruct(int(A.n), rp.ctypes.data, ci.ctypes.data, va.ctypes.data, MEM_HOST), [rp, ci, va]


class PartitionStruct(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("dofs_per_node", C.c_int32),
                ("ncut", C.c_int32 * 3), ("cut", C.c_void_p * 3)]


class Options(C.Structure):
    _fields_ = [("local_solver", C.c_int32), ("trsv", C.c_int32), ("sweeps_factor", C.c_int32),
                ("sweeps_trsv", C.c_int32), ("overlap", C.c_int32), ("precision", C.c_int32),
                ("krylov", C.c_int32), ("restart", C.c_int32), ("maxit", C.c_int32),
                ("coarse", C.c_int32), ("fill_level", C.c_int32), ("autotune", C.c_int32),
                ("gmres_orth", C.c_int32), ("flexible", C.c_int32), ("tol", C.c_double),
                ("wait_budget_cycles", C.c_int64)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("true_relres", C.c_double),
                ("seconds", C.c_double)]


class Stats(C.Structure):
    _fields_ = [(name, C.c_int64) for name in (
        "n", "nnz", "n_sub", "n0", "n_comp", "sum_omega", "max_omega", "nnz_L", "nnz_U", "ell_L",
        "ell_U", "nnz_phi", "n_levels_L", "n_levels_U", "max_levels", "dense_local", "n_blocks",
        "device_bytes", "n_problems", "a0_entries", "local_stages", "local_threads", "mf_supernodes", "mf_levels")] + [("setup_seconds", C.c_double), ("setup_phase_seconds", C.c_double * 8),
                                                          ("local_kernel", C.c_int64),
                                                          ("pcg_persistent_grid", C.c_int64),
                                                          ("phi_beside_local", C.c_int64),
                                                          ("phiT_wide", C.c_int64)]

    def as_dict(self) -> dict:
        d = {name: getattr(self, name) for name, _ in self._fields_ if name != "setup_phase_seconds"}
        d["setup_phase_seconds"] = list(self.setup_phase_seconds)
        return d


class GdswError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


_lib = None

# exported symbol -> (restype, argtypes)
SIGNATURES = {
    "gdsw_default_options": (None, [C.POINTER(Options)]),
    "gdsw_setup": (C.c_int, [C.POINTER(CSRStruct), C.POINTER(PartitionStruct), C.c_void_p, C.c_int32,
                             C.POINTER(Options), C.c_void_p, C.POINTER(C.c_void_p)]),
    "gdsw_setup_batch": (C.c_int, [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.POINTER(Options), C.c_void_p, C.POINTER(C.c_void_p)]),
    "gdsw_solve_batch": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gdsw_batch_start": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "gdsw_batch_iterate": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p]),
    "gdsw_batch_status": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gdsw_batch_finish": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(SolveInfo),
                                    C.POINTER(C.c_int32), C.c_void_p]),
    "gdsw_apply": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gdsw_apply_timed": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "gdsw_spmv": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gdsw_pcg_iteration_timed": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "gdsw_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(SolveInfo), C.c_void_p]),
    "gdsw_solve_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(SolveInfo), C.c_void_p]),
    "gdsw_solve_host_zero_guess": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(SolveInfo),
                                             C.c_void_p]),
    "gdsw_get_stats": (C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    "gdsw_destroy": (C.c_int, [C.c_void_p]),
    "gdsw_refactor": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "gdsw_bytes_required": (C.c_int, [C.POINTER(CSRStruct), C.POINTER(PartitionStruct), C.c_void_p, C.c_int32,
                                      C.POINTER(Options), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "gdsw_mf_plan_export": (C.c_int, [C.POINTER(CSRStruct), C.POINTER(PartitionStruct), C.POINTER(Options),
                                      C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                      C.POINTER(C.c_int64), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    "gdsw_spmv_dot_noalloc": (C.c_int, [C.c_int32, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "gdsw_measure_fma_rate": (C.c_int, [C.c_int32, C.POINTER(C.c_double), C.c_void_p]),
    "gdsw_check_conversions": (C.c_int, [C.c_uint64, C.c_int64, C.POINTER(C.c_uint64), C.c_void_p]),
    "gdsw_status_string": (C.c_char_p, [C.c_int]),
    "gdsw_last_error": (C.c_char_p, []),
}


def load(path: str = LIB_PATH):
    """Load libgdsw.so (built in-tree by ``paper_2304_04876_b300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libgdsw.so not found at {path}; run `python -m paper_2304_04876_b300.build`")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, what: str):
    if status != OK:
        lib = load()
        raise GdswError(status, f"{what}: {lib.gdsw_status_string(status).decode()}: "
                                f"{lib.gdsw_last_error().decode()}")


def default_options() -> Options:
    o = Options()
    load().gdsw_default_options(C.byref(o))
    return o


def make_options(**kw) -> Options:
    o = default_options()
    for k, v in kw.items():
        table = {"local_solver": LOCAL, "trsv": TRSV, "precision": PRECISION, "krylov": KRYLOV,
                 "coarse": COARSE, "gmres_orth": GMRES_ORTH}.get(k)
        if table is not None and isinstance(v, str):
            v = table[v]
        setattr(o, k, v)
    return o


def _ptr(t) -> int:
    """Device pointer of a torch tensor (contiguous float64)."""
    assert t.is_cuda and t.is_contiguous() and t.dtype.is_floating_point, "expected a contiguous CUDA tensor"
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(getattr(stream, "cuda_stream", stream))


class Handle:
    """One set-up problem: factors, Phi and A0^-1 resident on the device."""

    def __init__(self, A, part, Z: Optional[np.ndarray] = None, stream=None, _batch=None, **options):
        lib = load()
        if _batch is not None:
            self._init_batch(_batch, stream, options)
            return
        csr, ps, zp, nn, keep = _marshal(A, part, Z)
        self.options = make_options(**options)
        h = C.c_void_p()
        _check(lib.gdsw_setup(C.byref(csr), C.byref(ps), zp, nn, C.byref(self.options),
                              _stream(stream) if stream is not False else None, C.byref(h)), "gdsw_setup")
        del keep                      # the library copied the matrix, partition and null space
        self._h = h
        self.n = int(A.n)

    def _init_batch(self, members, stream, options):
        """members: list of (A, part, Z or None)."""
        lib = load()
        count = len(members)
        keep = []
        csrs = (CSRStruct * count)()
        parts = (PartitionStruct * count)()
        zs = (C.c_void_p * count)()
        nns = (C.c_int32 * count)()
        for i, (A, part, Z) in enumerate(members):
            csrs[i], bufs = _csr_struct(A)
            keep += bufs
            cuts = [np.ascontiguousarray(c, dtype=np.int32) for c in part.cuts]
            keep += cuts
            parts[i] = PartitionStruct(int(part.nx), int(part.ny), int(part.nz), int(part.dpn))
            for a in range(3):
                parts[i].ncut[a] = len(cuts[a])
                parts[i].cut[a] = cuts[a].ctypes.data if len(cuts[a]) else None
            if Z is None:
                zs[i], nns[i] = None, 0
            else:
                Zc = np.asfortranarray(np.asarray(Z, dtype=np.float64).reshape(A.n, -1))
                keep.append(Zc)
                zs[i], nns[i] = Zc.ctypes.data, Zc.shape[1]
        self.options = make_options(**options)
        h = C.c_void_p()
        _check(lib.gdsw_setup_batch(count, C.cast(csrs, C.c_void_p), C.cast(parts, C.c_void_p),
                                    C.cast(zs, C.c_void_p), C.cast(nns, C.c_void_p), C.byref(self.options),
                                    _stream(stream) if stream is not False else None, C.byref(h)),
               "gdsw_setup_batch")
        self._h = h
        self.count = count
        self.n = sum(int(m[0].n) for m in members)

    @classmethod
    def batch(cls, members, stream=None, **options):
        """One handle for independent problems [(A, part, Z), ...] (block-diagonal union)."""
        return cls(None, None, None, stream=stream, _batch=members, **options)

    def solve_batch(self, b, x, stream=None, raise_on_nonconvergence=True):
        infos = (SolveInfo * self.count)()
        st = load().gdsw_solve_batch(self._handle(), _ptr(b), _ptr(x), C.cast(infos, C.c_void_p), _stream(stream))
        if st != ERR_NOT_CONVERGED or raise_on_nonconvergence:
            _check(st, "gdsw_solve_batch")
        return list(infos)

    # ---- continuous batching (members of a batched handle as solve slots) ----
    def batch_start(self, member: int, b, stream=None):
        """Start member `member` on right-hand side b (CUDA float64 tensor of its n entries)."""
        _check(load().gdsw_batch_start(self._handle(), int(member), _ptr(b), _stream(stream)), "gdsw_batch_start")

    def batch_iterate(self, iterations: int, stream=None):
        """Enqueue `iterations` PCG iterations of every running member (asynchronous)."""
        _check(load().gdsw_batch_iterate(self._handle(), int(iterations), _stream(stream)), "gdsw_batch_iterate")

    def batch_status(self, stream=None):
        """(done, iters, relres) arrays over the members (waits for the stream)."""
        done = np.zeros(self.count, np.int32)
        iters = np.zeros(self.count, np.int32)
        rel = np.zeros(self.count, np.float64)
        _check(load().gdsw_batch_status(self._handle(), done.ctypes.data, iters.ctypes.data, rel.ctypes.data,
                                        _stream(stream)), "gdsw_batch_status")
        return done, iters, rel

    def batch_finish(self, member: int, x=None, stream=None):
        """For a stopped member: (info, continued).  continued = True when its true
        residual missed the tolerance and it went on iterating; otherwise x (CUDA
        float64 tensor, or None) receives its solution."""
        info = SolveInfo()
        cont = C.c_int32()
        _check(load().gdsw_batch_finish(self._handle(), int(member), _ptr(x) if x is not None else None,
                                        C.byref(info), C.byref(cont), _stream(stream)), "gdsw_batch_finish")
        return info, bool(cont.value)

    def _handle(self):
        if self._h is None:
            raise RuntimeError("handle destroyed")
        return self._h

    def apply(self, r, z, stream=None):
        _check(load().gdsw_apply(self._handle(), _ptr(r), _ptr(z), _stream(stream)), "gdsw_apply")
        return z

    def apply_timed(self, r, z, stream=None):
        ms = (C.c_double * 4)()
        _check(load().gdsw_apply_timed(self._handle(), _ptr(r), _ptr(z), _stream(stream), ms),
               "gdsw_apply_timed")
        return list(ms)

    PCG_KERNELS = ("spmv", "update", "local", "phiT", "coarse", "combine", "pupdate", "xupdate")

    def pcg_iteration_timed(self, b, stream=None) -> dict:
        """Device ms of each kernel of one PCG iteration from right-hand side b (CUDA events)."""
        ms = (C.c_double * len(self.PCG_KERNELS))()
        _check(load().gdsw_pcg_iteration_timed(self._handle(), _ptr(b), _stream(stream), ms),
               "gdsw_pcg_iteration_timed")
        return dict(zip(self.PCG_KERNELS, list(ms)))

    def spmv(self, x, y, stream=None):
        _check(load().gdsw_spmv(self._handle(), _ptr(x), _ptr(y), _stream(stream)), "gdsw_spmv")
        return y

    def solve(self, b, x, stream=None, raise_on_nonconvergence=True) -> SolveInfo:
        info = SolveInfo()
        st = load().gdsw_solve(self._handle(), _ptr(b), _ptr(x), C.byref(info), _stream(stream))
        if st != ERR_NOT_CONVERGED or raise_on_nonconvergence:
            _check(st, "gdsw_solve")
        return info

    def solve_host(self, b: np.ndarray, x: np.ndarray, stream=None, raise_on_nonconvergence=True,
                   zero_guess: bool = False) -> SolveInfo:
        """b, x: host float64 arrays (page-locked memory makes the copies asynchronous).
        x holds the initial guess, or with zero_guess=True is only written (x0 = 0)."""
        info = SolveInfo()
        name = "gdsw_solve_host_zero_guess" if zero_guess else "gdsw_solve_host"
        st = getattr(load(), name)(self._handle(), C.c_void_p(_host_ptr(b)), C.c_void_p(_host_ptr(x)),
                                   C.byref(info), _stream(stream))
        if st != ERR_NOT_CONVERGED or raise_on_nonconvergence:
            _check(st, name)
        return info

    def refactor(self, val: np.ndarray, stream=None):
        """New matrix values on the setup's pattern (host float64, CSR order): numeric phase only."""
        v = np.ascontiguousarray(val, dtype=np.float64)
        _check(load().gdsw_refactor(self._handle(), v.ctypes.data, _stream(stream)), "gdsw_refactor")

    def stats(self) -> dict:
        s = Stats()
        _check(load().gdsw_get_stats(self._handle(), C.byref(s)), "gdsw_get_stats")
        return s.as_dict()

    def close(self):
        if self._h is not None:
            load().gdsw_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _marshal(A, part, Z):
    """C structs for a CSR matrix, its partition and null space; the last item
    keeps the numpy buffers alive while the structs are in use."""
    csr, keep = _csr_struct(A)
    cuts = [np.ascontiguousarray(c, dtype=np.int32) for c in part.cuts]
    ps = PartitionStruct(int(part.nx), int(part.ny), int(part.nz), int(part.dpn))
    for a in range(3):
        ps.ncut[a] = len(cuts[a])
        ps.cut[a] = cuts[a].ctypes.data if len(cuts[a]) else None
    keep = keep + cuts
    if Z is None:
        zp, nn = None, 0
    else:
        Zc = np.asfortranarray(np.asarray(Z, dtype=np.float64).reshape(A.n, -1))
        keep.append(Zc)
        zp, nn = Zc.ctypes.data, Zc.shape[1]
    return csr, ps, zp, nn, keep


def bytes_required(A, part, Z: Optional[np.ndarray] = None, **options):
    """(resident, setup_scratch) device bytes of gdsw_setup on these arguments (host work only)."""
    csr, ps, zp, nn, keep = _marshal(A, part, Z)
    o = make_options(**options)
    res, scr = C.c_int64(), C.c_int64()
    _check(load().gdsw_bytes_required(C.byref(csr), C.byref(ps), zp, nn, C.byref(o), C.byref(res), C.byref(scr)),
           "gdsw_bytes_required")
    del keep
    return int(res.value), int(scr.value)


def mf_plan(A, part, subdomain: int, **options) -> dict:
    """The nested-dissection plan of the multifrontal exact solver for one subdomain
    (gdsw_mf_plan_export; host work only): nd_dof, sn_ptr, parent, b_ptr, b_pos."""
    csr, ps, _, _, keep = _marshal(A, part, None)
    o = make_options(**options)
    m, nsn, nbt = C.c_int32(), C.c_int32(), C.c_int64()
    lib = load()
    args = (C.byref(csr), C.byref(ps), C.byref(o), int(subdomain), C.byref(m), C.byref(nsn), C.byref(nbt))
    _check(lib.gdsw_mf_plan_export(*args, None, None, None, None, None), "gdsw_mf_plan_export")
    out = dict(nd_dof=np.zeros(m.value, np.int32), sn_ptr=np.zeros(nsn.value + 1, np.int32),
               parent=np.zeros(nsn.value, np.int32), b_ptr=np.zeros(nsn.value + 1, np.int64),
               b_pos=np.zeros(max(nbt.value, 1), np.int32))
    _check(lib.gdsw_mf_plan_export(*args, *(out[k].ctypes.data for k in ("nd_dof", "sn_ptr", "parent", "b_ptr",
                                                                          "b_pos"))), "gdsw_mf_plan_export")
    out["b_pos"] = out["b_pos"][:nbt.value]
    del keep
    return out


def _host_ptr(a) -> int:
    if hasattr(a, "data_ptr"):           # a pinned torch CPU tensor
        assert not a.is_cuda and a.is_contiguous() and a.dtype.is_floating_point
        return a.data_ptr()
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data


def measure_fma_rate(precision: str = "fp64", stream=None) -> float:
    """FMAs per second of the device in "fp64" or "fp32" (gdsw_measure_fma_rate)."""
    out = C.c_double()
    _check(load().gdsw_measure_fma_rate(PRECISION[precision], C.byref(out), _stream(stream)),
           "gdsw_measure_fma_rate")
    return out.value


def check_conversions(seed: int, count: int, stream=None) -> tuple:
    """(double->float, float->double) mismatch counts of the library's integer-ALU
    conversions against the hardware ones on `count` random bit patterns."""
    out = (C.c_uint64 * 2)()
    _check(load().gdsw_check_conversions(seed, count, out, _stream(stream)), "gdsw_check_conversions")
    return int(out[0]), int(out[1])


def spmv_dot_noalloc(rowptr, colind, val, x, y, dot, nnz: int, stream=None):
    """y = A x and dot[0] = (x, y) through gdsw_spmv_dot_noalloc (no device allocation).

    rowptr/colind (int32) and val, x, y, dot (float64) are CUDA tensors owned by the caller;
    their dtypes, sizes, layout and device are checked here, since the library reads the
    raw pointers (a float32 vector or a short index array would be read out of bounds).
    """
    import torch
    n = x.numel()
    dev = torch.device("cuda", torch.cuda.current_device())
    for name, t, dtype, size in (("rowptr", rowptr, torch.int32, n + 1), ("colind", colind, torch.int32, nnz),
                                 ("val", val, torch.float64, nnz), ("x", x, torch.float64, n),
                                 ("y", y, torch.float64, n), ("dot", dot, torch.float64, 1)):
        if t.dtype != dtype or not t.is_contiguous() or t.device != dev:
            raise ValueError(f"{name}: expected a contiguous {dtype} tensor on {dev}, got {t.dtype} on {t.device}")
        if (t.numel() < size) if name == "dot" else (t.numel() != size):
            raise ValueError(f"{name}: expected {size} elements, got {t.numel()}")
    _check(load().gdsw_spmv_dot_noalloc(n, int(nnz), rowptr.data_ptr(), colind.data_ptr(), _ptr(val),
                                        _ptr(x), _ptr(y), _ptr(dot), _stream(stream)),
           "gdsw_spmv_dot_noalloc")
    return y, dot
