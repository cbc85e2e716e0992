"""Helpers for the GPU parity tests: run the CUDA path through the C ABI binding and
the oracle on the same seeded inputs."""
import numpy as np

from oracle import gdsw_oracle as O
from paper_2304_04876_b300 import gdsw as G

LOCAL = {"exact": O.EXACT, "ic0": O.IC0, "ilu0": O.ILU0}
TRSV = {"levelsched": O.LEVELSCHED, "jacobi": O.JACOBI}


def oracle_for(prob, local="ic0", trsv="levelsched", sweeps_factor=3, sweeps_trsv=5, overlap=1,
               coarse="gdsw", fill_level=0):
    return O.GDSW(prob.A, prob.part, prob.Z, local=LOCAL[local], trsv=TRSV[trsv],
                  sweeps_factor=sweeps_factor, sweeps_trsv=sweeps_trsv, overlap=overlap,
                  coarse=(coarse != "none"), coarse_variant=("rgdsw" if coarse == "rgdsw" else "gdsw"),
                  fill_level=fill_level)


def gpu_handle(prob, **opts):
    Z = None if prob.Z is None or prob.Z.shape[1] == 1 and np.all(prob.Z == 1) else prob.Z
    return G.Handle(prob.A, prob.part, Z, **opts)


def gpu_apply(h, r):
    import torch
    rt = torch.tensor(r, dtype=torch.float64, device="cuda")
    zt = torch.empty_like(rt)
    h.apply(rt, zt)
    torch.cuda.synchronize()
    return zt.cpu().numpy()


def gpu_spmv(h, x):
    import torch
    xt = torch.tensor(x, dtype=torch.float64, device="cuda")
    yt = torch.empty_like(xt)
    h.spmv(xt, yt)
    torch.cuda.synchronize()
    return yt.cpu().numpy()


def gpu_solve(h, b, x0=None, raise_on_nonconvergence=True):
    import torch
    bt = torch.tensor(b, dtype=torch.float64, device="cuda")
    xt = torch.zeros_like(bt) if x0 is None else torch.tensor(x0, dtype=torch.float64, device="cuda")
    info = h.solve(bt, xt, raise_on_nonconvergence=raise_on_nonconvergence)
    torch.cuda.synchronize()
    return xt.cpu().numpy(), info


def relerr(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
