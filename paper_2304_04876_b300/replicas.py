"""Replicas on several GPUs of one node: every rank solves its own problems (no
collective on the data path); only the timing is combined.

The solve shards by subdomain in principle (the paper's MPI design), but each
rank here holds whole problems, so a run on N GPUs is N independent replicas:
the whole-job rate is the units all ranks processed divided by the slowest
rank's time (max over ranks, after a barrier on both sides of the timed region).
"""
from __future__ import annotations


def rhs_seed(rank: int, k: int) -> int:
    """Seed of the k-th right-hand side of a rank (distinct across ranks)."""
    return (rank * 5 + k) % 997


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The largest `value` over all ranks (the value itself without a process group)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, seconds: float, world: int) -> float:
    """Whole-job throughput: every rank processed `units_per_rank` in at most `seconds`."""
    return world * units_per_rank / seconds
