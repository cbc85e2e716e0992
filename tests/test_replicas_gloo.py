"""The multi-GPU path is replicas (each rank solves its own problems; no collective on
the data path): its host logic, the max-over-ranks timing and the whole-job rate, run
here as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2304_04876_b300 import replicas as R


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = [0.5, 2.0][rank]               # the slow rank decides the job's time
        t = R.max_over_ranks(elapsed, dist, "cpu")
        out[rank] = (t, R.job_rate(10, t, world), R.rhs_seed(rank, 0), R.rhs_seed(rank, 4))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.0
    assert res[0][1] == res[1][1] == pytest.approx(world * 10 / 2.0)
    # every rank draws its own right-hand sides
    seeds = {res[r][2] for r in range(world)} | {res[r][3] for r in range(world)}
    assert len(seeds) == 4


def test_single_process_needs_no_group():
    assert R.max_over_ranks(1.5) == 1.5
    assert R.job_rate(6, 2.0, 1) == 3.0
