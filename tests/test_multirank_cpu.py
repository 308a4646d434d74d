"""The multi-rank host logic of bench.py on CPU: two gloo ranks (spawned processes).

Under torchrun every rank solves its own replica; the job's time is the slowest rank's (an
all-reduce MAX over the ranks' times) and the whole-job rate counts every rank's units.  No GPU
is involved: the reduction runs on gloo with host tensors.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        total = bench.max_over_ranks(ms, dist)
        out[rank] = (total, bench.job_rate(8, 10, world, total))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_rank_and_the_job_rate():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        total, rate = res[r]
        assert total == 150.0  # max over ranks
        assert rate == pytest.approx(8 * 10 * world / 0.150)


def test_without_a_process_group_the_rank_is_the_job():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(123.0, None) == 123.0
    assert bench.job_rate(8, 10, 1, 80.0) == pytest.approx(1000.0)
