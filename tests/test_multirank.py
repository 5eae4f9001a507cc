"""The replica (N > 1) path of bench.py, as world_size-2 gloo ranks on CPU:
the job is timed by its slowest rank and its rate counts every rank's units."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms_by_rank, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(ms_by_rank[rank], world)
        value = bench.job_throughput(1000.0, world, ms)
        dist.barrier()
        out[rank] = (ms, value)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ms_by_rank", [(2.0, 3.0), (5.0, 1.0)])
def test_slowest_rank_times_the_job(ms_by_rank):
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), ms_by_rank, out), nprocs=world, join=True)
        res = dict(out)
    slow = max(ms_by_rank)
    for r in range(world):
        assert res[r][0] == slow
        assert res[r][1] == pytest.approx(world * 1000.0 / (slow * 1e-3))


def test_single_rank_is_unchanged():
    assert bench.max_over_ranks(4.0, 1) == 4.0
    assert bench.job_throughput(10.0, 1, 2.0) == pytest.approx(5000.0)
