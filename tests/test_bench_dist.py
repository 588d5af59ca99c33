"""The bench's multi-replica aggregation on CPU with two gloo ranks: the step
time is the slowest rank's and the throughput counts every rank's units."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms_local = 100.0 if rank == 0 else 250.0  # rank 1 is slower
    ms_step, rate = bench.job_time_and_rate(ms_local, units_per_rank=1e9, steps=5, dist=dist)
    out[rank] = (ms_step, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replica_aggregation_gloo():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in (0, 1):
        ms_step, rate = out[r]
        assert ms_step == pytest.approx(50.0)        # max over ranks: 250 ms / 5 steps
        assert rate == pytest.approx(2 * 1e9 / 0.05)  # both ranks' units over the slowest time


def test_single_process_aggregation():
    import bench

    ms_step, rate = bench.job_time_and_rate(40.0, units_per_rank=2e9, steps=4, dist=None)
    assert ms_step == 10.0 and rate == pytest.approx(2e11)
