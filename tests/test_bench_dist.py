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


def test_fengine_fp32_rate():
    """Nominal FFT arithmetic of the F-engine line: 5 N log2 N flop per FFT over
    152 x 128 FP32 lanes x 2 flop at the sampled clock."""
    import bench

    r = bench.fengine_fp32_rate(1024, 2 * 2 ** 20, 4.0, {"sm_mhz": 2000.0, "sm_max_mhz": 2070.0})
    flop = 5 * 1024 * 10 * 2 * 2 ** 20
    assert r["flop_per_launch"] == flop
    assert r["achieved_tflops"] == pytest.approx(flop / 4e-3 / 1e12)
    assert r["peak_tflops"] == pytest.approx(152 * 128 * 2 * 2.0e9 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved_tflops"] / r["peak_tflops"])
    assert bench.fengine_fp32_rate(1024, 1, 1.0, None)["peak_tflops"] == pytest.approx(152 * 256 * 2.07e9 / 1e12)
