"""The N > 1 launch path of bench.py on CPU: two gloo ranks (no GPU).

The job's time is the slowest rank's, its units the sum over the ranks, so
value = units / time; the reference arm runs on rank 0 only and the other
ranks leave without work.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        ms, units = bench.job_timing(10.0 + 5.0 * rank, 100.0 * (rank + 1), dist)
        out[rank] = (ms, units)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_timing_max_time_sum_units():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        ps = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == out[1] == (15.0, 300.0)


def test_job_timing_single_process():
    import bench

    assert bench.job_timing(12.5, 7.0) == (12.5, 7.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    import argparse

    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(steps=1, warmup=3, gpus=2)
    assert bench.run_reference(args) == 0     # returns before touching the oracle
