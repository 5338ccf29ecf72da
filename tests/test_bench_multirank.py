"""The benchmark's multi-rank aggregation on CPU with gloo, world size 2:
throughput = work of all ranks / slowest rank's time; the reference arm runs
on rank 0 only."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = [100.0, 250.0][rank]           # rank 1 is the slow one
    units = [1000.0, 1000.0][rank]
    value, ms_max = bench.aggregate(ms, units, dist, "cpu")
    out[rank] = (value, ms_max)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_max_time_sum_work_world2():
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        value, ms_max = out[r]
        assert ms_max == 250.0
        assert value == pytest.approx(2000.0 / 0.25)


def test_reference_arm_non_zero_rank_exits_without_work(monkeypatch):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        gpus, steps, warmup = 2, 1, 0

    assert bench.run_reference(A()) == 0
