"""The multi-rank host logic of bench.py (replicas, max over ranks) on two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, values, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out[rank] = bench.max_over_ranks(values[rank], world)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks():
    world = 2
    values = [12.5, 40.25]
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), values, out), nprocs=world, join=True)
    assert out[0] == 40.25 and out[1] == 40.25


def test_single_rank_and_replica_scaling():
    import bench
    assert bench.max_over_ranks(3.0, 1) == 3.0
    assert bench.whole_job_ms_per_solve(40.0, 4) == 10.0
