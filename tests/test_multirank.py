"""Multi-rank host logic of bench.py on CPU: two gloo ranks, each with its own replica of the
work; the job time is the slowest rank's and the work is summed (weak scaling, no data exchange)."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as tmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, vi = bench.reduce_across_ranks(10.0 * (rank + 1), 1000.0 * (rank + 1), torch.device("cpu"), world)
    out[rank] = (ms, vi)
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_work():
    import random
    port = 29500 + random.randint(0, 2000)
    world = 2
    mgr = tmp.Manager()
    out = mgr.dict()
    tmp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        assert out[r] == (20.0, 3000.0)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_across_ranks(3.5, 7.0, None, 1) == (3.5, 7.0)
