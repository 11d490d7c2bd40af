"""bench.py's multi-rank accounting (the slowest rank's time, the work summed
over ranks: the column-sharded run's value) with two gloo ranks on the CPU."""
import os
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, by = bench.reduce_across_ranks(dist, 10.0 + rank * 5.0, 1e9 * (rank + 1))
    out[rank] = (ms, by)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction():
    port = 29500 + os.getpid() % 1000
    mgr = mp.get_context("spawn").Manager()  # no fork of a multi-threaded test process
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == (15.0, 3e9)


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_across_ranks(None, 7.0, 5.0) == (7.0, 5.0)
