"""The multi-rank path of the benchmark on CPU: two gloo ranks reduce their
timings and counts the way the GPU ranks do (max of time, sum of work)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, pts, launches = bench.reduce_ranks(1.5 + rank, 1000 * (rank + 1), 7 + rank, world, "cpu")
    out[rank] = (t, pts, launches)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        assert out[r] == (2.5, 3000.0, 15)


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_ranks(0.25, 10, 3, 1, "cpu") == (0.25, 10.0, 3)
