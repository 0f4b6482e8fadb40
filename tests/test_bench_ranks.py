"""The replicas-only aggregation of bench.py over two gloo ranks on CPU:
max of the per-rank times, sum of the per-rank bytes and launches."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, b, n = bench.combine_ranks(10.0 + rank, 100.0 * (rank + 1), 7 + rank)
    out[rank] = (t, b, n)
    dist.destroy_process_group()


def test_combine_ranks_two_gloo_ranks():
    world = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as m:   # no fork of a process with threads
        out = m.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True,
                           start_method="spawn")
        res = dict(out)
    for r in range(world):
        assert res[r] == (11.0, 300.0, 15)


def test_combine_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_ranks(3.0, 5.0, 2) == (3.0, 5.0, 2)
