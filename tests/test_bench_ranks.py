"""The replica aggregation of bench.py under torch.distributed (gloo, two
ranks on the CPU): max of the times, sum of the work."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    maxes, sums = bench.reduce_over_ranks([10.0 + rank, 1.0], [100.0 * (rank + 1)], "cpu")
    out[rank] = (maxes, sums)
    dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    import torch.multiprocessing as mp
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    os.environ["PYTHONPATH"] = root + os.pathsep + os.environ.get("PYTHONPATH", "")
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    for r in range(2):
        maxes, sums = out[r]
        assert maxes == [11.0, 1.0]
        assert sums == [300.0]


def test_single_process_is_identity():
    import bench
    assert bench.reduce_over_ranks([3.0], [4.0, 5.0], "cpu") == ([3.0], [4.0, 5.0])
