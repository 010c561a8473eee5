"""Replica aggregation of bench.py under a 2-rank process group (gloo, CPU): the
reported time is the slowest rank's and the value counts every rank's work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = [1200.0, 1500.0][rank]             # rank 1 is the slow one
        ms_max = bench.reduce_max(ms_local, dist, torch.device("cpu"))
        value = bench.replica_throughput(2.0e11, 5, ms_max, world)
        out[rank] = (ms_max, value)
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_time():
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1]
    ms_max, value = res[0]
    assert ms_max == 1500.0
    assert value == pytest.approx(2 * 2.0e11 * 5 / 1.5 / 1e9)


def test_single_process_needs_no_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, None, None) == 3.5
    assert bench.replica_throughput(1e9, 2, 1000.0, 1) == pytest.approx(2.0)
