"""The N > 1 path of bench.py on CPU: world_size 2 over gloo.  The solve does
not shard (replicas only), so the only exchange is the timing reduction: the
slowest rank's time and the sum of all ranks' units."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r solved 100 (r + 1) units in 10 (r + 1) ms
        ms, rate = bench.replica_throughput(dist, "cpu", 100.0 * (rank + 1), 10.0 * (rank + 1))
        out[rank] = (ms, rate)
    finally:
        dist.destroy_process_group()


def test_replica_throughput_two_ranks_gloo():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank, args=(2, _free_port(), out), nprocs=2, join=True)
    for r in range(2):
        ms, rate = out[r]
        assert ms == 20.0                       # the slowest rank
        assert rate == pytest.approx(300.0 / 0.020)  # all ranks' units over that time


def test_replica_throughput_one_process():
    import bench
    ms, rate = bench.replica_throughput(None, "cpu", 1000.0, 4.0)
    assert ms == 4.0 and rate == pytest.approx(250000.0)
