"""The multi-GPU form is replicas only (independent problems, no data-path
collective): the bench's whole-job value is every rank's point*RHS over the
slowest rank's time.  This checks that aggregation with two gloo ranks on CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 * (rank + 1)                  # rank 1 is the slow one
        m = bench.reduce_max_ms(local_ms, world, "cpu")
        out[rank] = (m, bench.aggregate_rate(2.0e6, world, 4, m))
    finally:
        dist.destroy_process_group()


def test_two_rank_replica_aggregation():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        m, rate = out[r]
        assert m == 200.0                               # max over ranks, on every rank
        assert abs(rate - 2.0e6 * 2 * 4 / 0.2 / 1e6) < 1e-9


def test_single_rank_is_identity():
    assert bench.reduce_max_ms(12.5, 1) == 12.5
    assert bench.aggregate_rate(1e6, 1, 2, 1000.0) == 2.0
