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


# ---- one job's RHS partitioned over replicas (paper_2108_08730_gb300.replicas)

from paper_2108_08730_gb300 import replicas as RP


def test_rhs_partition_covers_every_rhs_once():
    for nrhs in (0, 1, 5, 16, 64, 67):
        for world in (1, 2, 3, 4, 8):
            seen = []
            sizes = []
            for rank in range(world):
                lo, hi = RP.rhs_slice(nrhs, world, rank)
                seen.extend(range(lo, hi))
                sizes.append(hi - lo)
            assert seen == list(range(nrhs))               # contiguous, in order, each once
            assert max(sizes) - min(sizes) <= 1
    src = [(3, 4, 5, r, 1.0 + r) for r in range(7)] + [(6, 6, 6, 2, 0.5j)]   # two sources on RHS 2
    got = []
    for rank in range(3):
        mine, (lo, hi) = RP.local_sources(src, 7, 3, rank)
        assert all(0 <= s[3] < hi - lo for s in mine)
        got.extend((s[0], s[1], s[2], s[3] + lo, s[4]) for s in mine)
    assert sorted(got, key=str) == sorted(src, key=str)


def _oracle_solve(sources, nrhs):
    """CPU oracle (banded LU of the assembled matrix) standing in for each
    rank's GPU solve of its RHS slice."""
    import numpy as np
    from oracle import operator as O
    from oracle import solve as S
    from oracle import weights as W
    from paper_2108_08730_gb300 import synth
    nodes, T = W.fit_table()
    wl = synth.homogeneous(n=10, npml=2)
    wl.v = synth.random_velocity(wl.shape, 9, 1500.0, 2500.0)
    prof = O.profiles_for(wl.shape, wl.h, wl.npml, 2500.0, wl.r_coef)
    A = O.assemble_csr(wl.v, wl.h, wl.f, prof, T, nodes)
    rhs = np.zeros((nrhs,) + wl.shape, dtype=np.complex128)
    for ix, iy, iz, r, amp in sources:
        rhs[r] += S.point_sources(wl.shape, wl.h, [(ix, iy, iz)], amps=[amp])[0]
    if nrhs == 0:
        return torch.zeros((0,) + wl.shape, dtype=torch.complex128)
    x = S.solve_banded(A, rhs.reshape(nrhs, -1).T).T.reshape(rhs.shape)
    return torch.from_numpy(x)


_SOURCES = [(4, 4, 4, 0, 1.0), (5, 3, 6, 1, 1j), (3, 6, 5, 2, 2.0), (6, 5, 3, 3, -1.0), (4, 6, 4, 4, 0.5)]


def _partition_rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine, (lo, hi) = RP.local_sources(_SOURCES, 5, world, rank)
        local = _oracle_solve(mine, hi - lo)
        full = RP.gather_wavefields(local, 5, world, rank)
        if rank == 0:
            out["gathered"] = full.numpy()
        else:
            out[f"none{rank}"] = full is None
    finally:
        dist.destroy_process_group()


def test_two_rank_partitioned_solve_equals_one_rank():
    import numpy as np
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_partition_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    ref = _oracle_solve(_SOURCES, 5).numpy()
    assert out["none1"]
    assert np.array_equal(out["gathered"], ref)
