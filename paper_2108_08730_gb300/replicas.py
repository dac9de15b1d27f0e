"""One job's right-hand sides spread over replicas (one process per GPU).

The solve shards by independent units: every RHS (source) of a (model,
frequency) problem is solved independently, so each rank holds a replica of
the velocity, weight table and multigrid hierarchy and takes a disjoint,
contiguous slice of the RHS.  Nothing is exchanged on the data path; the
host gathers the wavefields at the end (or each rank writes its own).

Pure host logic (no arithmetic of the method), shared by bench.py and the
tests; it works with any torch.distributed backend (gloo on CPU in tests).
"""
from __future__ import annotations


def rhs_slice(nrhs: int, world: int, rank: int) -> tuple[int, int]:
    """[lo, hi) of the RHS owned by `rank`: contiguous, sizes differ by at
    most one, the first nrhs % world ranks take the larger share."""
    if world < 1 or not 0 <= rank < world or nrhs < 0:
        raise ValueError("need world >= 1, 0 <= rank < world, nrhs >= 0")
    q, r = divmod(nrhs, world)
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def local_sources(sources, nrhs: int, world: int, rank: int):
    """The rank's share of a source list [(ix, iy, iz, rhs, amp)] with its RHS
    renumbered from 0, and the slice (lo, hi) of the global RHS it covers."""
    lo, hi = rhs_slice(nrhs, world, rank)
    mine = [(ix, iy, iz, rhs - lo, amp) for ix, iy, iz, rhs, amp in sources if lo <= rhs < hi]
    return mine, (lo, hi)


def gather_wavefields(local, nrhs: int, world: int, rank: int, dst: int = 0):
    """Gather every rank's wavefields (a CPU torch tensor (hi - lo, ...)) into
    one (nrhs, ...) tensor on rank `dst` (None elsewhere).  Uses
    torch.distributed.gather_object, so it runs on gloo as well as on nccl
    process groups; world == 1 returns `local` itself."""
    if world == 1:
        return local
    import torch
    import torch.distributed as dist
    parts = [None] * world if rank == dst else None
    dist.gather_object((rank, local), parts, dst=dst)
    if rank != dst:
        return None
    out = None
    for r, part in parts:
        lo, hi = rhs_slice(nrhs, world, r)
        if part.shape[0] != hi - lo:
            raise RuntimeError(f"rank {r} returned {part.shape[0]} RHS, expected {hi - lo}")
        if out is None:
            out = torch.empty((nrhs,) + tuple(part.shape[1:]), dtype=part.dtype)
        out[lo:hi] = part
    return out
