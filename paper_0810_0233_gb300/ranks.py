"""Host-side logic of multi-process runs (one process per GPU).

The ensemble's samples are independent, so they are dealt round-robin over
the ranks and every rank steps its own share with no collective inside the
step; only the report reduces over ranks: the timed total by its maximum (the
slowest rank bounds the whole job) and the dipole counts by their sum.  A
single system is not sharded (every rank runs a replica).

`dist` is torch.distributed with an initialised process group (NCCL on the
GPUs, gloo in the CPU tests) or None for one process.
"""
from __future__ import annotations

import numpy as np


def shard(offsets, rank: int, world: int):
    """Samples i with i mod world == rank.  Returns (sample ids, local
    offsets of their concatenation, the global row ranges [start, end))."""
    off = np.asarray(offsets, dtype=np.int64)
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside 0..%d" % (rank, world - 1))
    ids = np.arange(rank, len(off) - 1, world, dtype=np.int64)
    sizes = off[ids + 1] - off[ids]
    local = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    rows = np.stack([off[ids], off[ids + 1]], axis=1) if len(ids) else np.zeros((0, 2), np.int64)
    return ids, local, rows


def gather_rows(x, rows):
    """The rows of the global array x that a shard owns, concatenated."""
    if len(rows) == 0:
        return x[:0]
    return np.concatenate([x[a:b] for a, b in rows])


def _reduce(value: float, op, dist, device):
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op(dist))
    return float(t.item())


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The largest value over the ranks (timed totals)."""
    return _reduce(value, lambda d: d.ReduceOp.MAX, dist, device)


def sum_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The sum over the ranks (dipoles processed)."""
    return _reduce(value, lambda d: d.ReduceOp.SUM, dist, device)
