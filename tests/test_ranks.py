"""Multi-process host logic (ranks.py) with two gloo ranks on the CPU: the
ensemble's samples are dealt so that every sample is stepped by exactly one
rank, each rank's rows are its samples in order, and the report's reductions
(maximum of the timed totals, sum of the dipole counts) agree on every rank."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_0810_0233_gb300 import ranks as R
from paper_0810_0233_gb300 import workloads as W


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, off, q):
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank,
                            world_size=world)
    try:
        ids, local, rows = R.shard(off, rank, world)
        x = np.arange(int(off[-1]), dtype=np.float64)
        mine = R.gather_rows(x, rows)
        t = R.max_over_ranks(1.5 + rank, dist)
        n = R.sum_over_ranks(float(local[-1]), dist)
        q.put((rank, ids.tolist(), local.tolist(), mine.tolist(), t, n))
    finally:
        dist.destroy_process_group()


def test_shard_single_process():
    off = np.array([0, 3, 3, 10, 12], dtype=np.int64)
    ids, local, rows = R.shard(off, 0, 1)
    assert ids.tolist() == [0, 1, 2, 3] and local.tolist() == [0, 3, 3, 10, 12]
    ids, local, rows = R.shard(off, 1, 3)
    assert ids.tolist() == [1] and local.tolist() == [0, 0] and rows.tolist() == [[3, 3]]
    with pytest.raises(ValueError):
        R.shard(off, 2, 2)
    assert R.max_over_ranks(2.5) == 2.5 and R.sum_over_ranks(4.0) == 4.0


def test_two_gloo_ranks():
    sizes = W.ensemble_sizes(count=9, n_lo=10, n_hi=200, seed=5)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, off, q)) for r in range(world)]
    for p_ in procs:
        p_.start()
    res = {}
    for _ in range(world):
        r, ids, local, mine, t, n = q.get(timeout=120)
        res[r] = (ids, local, mine, t, n)
    for p_ in procs:
        p_.join(timeout=60)
        assert p_.exitcode == 0
    # every sample exactly once, dealt round-robin
    all_ids = sorted(res[0][0] + res[1][0])
    assert all_ids == list(range(len(sizes)))
    assert res[0][0] == list(range(0, len(sizes), 2)) and res[1][0] == list(range(1, len(sizes), 2))
    x = np.arange(int(off[-1]), dtype=np.float64)
    for r in range(world):
        ids, local, mine, t, n = res[r]
        expect = np.concatenate([x[off[i]:off[i + 1]] for i in ids])
        assert np.array_equal(np.asarray(mine), expect)
        assert local[-1] == len(expect)
        assert t == 2.5  # the slowest rank
        assert n == float(off[-1])  # all dipoles
