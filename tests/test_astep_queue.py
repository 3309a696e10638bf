"""The persistent step's task queue (fmm_adaptive_queue, host only): the
properties the kernel relies on, checked on random forest shapes.

- need[ph] is the number of tasks of phase ph;
- every phase a task waits for lies wholly before it in the queue (blocks
  take tasks in queue order, so the earliest unfinished task never waits on
  a later one: the queue cannot deadlock whatever number of blocks runs);
- every dipole chunk, leaf, cell of each level, M2L item and sample is
  covered exactly once by its stage's tasks;
- the stages depend on one another as the evaluation does: permutation after
  rotation, P2M after it, M2M from the deepest level up, the fold, M2L, L2L
  from the roots down, the near field after the permutation, L2P after the
  last L2L level and the whole near field, then the unpermute and energies.
"""
import numpy as np
import pytest

from paper_0810_0233_gb300 import ccfmm as C

ROT, PERM, P2M, M2M, FOLD, BIG, SMALL, L2L, P2P, L2P, UNPERM, ENERGY = range(12)


def decode(tasks):
    typ = tasks[:, 0] & 255
    ph = tasks[:, 0] >> 8
    w1 = (tasks[:, 3] & 0xFFFF) - 1
    w2 = ((tasks[:, 3] >> 16) & 0xFFFF) - 1
    return typ, ph, tasks[:, 1], tasks[:, 2], w1, w2


def covered(ranges, n):
    hit = np.zeros(n, np.int64)
    for a, b in ranges:
        hit[a:b] += 1
    return hit


def check_queue(N, ns, nleaf, off, n_big, n_small):
    nc = int(off[-1])
    maxL = len(off) - 2
    tasks, need, (chunk, cells, groups) = C.adaptive_queue(N, ns, nleaf, nc, off, n_big, n_small)
    typ, ph, y, z, w1, w2 = decode(tasks)
    nph = len(need)
    # phase counts
    assert np.array_equal(np.bincount(ph, minlength=nph), need)
    # waits refer to phases wholly earlier in the queue
    last = np.full(nph, -1)
    for i, p in enumerate(ph):
        last[p] = i
    pos = np.arange(len(tasks))
    for w in (w1, w2):
        m = w >= 0
        assert np.all(w[m] < nph)
        assert np.all(last[w[m]] < pos[m])
    # one phase per stage, except M2M and L2L (one per non-empty level)
    for t in (ROT, PERM, P2M, FOLD, P2P, L2P, UNPERM, ENERGY):
        assert len(set(ph[typ == t])) == 1, t
    # coverage
    nch = (N + chunk - 1) // chunk
    for t in (ROT, PERM, UNPERM):
        assert sorted(y[typ == t]) == list(range(nch))
    for t in (P2M, L2P):
        r = [(a, min(b, a + cells)) for a, b in zip(y[typ == t], z[typ == t])]
        assert np.all(z[typ == t] == nleaf)
        assert np.all(covered(r, nleaf) == 1)
    assert sorted(y[typ == P2P]) == list(range(nleaf))
    r = [(a, min(b, a + cells)) for a, b in zip(y[typ == FOLD], z[typ == FOLD])]
    assert np.all(covered(r, nc) == 1)
    assert sorted(y[typ == BIG]) == list(range(n_big))
    ng = (n_small + 3) // 4
    r = [(a, min(b, a + groups)) for a, b in zip(y[typ == SMALL], z[typ == SMALL])]
    assert np.all(covered(r, ng) == 1) and np.all(z[typ == SMALL] == ng)
    assert sorted(y[typ == ENERGY]) == list(range(ns))
    for t, levels in ((M2M, range(maxL)), (L2L, range(maxL + 1))):
        want = np.zeros(nc, np.int64)
        for l in levels:
            want[off[l]:off[l + 1]] = 1
        sel = typ == t
        r = [(a, min(b, a + cells)) for a, b in zip(y[sel], z[sel])]
        assert np.array_equal(covered(r, nc), want), t
        # every tile lies in one level, and a level's tiles share a phase
        lev = np.searchsorted(off, y[sel], side="right") - 1
        assert np.all(z[sel] == off[lev + 1])
        for l in set(lev):
            assert len(set(ph[sel][lev == l])) == 1
    # dependencies between the stages
    def phase_of(t):
        return ph[typ == t][0]
    assert np.all(w1[typ == ROT] == -1) and np.all(w2[typ == ROT] == -1)
    assert np.all(w1[typ == PERM] == phase_of(ROT))
    assert np.all(w1[typ == P2P] == phase_of(PERM))
    # the far chain's phases are consecutive and each waits for the one
    # before it: P2M, M2M from the deepest level, the fold, M2L (a phase
    # even when it has no items), L2L from the roots
    first, final = phase_of(P2M), w1[typ == L2P][0]
    assert np.all(w1[typ == P2M] == phase_of(PERM))
    chain = (ph > first) & (ph <= final)
    assert np.all(w1[chain] == ph[chain] - 1) and np.all(w2[chain] == -1)
    assert set(typ[chain]) <= {M2M, FOLD, BIG, SMALL, L2L}
    fold = phase_of(FOLD)
    for t, sign in ((M2M, -1), (L2L, 1)):
        sel = typ == t
        lev = np.searchsorted(off, y[sel], side="right") - 1
        order = [ph[sel][lev == l][0] for l in sorted(set(lev), key=lambda l: sign * l)]
        assert order == sorted(order)
        if t == M2M:
            assert all(f < fold for f in order)
        else:
            assert all(f > fold + 1 for f in order)
    m2l = (typ == BIG) | (typ == SMALL)
    assert np.all(ph[m2l] == fold + 1)
    far = [final]
    assert np.all(w1[typ == L2P] == far[-1]) and np.all(w2[typ == L2P] == phase_of(P2P))
    assert np.all(w1[typ == UNPERM] == phase_of(L2P))
    assert np.all(w1[typ == ENERGY] == phase_of(UNPERM))


@pytest.mark.parametrize("seed", range(12))
def test_queue_properties_on_random_shapes(seed):
    rng = np.random.default_rng(seed)
    maxL = int(rng.integers(0, 14))
    counts = rng.integers(0, 400, maxL + 1)
    counts[0] = max(counts[0], 1)
    if seed % 3 == 0 and maxL > 2:
        counts[rng.integers(1, maxL)] = 0  # an empty level
    off = np.concatenate([[0], np.cumsum(counts)])
    nc = int(off[-1])
    nleaf = int(rng.integers(1, nc + 1))
    N = int(rng.integers(1, 50_000))
    ns = int(rng.integers(1, 6))
    check_queue(N, ns, nleaf, off, int(rng.integers(0, 300)), int(rng.integers(0, 2000)))


def test_queue_of_single_leaves_and_no_m2l():
    """Every sample a single root leaf: no M2M level, no M2L item."""
    check_queue(5, 5, 5, np.array([0, 5]), 0, 0)


def test_queue_rejects_inconsistent_shapes():
    with pytest.raises(C.CCFMMError):
        C.adaptive_queue(100, 1, 10, 20, [1, 10, 20], 0, 0)  # offsets not from 0
    with pytest.raises(C.CCFMMError):
        C.adaptive_queue(100, 1, 10, 20, [0, 12, 10, 20], 0, 0)  # decreasing
    with pytest.raises(C.CCFMMError):
        C.adaptive_queue(100, 1, 10, 20, [0, 10, 19], 0, 0)  # not ending at ncells
    with pytest.raises(C.CCFMMError):
        C.adaptive_queue(100, 1, 30, 20, [0, 10, 20], 0, 0)  # more leaves than cells
