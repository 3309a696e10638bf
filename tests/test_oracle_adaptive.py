"""Pins of the oracle's adaptive-depth tree (a project extension: the paper's
tree is complete, Sec. II and Appendix).

Independent statements it is checked against:
  * on inputs where every leaf lands at one depth it is the uniform oracle
    (itself pinned in ``test_oracle_pins.py``): same lists, same field;
  * brute force over every ordered pair of points: each pair (i, j), i != j,
    is covered exactly once, either by a nearPartners leaf of i's leaf or by
    exactly one far pair (T, S) with T holding i and S holding j;
  * the direct dipole sum: the error falls with p, and with every pair near
    (a tiny opening angle) the method is the direct sum;
  * the tree's own definition: leaves hold at most s points, split cells more;
  * symmetry of the near and far relations, which the near test implies.
"""
import numpy as np

import oracle as O
from paper_0810_0233_gb300 import workloads as W


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def _clustered(n, seed):
    return W.clustered(n, seed=seed, blob_size=60, chain_len=10)


def _points_of(cells, perm, c):
    p0, np_ = cells[c, 4], cells[c, 5]
    return perm[p0:p0 + np_]


def pin_adaptive_matches_uniform():
    """8^3 and 16 x 8 x 8 lattices at s = 8: every leaf holds 8 points at one
    depth, so the adaptive tree is the complete tree of the uniform oracle."""
    ok = True
    for dims in ((8, 8, 8), (16, 8, 8)):
        pos, mom, box = W.lattice(*dims, seed=W.BASE_SEED + 60)
        Hu, Eu, fu = O.fmm_field(pos, mom, 5, 0.5, 8.0, box=box)
        Ha, Ea, fa = O.afmm_field(pos, mom, 5, 0.5, 8.0, box=box)
        cells = fa.cells()
        leaf_levels = np.unique(cells[cells[:, 6] == 1, 0])
        ok &= list(leaf_levels) == [fu.depth]
        ok &= len(fa.pairs("far")) == len(fu.far_pairs())
        ok &= len(fa.pairs("near")) == len(fu.near_pairs())
        ok &= _rel(Ha, Hu) < 1e-13 and abs(Ea - Eu) <= 1e-12 * abs(Eu)
    return bool(ok)


def pin_adaptive_coverage():
    """Clustered points, s = 4 (leaves at many depths): exact pair coverage."""
    pos, mom = _clustered(300, 61)
    f = O.OracleAFMM(pos, mom, 3, 0.5, 4.0)
    cells, perm = f.cells(), f.perm()
    n = len(pos)
    cover = np.zeros((n, n), dtype=np.int64)
    for t, s in f.pairs("far"):
        cover[np.ix_(_points_of(cells, perm, t), _points_of(cells, perm, s))] += 1
    far_only = cover.copy()
    for t, s in f.pairs("near"):
        cover[np.ix_(_points_of(cells, perm, t), _points_of(cells, perm, s))] += 1
    off = ~np.eye(n, dtype=bool)
    levels = cells[:, 0]
    far = f.pairs("far")
    near = f.pairs("near")
    unequal = (levels[far[:, 0]] != levels[far[:, 1]]).any() and \
        (levels[near[:, 0]] != levels[near[:, 1]]).any()
    return bool(np.all(cover[off] == 1) and np.all(np.diag(far_only) == 0) and unequal)


def pin_adaptive_converges():
    """Clustered points: the field error against the direct sum falls with p."""
    pos, mom = _clustered(600, 62)
    Hd = O.direct_field(pos, mom)
    errs = []
    for p in (2, 4, 6, 8):
        H, E, f = O.afmm_field(pos, mom, p, 0.5, 6.0)
        errs.append(_rel(H, Hd))
    return all(b < a for a, b in zip(errs, errs[1:])) and errs[-1] < 1e-5


def pin_adaptive_all_near_is_direct():
    """theta so small that no pair is far: the method is the direct sum."""
    pos, mom = _clustered(240, 63)
    H, E, f = O.afmm_field(pos, mom, 3, 0.02, 4.0)
    Hd = O.direct_field(pos, mom)
    return len(f.pairs("far")) == 0 and _rel(H, Hd) < 1e-13


def pin_adaptive_symmetry():
    """The lists are symmetric: (A, B) is a near pair iff (B, A) is, and the
    same for far pairs, including pairs of unequal levels (both sides stop
    at the same cell of the other's subtree: the near test is symmetric)."""
    pos, mom = _clustered(400, 65)
    f = O.OracleAFMM(pos, mom, 2, 0.5, 4.0)
    ok = True
    for kind in ("near", "far"):
        pr = {tuple(map(int, x)) for x in f.pairs(kind)}
        ok &= all((b, a) in pr for a, b in pr)
    return bool(ok)


def pin_adaptive_tree():
    """Leaves hold at most s points; split cells more; children partition."""
    pos, mom = _clustered(500, 64)
    s = 5.0
    f = O.OracleAFMM(pos, mom, 2, 0.5, s)
    cells, perm = f.cells(), f.perm()
    ok = sorted(perm.tolist()) == list(range(len(pos)))
    for c, (lev, par, c0, c1, p0, cnt, leaf) in enumerate(cells):
        if leaf:
            ok &= cnt <= s
        else:
            ok &= cnt > s
            kids = [k for k in (c0, c1) if k >= 0]
            ok &= sum(cells[k, 5] for k in kids) == cnt
            ok &= all(cells[k, 0] == lev + 1 and cells[k, 1] == c for k in kids)
    return bool(ok)


def test_adaptive_matches_uniform():
    assert pin_adaptive_matches_uniform()


def test_adaptive_coverage():
    assert pin_adaptive_coverage()


def test_adaptive_converges():
    assert pin_adaptive_converges()


def test_adaptive_all_near_is_direct():
    assert pin_adaptive_all_near_is_direct()


def test_adaptive_symmetry():
    assert pin_adaptive_symmetry()


def test_adaptive_tree():
    assert pin_adaptive_tree()
