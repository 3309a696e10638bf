"""Full-size workloads in the benchmark's launch configuration, checked on
samples the oracle can afford: the whole tree and list sizes exactly, and the
field of randomly sampled leaves (the oracle evaluates only those leaves and
the cells above them).  The 10^6 ferrofluid is the benchmark workload; the
4.2 x 10^6 ring is the nanomagnet workload."""
import numpy as np
import pytest

import oracle as O
from paper_0810_0233_gb300 import ccfmm as C
from paper_0810_0233_gb300 import workloads as W

import local_parity as LP

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def _sampled(pos, mom, p, theta, nleaves, seed, precisions=("mixed",)):
    f = O.OracleFMM(pos, mom, p, theta, 0.0)
    f.upward()
    L = f.depth
    leaf_of = f.leaf_of()
    occupied = np.unique(leaf_of)
    rng = np.random.default_rng(seed)
    pick = rng.choice(occupied, size=min(nleaves, len(occupied)), replace=False)
    mask = np.zeros(1 << L, np.uint8)
    mask[pick] = 1
    f.downward(mask)
    Href = f.field()
    sel = np.isin(leaf_of, pick)
    out = {}
    # the cells the oracle evaluated: ancestors (levels >= 2) of the picked leaves
    cells = sorted({(1 << l) + int(k >> (L - l)) for k in pick for l in range(2, L + 1)})
    cols = np.array([O.index(n) for n in C.multi_indices(p)])
    for prec in precisions:
        with C.FMM(pos, mom, p, theta, 0.0, precision=prec) as g:
            H = g.field()
            st = g.stats()
            assert st["depth"] == L
            assert np.array_equal(g.leaf_of(), leaf_of)
            if prec == "mixed":
                # local bounds: every sampled dipole and every evaluated cell
                assert LP.dipole_max_err(H[sel], Href[sel]) < LP.DIPOLE_TOL
                err = LP.cell_errors(g.expansions("V"), f.locals()[:, cols], cells,
                                     C.multi_indices(p), f.box(), f.axes())
                assert max(err.values()) < LP.CELL_TOL, err
        out[prec] = (H, st)
    ne = np.zeros(1 << (L + 1), dtype=bool)
    for l in range(L + 1):
        ne[(1 << l) + np.unique(leaf_of >> (L - l))] = True
    far, near = f.far_pairs(), f.near_pairs()
    nfar = int((ne[far[:, 0]] & ne[far[:, 1]]).sum())
    nnear = int((ne[near[:, 0]] & ne[near[:, 1]]).sum())
    return Href, sel, out, nfar, nnear


def test_ferrofluid_1e6_p6():
    pos, mom = W.ferrofluid()
    Href, sel, out, nfar, nnear = _sampled(pos, mom, 6, 0.5, 24, 5, ("mixed", "fp64"))
    Hm, st = out["mixed"]
    H64, _ = out["fp64"]
    assert st["far_pairs"] == nfar and st["near_leaf_pairs"] == nnear
    assert rel(H64[sel], Href[sel]) < 1e-12
    assert rel(Hm[sel], Href[sel]) < 1e-5
    # FP32 mixed against the FP64 path on every dipole
    assert rel(Hm, H64) < 1e-5
    # against the direct sum on a random subset
    sub = W.subset(len(pos), 2000, 3)
    Hd = C.direct_field(pos, mom, targets=sub)
    assert rel(Hm[sub], Hd) < 1e-4


def test_ring_4m_p6_theta04():
    pos, mom = W.ring()
    assert len(pos) == 4_194_432
    Href, sel, out, nfar, nnear = _sampled(pos, mom, 6, 0.4, 12, 6)
    Hm, st = out["mixed"]
    assert st["far_pairs"] == nfar and st["near_leaf_pairs"] == nnear
    assert rel(Hm[sel], Href[sel]) < 1e-5
    sub = W.subset(len(pos), 1000, 4)
    assert rel(Hm[sub], C.direct_field(pos, mom, targets=sub)) < 1e-4


def test_ensemble_512_p5():
    """The ensemble in the bench's configuration: all 512 samples (sum N =
    18,752,310) stepped by one graph launch per step.  After two steps every
    rotated moment against the oracle's rotation, and the field and energy of
    sampled samples (the six smallest and two random ones) against the oracle
    FMM on the rotated moments."""
    pos, mom, off = W.ensemble()
    assert len(off) == 513 and off[-1] == 18_752_310
    p, theta, seed = 5, 0.5, 810237
    with C.Batch(pos, mom, off, p, theta) as b:
        H = np.zeros((b.total, 3))
        E = np.zeros(b.ns)
        for step in range(2):
            b.step(seed=seed, step=step, max_angle=0.05, H_out=H, E_out=E)
        M = b.moments()
    ref_m = mom
    for step in range(2):
        ref_m = O.rotate_moments(ref_m, seed, step, 0.05)
    assert np.abs(M - ref_m).max() < 1e-14
    sizes = np.diff(off)
    rng = np.random.default_rng(9)
    pick = list(np.argsort(sizes)[:6]) + list(rng.choice(np.where(sizes < 40000)[0], 2,
                                                          replace=False))
    for s in pick:
        sl = slice(off[s], off[s + 1])
        Hr, Er, _ = O.fmm_field(pos[sl], ref_m[sl], p, theta)
        assert rel(H[sl], Hr) < 1e-5, s
        assert LP.dipole_max_err(H[sl], Hr) < LP.DIPOLE_TOL, s
        assert abs(E[s] - Er) <= 1e-4 * abs(Er), s
