"""Adaptive-depth tree on the GPU (fmm_adaptive_*, through the C-ABI)
against the CPU oracle's adaptive mode (oracle/ccfmm_oracle.c, orc_afmm_*).

Bars: cells (level, parent, children, dipole range, leaf flag) equal to the
oracle's, cell for cell in creation order; each cell's dipoles the same set;
near and far pairs equal as sets; FP64 fields, energies, Q and V within
1e-12 (relative RMS); the mixed path within 1e-5 plus the local bounds of
``local_parity`` (every dipole, every cell's V against the oracle's).
Several samples in one handle are checked sample by sample.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_0810_0233_gb300 import ccfmm as C
from paper_0810_0233_gb300 import workloads as W

import local_parity as LP

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOLMIX = 1e-5


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


def lib_to_oracle_cols(p):
    """Oracle columns of the library's coefficient columns (multi-indices
    1 .. T(p) - 1 in library order)."""
    return np.array([O.index(n) for n in C.multi_indices(p)[1:]])


def check_structure(g, f, c0=0, p0=0):
    """Library cells [c0, c0 + nc) and dipoles [p0, p0 + n) against one
    sample's oracle tree."""
    oc = f.cells()
    nc = len(oc)
    gc = g.cells()[c0:c0 + nc].copy()
    for k in (1, 2, 3):
        m = gc[:, k] >= 0
        gc[m, k] -= c0
    gc[:, 4] -= p0
    assert np.array_equal(gc[:, :7], oc), "cells differ from the oracle's"
    gp = g.perm()
    op = f.perm()
    for c in np.nonzero(oc[:, 6])[0]:
        a, n = oc[c, 4], oc[c, 5]
        assert set(gp[p0 + a:p0 + a + n] - p0) == set(op[a:a + n])
    for kind in ("near", "far"):
        gpairs = g.pairs(kind)
        sel = (gpairs[:, 0] >= c0) & (gpairs[:, 0] < c0 + nc)
        gs = {(int(a) - c0, int(b) - c0) for a, b in gpairs[sel]}
        os_ = {(int(a), int(b)) for a, b in f.pairs(kind)}
        assert gs == os_, kind
        assert sel.sum() == len(f.pairs(kind)), "duplicate pairs"


def check_fp64(H, E, Q, V, f, pos_n, p):
    cols = lib_to_oracle_cols(p)
    assert rel(H, f.field()) < TOL64
    assert abs(E - f.energy()) <= TOL64 * abs(f.energy()) * 10
    assert rel(Q, f.moments()[:, cols]) < TOL64
    assert rel(V, f.locals()[:, cols]) < TOL64


def energy_bar(f, Href):
    """Bar on the mixed energy: 10 TOLMIX |E|, or, where the sum -1/2 sum m.H
    cancels, what the field bar implies: |dE| = 1/2 |sum m.dH| <=
    1/2 |m| |dH| (Cauchy-Schwarz) with |dH| < TOLMIX |H|."""
    cs = 0.5 * np.linalg.norm(f.mom) * np.linalg.norm(Href)
    return max(10 * TOLMIX * abs(f.energy()), TOLMIX * cs)


def check_mixed(H, E, V, f, p):
    Href = f.field()
    assert rel(H, Href) < TOLMIX
    assert abs(E - f.energy()) <= energy_bar(f, Href)
    assert LP.dipole_max_err(H, Href) < LP.DIPOLE_TOL
    oc = f.cells()
    Vo = f.locals()[:, lib_to_oracle_cols(p)]
    rows = np.arange(len(oc))
    w = f.widths()
    rho = 0.5 * np.sqrt((w ** 2).sum(1))
    if np.abs(Vo).max() > 0:
        err = LP.cell_errors_levels(V, Vo, rows, oc[:, 0], rho, C.multi_indices(p)[1:])
        assert max(err.values()) < LP.CELL_TOL, err


CASES = [
    ("clustered", 3000, 4, 0.5, 12.0),
    ("clustered", 8000, 5, 0.5, 26.0),
    ("clustered", 6000, 6, 0.4, 18.0),
    ("ferrofluid", 5000, 5, 0.5, 20.0),
    ("ring", 0, 4, 0.5, 10.0),
    ("lattice", 0, 3, 0.5, 8.0),
    ("clustered", 2500, 7, 0.5, 20.0),  # FP32 FMA contraction (no tensor-core form at p = 7)
    ("clustered", 1500, 8, 0.6, 16.0),
]


def workload(kind, n):
    if kind == "clustered":
        return W.clustered(n, seed=n + 17), None
    if kind == "ferrofluid":
        return W.ferrofluid(n, side=100.0 * (n / 1e6) ** (1 / 3), seed=W.BASE_SEED + 31), None
    if kind == "ring":
        return W.ring(r_out=30.0, r_in=10.0, layers=2), None
    pos, mom, box = W.lattice(12)
    return (pos, mom), box


@pytest.mark.parametrize("kind,n,p,theta,s", CASES)
def test_single_system_equals_oracle(kind, n, p, theta, s):
    (pos, mom), box = workload(kind, n)
    f = O.OracleAFMM(pos, mom, p, theta, s, box=box)
    f.run()
    with C.Adaptive(pos, mom, p, theta, split=s, box=box, precision="fp64") as g:
        check_structure(g, f)
        H, E = g.evaluate()
        Q, V = g.expansions()
        check_fp64(H, E[0], Q, V, f, len(pos), p)
        st = g.stats()
        assert st["ncells"] == len(f.cells())
        assert st["far_pairs"] == len(f.pairs("far"))
    with C.Adaptive(pos, mom, p, theta, split=s, box=box, precision="mixed") as g:
        H, E = g.evaluate()
        Q, V = g.expansions()
        check_mixed(H, E[0], V, f, p)
        # repeated evaluations agree to rounding (atomic accumulation order)
        H2, E2 = g.evaluate()
        assert rel(H2, H) < 1e-6


def test_ensemble_equals_oracle_per_sample():
    """Six clustered samples of different sizes and split thresholds in one
    handle: every sample's tree, lists and fields as the oracle's."""
    rng = np.random.default_rng(5)
    sizes = [400, 1500, 900, 5000, 2500, 3000]
    split = [8.0, 12.0, 26.0, 18.0, 40.0, 12.0]
    ps, ms = [], []
    for i, n in enumerate(sizes):
        pos, mom = W.clustered(n, seed=900 + i)
        ps.append(pos + rng.uniform(-1e3, 1e3, 3))
        ms.append(mom)
    off = np.concatenate([[0], np.cumsum(sizes)])
    pos, mom = np.concatenate(ps), np.concatenate(ms)
    p, theta = 5, 0.5
    for prec in ("fp64", "mixed"):
        with C.Adaptive(pos, mom, p, theta, split=split, offsets=off, precision=prec) as g:
            H, E = g.evaluate()
            Q, V = g.expansions()
            cells = g.cells()
            c0 = 0
            for i in range(len(sizes)):
                f = O.OracleAFMM(ps[i], ms[i], p, theta, split[i])
                f.run()
                nc = len(f.cells())
                assert np.all(cells[c0:c0 + nc, 7] == i)
                sl = slice(off[i], off[i + 1])
                if prec == "fp64":
                    check_structure(g, f, c0, off[i])
                    check_fp64(H[sl], E[i], Q[c0:c0 + nc], V[c0:c0 + nc], f, sizes[i], p)
                else:
                    check_mixed(H[sl], E[i], V[c0:c0 + nc], f, p)
                c0 += nc
            assert c0 == len(cells)


def test_step_is_rotation_then_evaluation():
    """fmm_adaptive_step = the oracle's Philox rotation of every moment, then
    an evaluation (FP64 path against the oracle on the rotated moments)."""
    sizes = [700, 1300]
    ps = [W.clustered(n, seed=40 + i)[0] + 500.0 * i for i, n in enumerate(sizes)]
    ms = [W.clustered(n, seed=40 + i)[1] for i, n in enumerate(sizes)]
    off = np.concatenate([[0], np.cumsum(sizes)])
    pos, mom = np.concatenate(ps), np.concatenate(ms)
    with C.Adaptive(pos, mom, 4, 0.5, split=10.0, offsets=off, precision="fp64") as g:
        for step in range(2):
            H, E = g.step(seed=11, step=step, max_angle=0.05)
            mom = O.rotate_moments(mom, 11, step, 0.05)
            assert np.allclose(g.moments(), mom, rtol=0, atol=1e-14)
            for i in range(2):
                sl = slice(off[i], off[i + 1])
                f = O.OracleAFMM(pos[sl], mom[sl], 4, 0.5, 10.0)
                f.run()
                assert rel(H[sl], f.field()) < TOL64
                assert abs(E[i] - f.energy()) <= 1e-11 * abs(f.energy())


def test_degenerate_inputs():
    """A single dipole (root leaf, no lists beyond itself); all dipoles in one
    leaf (no far pairs, no D rows); coincident dipoles deeper than the
    40-level cap (a leaf above s at level 40)."""
    rng = np.random.default_rng(2)
    one = (np.array([[1.0, 2.0, 3.0]]), np.array([[0.0, 0.0, 1.0]]))
    few = (rng.uniform(0, 1, (7, 3)), rng.standard_normal((7, 3)))
    pos = rng.uniform(0, 10, (300, 3))
    pos[:5] = pos[0]  # five dipoles on one point: the r = 0 terms vanish
    dup = (pos, rng.standard_normal((300, 3)))
    for (pos, mom), s in ((one, 8.0), (few, 8.0), (dup, 3.0)):
        f = O.OracleAFMM(pos, mom, 3, 0.5, s)
        f.run()
        with C.Adaptive(pos, mom, 3, 0.5, split=s, precision="fp64") as g:
            check_structure(g, f)
            H, E = g.evaluate()
            assert rel(H, f.field()) < TOL64
            assert abs(E[0] - f.energy()) <= 1e-11 * max(abs(f.energy()), 1e-300)
    with C.Adaptive(dup[0], dup[1], 3, 0.5, split=3.0, precision="fp64") as g:
        assert g.stats()["max_level"] == 40


def test_bad_arguments_rejected():
    pos, mom = W.clustered(500, seed=1)
    with pytest.raises(C.CCFMMError):
        C.Adaptive(pos, mom, 9, 0.5)
    with pytest.raises(C.CCFMMError):
        C.Adaptive(pos, mom, 4, 1.5)
    with pytest.raises(C.CCFMMError):
        C.Adaptive(pos, mom, 4, 0.5, split=0.5)
    bad = pos.copy()
    bad[3, 1] = np.nan
    with pytest.raises(C.CCFMMError):
        C.Adaptive(bad, mom, 4, 0.5)
    with pytest.raises(C.CCFMMError):
        C.Adaptive(pos, mom, 4, 0.5, offsets=[0, 200, 200, 500])


def test_near_pair_cut_on_clustered_sample():
    """On a 20k clustered sample of the ensemble generator (p = 5, theta =
    0.5) the adaptive tree at s = 18 needs far fewer near-field dipole pairs
    than the complete tree at the Eq. so leaf occupancy, and fewer far
    pairs, at an error against the direct sum of the same order."""
    pos, mom = W.clustered(20000, seed=7)
    with C.FMM(pos, mom, 5, 0.5, 0.0, precision="mixed") as u:
        Hu, _ = u.field_energy()
        su = u.stats()
    with C.Adaptive(pos, mom, 5, 0.5, split=18.0, precision="mixed") as g:
        Ha, _ = g.evaluate()
        sa = g.stats()
    assert sa["near_pairs"] < 0.67 * su["p2p_pairs"], (sa, su)
    assert sa["far_pairs"] < su["far_pairs"]
    idx = np.random.default_rng(0).choice(len(pos), 1500, replace=False)
    Hd = O.direct_field(pos, mom, targets=idx)
    eu, ea = rel(Hu[idx], Hd), rel(Ha[idx], Hd)
    assert ea < 1e-4 and eu < 1e-4, (eu, ea)


def test_autotuner_picks_per_class_and_stays_exact():
    """The library's split autotuner: one threshold per size class from the
    candidate set, and the forest it builds agrees with the oracle run at
    each sample's chosen threshold (mixed bounds)."""
    sizes = [600, 700, 2500, 3100, 9000]
    ps, ms = [], []
    for i, n in enumerate(sizes):
        pos, mom = W.clustered(n, seed=300 + i)
        ps.append(pos)
        ms.append(mom)
    off = np.concatenate([[0], np.cumsum(sizes)])
    pos, mom = np.concatenate(ps), np.concatenate(ms)
    p, theta = 5, 0.5
    s0 = O.leaf_size_rule(p)
    cand = [s0 * m for m in (1.0, math.sqrt(2), 2.0, 2 * math.sqrt(2), 4.0)]
    with C.Adaptive(pos, mom, p, theta, offsets=off, autotune=True, trials=1) as g:
        tune = g.tuning()
        assert [c[0] for c in tune] == [600, 2500, 9000]
        for _, sv in tune:
            assert min(abs(sv - c) for c in cand) < 1e-9 * sv
        H, E = g.evaluate()
        Q, V = g.expansions()
        c0 = 0
        for i, n in enumerate(sizes):
            sv = [sv for nmin, sv in tune if nmin <= n][-1]
            f = O.OracleAFMM(ps[i], ms[i], p, theta, sv)
            f.run()
            nc = len(f.cells())
            check_mixed(H[off[i]:off[i + 1]], E[i], V[c0:c0 + nc], f, p)
            c0 += nc


def _forest(sizes, seed0):
    rng = np.random.default_rng(seed0)
    ps, ms = [], []
    for i, n in enumerate(sizes):
        pos, mom = W.clustered(n, seed=seed0 + i)
        ps.append(pos + rng.uniform(-1e3, 1e3, 3))
        ms.append(mom)
    off = np.concatenate([[0], np.cumsum(sizes)])
    return ps, ms, off, np.concatenate(ps), np.concatenate(ms)


@pytest.mark.parametrize("p,theta,split", [(3, 0.5, 10.0), (5, 0.5, 18.0), (6, 0.4, 26.0)])
def test_persistent_step_equals_oracle(p, theta, split):
    """The persistent step kernel (one launch, task queue over all samples'
    stages): every sample within the mixed bounds of the oracle, the same
    fields as the graph of stage kernels to rounding, and a step = the
    oracle's rotation then an evaluation."""
    sizes = [300, 2200, 900, 5000, 1700]
    ps, ms, off, pos, mom = _forest(sizes, 620 + p)
    with C.Adaptive(pos, mom, p, theta, split=split, offsets=off, persistent=True) as g, \
            C.Adaptive(pos, mom, p, theta, split=split, offsets=off) as r:
        assert g.stats()["kernels_per_eval"] == 1
        H, E = g.evaluate()
        Hr, Er = r.evaluate()
        assert rel(H, Hr) < 1e-6
        for i in range(len(sizes)):
            # both energies are -1/2 sum m.H of their own fields (FP64 sums):
            # |E - Er| <= 1/2 |m| |H - Hr| (Cauchy-Schwarz) + rounding
            sl = slice(off[i], off[i + 1])
            mn = np.linalg.norm(mom[sl])
            bound = 0.5 * mn * (np.linalg.norm(H[sl] - Hr[sl]) + 1e-12 * np.linalg.norm(Hr[sl]))
            assert abs(E[i] - Er[i]) <= bound, (i, E[i], Er[i], bound)
        Q, V = g.expansions()
        c0 = 0
        for i in range(len(sizes)):
            f = O.OracleAFMM(ps[i], ms[i], p, theta, split)
            f.run()
            nc = len(f.cells())
            check_mixed(H[off[i]:off[i + 1]], E[i], V[c0:c0 + nc], f, p)
            c0 += nc
        for step in range(2):
            H, E = g.step(seed=21, step=step, max_angle=0.05)
            Hr, Er = r.step(seed=21, step=step, max_angle=0.05)
            mom = O.rotate_moments(mom, 21, step, 0.05)
            assert np.allclose(g.moments(), mom, rtol=0, atol=1e-14)
            assert rel(H, Hr) < 1e-6
        i = 3
        sl = slice(off[i], off[i + 1])
        f = O.OracleAFMM(pos[sl], mom[sl], p, theta, split)
        f.run()
        assert rel(H[sl], f.field()) < TOLMIX
        assert LP.dipole_max_err(H[sl], f.field()) < LP.DIPOLE_TOL


def test_persistent_step_needs_the_mixed_tensor_core_path():
    pos, mom = W.clustered(800, seed=3)
    with pytest.raises(C.CCFMMError):
        C.Adaptive(pos, mom, 4, 0.5, split=10.0, precision="fp64", persistent=True)
    with pytest.raises(C.CCFMMError):
        C.Adaptive(pos, mom, 7, 0.5, split=10.0, persistent=True)


def test_persistent_step_wait_gives_up(monkeypatch):
    """CCFMM_ASTEP_STALL=1 asks one task more of the M2L phase than the queue
    holds, so the L2L tasks' bounded waits run out: the evaluation reports
    CCFMM_ERR_TIMEOUT, and a handle built afterwards evaluates exactly."""
    sizes = [500, 1200]
    ps, ms, off, pos, mom = _forest(sizes, 77)
    monkeypatch.setenv("CCFMM_ASTEP_STALL", "1")
    with C.Adaptive(pos, mom, 4, 0.5, split=10.0, offsets=off, persistent=True) as g:
        with pytest.raises(C.CCFMMError) as e:
            g.evaluate()
        assert e.value.status == C.ERR_TIMEOUT, e.value
    monkeypatch.delenv("CCFMM_ASTEP_STALL")
    with C.Adaptive(pos, mom, 4, 0.5, split=10.0, offsets=off, persistent=True) as g:
        H, E = g.evaluate()
        f = O.OracleAFMM(ps[1], ms[1], 4, 0.5, 10.0)
        f.run()
        assert rel(H[off[1]:off[2]], f.field()) < TOLMIX
