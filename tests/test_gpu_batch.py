"""Ensemble step (fmm_batch_*): the Philox rotation of every moment against
the oracle's rotation, and every sample's field against a single-system
evaluation and the oracle FMM, over several steps."""
import numpy as np
import pytest

import oracle as O
from paper_0810_0233_gb300 import ccfmm as C
from paper_0810_0233_gb300 import workloads as W

import local_parity as LP

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def _ensemble(ns=5, seed=77):
    rng = np.random.default_rng(seed)
    sizes = rng.integers(800, 4000, size=ns)
    pos, mom = [], []
    for i, n in enumerate(sizes):
        p_, m_ = W.clustered(int(n), seed=seed * 100 + i)
        pos.append(p_)
        mom.append(m_)
    off = np.concatenate([[0], np.cumsum([len(x) for x in pos])]).astype(np.int64)
    return np.concatenate(pos), np.concatenate(mom), off


def check_member_local(b, s, H, Href, f, p):
    """Local bounds of one ensemble member: every dipole, and every cell of
    levels >= 2 against the oracle's Taylor coefficients."""
    assert LP.dipole_max_err(H, Href) < LP.DIPOLE_TOL, s
    L = f.depth
    lo = f.leaf_of()
    cells = sorted({(1 << l) + int(k) for l in range(2, L + 1) for k in np.unique(lo >> (L - l))})
    if not cells:
        return
    cols = np.array([O.index(n) for n in C.multi_indices(p)])
    err = LP.cell_errors(b.sample(s).expansions("V"), f.locals()[:, cols], cells,
                         C.multi_indices(p), f.box(), f.axes())
    if err:
        assert max(err.values()) < LP.CELL_TOL, (s, err)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("mixed", 1e-5)])
def test_batch_steps_match_oracle(prec, tol):
    pos, mom, off = _ensemble()
    p, theta = 5, 0.5
    ref_m = mom.copy()
    with C.Batch(pos, mom, off, p, theta, precision=prec) as b:
        assert b.kernels_per_step() == 0  # graph not captured yet
        for step in range(3):
            H = np.zeros((b.total, 3))
            E = np.zeros(b.ns)
            b.step(seed=99, step=step, max_angle=0.05, H_out=H, E_out=E)
            ref_m = O.rotate_moments(ref_m, 99, step, 0.05)
            assert np.abs(b.moments() - ref_m).max() < 1e-14
            for s in range(b.ns):
                sl = slice(off[s], off[s + 1])
                Hr, Er, f = O.fmm_field(pos[sl], ref_m[sl], p, theta)
                assert rel(H[sl], Hr) < tol, (prec, step, s)
                if prec == "mixed":
                    check_member_local(b, s, H[sl], Hr, f, p)
                assert abs(E[s] - Er) <= 10 * tol * abs(Er)
        if prec == "mixed":
            # one launch per stage over every sample (tensor-core M2L path)
            assert 5 < b.kernels_per_step() < 40
        else:
            assert b.kernels_per_step() > b.ns


@pytest.mark.parametrize("engine", ["fma", "tc"])
def test_batch_equals_single_systems_bitwise(monkeypatch, engine):
    """Ensemble members and standalone handles with the same M2L engine
    give the same bits."""
    monkeypatch.setenv("CCFMM_M2L", engine)
    pos, mom, off = _ensemble(ns=4, seed=78)
    with C.Batch(pos, mom, off, 4, 0.5) as b:
        H = np.zeros((b.total, 3))
        b.evaluate(H_out=H)
        H2 = np.zeros((b.total, 3))
        b.evaluate(H_out=H2)
    assert np.array_equal(H, H2)
    for s in range(4):
        sl = slice(off[s], off[s + 1])
        with C.FMM(pos[sl], mom[sl], 4, 0.5) as f:
            assert np.array_equal(f.field(), H[sl])


def test_batch_rejects_bad_offsets():
    pos = np.random.default_rng(0).uniform(0, 5, (10, 3))
    mom = np.ones((10, 3))
    with pytest.raises(C.CCFMMError):
        C.Batch(pos, mom, [0, 5, 5, 10], 4, 0.5)
    with pytest.raises(C.CCFMMError):
        C.Batch(pos, mom, [1, 10], 4, 0.5)


def test_fp64_pair_with_levels_without_m2l_entries():
    """Two clustered samples whose first has levels with far offsets but no
    M2L entries: that tile's epilogue must not depend on the entry loop's
    barriers (it once read scale factors other warps had not yet written)."""
    pos, mom, off = _ensemble()
    o = off[:3]
    P, M = pos[:o[-1]], mom[:o[-1]]
    with C.Batch(P, M, o, 5, 0.5, precision="fp64") as b:
        H = np.zeros((b.total, 3))
        b.evaluate(H_out=H)
        tiles = b.sample(0).m2l_data()[3]
    assert np.any(tiles[:, 5] == 0)  # a tile with no entries
    assert np.all(np.isfinite(H))
    for s in range(2):
        sl = slice(o[s], o[s + 1])
        with C.FMM(P[sl], M[sl], 5, 0.5, precision="fp64") as f:
            assert rel(H[sl], f.field()) < 1e-13


@pytest.mark.parametrize("mode", ["batched", "graph"])
def test_batched_stages_equal_member_graph_bitwise(monkeypatch, mode):
    """The batched stages (one launch per stage over all samples) run each
    sample's arithmetic unchanged: the same bits as the graph of per-sample
    launches (CCFMM_BATCH_MODE=graph) and as standalone handles."""
    pos, mom, off = _ensemble(ns=6, seed=79)
    monkeypatch.delenv("CCFMM_M2L", raising=False)
    if mode == "graph":
        monkeypatch.setenv("CCFMM_BATCH_MODE", "graph")
    with C.Batch(pos, mom, off, 5, 0.5) as b:
        H = np.zeros((b.total, 3))
        E = np.zeros(b.ns)
        b.step(seed=5, step=0, max_angle=0.05, H_out=H, E_out=E)
        M = b.moments()
        k = b.kernels_per_step()
    assert (k < 40) == (mode == "batched")
    for s in range(b.ns):
        sl = slice(off[s], off[s + 1])
        with C.FMM(pos[sl], M[sl], 5, 0.5) as f:
            Hs, Es = f.field_energy()
        assert np.array_equal(Hs, H[sl]), s
        assert Es == E[s], s


def test_autotuner_picks_per_class_and_stays_exact():
    """fmm_batch_create_ex with autotune: one (leaf, item length) per size
    class, chosen from the candidates; the tuned ensemble still matches the
    oracle."""
    rng = np.random.default_rng(81)
    sizes = [900, 1100, 3000, 3500, 9000]
    pos, mom = [], []
    for i, n in enumerate(sizes):
        p_, m_ = W.clustered(n, seed=8100 + i)
        pos.append(p_)
        mom.append(m_)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pos, mom = np.concatenate(pos), np.concatenate(mom)
    rule = C.leaf_size_rule(5)
    with C.Batch(pos, mom, off, 5, 0.5, autotune=True, trials=2) as b:
        tun = b.tuning()
        H = np.zeros((b.total, 3))
        b.evaluate(H_out=H)
    octaves = sorted({int(np.floor(np.log2(n))) for n in sizes})
    assert len(tun) == len(octaves)
    for nmin, leaf, il in tun:
        assert il in (32, 64)
        assert any(abs(leaf - max(1.0, rule * f)) < 1e-9
                   for f in (0.5, 2 ** -0.5, 1.0, 2 ** 0.5, 2.0))
    leaf_of_octave = {int(np.floor(np.log2(nmin))): leaf for nmin, leaf, _ in tun}
    for s, n in enumerate(sizes):
        sl = slice(off[s], off[s + 1])
        leaf = leaf_of_octave[int(np.floor(np.log2(n)))]
        Hr = O.fmm_field(pos[sl], mom[sl], 5, 0.5, leaf)[0]
        assert rel(H[sl], Hr) < 1e-5, (s, leaf)
