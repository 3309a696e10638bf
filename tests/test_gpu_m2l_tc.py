"""The tensor-core M2L (tcgen05, TF32 three-product split) against the FP32
FMA M2L and the FP64 oracle, for every order it supports (p = 4..7).  Besides
the relative RMS, every dipole's field and every cell's Taylor coefficients
are held to the local bounds of ``local_parity`` against the oracle, so that
one partner row or one entry run lost at a tile or item boundary fails."""
import os

import numpy as np
import pytest

import oracle as O
from paper_0810_0233_gb300 import ccfmm as C
from paper_0810_0233_gb300 import workloads as W

import local_parity as LP

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def check_local_vs_oracle(H, V, pos, mom, p, theta):
    """Per-dipole and per-cell bounds against the oracle FMM (square
    truncation, all cells)."""
    Href, _, f = O.fmm_field(pos, mom, p, theta)
    assert rel(H, Href) < 1e-5
    assert LP.dipole_max_err(H, Href) < LP.DIPOLE_TOL
    L = f.depth
    lo = f.leaf_of()
    cells = sorted({(1 << l) + int(k) for l in range(2, L + 1) for k in np.unique(lo >> (L - l))})
    cols = np.array([O.index(n) for n in C.multi_indices(p)])
    Vo = f.locals()[:, cols]
    err = LP.cell_errors(V, Vo, cells, C.multi_indices(p), f.box(), f.axes())
    assert max(err.values()) < LP.CELL_TOL, err
    return Href


def _run(engine, pos, mom, p, theta):
    old = os.environ.get("CCFMM_M2L")
    os.environ["CCFMM_M2L"] = engine
    try:
        with C.FMM(pos, mom, p, theta) as f:
            H = f.field()
            V = f.expansions("V")
    finally:
        if old is None:
            del os.environ["CCFMM_M2L"]
        else:
            os.environ["CCFMM_M2L"] = old
    return H, V


@pytest.mark.parametrize("p", [4, 5, 6, 7])
def test_tensor_core_m2l_matches(p):
    pos, mom = W.ferrofluid(20000, side=100.0 * 0.02 ** (1 / 3), seed=W.BASE_SEED + 30 + p)
    Hf, Vf = _run("fma", pos, mom, p, 0.5)
    Ht, Vt = _run("tc", pos, mom, p, 0.5)
    nz = np.abs(Vf).sum(1) > 0
    assert rel(Vt[nz], Vf[nz]) < 2e-5
    assert rel(Ht, Hf) < 2e-6
    check_local_vs_oracle(Ht, Vt, pos, mom, p, 0.5)


@pytest.mark.parametrize("kind", ["clustered", "ring"])
def test_tensor_core_m2l_irregular(kind):
    """Clustered and flat point sets: tiles with many cells lacking a given
    partner (zero rows) and boxes whose levels are not cubes."""
    if kind == "clustered":
        pos, mom = W.clustered(30000, seed=W.BASE_SEED + 41)
    else:
        pos, mom = W.ring(r_out=60.0, r_in=20.0, seed=W.BASE_SEED + 42)
    Hf, Vf = _run("fma", pos, mom, 6, 0.5)
    Ht, Vt = _run("tc", pos, mom, 6, 0.5)
    nz = np.abs(Vf).sum(1) > 0
    assert rel(Vt[nz], Vf[nz]) < 2e-5
    assert rel(Ht, Hf) < 2e-6
    check_local_vs_oracle(Ht, Vt, pos, mom, 6, 0.5)
    sub = W.subset(len(pos), 300, 5)
    Hd = C.direct_field(pos, mom, targets=sub)
    assert rel(Ht[sub], Hd) < 1e-4


def _run_gather(mode, pos, mom, p, theta, where="smem"):
    saved = {k: os.environ.get(k) for k in ("CCFMM_TC_GATHER", "CCFMM_TC_A")}
    os.environ["CCFMM_TC_GATHER"] = mode
    os.environ["CCFMM_TC_A"] = where
    try:
        return _run("tc", pos, mom, p, theta)
    finally:
        for k, v in saved.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v


@pytest.mark.parametrize("case", ["p4", "p5", "p6", "p7", "clustered", "ring"])
def test_operand_paths_are_bitwise(case):
    """The TMA row gather (tile::gather4 copies; an absent partner reads the
    zero row 0) fills the operand stages with the same bytes as the cp.async
    gather, and the tensor-memory operand (moments split in registers and
    stored with tcgen05.st) holds the same TF32 pairs, so the MMAs, and the
    whole field, agree bit for bit on all three paths."""
    if case == "clustered":
        pos, mom = W.clustered(30000, seed=W.BASE_SEED + 41)
        p = 6
    elif case == "ring":
        pos, mom = W.ring(r_out=60.0, r_in=20.0, seed=W.BASE_SEED + 42)
        p = 6
    else:
        p = int(case[1])
        pos, mom = W.ferrofluid(20000, side=100.0 * 0.02 ** (1 / 3), seed=W.BASE_SEED + 30 + p)
    Hc, Vc = _run_gather("cp", pos, mom, p, 0.5)
    Ht, Vt = _run_gather("tma", pos, mom, p, 0.5)
    assert np.array_equal(Vt, Vc)
    assert np.array_equal(Ht, Hc)
    Hm, Vm = _run_gather("cp", pos, mom, p, 0.5, where="tmem")
    assert np.array_equal(Vm, Vc)
    assert np.array_equal(Hm, Hc)
