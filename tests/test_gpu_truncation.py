"""Total-degree truncation of Eq. taylorcalc on the GPU against the oracle.

``fmm_set_truncation(h, P)`` keeps only the M2L terms with |n|+|k| <= P
(the oracle's ``max_degree``, pinned in ``test_oracle_pins.py`` against the
Taylor polynomial of the dipole field).  Every M2L engine is checked: the
FP64 FMA kernel (1e-12 relative RMS), and on the mixed path the tensor-core
kernel and the FP32 FMA kernel (1e-5).  The bound 2p, and a return to the
default, must reproduce the square truncation bit for bit (the index table
and the tensor-core operators are rebuilt).  Input: the ferrofluid recipe at
its benchmark density (one dipole per unit volume, minimum separation 0.5),
30,000 dipoles: several tiles per level and ragged leaves.
"""
import functools

import numpy as np
import pytest

import oracle as O
from paper_0810_0233_gb300 import ccfmm as C
from paper_0810_0233_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N = 30_000
THETA = 0.5
TOL = {"fp64": 1e-12, "mixed": 1e-5}
ENGINES = [("fp64", None), ("mixed", "tc"), ("mixed", "fma")]
CASES = [(4, 5), (4, 7), (6, 7), (6, 10)]


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


@functools.lru_cache(maxsize=None)
def inputs():
    return W.ferrofluid(N, side=N ** (1.0 / 3.0), seed=810233 + 40)


@functools.lru_cache(maxsize=None)
def oracle_field(p, bound):
    pos, mom = inputs()
    H, E, _ = O.fmm_field(pos, mom, p, THETA, max_degree=bound)
    return H, E


def _engine(monkeypatch, eng):
    if eng is None:
        monkeypatch.delenv("CCFMM_M2L", raising=False)
    else:
        monkeypatch.setenv("CCFMM_M2L", eng)


@pytest.mark.parametrize("prec,eng", ENGINES)
@pytest.mark.parametrize("p,bound", CASES)
def test_total_degree_matches_oracle(monkeypatch, prec, eng, p, bound):
    _engine(monkeypatch, eng)
    pos, mom = inputs()
    Href, Eref = oracle_field(p, bound)
    with C.FMM(pos, mom, p, THETA, precision=prec) as f:
        f.set_truncation(bound)
        assert f.max_degree == bound
        H, E = f.field_energy()
    err = rel(H, Href)
    assert err < TOL[prec], (prec, eng, p, bound, err)
    assert abs(E - Eref) <= 10 * TOL[prec] * abs(Eref)


def test_truncation_is_not_vacuous():
    """The bounds tested change the result well above both tolerances."""
    for p, bound in CASES:
        Hs, _ = oracle_field(p, None)
        Ht, _ = oracle_field(p, bound)
        assert rel(Ht, Hs) > 1e-8, (p, bound)


@pytest.mark.parametrize("prec,eng", ENGINES)
def test_square_bound_and_reset_are_bitwise(monkeypatch, prec, eng):
    _engine(monkeypatch, eng)
    pos, mom = inputs()
    p = 6
    with C.FMM(pos, mom, p, THETA, precision=prec) as f:
        assert f.max_degree == 2 * p
        H0 = f.field()
        f.set_truncation(p + 1)
        H1 = f.field()
        f.set_truncation(2 * p)
        H2 = f.field()
        f.set_truncation(p + 1)
        f.set_truncation(None)
        H3 = f.field()
        # new positions keep the bound
        f.set_truncation(p + 1)
        f.set_positions(pos, mom)
        H4 = f.field()
    assert np.array_equal(H0, H2) and np.array_equal(H0, H3)
    assert np.array_equal(H1, H4)
    assert not np.array_equal(H0, H1)


def test_bad_bounds_rejected():
    pos, mom = inputs()
    p = 4
    with C.FMM(pos[:2000], mom[:2000], p, THETA) as f:
        for bad in (1, 2 * p + 1):
            with pytest.raises(C.CCFMMError):
                f.set_truncation(bad)
        assert f.max_degree == 2 * p
        f.set_truncation(2)
        assert f.max_degree == 2
