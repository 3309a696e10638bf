"""Scaling experiments of Sec. IV (experiments.py) on small lattices: the
measurements are well formed and the tree responds to the occupancy."""
import pytest

from paper_0810_0233_gb300 import ccfmm as C
from paper_0810_0233_gb300 import experiments as X

pytestmark = pytest.mark.gpu


def test_scaling_rows():
    rows = X.scaling(sizes=(8, 12), params=((4, 0.5),), direct_max=10_000)
    assert [r["N"] for r in rows] == [512, 1728]
    for r in rows:
        assert r["fmm_p4_a0.50_ms"] > 0 and r["direct_ms"] > 0 and r["depth_p4"] >= 1


def test_leaf_sweep_depth_falls_with_occupancy():
    res = X.leaf_sweep(n=16, p=3, theta=0.54, leaves=(2, 8, 32))
    depths = [r["depth"] for r in res]
    assert depths == sorted(depths, reverse=True) and depths[0] > depths[-1]
    # the paper's 32^3 example: s = 8 gives 8 x 8 x 8 leaves of 8 points (Sec. IV)
    assert X.leaf_sweep(n=32, p=3, theta=0.54, leaves=(8,))[0]["depth"] == 12


def test_optimal_leaf_small():
    res = X.optimal_leaf(ps=(3,), sizes=(30,))
    assert res[3]["rule"] == C.leaf_size_rule(3)
    assert 1.0 <= res[3]["s_o"] <= 512.0


def test_error_budget_small():
    """Table II's construction: alpha from the estimate e = [a/(2-a)]^p, and
    at e = 0.05 the errors reached stay inside the estimate, with the energy
    error below 1 % (Sec. IV)."""
    res = X.error_budget(n=16, es=(0.05,), ps=(3, 5))
    for r in res["rows"]:
        a = r["alpha"]
        assert abs((a / (2 - a)) ** r["p"] - 0.05) < 1e-12
        assert r["rms_field_error"] < 0.05
        assert r["energy_error"] < 0.01
    assert res["fastest"][0.05]["p"] in (3, 5)


def test_truncation_small():
    rows = X.truncation(n=20_000, ps=(4,), evals=2)
    assert [(r["p"], r["max_degree"]) for r in rows] == [(4, 8), (4, 5)]
    sq, td = rows
    for r in rows:
        assert 0.0 < r["rms_field_error"] < 5e-2
        assert r["tc_eval_ms"] > 0 and r["fma_m2l_ms"] > 0
    # fewer far-field terms cannot make the field markedly more accurate
    assert td["rms_field_error"] > 0.5 * sq["rms_field_error"]


def test_fft_comparator_small():
    """FFT and fast method on small lattices: the FFT (FP64) is exact to
    rounding, the fast method within its truncation error."""
    rows = X.fft_comparator(sizes=(12, 20), repeats=1, nsub=300)
    for r in rows:
        assert r["fft_fp64_error"] < 1e-12 and r["fft_mixed_error"] < 1e-5
        assert r["fmm_p6_error"] < 1e-3 and r["fmm_p5_error"] < 1e-2
        assert r["fft_fp64_ms"] > 0 and r["fmm_p5_ms"] > 0
