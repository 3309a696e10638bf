"""The local parity bounds are tight enough to see one dropped far partner.

For the inputs the GPU parity tests use, the oracle computes what leaving out
any single far partner A of any single cell B would do:

* to B's Taylor coefficients: the whole M2L term of the pair, Eq. taylorcalc,
  V_n += (-1)^|n| sum_k D_(n+k)(c_B - c_A) Q_k^A;
* to the field of B's dipoles (leaf cells): the direct field of A's dipoles,
  which the far-field expansion reproduces to far better than the bound.

Every such change must exceed the bounds of ``local_parity`` by a wide margin,
so that a lost partner row, entry or item in the grouped M2L fails the GPU
tests even when the relative RMS over all dipoles barely moves."""
import numpy as np
import pytest

import oracle as O
from paper_0810_0233_gb300 import workloads as W

import local_parity as LP

CASES = {
    "ferrofluid": lambda: W.ferrofluid(20000, side=100.0 * 0.02 ** (1 / 3),
                                       seed=W.BASE_SEED + 12),
    "clustered": lambda: W.clustered(30000, seed=W.BASE_SEED + 41),
    "ring": lambda: W.ring(r_out=60.0, r_in=20.0, seed=W.BASE_SEED + 42),
}


def _tree(pos, mom, p, theta):
    f = O.OracleFMM(pos, mom, p, theta)
    f.upward()
    f.downward()
    L = f.depth
    lo = f.leaf_of()
    ne = np.zeros(1 << (L + 1), bool)
    for l in range(L + 1):
        ne[(1 << l) + np.unique(lo >> (L - l))] = True
    far = f.far_pairs()
    far = far[ne[far[:, 0]] & ne[far[:, 1]]]
    cen = np.array([f.cell_center(c) if c > 0 else np.zeros(3) for c in range(1 << (L + 1))])
    return f, ne, far, cen


def _operators(p):
    """Index table n + k and the sign (-1)^|n| of Eq. taylorcalc."""
    mi = O.multi_indices(p)
    T = len(mi)
    idx = np.array([[O.index(mi[a] + mi[b]) for b in range(T)] for a in range(T)])
    return mi, idx, (-1.0) ** mi.sum(1)


def cell_detection(pos, mom, p, theta):
    """min over far pairs (B, A) of |w dV| / RMS_level |w V| (cell measure)."""
    f, ne, far, cen = _tree(pos, mom, p, theta)
    Q, V = f.moments(), f.locals()
    mi, idx, sign = _operators(p)
    rho = LP.level_half_diagonals(f.box(), f.axes())
    off = cen[far[:, 0]] - cen[far[:, 1]]
    lev = np.floor(np.log2(far[:, 0])).astype(int)
    key = np.c_[lev, np.round(off * 1e9).astype(np.int64)]
    uk, inv = np.unique(key, axis=0, return_inverse=True)
    inv = inv.ravel()
    worst = np.inf
    for u in range(len(uk)):
        sel = np.where(inv == u)[0]
        l = lev[sel[0]]
        M = sign[:, None] * O.D_tensors(2 * p, off[sel[0]])[idx]
        M[0, :] = 0.0  # V_0 is not kept
        w = LP.term_weights(mi, rho[l])
        rows = np.where(ne[(1 << l):(1 << (l + 1))])[0] + (1 << l)
        scale = np.sqrt(((V[rows] * w) ** 2).sum(1).mean())
        dV = Q[far[sel, 1]] @ M.T
        worst = min(worst, float((np.sqrt(((dV * w) ** 2).sum(1)) / scale).min()))
    # the table-built operator is the oracle's M2L
    B, A = far[len(far) // 2]
    M = sign[:, None] * O.D_tensors(2 * p, cen[B] - cen[A])[idx]
    M[0, :] = 0.0
    ref = O.m2l(p, cen[B] - cen[A], Q[A])
    assert np.abs(M @ Q[A] - ref).max() <= 1e-12 * np.abs(ref).max()
    return worst, len(far)


def dipole_detection(pos, mom, p, theta):
    """For every leaf-level far pair (B, A): max_{i in B} |H_A(x_i)| /
    max(|H_i|, RMS |H|) (the dipole measure of leaving A out of B's list);
    H_A = direct field of A's dipoles."""
    f, ne, far, cen = _tree(pos, mom, p, theta)
    L = f.depth
    Href = f.field()
    mag = np.sqrt((Href ** 2).sum(1))
    floor = np.maximum(mag, np.sqrt((mag ** 2).mean()))
    lo = f.leaf_of()
    order = np.argsort(lo, kind="stable")
    starts = np.searchsorted(lo[order], np.arange((1 << L) + 1))
    leafp = far[np.floor(np.log2(far[:, 0])).astype(int) == L] - (1 << L)
    seen = np.zeros(len(leafp))
    for k, (B, A) in enumerate(leafp):
        tb = order[starts[B]:starts[B + 1]]
        sa = order[starts[A]:starts[A + 1]]
        hA = O.direct_field(np.concatenate([pos[sa], pos[tb]]),
                            np.concatenate([mom[sa], np.zeros((len(tb), 3))]),
                            targets=np.arange(len(sa), len(sa) + len(tb)))
        seen[k] = float((np.sqrt((hA ** 2).sum(1)) / floor[tb]).max())
    return seen


@pytest.mark.parametrize("case", sorted(CASES))
def test_one_dropped_partner_moves_a_cell_past_the_bound(case):
    pos, mom = CASES[case]()
    worst, npairs = cell_detection(pos, mom, 6, 0.5)
    assert npairs > 10000
    assert worst > 2 * LP.CELL_TOL, (case, worst)


def test_most_dropped_leaf_partners_move_a_dipole_past_the_bound():
    """The dipole bound alone already sees almost every lost leaf-level
    partner (the cell bound sees all of them)."""
    pos, mom = CASES["ferrofluid"]()
    seen = dipole_detection(pos, mom, 6, 0.5)
    assert len(seen) > 10000
    assert (seen > LP.DIPOLE_TOL).mean() > 0.9, np.percentile(seen, [1, 5, 50])


def test_measures_are_zero_on_identical_inputs_and_scale_free():
    rng = np.random.default_rng(3)
    H = rng.standard_normal((50, 3))
    assert LP.dipole_max_err(H, H) == 0.0
    assert LP.dipole_max_err(3 * (H + 1e-3), 3 * H) == pytest.approx(LP.dipole_max_err(H + 1e-3, H))
    mi = O.multi_indices(3)
    w = LP.term_weights(mi, 2.0)
    assert w[0] == 0.0 and w[O.index((1, 0, 0))] == 2.0 and w[O.index((2, 1, 0))] == 4.0
    rho = LP.level_half_diagonals([0, 0, 0, 4, 2, 2], [0, 0, 1])
    assert np.allclose(rho, 0.5 * np.sqrt([24, 12, 9, 6]))
