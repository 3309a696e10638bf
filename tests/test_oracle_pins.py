"""Pins of the FP64 CPU oracle against facts the paper and mathematics fix.

None of these tests retype the oracle's formulas: each compares it with an
independent statement (a textbook closed form, symbolic differentiation, a
finite difference of the potential, the +-q limit that defines a dipole,
brute force, the paper's printed examples and tables, or an exact identity).
``tests/test_oracle_mutants.py`` plants plausible mistakes in a copy of the
oracle and checks that these pins catch each of them.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_0810_0233_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rng(s=7):
    return np.random.default_rng(s)


def _rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.sqrt(((a - b) ** 2).sum() / max((b ** 2).sum(), 1e-300)))


# --------------------------------------------------------------------------
# Direct dipole sum (Sec. I brute force; Eq. H2 as read)
# --------------------------------------------------------------------------

def pin_axial_equatorial():
    """On the dipole axis the field is 2m/r^3, on its equator -m/r^3."""
    d = 1.7
    pos = np.array([[0.0, 0, 0], [d, 0, 0], [0, d, 0]])
    mom = np.array([[1.0, 0, 0], [0, 0, 0], [0, 0, 0]])
    H = O.direct_field(pos, mom)
    ok = np.allclose(H[1], [2.0 / d**3, 0, 0], rtol=1e-14, atol=1e-16)
    ok &= np.allclose(H[2], [-1.0 / d**3, 0, 0], rtol=1e-14, atol=1e-16)
    return bool(ok)


def pin_field_is_minus_grad_potential():
    """H_i = -grad phi at r_i, phi(r) = sum_j m_j.(r-r_j)/|r-r_j|^3 (the dipole
    potential), by a 4th-order central difference."""
    rng = _rng(3)
    pos = rng.uniform(0, 4, size=(12, 3))
    mom = W.unit_vectors(12, rng)
    H = O.direct_field(pos, mom)

    def phi(r, i):
        s = 0.0
        for j in range(len(pos)):
            if j == i:
                continue
            d = r - pos[j]
            s += mom[j] @ d / np.linalg.norm(d) ** 3
        return s

    h = 1e-3
    worst = 0.0
    for i in range(len(pos)):
        g = np.zeros(3)
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            g[a] = (-phi(pos[i] + 2 * e, i) + 8 * phi(pos[i] + e, i) - 8 * phi(pos[i] - e, i)
                    + phi(pos[i] - 2 * e, i)) / (12 * h)
        worst = max(worst, np.abs(-g - H[i]).max() / np.abs(H[i]).max())
    return worst < 1e-7


def pin_pair_energy():
    """E from -1/2 sum m.H equals the sum over pairs of the dipole-dipole
    energy (m_i.m_j - 3 (m_i.u)(m_j.u)) / r^3."""
    rng = _rng(5)
    pos = rng.uniform(0, 3, size=(20, 3))
    mom = W.unit_vectors(20, rng)
    H = O.direct_field(pos, mom)
    E = O.energy_from_field(mom, H)
    Ep = 0.0
    for i, j in itertools.combinations(range(20), 2):
        d = pos[i] - pos[j]
        r = np.linalg.norm(d)
        u = d / r
        Ep += (mom[i] @ mom[j] - 3 * (mom[i] @ u) * (mom[j] @ u)) / r**3
    return abs(E - Ep) < 1e-12 * abs(Ep)


def pin_lorentz_sphere():
    """A sphere cut from a simple-cubic lattice with parallel moments has zero
    dipolar field at its centre (cubic symmetry, sum over each shell of
    u_a u_b = delta_ab / 3)."""
    R = 6
    g = np.arange(-R, R + 1, dtype=float)
    P = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    P = P[(P**2).sum(1) <= R * R]
    c = int(np.flatnonzero((P**2).sum(1) == 0)[0])
    mom = np.tile(np.array([0.3, -0.5, 0.81]), (len(P), 1))
    H = O.direct_field(P, mom, targets=[c])
    return np.abs(H).max() < 1e-12


def test_direct_axial_equatorial():
    assert pin_axial_equatorial()


def test_direct_minus_grad_potential():
    assert pin_field_is_minus_grad_potential()


def test_direct_pair_energy():
    assert pin_pair_energy()


def test_direct_lorentz_sphere():
    assert pin_lorentz_sphere()


def test_direct_targets_and_coincident():
    rng = _rng(9)
    pos = rng.uniform(0, 3, size=(30, 3))
    mom = W.unit_vectors(30, rng)
    H = O.direct_field(pos, mom)
    Ht = O.direct_field(pos, mom, targets=[4, 17, 29])
    assert np.array_equal(Ht, H[[4, 17, 29]])
    # a second dipole on the field point is skipped (Appendix: "except when the
    # dipole is located at the field point")
    pos2 = np.vstack([pos, pos[:1]])
    mom2 = np.vstack([mom, [[0.0, 0.0, 1.0]]])
    H2 = O.direct_field(pos2, mom2, targets=[0])
    Hextra = O.direct_field(np.vstack([pos, pos[:1] + 0.0]), mom2, targets=[30])
    assert np.allclose(H2[0], H[0], rtol=0, atol=1e-15)
    assert np.all(np.isfinite(Hextra))


# --------------------------------------------------------------------------
# Derivative tensors D_n (Eqs. Vm, Dn, Dnr)
# --------------------------------------------------------------------------

def pin_D_closed_forms():
    r = np.array([0.7, -1.3, 2.1])
    rr = np.linalg.norm(r)
    D = O.D_tensors(12, r)
    ok = abs(D[O.index((0, 0, 0))] - 1 / rr) < 1e-15
    for a in range(3):
        n = [0, 0, 0]
        n[a] = 1
        ok &= abs(D[O.index(n)] - r[a] / rr**3) < 1e-15
    x = 1.9
    Dx = O.D_tensors(12, [x, 0, 0])
    for k in range(13):
        ok &= abs(Dx[O.index((k, 0, 0))] - math.factorial(k) / x ** (k + 1)) <= 1e-13 * math.factorial(k) / x ** (k + 1)
    return bool(ok)


def pin_D_symbolic(order=6):
    """D_n = (-1)^|n| d^n (1/r) by sympy, every |n| <= order."""
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    f = 1 / sp.sqrt(x**2 + y**2 + z**2)
    r = (0.9, -0.4, 1.3)
    D = O.D_tensors(order, r)
    worst = 0.0
    for n in O.multi_indices(order):
        e = f
        for v, k in zip((x, y, z), n):
            if k:
                e = sp.diff(e, v, int(k))
        val = float(e.subs({x: r[0], y: r[1], z: r[2]})) * (-1) ** int(sum(n))
        got = D[O.index(n)]
        worst = max(worst, abs(got - val) / max(abs(val), 1e-12))
    return worst < 1e-12


def pin_D_laplace_parity():
    r = np.array([1.1, 0.3, -0.8])
    D = O.D_tensors(12, r)
    Dm = O.D_tensors(12, -r)
    ok = True
    scale = np.abs(D).max()
    for n in O.multi_indices(10):
        lap = sum(D[O.index(n + 2 * np.eye(3, dtype=int)[a])] for a in range(3))
        ok &= abs(lap) < 1e-12 * scale
    for t, n in enumerate(O.multi_indices(12)):
        ok &= abs(Dm[t] - (-1) ** int(sum(n)) * D[t]) <= 1e-13 * abs(D[t]) + 1e-300
    return bool(ok)


def test_D_closed_forms():
    assert pin_D_closed_forms()


def test_D_symbolic():
    assert pin_D_symbolic(6)


def test_D_laplace_parity():
    assert pin_D_laplace_parity()


def test_F_table_sparse():
    # the paper: F_n(q) is non-zero for only a few q; at order 12 at most 28
    mi = O.multi_indices(12)
    counts = [O.F_nnz(12, t) for t in range(len(mi)) if sum(mi[t]) == 12]
    assert max(counts) <= 28
    assert O.nterms(12) == 455 and O.nterms(6) == 84


def test_multi_index_enumeration():
    for order in (0, 1, 4, 12):
        mi = O.multi_indices(order)
        assert len(mi) == O.nterms(order) == (order + 1) * (order + 2) * (order + 3) // 6
        assert len({tuple(n) for n in mi}) == len(mi)
        assert all(O.index(n) == t for t, n in enumerate(mi))
        assert list(mi.sum(1)) == sorted(mi.sum(1))


# --------------------------------------------------------------------------
# Moments and shifts (Eqs. multipolemoments, momentshift, taylorshift, H)
# --------------------------------------------------------------------------

def _charge_moments(p, c, pos, q):
    """Q_n = (1/n!) sum q r^n about c (the charge definition, Sec. III)."""
    out = np.zeros(O.nterms(p))
    for t, n in enumerate(O.multi_indices(p)):
        r = pos - c
        out[t] = (q * np.prod(r ** n, axis=1)).sum() / np.prod([math.factorial(k) for k in n])
    return out


def pin_p2m_single_dipole():
    """A dipole at the centre has only Q_(1,0,0)=m_x, Q_(0,1,0)=m_y, Q_(0,0,1)=m_z."""
    m = np.array([0.3, -0.7, 0.2])
    Q = O.p2m(6, [1.0, 2.0, 3.0], [[1.0, 2.0, 3.0]], [m])
    ref = np.zeros_like(Q)
    ref[O.index((1, 0, 0))], ref[O.index((0, 1, 0))], ref[O.index((0, 0, 1))] = m
    return np.allclose(Q, ref, rtol=0, atol=1e-15)


def pin_p2m_charge_limit():
    """Eq. multipolemoments is the d -> 0 limit of charges +-q at r +- d with
    m = 2 q d; Richardson-extrapolated charge moments must agree."""
    rng = _rng(11)
    c = np.array([0.2, -0.1, 0.4])
    pos = rng.uniform(-1, 1, size=(5, 3))
    mom = W.unit_vectors(5, rng)
    p = 6
    Q = O.p2m(p, c, pos, mom)

    def pair(h):
        d = mom * h
        q = 1.0 / (2 * h)
        P = np.vstack([pos + d, pos - d])
        qq = np.concatenate([np.full(5, q), np.full(5, -q)])
        return _charge_moments(p, c, P, qq)

    h = 1e-3
    Qr = (4 * pair(h / 2) - pair(h)) / 3
    return np.abs(Qr - Q).max() < 1e-8 * np.abs(Q).max()


def pin_multipole_potential():
    """V(r) = sum_n D_n(r) Q_n (Eq. Vm) converges to the direct dipole
    potential as p grows."""
    rng = _rng(12)
    pos = rng.uniform(-0.5, 0.5, size=(20, 3))
    mom = W.unit_vectors(20, rng)
    r = np.array([2.5, 1.0, -1.5])
    exact = sum(mom[j] @ (r - pos[j]) / np.linalg.norm(r - pos[j]) ** 3 for j in range(20))
    errs = []
    for p in (2, 4, 6, 8):
        Q = O.p2m(p, [0, 0, 0], pos, mom)
        D = O.D_tensors(p, r)
        errs.append(abs(D @ Q - exact) / abs(exact))
    return all(b < a for a, b in zip(errs, errs[1:])) and errs[-1] < 5e-5


def pin_m2m_exact():
    """Shifted child moments equal direct moments about the new centre."""
    rng = _rng(13)
    pos = rng.uniform(-1, 1, size=(9, 3))
    mom = W.unit_vectors(9, rng)
    p = 6
    cc = np.array([0.25, -0.5, 0.125])
    cp = np.array([-0.75, 0.5, 0.375])
    Qc = O.p2m(p, cc, pos, mom)
    Qp = O.m2m(p, cc - cp, Qc)
    Qd = O.p2m(p, cp, pos, mom)
    return np.abs(Qp - Qd).max() < 1e-13 * np.abs(Qd).max()


def pin_l2l_l2p():
    """L2P from the parent equals L2L to the child then L2P (the shift of a
    degree-p polynomial is exact)."""
    rng = _rng(14)
    p = 6
    V = rng.standard_normal(O.nterms(p))
    V[0] = 0.0
    c = np.array([0.4, -0.2, 0.3])
    Vc = O.l2l(p, c, V)
    worst = 0.0
    for _ in range(5):
        x = rng.uniform(-0.5, 0.5, 3)
        a = O.l2p(p, c + x, V)
        b = O.l2p(p, x, Vc)
        worst = max(worst, np.abs(a - b).max() / np.abs(a).max())
    return worst < 1e-12


def pin_l2p_gradient():
    """L2P is -grad of the Taylor polynomial V(r) = sum V_n r^n / n!
    (Eq. taylorexpansion), by central differences."""
    rng = _rng(15)
    p = 5
    V = rng.standard_normal(O.nterms(p))
    mi = O.multi_indices(p)
    fac = np.array([np.prod([math.factorial(k) for k in n]) for n in mi])

    def poly(r):
        return float((V * np.prod(r ** mi, axis=1) / fac)[1:].sum())

    x = np.array([0.3, -0.2, 0.1])
    h = 1e-5
    g = np.array([(poly(x + h * e) - poly(x - h * e)) / (2 * h) for e in np.eye(3)])
    H = O.l2p(p, x, V)
    return np.abs(H + g).max() < 1e-7 * np.abs(g).max()


def pin_m2l_convergence():
    """One source cell, one field cell at d/r ~ 6: the field at target points
    from M2L + L2P converges to the direct field as p grows, inside the
    estimate [alpha/(2-alpha)]^p up to a constant."""
    rng = _rng(16)
    src = rng.uniform(-0.5, 0.5, size=(30, 3))
    mom = W.unit_vectors(30, rng)
    tc = np.array([6.0, 0.5, -0.3])
    tgt = tc + rng.uniform(-0.5, 0.5, size=(10, 3))
    P = np.vstack([src, tgt])
    M = np.vstack([mom, np.zeros((10, 3))])
    Hd = O.direct_field(P, M, targets=np.arange(30, 40))
    alpha = 2 * (math.sqrt(3) / 2) / np.linalg.norm(tc)
    errs = []
    for p in (2, 4, 6, 8):
        Q = O.p2m(p, [0, 0, 0], src, mom)
        V = O.m2l(p, tc, Q)
        H = np.array([O.l2p(p, x - tc, V) for x in tgt])
        errs.append(_rel(H, Hd))
    mono_ok = all(b < a for a, b in zip(errs, errs[1:]))
    bound_ok = all(e < 10 * (alpha / (2 - alpha)) ** p for e, p in zip(errs, (2, 4, 6, 8)))
    return mono_ok and bound_ok and errs[-1] < 1e-5


def test_p2m_single_dipole():
    assert pin_p2m_single_dipole()


def test_p2m_charge_limit():
    assert pin_p2m_charge_limit()


def test_multipole_potential():
    assert pin_multipole_potential()


def test_m2m_exact():
    assert pin_m2m_exact()


def test_l2l_l2p():
    assert pin_l2l_l2p()


def test_l2p_gradient():
    assert pin_l2p_gradient()


def test_m2l_convergence():
    assert pin_m2l_convergence()


# --------------------------------------------------------------------------
# Total-degree truncation of Eq. taylorcalc (the alternative reading of the
# "terms after the p_m-th order" of Sec. II)
# --------------------------------------------------------------------------

def _dipole_field(w, m):
    """Field of a dipole m at offset w (rows), real or complex w:
    (3 (m.w) w - m (w.w)) / (w.w)^(5/2)."""
    ww = (w * w).sum(-1)[..., None]
    mw = (w * m).sum(-1)[..., None]
    return (3 * mw * w - m * ww) / ww ** 2.5


def _taylor_field(R, z, m, deg, M=64):
    """Taylor polynomial of degree ``deg`` of H(R + z) in z, evaluated at z,
    for dipoles m (rows) and offsets z (rows) against one centre offset R.
    The coefficients of f(t) = H(R + t z) are Cauchy integrals over the unit
    circle, taken by the trapezoid rule (Lyness & Moler, SIAM J. Numer. Anal.
    4 (1967) 202); the sum of the first deg+1 of them is the polynomial at
    t = 1.  With |z| < 0.45 |R|, w.w keeps a positive real part on the
    circle, so the principal power is analytic there."""
    z = np.atleast_2d(z)
    m = np.atleast_2d(m)
    th = 2 * np.pi * np.arange(M) / M
    t = np.exp(1j * th)                                           # (M,)
    w = R[None, None, :] + t[:, None, None] * z[None, :, :]      # (M, n, 3)
    f = _dipole_field(w, m[None, :, :])
    j = np.arange(deg + 1)
    a = np.einsum("mnc,jm->jnc", f, np.exp(-1j * np.outer(j, th))) / M
    return a.sum(0).real


def pin_total_degree_is_taylor():
    """One source dipole at c_s + y, one target at c_t + x, R = c_t - c_s:
    P2M, M2L with the terms |n|+|k| <= P (2 <= P <= p+1), then L2P give the
    Taylor polynomial of degree P-2 of the dipole field H(R + z) in
    z = x - y (the multinomial theorem regroups the double series of Eq.
    taylorcalc by |n|+|k|).  The square truncation is not that polynomial,
    so the check tells the two readings apart."""
    rng = _rng(41)
    R = np.array([4.0, -2.5, 3.0])
    worst, gap = 0.0, np.inf
    for p in (2, 3, 4, 6):
        for P in range(2, p + 2):
            y = rng.uniform(-0.5, 0.5, 3)
            x = rng.uniform(-0.5, 0.5, 3)
            m = W.unit_vectors(1, rng)[0]
            Q = O.p2m(p, [0.0, 0.0, 0.0], y[None], m[None])
            H = O.l2p(p, x, O.m2l(p, R, Q, max_degree=P))
            T = _taylor_field(R, x - y, m, P - 2)[0]
            worst = max(worst, np.abs(H - T).max() / np.linalg.norm(T))
            if P == p + 1:
                Hs = O.l2p(p, x, O.m2l(p, R, Q))
                gap = min(gap, np.abs(Hs - T).max() / np.linalg.norm(T))
    return worst < 1e-12 and gap > 1e-8


def pin_fmm_total_degree_brute_force():
    """The whole FMM with the total-degree bound P = p+1 at a sample of
    targets equals, to rounding, the brute-force sum over the oracle's lists:
    the exact field of every source in the target leaf's Near leaves, plus,
    for every ancestor cell c of the target leaf (the leaf included) and every
    Far partner A of c, the Taylor polynomial of degree p-1 of each source's
    field about R = c - A (centres).  M2M and L2L are exact, so every far
    interaction reaches the target as that polynomial."""
    pos, mom, box = W.lattice(7, seed=77)
    p, P = 4, 5
    f = O.OracleFMM(pos, mom, p, 0.5, 4.0, box=box)
    f.set_truncation(P)
    f.upward()
    f.downward()
    H = f.field()
    L = f.depth
    heap = (1 << L) + f.leaf_of()
    far, near = f.far_pairs(), f.near_pairs()
    rng = _rng(42)
    worst = 0.0
    for i in rng.choice(len(pos), 12, replace=False):
        h = np.zeros(3)
        for a in near[near[:, 0] == heap[i], 1]:
            js = np.flatnonzero((heap == a) & (np.arange(len(pos)) != i))
            h += _dipole_field(pos[i] - pos[js], mom[js]).sum(0)
        for l in range(L + 1):
            c = heap[i] >> (L - l)
            cc = f.cell_center(c)
            for a in far[far[:, 0] == c, 1]:
                js = np.flatnonzero((heap >> (L - l)) == a)
                ca = f.cell_center(a)
                z = (pos[i] - cc)[None, :] - (pos[js] - ca)
                h += _taylor_field(cc - ca, z, mom[js], P - 2).sum(0)
        worst = max(worst, np.linalg.norm(H[i] - h) / np.linalg.norm(h))
    return worst < 1e-11


def test_total_degree_is_taylor():
    assert pin_total_degree_is_taylor()


def test_fmm_total_degree_brute_force():
    assert pin_fmm_total_degree_brute_force()


def test_truncation_bounds():
    pos, mom, box = W.lattice(4)
    f = O.OracleFMM(pos, mom, 3, 0.5, 4.0, box=box)
    for bad in (1, 7):
        with pytest.raises(ValueError):
            f.set_truncation(bad)
    f.set_truncation(6)   # 2p: the square truncation
    f.set_truncation(None)


# --------------------------------------------------------------------------
# Tree and rule of thumb (Sec. II, Sec. IV, Eq. so, Tables I and II)
# --------------------------------------------------------------------------

def pin_worked_examples():
    g = json.load(open(os.path.join(GOLD, "worked_examples.json")))
    ok = True
    for ex in g["examples"]:
        nx, ny, nz = ex["lattice"]
        pos, mom, box = W.lattice(nx, ny, nz)
        f = O.OracleFMM(pos, mom, ex["p"], 0.5, 0.0, box=box)
        ok &= np.allclose(f.leaf_widths(), ex["leaf_widths"], rtol=1e-12)
        occ = len(pos) / f.nonempty_leaves()
        ok &= abs(occ - ex["mean_occupancy"]) < 0.01 * ex["mean_occupancy"]
    return bool(ok)


def pin_eq_so():
    g = json.load(open(os.path.join(GOLD, "eq_so.json")))
    ok = all(abs(O.leaf_size_rule(int(p)) - v) < 1e-12 for p, v in g["s_o"].items())
    t1 = g["table1"]
    ok &= O.leaf_size_rule(t1["p"]) == t1["optimal_s"]
    return bool(ok)


def test_worked_examples():
    assert pin_worked_examples()


def test_eq_so():
    assert pin_eq_so()


def test_table2_error_estimate():
    g = json.load(open(os.path.join(GOLD, "table2.json")))
    for row in g["rows"]:
        e = O.error_estimate(row["p"], row["alpha"])
        assert 0.046 <= e <= 0.054, (row, e)


def test_c1_tree_and_boundary_rule():
    """The 10^3 lattice at s = 8: L = 7, leaves 8 x 4 x 4 of 1.25 x 2.5 x 2.5;
    the lattice plane x = 2 lies on a cell boundary and goes to the upper cell."""
    pos, mom, box = W.lattice(10)
    f = O.OracleFMM(pos, mom, 4, 0.5, 8.0, box=box)
    assert f.depth == 7
    assert np.allclose(f.leaf_widths(), [1.25, 2.5, 2.5])
    assert list(f.axes()) == [0, 1, 2, 0, 1, 2, 0]
    leaf = f.leaf_of()
    # x-cell index of a leaf key: bits of levels 1, 4, 7 (x splits)
    xcell = ((leaf >> 6) & 1) * 4 + ((leaf >> 3) & 1) * 2 + (leaf & 1)
    on = pos[:, 0] == 2.0
    assert np.all(xcell[on] == 2)
    assert np.all(xcell[pos[:, 0] == 1.0] == 1)


# --------------------------------------------------------------------------
# Interaction lists (Sec. II step 1, Appendix createPartners)
# --------------------------------------------------------------------------

def _lists_ok(f, theta):
    L = f.depth
    nleaf = 1 << L
    far = [(int(a), int(b)) for a, b in f.far_pairs()]
    near = [(int(a), int(b)) for a, b in f.near_pairs()]
    far_set = {tuple(x) for x in far}
    near_set = {tuple(x) for x in near}
    ok = len(far_set) == len(far) and len(near_set) == len(near)
    # symmetric
    ok &= all((b, a) in far_set for a, b in far_set)
    ok &= all((b, a) in near_set for a, b in near_set)
    # every ordered pair of leaves is covered exactly once
    cover = np.zeros((nleaf, nleaf), dtype=np.int32)
    for a, b in near:
        cover[a - nleaf, b - nleaf] += 1
    for a, b in far:
        la = a.bit_length() - 1
        s = 1 << (L - la)
        ka, kb = (a - (1 << la)) * s, (b - (1 << la)) * s
        cover[ka:ka + s, kb:kb + s] += 1
    ok &= bool(np.all(cover == 1))
    # far pairs have alpha <= theta, near pairs of distinct leaves alpha > theta
    w_leaf = f.leaf_widths()
    for a, b in list(far)[:2000]:
        la = a.bit_length() - 1
        ca, cb = f.cell_center(a), f.cell_center(b)
        wl = _level_widths(f, la)
        al = np.linalg.norm(wl) / np.linalg.norm(ca - cb)
        ok &= al <= theta * (1 + 1e-9)
    for a, b in list(near)[:2000]:
        if a == b:
            continue
        al = np.linalg.norm(w_leaf) / np.linalg.norm(f.cell_center(a) - f.cell_center(b))
        ok &= al > theta
    return bool(ok)


def _level_widths(f, l):
    box = f.box()
    ext = box[3:] - box[:3]
    ax = f.axes()
    n = np.zeros(3, int)
    for a in ax[:l]:
        n[a] += 1
    return ext / 2.0 ** n


def test_lists_cover_once_c1():
    pos, mom, box = W.lattice(10)
    f = O.OracleFMM(pos, mom, 4, 0.5, 8.0, box=box)
    assert _lists_ok(f, 0.5)
    assert len(f.far_pairs()) == 4008


def test_lists_cover_once_random():
    rng = _rng(21)
    pos = rng.uniform(0, 7, size=(700, 3)) * np.array([1.0, 0.6, 0.3])
    mom = W.unit_vectors(700, rng)
    for theta in (0.3, 0.55, 0.8):
        f = O.OracleFMM(pos, mom, 3, theta, 4.0)
        assert _lists_ok(f, theta)


def test_tie_is_far():
    """C1 leaves are 1.25 x 2.5 x 2.5 (|w| = 3.75); at offset 6 along x, d = 7.5
    and alpha = theta = 0.5 exactly: the pair is far (near means larger than)."""
    pos, mom, box = W.lattice(10)
    f = O.OracleFMM(pos, mom, 4, 0.5, 8.0, box=box)
    far = {tuple(x) for x in f.far_pairs()}
    nleaf = 1 << f.depth
    # leaf with x-cell 0 and leaf with x-cell 6, same y/z cells
    def key(xc, yc, zc):
        k = 0
        cnt = {0: 0, 1: 0, 2: 0}
        coords = {0: xc, 1: yc, 2: zc}
        nb = {0: 3, 1: 2, 2: 2}
        for a in f.axes():
            bit = (coords[a] >> (nb[a] - 1 - cnt[a])) & 1
            cnt[a] += 1
            k = 2 * k + bit
        return k
    a, b = nleaf + key(0, 1, 1), nleaf + key(6, 1, 1)
    near = {tuple(x) for x in f.near_pairs()}
    assert (a, b) not in near
    # covered as far at the leaf level or above
    anc = [(a >> s, b >> s) for s in range(f.depth + 1)]
    assert any(x in far for x in anc)


def test_small_theta_is_direct():
    """theta -> 0 makes every pair near: the FMM is the direct sum."""
    rng = _rng(22)
    pos = rng.uniform(0, 5, size=(300, 3))
    mom = W.unit_vectors(300, rng)
    H, E, f = O.fmm_field(pos, mom, 3, 1e-3, 4.0)
    assert len(f.far_pairs()) == 0
    Hd = O.direct_field(pos, mom)
    assert _rel(H, Hd) < 1e-14


def test_single_leaf_is_direct():
    rng = _rng(23)
    pos = rng.uniform(0, 5, size=(64, 3))
    mom = W.unit_vectors(64, rng)
    H, E, f = O.fmm_field(pos, mom, 4, 0.5, 1000.0)
    assert f.depth == 0
    assert _rel(H, O.direct_field(pos, mom)) < 1e-14


# --------------------------------------------------------------------------
# The whole method
# --------------------------------------------------------------------------

def pin_fmm_converges():
    pos, mom, box = W.lattice(10)
    Hd = O.direct_field(pos, mom)
    errs = []
    for p in (2, 4, 6):
        H, E, f = O.fmm_field(pos, mom, p, 0.5, 8.0, box=box)
        errs.append(_rel(H, Hd))
    return all(b < a for a, b in zip(errs, errs[1:])) and errs[-1] < 1e-4


def pin_root_moments():
    """Root moments by the upward pass equal P2M of all points about the root
    centre (Eq. momentshift is exact); Q_(e_a) of the root = total moment."""
    rng = _rng(24)
    pos = rng.uniform(0, 4, size=(200, 3))
    mom = W.unit_vectors(200, rng)
    f = O.OracleFMM(pos, mom, 5, 0.5, 6.0)
    f.upward()
    Q = f.moments()
    Qd = O.p2m(5, f.cell_center(1), pos, mom)
    ok = np.abs(Q[1] - Qd).max() < 1e-12 * np.abs(Qd).max()
    ok &= np.allclose([Q[1][O.index(e)] for e in np.eye(3, dtype=int)], mom.sum(0), atol=1e-12)
    return bool(ok)


def test_fmm_converges_with_p():
    assert pin_fmm_converges()


def test_root_moments():
    assert pin_root_moments()


def test_energy_error_at_e005():
    """Sec. IV: at e = 0.05 the energy error is below 1 % (configurations
    whose energy is near zero excepted); (p, alpha) = (5, 0.71), (3, 0.54)."""
    pos, mom, box = W.lattice(12, seed=99)
    Hd = O.direct_field(pos, mom)
    Ed = O.energy_from_field(mom, Hd)
    for p, a in ((5, 0.71), (3, 0.54)):
        H, E, f = O.fmm_field(pos, mom, p, a, 0.0, box=box)
        assert abs(E - Ed) < 0.01 * abs(Ed), (p, a, E, Ed)


def test_average_error_p6_048():
    """Sec. IV: (p, alpha) = (6, 0.48) gives about 0.02 % average error."""
    pos, mom, box = W.lattice(12, seed=98)
    Hd = O.direct_field(pos, mom)
    H, E, f = O.fmm_field(pos, mom, 6, 0.48, 0.0, box=box)
    rel = np.linalg.norm(H - Hd, axis=1) / np.linalg.norm(Hd, axis=1)
    assert rel.mean() < 2e-3


def test_sampled_downward_matches_full():
    pos, mom, box = W.lattice(10)
    H, E, f = O.fmm_field(pos, mom, 4, 0.5, 8.0, box=box)
    mask = np.zeros(1 << f.depth, np.uint8)
    mask[[3, 77, 100]] = 1
    f.downward(mask)
    Hs = f.field()
    sel = np.isin(f.leaf_of(), [3, 77, 100])
    assert np.array_equal(Hs[sel], H[sel])
    assert np.all(np.isnan(Hs[~sel]))


# --------------------------------------------------------------------------
# Ensemble time step: Philox4x64-10 and the random rotation
# --------------------------------------------------------------------------

def test_philox_matches_numpy():
    """The oracle's Philox4x64-10 equals numpy's Philox bit generator, which
    increments its counter before each block."""
    for key, ctr in (((7, 11), 5), ((0, 0), 0), ((810233, 3), 123456789)):
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                              counter=np.array([ctr, 0, 0, 0], dtype=np.uint64))
        want = bg.random_raw(4)
        got = O.philox4x64([ctr + 1, 0, 0, 0], key)
        assert np.array_equal(got, want)


def test_rotation_properties():
    """Rotations keep |m|, turn by at most max_angle, and are reproducible;
    axes are isotropic and angles uniform over many draws."""
    rng = np.random.default_rng(31)
    m = W.unit_vectors(20000, rng)
    r = O.rotate_moments(m, seed=5, step=2, max_angle=0.05)
    assert np.allclose(np.linalg.norm(r, axis=1), 1.0, atol=1e-14)
    ang = np.arccos(np.clip((m * r).sum(1), -1, 1))
    assert ang.max() <= 0.05 + 1e-12 and ang.mean() > 0.01
    assert np.array_equal(r, O.rotate_moments(m, 5, 2, 0.05))
    assert not np.array_equal(r, O.rotate_moments(m, 5, 3, 0.05))
    # the first 10 dipoles drawn as a slice equal the same dipoles in the full call
    assert np.array_equal(O.rotate_moments(m[100:110], 5, 2, 0.05, first=100), r[100:110])
    # a large angle: the rotation of the axis itself is the identity
    e = np.tile([0.0, 0.0, 1.0], (5000, 1))
    big = O.rotate_moments(e, 9, 0, np.pi)
    assert np.abs((big ** 2).sum(1) - 1).max() < 1e-14
    # isotropy of the drawn axes: the mean of m' - m over random directions
    assert np.abs((big - e).mean(0)[:2]).max() < 0.05
