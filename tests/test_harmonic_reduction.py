"""The harmonic reduction the tensor-core M2L engines contract (CPU, against
the oracle's M2L, Eq. taylorcalc).

The D tensors are derivatives of 1/r, so sum_a D_{m+2e_a} = 0 (Laplace).
Hence a moment Q_k with k_z >= 2 may be folded into Q_{k-2e_z+2e_x} and
Q_{k-2e_z+2e_y} (minus sign) without changing any V_n, and V_n with n_z >= 2
equals -V_{n-2e_z+2e_x} - V_{n-2e_z+2e_y}.  These tests restate the fold and
the completion in NumPy and check them against the oracle's full M2L, for
every order the engines use and both truncations; they pin the arithmetic
the GPU kernels implement, not the kernels themselves."""
import numpy as np
import pytest

import oracle as O


def fold(p, Q):
    """Q (oracle order, T(p) entries) -> Q folded: entries with k_z >= 2 moved."""
    mi = O.multi_indices(p)
    idx = {tuple(int(v) for v in m): i for i, m in enumerate(mi)}
    Q = np.array(Q, dtype=float)
    # by decreasing k_z, so that every moved value is already final
    for i in sorted(range(len(mi)), key=lambda i: -int(mi[i][2])):
        x, y, z = (int(v) for v in mi[i])
        if z < 2:
            continue
        v = Q[i]
        Q[idx[(x + 2, y, z - 2)]] -= v
        Q[idx[(x, y + 2, z - 2)]] -= v
        Q[i] = 0.0
    return Q


def complete(p, V):
    """V with the n_z >= 2 entries recomputed from the others."""
    mi = O.multi_indices(p)
    idx = {tuple(int(v) for v in m): i for i, m in enumerate(mi)}
    V = np.array(V, dtype=float)
    for i in sorted(range(len(mi)), key=lambda i: int(mi[i][2])):
        x, y, z = (int(v) for v in mi[i])
        if z >= 2:
            V[i] = -V[idx[(x + 2, y, z - 2)]] - V[idx[(x, y + 2, z - 2)]]
    return V


@pytest.mark.parametrize("p", [2, 4, 5, 6, 7])
def test_fold_leaves_every_coefficient_unchanged(p):
    rng = np.random.default_rng(p)
    mi = O.multi_indices(p)
    deg = mi.sum(1)
    for trial in range(4):
        c = rng.uniform(-3, 3, 3) + np.array([5.0, 0.0, 0.0]) * (trial + 1)
        Q = rng.standard_normal(len(mi)) * 0.5 ** deg
        Q[0] = 0.0
        V_full = O.m2l(p, c, Q)
        V_fold = O.m2l(p, c, fold(p, Q))
        scale = np.abs(V_full).max()
        assert np.abs(V_fold - V_full).max() <= 1e-12 * scale
        # the folded moments live on the (p+1)^2 multi-indices with k_z <= 1
        assert np.all(fold(p, Q)[mi[:, 2] >= 2] == 0.0)
        assert int((mi[:, 2] <= 1).sum()) == (p + 1) ** 2


@pytest.mark.parametrize("p,P", [(4, 6), (6, 9), (6, 12)])
def test_fold_under_total_degree_truncation(p, P):
    """The fold keeps |k|, so the bound |n| + |k| <= P is unaffected."""
    rng = np.random.default_rng(10 * p + P)
    mi = O.multi_indices(p)
    Q = rng.standard_normal(len(mi)) * 0.4 ** mi.sum(1)
    Q[0] = 0.0
    c = np.array([4.0, -2.5, 3.0])
    V_full = O.m2l(p, c, Q, max_degree=P)
    V_fold = O.m2l(p, c, fold(p, Q), max_degree=P)
    assert np.abs(V_fold - V_full).max() <= 1e-12 * np.abs(V_full).max()


@pytest.mark.parametrize("p", [3, 5, 6])
def test_completion_recovers_the_dropped_coefficients(p):
    """V computed only on n_z <= 1 and completed by the Laplace identity equals
    the oracle's full V; a wrong sign or source index would not."""
    rng = np.random.default_rng(100 + p)
    mi = O.multi_indices(p)
    Q = rng.standard_normal(len(mi)) * 0.5 ** mi.sum(1)
    Q[0] = 0.0
    c = np.array([-3.0, 4.5, 2.0])
    V = O.m2l(p, c, fold(p, Q))
    part = V.copy()
    part[mi[:, 2] >= 2] = 0.0
    got = complete(p, part)
    assert np.abs(got - V).max() <= 1e-12 * np.abs(V).max()
    # planted mistake: the completion with one source instead of two fails
    bad = part.copy()
    idx = {tuple(int(v) for v in m): i for i, m in enumerate(mi)}
    for i in sorted(range(len(mi)), key=lambda i: int(mi[i][2])):
        x, y, z = (int(v) for v in mi[i])
        if z >= 2:
            bad[i] = -bad[idx[(x + 2, y, z - 2)]]
    assert np.abs(bad - V).max() > 1e-3 * np.abs(V).max()
