"""Pins of the selector network's CPU oracle (oracle/mlp.py): the analytic
gradient against central finite differences, BF16 rounding against its
definition, and the loss against a hand computation for a one-hidden-unit
case."""
import numpy as np

from oracle import mlp as M


def _setup(seed=0, B=37):
    rng = np.random.default_rng(seed)
    theta = rng.standard_normal(M.n_params()) * 0.2
    X = rng.standard_normal((B, 12)) * 3 + 1
    T = rng.standard_normal((B, 2))
    mask = (rng.uniform(size=(B, 2)) > 0.2).astype(float)
    norm = (X.mean(0), X.std(0) + 0.1, T.mean(0), T.std(0) + 0.1)
    return theta, X, T, mask, norm


def test_gradient_matches_finite_differences():
    theta, X, T, mask, norm = _setup()
    L, g = M.loss_and_grad(theta, X, T, mask, norm)
    rng = np.random.default_rng(1)
    idx = rng.choice(len(theta), size=60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (M.loss_and_grad(theta + e, X, T, mask, norm)[0] -
              M.loss_and_grad(theta - e, X, T, mask, norm)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.140625, 1e-3], dtype=np.float32)
    r = M.bf16(x)
    assert r[0] == 1.0
    # BF16 keeps 7 fraction bits (step 2^-7 near 1): 1 + 2^-8 is a tie and
    # rounds to the even neighbour 1; 1 + 3*2^-9 = 1 + 0.75*2^-7 rounds up
    assert r[1] == 1.0
    assert r[2] == 1.0 + 2 ** -7
    assert r[3] == -3.140625
    # the relative error of BF16 rounding is at most 2^-8
    y = np.random.default_rng(3).standard_normal(1000).astype(np.float32)
    assert np.all(np.abs(M.bf16(y) - y) <= 2 ** -8 * np.abs(y) + 1e-45)


def test_shapes_and_zero_mask():
    theta, X, T, mask, norm = _setup(B=5)
    Y, acts = M.forward(theta, X, norm)
    assert Y.shape == (5, 2) and len(acts) == 5
    L, g = M.loss_and_grad(theta, X, T, np.zeros_like(mask), norm)
    assert L == 0.0 and np.all(g == 0.0)
    assert M.n_params() == 12 * 64 + 64 + 2 * (64 * 64 + 64) + 64 * 2 + 2
