"""TEST INFRASTRUCTURE ONLY: plain NumPy FP64 statement of the parameter
selector's network (a project addition; the paper chooses s by Eq. so and
(p, alpha_m) from Table II / Fig. 3 by hand).

Network: 12 inputs -> 64 -> 64 -> 64 -> 2 outputs, ReLU after each hidden
layer, linear output.  Inputs are standardised, x_n = (x - mu_x) / sd_x;
targets likewise, t_n = (t - mu_y) / sd_y.  Loss: mean squared error over the
masked outputs, L = sum(mask * (y - t_n)^2) / max(sum(mask), 1).
Weights are used as BF16 values (round to nearest even from FP32 masters),
the arithmetic here is FP64.

Only the tests import this module; it shares nothing with the GPU library.
Pinned in tests/test_oracle_mlp.py against central finite differences.
"""
import numpy as np

SIZES = (12, 64, 64, 64, 2)


def n_params():
    return sum(a * b + b for a, b in zip(SIZES[:-1], SIZES[1:]))


def unpack(theta):
    """Flat parameter vector -> [(W (in x out), b (out))] per layer."""
    out, k = [], 0
    for a, b in zip(SIZES[:-1], SIZES[1:]):
        W = theta[k:k + a * b].reshape(a, b)
        k += a * b
        bb = theta[k:k + b]
        k += b
        out.append((W, bb))
    return out


def bf16(x):
    """Round FP32 values to the nearest BF16 value (ties to even), as FP64."""
    u = np.ascontiguousarray(np.asarray(x, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def forward(theta, X, norm):
    """Returns (outputs in standardised units, list of layer activations)."""
    mu_x, sd_x = norm[0], norm[1]
    h = (np.asarray(X, np.float64) - mu_x) / sd_x
    acts = [h]
    layers = unpack(np.asarray(theta, np.float64))
    for li, (W, b) in enumerate(layers):
        z = h @ W + b
        h = np.maximum(z, 0.0) if li < len(layers) - 1 else z
        acts.append(h)
    return h, acts


def loss_and_grad(theta, X, T, mask, norm):
    """MSE loss in standardised units and its gradient with respect to theta."""
    mu_y, sd_y = norm[2], norm[3]
    Tn = (np.asarray(T, np.float64) - mu_y) / sd_y
    Y, acts = forward(theta, X, norm)
    m = np.asarray(mask, np.float64)
    cnt = max(m.sum(), 1.0)
    L = float((m * (Y - Tn) ** 2).sum() / cnt)
    layers = unpack(np.asarray(theta, np.float64))
    dh = 2.0 * m * (Y - Tn) / cnt
    grads = []
    for li in range(len(layers) - 1, -1, -1):
        W, b = layers[li]
        a_in = acts[li]
        if li < len(layers) - 1:
            dh = dh * (acts[li + 1] > 0.0)
        grads.append((a_in.T @ dh, dh.sum(0)))
        dh = dh @ W.T
    grads.reverse()
    g = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    return L, g
