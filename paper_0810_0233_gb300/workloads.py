"""Seeded synthetic dipole sets.

This module only draws inputs: positions, unit moments and the random numbers
of the ensemble time step.  It holds none of the multipole method's
arithmetic, so it can feed both the GPU library and the CPU oracle.

Workloads (sizes and distributions of the paper's lattice benchmark, Sec. IV,
and of the ferrofluid / nanomagnet / ensemble settings built on it):

* ``lattice``      simple-cubic lattice, spacing 1, random unit moments
                   (the paper's benchmark system).
* ``ferrofluid``   N uniform points in a cube, minimum separation enforced by
                   rejection sampling, random unit moments.
* ``ring``         thin-film ring cut from a square lattice, vortex moments
                   with Gaussian tilt noise.
* ``clustered``    Gaussian blobs plus straight chains of touching dipoles.

Seeds: base 810233; workload k of the benchmark suite uses 810233 + k.
"""
from __future__ import annotations

import math

import numpy as np

BASE_SEED = 810233


def unit_vectors(n: int, rng: np.random.Generator) -> np.ndarray:
    """n directions uniform on the unit sphere (normalised Gaussians)."""
    v = rng.standard_normal((n, 3))
    norm = np.linalg.norm(v, axis=1, keepdims=True)
    bad = norm[:, 0] == 0.0
    while bad.any():
        v[bad] = rng.standard_normal((int(bad.sum()), 3))
        norm = np.linalg.norm(v, axis=1, keepdims=True)
        bad = norm[:, 0] == 0.0
    return v / norm


def lattice(nx: int, ny: int | None = None, nz: int | None = None, spacing: float = 1.0,
            seed: int = BASE_SEED + 1):
    """Simple-cubic lattice (points at 0..n-1) with random unit moments.

    Returns (pos, mom, box) where box = [lo, hi] is the lattice-cell box
    [-spacing/2, (n-1/2) spacing] used by the paper's examples."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    rng = np.random.default_rng(seed)
    gx, gy, gz = (np.arange(k, dtype=np.float64) * spacing for k in (nx, ny, nz))
    pos = np.stack(np.meshgrid(gx, gy, gz, indexing="ij"), axis=-1).reshape(-1, 3)
    mom = unit_vectors(len(pos), rng)
    box = np.array([-0.5 * spacing] * 3 + [(nx - 0.5) * spacing, (ny - 0.5) * spacing,
                                           (nz - 0.5) * spacing])
    return np.ascontiguousarray(pos), mom, box


def ferrofluid(n: int = 1_000_000, side: float = 100.0, dmin: float = 0.5,
               seed: int = BASE_SEED + 2):
    """n points uniform in [0, side]^3 with pairwise distance >= dmin.

    Rejection sampling in batches: a candidate is rejected if it lies closer
    than dmin to an accepted point, or to an earlier candidate of its own
    batch.  Returns (pos, mom)."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    acc = np.zeros((0, 3))
    while len(acc) < n:
        need = n - len(acc)
        cand = rng.uniform(0.0, side, size=(int(need * 1.25) + 64, 3))
        if len(acc):
            d, _ = cKDTree(acc).query(cand, k=1, distance_upper_bound=dmin)
            cand = cand[~(d < dmin)]
        if len(cand) > 1:
            pairs = cKDTree(cand).query_pairs(dmin, output_type="ndarray")
            if len(pairs):
                drop = np.zeros(len(cand), dtype=bool)
                # the later candidate of each close pair is rejected
                drop[np.maximum(pairs[:, 0], pairs[:, 1])] = True
                cand = cand[~drop]
        acc = np.concatenate([acc, cand[:need]])
    pos = np.ascontiguousarray(acc[:n])
    mom = unit_vectors(n, rng)
    return pos, mom


def ring(r_out: float = 707.58, r_in: float = 235.86, layers: int = 3, spacing: float = 1.0,
         tilt_sigma: float = 0.1, seed: int = BASE_SEED + 3):
    """Thin-film ring: square-lattice points with r_in <= rho <= r_out in each
    of ``layers`` planes z = 0, 1, ...; moments follow the in-plane vortex
    (-sin phi, cos phi, 0) plus a Gaussian tilt of ``tilt_sigma`` drawn
    perpendicular to the vortex direction, renormalised to unit length.
    Returns (pos, mom)."""
    rng = np.random.default_rng(seed)
    m = int(math.ceil(r_out / spacing))
    g = np.arange(-m, m + 1, dtype=np.float64) * spacing
    X, Y = np.meshgrid(g, g, indexing="ij")
    rho2 = X * X + Y * Y
    keep = (rho2 >= r_in * r_in) & (rho2 <= r_out * r_out)
    x, y = X[keep], Y[keep]
    n2 = len(x)
    pos = np.empty((n2 * layers, 3))
    for k in range(layers):
        pos[k * n2:(k + 1) * n2, 0] = x
        pos[k * n2:(k + 1) * n2, 1] = y
        pos[k * n2:(k + 1) * n2, 2] = k * spacing
    phi = np.arctan2(pos[:, 1], pos[:, 0])
    m0 = np.stack([-np.sin(phi), np.cos(phi), np.zeros_like(phi)], axis=1)
    # two unit vectors perpendicular to the vortex direction: radial and z
    e1 = np.stack([np.cos(phi), np.sin(phi), np.zeros_like(phi)], axis=1)
    e2 = np.zeros_like(m0)
    e2[:, 2] = 1.0
    g2 = rng.standard_normal((len(pos), 2)) * tilt_sigma
    mom = m0 + g2[:, :1] * e1 + g2[:, 1:] * e2
    mom /= np.linalg.norm(mom, axis=1, keepdims=True)
    return np.ascontiguousarray(pos), np.ascontiguousarray(mom)


def clustered(n: int, seed: int, blob_sigma: float = 3.0, blob_size: int = 500,
              chain_len: int = 20, chain_frac: float = 0.2, dmin: float = 0.5):
    """Clustered set of n points: (1-chain_frac) of them in Gaussian blobs of
    ``blob_size`` points (sigma ``blob_sigma``, centres uniform in a cube of
    side 4 n^(1/3)), the rest in straight chains of ``chain_len`` touching
    dipoles (spacing 1, random direction).  Points closer than dmin to an
    earlier point are redrawn.  Returns (pos, mom)."""
    from scipy.spatial import cKDTree

    rng = np.random.default_rng(seed)
    side = 4.0 * n ** (1.0 / 3.0)
    n_chain = int(round(chain_frac * n)) // chain_len * chain_len
    n_blob = n - n_chain
    pts = []
    nb = max(1, int(math.ceil(n_blob / blob_size)))
    centres = rng.uniform(0.0, side, size=(nb, 3))
    left = n_blob
    for b in range(nb):
        k = min(blob_size, left)
        if k <= 0:
            break
        pts.append(centres[b] + rng.standard_normal((k, 3)) * blob_sigma)
        left -= k
    for _ in range(n_chain // chain_len):
        start = rng.uniform(0.0, side, size=3)
        d = unit_vectors(1, rng)[0]
        pts.append(start + np.arange(chain_len)[:, None] * d[None, :])
    pos = np.concatenate(pts) if pts else np.zeros((0, 3))
    # enforce the minimum separation by redrawing offenders uniformly
    for _ in range(64):
        pairs = cKDTree(pos).query_pairs(dmin, output_type="ndarray")
        if len(pairs) == 0:
            break
        bad = np.unique(np.maximum(pairs[:, 0], pairs[:, 1]))
        pos[bad] = rng.uniform(0.0, side, size=(len(bad), 3))
    mom = unit_vectors(len(pos), rng)
    return np.ascontiguousarray(pos), mom


def ensemble_sizes(count: int = 512, n_lo: int = 1_000, n_hi: int = 200_000,
                   seed: int = BASE_SEED + 4) -> np.ndarray:
    """Per-sample N, log-uniform in [n_lo, n_hi]."""
    rng = np.random.default_rng(seed)
    return np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count)).astype(np.int64)


def ensemble(count: int = 512, seed: int = BASE_SEED + 4):
    """The ensemble workload: `count` clustered samples with log-uniform sizes
    (ensemble_sizes), sample i drawn by clustered(N_i, seed * 1000 + i).
    Returns (positions, moments, offsets), offsets of length count + 1."""
    sizes = ensemble_sizes(count, seed=seed)
    pos, mom = [], []
    for i, n in enumerate(sizes):
        p_, m_ = clustered(int(n), seed=seed * 1000 + i)
        pos.append(p_)
        mom.append(m_)
    off = np.concatenate([[0], np.cumsum([len(x) for x in pos])]).astype(np.int64)
    return np.ascontiguousarray(np.concatenate(pos)), np.ascontiguousarray(np.concatenate(mom)), off


def rotation_draws(n: int, max_angle: float, rng: np.random.Generator):
    """Random rotation per moment: axis uniform on the sphere and angle
    uniform in [0, max_angle].  Returns (axis n x 3, angle n)."""
    return unit_vectors(n, rng), rng.uniform(0.0, max_angle, size=n)


def subset(n: int, k: int, seed: int) -> np.ndarray:
    """k distinct indices out of n, sorted (error-evaluation subsets)."""
    rng = np.random.default_rng(seed)
    k = min(k, n)
    return np.sort(rng.choice(n, size=k, replace=False)).astype(np.int64)
