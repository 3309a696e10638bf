"""Local parity measures for the FP32 mixed path (test helpers).

A relative RMS over all dipoles can hide a fault that touches few of them:
one far partner dropped from one cell (an item or tile boundary slip in the
grouped M2L) changes only the field of that cell's dipoles.  Two local
measures bound every dipole and every cell instead:

* dipole:  max_i |H_i - H_i^ref| / max(|H_i^ref|, RMS_j |H_j^ref|), i.e.
  Eq. H2 plus Eq. H read per field point, relative to the point's own field
  (with the RMS field as the floor, so that a point where the field happens
  to vanish is held to the absolute scale of the system);
* cell:    the Taylor coefficients V of a cell (Eq. taylorcalc plus
  Eq. taylorshift) weighted by the size of each term at the cell's half
  diagonal rho, w_n = rho^|n| / n! (w_n V_n is the term's share of the
  potential at the cell's corner), compared with the oracle's as
  |w (V_c - V_c^ref)| / RMS over the level's cells of |w V^ref|.

``tests/test_local_parity.py`` computes, on the CPU and for the inputs the
GPU tests use, how far dropping any single far partner of any single cell
moves these measures, and checks that it is far above the bounds below.
"""
import math

import numpy as np

# bounds applied to every mixed-path (FP32 bulk, TF32x3 or FP32 FMA M2L,
# FP64 tables and local accumulation) result
DIPOLE_TOL = 5e-5
CELL_TOL = 1e-4


def dipole_errors(H, Href):
    """|H_i - H_i^ref| / max(|H_i^ref|, RMS_j |H_j^ref|) for every row."""
    H = np.asarray(H, float).reshape(-1, 3)
    Href = np.asarray(Href, float).reshape(-1, 3)
    mag = np.sqrt((Href ** 2).sum(1))
    rms = math.sqrt(float((mag ** 2).mean()))
    return np.sqrt(((H - Href) ** 2).sum(1)) / np.maximum(mag, max(rms, 1e-300))


def dipole_max_err(H, Href):
    return float(dipole_errors(H, Href).max())


def level_half_diagonals(box, axes):
    """Half diagonal of the cells of every level 0..L of the bisection tree
    (axes[l-1] is the axis split to make level l)."""
    w = np.array(box[3:], float) - np.array(box[:3], float)
    out = [0.5 * float(np.linalg.norm(w))]
    for a in axes:
        w[int(a)] *= 0.5
        out.append(0.5 * float(np.linalg.norm(w)))
    return np.array(out)


def term_weights(mi, rho):
    """w_n = rho^|n| / n! for the multi-indices mi (T x 3); w_0 = 0 (V_0
    never reaches the field)."""
    mi = np.asarray(mi)
    deg = mi.sum(1)
    fact = np.array([math.factorial(a) * math.factorial(b) * math.factorial(c) for a, b, c in mi],
                    float)
    w = rho ** deg / fact
    w[deg == 0] = 0.0
    return w


def cell_errors(V, Vref, cells, mi, box, axes):
    """Per-cell weighted error of V against Vref (both T columns ordered as
    mi) for the heap ids ``cells``; returns {level: max error}."""
    rho = level_half_diagonals(box, axes)
    cells = np.asarray(sorted(cells), dtype=np.int64)
    lev = np.floor(np.log2(cells)).astype(int)
    out = {}
    for l in np.unique(lev):
        rows = cells[lev == l]
        w = term_weights(mi, rho[l])
        ref = Vref[rows] * w
        scale = math.sqrt(float((ref ** 2).sum(1).mean()))
        if scale == 0.0:
            continue
        d = (V[rows] - Vref[rows]) * w
        out[int(l)] = float(np.sqrt((d ** 2).sum(1)).max() / scale)
    return out


def cell_max_err(V, Vref, cells, mi, box, axes):
    e = cell_errors(V, Vref, cells, mi, box, axes)
    return max(e.values()) if e else 0.0


def cell_errors_levels(V, Vref, rows, levels, rho, mi):
    """cell_errors for trees whose cells are not heap-numbered (the adaptive
    tree): rows are cell numbers, levels their levels, rho[l] the half
    diagonal of level l; returns {level: max error}."""
    rows = np.asarray(rows, dtype=np.int64)
    levels = np.asarray(levels, dtype=np.int64)
    out = {}
    for l in np.unique(levels):
        r = rows[levels == l]
        w = term_weights(mi, rho[int(l)])
        ref = Vref[r] * w
        scale = math.sqrt(float((ref ** 2).sum(1).mean()))
        if scale == 0.0:
            continue
        d = (V[r] - Vref[r]) * w
        out[int(l)] = float(np.sqrt((d ** 2).sum(1)).max() / scale)
    return out
