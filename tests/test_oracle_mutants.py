"""The oracle's pins catch plausible mistakes.

Each case copies the oracle source, plants one mistake (a dropped term, a
wrong sign, a wrong index, a transposed operand, a wrong factor, a wrong tie
rule), compiles the copy on the CPU and runs the pins of
``test_oracle_pins.py`` against it: at least one pin must fail.  The oracle
source itself is never modified.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle as O
from paper_0810_0233_gb300 import workloads as W
import test_oracle_adaptive as A
import test_oracle_pins as P

SRC = os.path.join(os.path.dirname(O.__file__), "ccfmm_oracle.c")

MUTANTS = {
    "p2m_dropped_derivative": (
        "if (n[0] > 0) s += m[0] * mono(r, n[0] - 1, n[1], n[2]);",
        "if (n[0] > 0) s += m[0] * mono(r, n[0], n[1], n[2]);"),
    "m2l_sign": (
        "V[t] += ((kn % 2) ? -1.0 : 1.0) * s;",
        "V[t] += s;"),
    "l2p_sign": (
        "if (n[0] > 0) H[0] -= V[t] * mono(r, n[0] - 1, n[1], n[2]);",
        "if (n[0] > 0) H[0] += V[t] * mono(r, n[0] - 1, n[1], n[2]);"),
    "direct_factor": (
        "H[0] += (3.0 * mu * u[0] - mj[0]) / r3;",
        "H[0] += (2.0 * mu * u[0] - mj[0]) / r3;"),
    "ftable_term": (
        "(double)(2 * km + 1 - q[v]) * f",
        "(double)(2 * km - q[v]) * f"),
    "l2l_transposed": (
        "Vp[orc_index(n[0] + k[0], n[1] + k[1], n[2] + k[2])]",
        "Vp[orc_index(n[0] + k[1], n[1] + k[0], n[2] + k[2])]"),
    "m2m_transposed": (
        "s += mono(c, kx, ky, kz) * Qc",
        "s += mono(c, ky, kx, kz) * Qc"),
    "energy_no_half": (
        "return -0.5 * e;",
        "return -1.0 * e;"),
    "near_test_theta": (
        "return w2 > f->theta * f->theta * d2 * (1.0 + 1e-12);",
        "return w2 > f->theta * d2 * (1.0 + 1e-12);"),
    "boundary_to_lower_cell": (
        "i64 ca = (i64)floor(t);",
        "i64 ca = (i64)ceil(t) - 1;"),
    "split_tie_y_first": (
        "if (w[1] > w[a]) a = 1;",
        "if (w[1] >= w[a]) a = 1;"),
    "sibling_dropped": (
        "ivec_push(&f->partners[2 * c], 2 * c + 1);\n",
        "\n"),
    "m2l_offset_reversed": (
        "for (int a = 0; a < 3; ++a) rel[a] = cen[a] - ca[a];",
        "for (int a = 0; a < 3; ++a) rel[a] = ca[a] - cen[a];"),
    "degree_bound_off_by_one": (
        "if (kn + k[0] + k[1] + k[2] > maxdeg) continue;",
        "if (kn + k[0] + k[1] + k[2] >= maxdeg) continue;"),
    "fmm_ignores_truncation": (
        "m2l_one(&f->F, f->p, f->maxdeg, rel,",
        "m2l_one(&f->F, f->p, 2 * f->p, rel,"),
    "adaptive_far_descendant_dropped": (
        "            ivec_push(&f->c[c].farp, b);",
        "            (void)b;"),
    "adaptive_coarse_leaf_dropped": (
        "                a_consider(f, ci, a);",
        "                (void)ci;"),
    "adaptive_m2m_offset_reversed": (
        "for (int a = 0; a < 3; ++a) rel[a] = cc[a] - cen[a];",
        "for (int a = 0; a < 3; ++a) rel[a] = cen[a] - cc[a];"),
    "adaptive_splits_at_s": (
        "if ((double)f->c[c].np <= f->s",
        "if ((double)f->c[c].np < f->s"),
    "leaf_not_self_near": (
        "ivec_push(&f->nearp[c], c);",
        "(void)0;"),
}


def _c1_checks():
    pos, mom, box = W.lattice(10)
    f = O.OracleFMM(pos, mom, 4, 0.5, 8.0, box=box)
    ok = f.depth == 7 and list(f.axes()) == [0, 1, 2, 0, 1, 2, 0]
    leaf = f.leaf_of()
    xcell = ((leaf >> 6) & 1) * 4 + ((leaf >> 3) & 1) * 2 + (leaf & 1)
    ok &= bool(np.all(xcell[pos[:, 0] == 2.0] == 2))
    ok &= P._lists_ok(f, 0.5)
    return bool(ok)


PINS = [P.pin_axial_equatorial, P.pin_field_is_minus_grad_potential, P.pin_pair_energy,
        P.pin_lorentz_sphere, P.pin_D_closed_forms, P.pin_D_laplace_parity,
        P.pin_p2m_single_dipole, P.pin_p2m_charge_limit, P.pin_multipole_potential,
        P.pin_m2m_exact, P.pin_l2l_l2p, P.pin_l2p_gradient, P.pin_m2l_convergence,
        P.pin_worked_examples, P.pin_eq_so, P.pin_fmm_converges, P.pin_root_moments,
        P.pin_total_degree_is_taylor, P.pin_fmm_total_degree_brute_force, _c1_checks,
        A.pin_adaptive_matches_uniform, A.pin_adaptive_coverage, A.pin_adaptive_converges,
        A.pin_adaptive_all_near_is_direct, A.pin_adaptive_symmetry, A.pin_adaptive_tree]


def _run_pins():
    failed = []
    for pin in PINS:
        try:
            with np.errstate(all="ignore"):
                ok = bool(pin())
        except Exception:  # a mistake that breaks a pin outright also counts
            ok = False
        if not ok:
            failed.append(pin.__name__)
    return failed


def test_unmodified_oracle_passes_all_pins():
    assert _run_pins() == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, "mutation anchor not found: %s" % name
    mutated = src.replace(old, new)
    c = tmp_path / ("m_%s.c" % name)
    so = tmp_path / ("m_%s.so" % name)
    c.write_text(mutated)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp", str(c),
                           "-o", str(so), "-lm"])
    with O.using_library(str(so)):
        failed = _run_pins()
    assert failed, "no pin caught mutant %s" % name
