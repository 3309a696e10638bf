"""TEST INFRASTRUCTURE ONLY: Python bindings of the FP64 CPU oracle.

The oracle (``ccfmm_oracle.c``) is a plain, slow statement of the Cartesian
FMM for point dipoles of Zhang & Haas and of the O(N^2) direct dipole sum.
Only the test suite, the package smoke check and the benchmark's CPU-baseline
leg may import this module.  It shares no code with the GPU library and
never imports it.

Pins: every routine is checked in ``tests/test_oracle_*.py`` against
closed forms, the paper's worked examples and tables, symbolic
differentiation and brute force (see the docstrings there); the
adaptive-depth tree (``OracleAFMM``, a project extension) in
``tests/test_oracle_adaptive.py``.  Parity
unpinned: none of the functions exported here.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ccfmm_oracle.c")
_LIB = os.path.join(_HERE, "libccfmm_oracle.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lp = ctypes.POINTER(ctypes.c_int64)
_up = ctypes.POINTER(ctypes.c_uint8)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/libccfmm_oracle.so`` (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _bind(path):
    lib = ctypes.CDLL(path)
    sig = {
        "orc_nterms": (ctypes.c_int, [ctypes.c_int]),
        "orc_index": (ctypes.c_int, [ctypes.c_int] * 3),
        "orc_multi_indices": (None, [ctypes.c_int, _ip]),
        "orc_D_tensors": (None, [ctypes.c_int, _dp, _dp]),
        "orc_F_nnz": (ctypes.c_int, [ctypes.c_int, ctypes.c_int]),
        "orc_p2m": (None, [ctypes.c_int, _dp, _i64, _dp, _dp, _dp]),
        "orc_m2m": (None, [ctypes.c_int, _dp, _dp, _dp]),
        "orc_l2l": (None, [ctypes.c_int, _dp, _dp, _dp]),
        "orc_m2l": (None, [ctypes.c_int, _dp, _dp, _dp]),
        "orc_m2l_degree": (None, [ctypes.c_int, ctypes.c_int, _dp, _dp, _dp]),
        "orc_fmm_set_truncation": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
        "orc_l2p": (None, [ctypes.c_int, _dp, _dp, _dp]),
        "orc_direct_field": (None, [_i64, _dp, _dp, _i64, _lp, _dp]),
        "orc_energy_from_field": (ctypes.c_double, [_i64, _dp, _dp]),
        "orc_leaf_size_rule": (ctypes.c_double, [ctypes.c_int]),
        "orc_error_estimate": (ctypes.c_double, [ctypes.c_int, ctypes.c_double]),
        "orc_threads": (ctypes.c_int, []),
        "orc_set_threads": (None, [ctypes.c_int]),
        "orc_fmm_new": (ctypes.c_void_p, [_i64, _dp, _dp, ctypes.c_int, ctypes.c_double,
                                          ctypes.c_double, _dp]),
        "orc_fmm_free": (None, [ctypes.c_void_p]),
        "orc_fmm_depth": (ctypes.c_int, [ctypes.c_void_p]),
        "orc_fmm_leaf_target": (ctypes.c_double, [ctypes.c_void_p]),
        "orc_fmm_box": (None, [ctypes.c_void_p, _dp]),
        "orc_fmm_axes": (None, [ctypes.c_void_p, _ip]),
        "orc_fmm_leaf_widths": (None, [ctypes.c_void_p, _dp]),
        "orc_fmm_leaf_of": (None, [ctypes.c_void_p, _lp]),
        "orc_fmm_nonempty_leaves": (_i64, [ctypes.c_void_p]),
        "orc_fmm_cell_center": (None, [ctypes.c_void_p, _i64, _dp]),
        "orc_fmm_far_pairs": (_i64, [ctypes.c_void_p, _lp]),
        "orc_fmm_near_pairs": (_i64, [ctypes.c_void_p, _lp]),
        "orc_fmm_upward": (None, [ctypes.c_void_p]),
        "orc_fmm_downward": (None, [ctypes.c_void_p, _up]),
        "orc_fmm_moments": (None, [ctypes.c_void_p, _dp]),
        "orc_fmm_locals": (None, [ctypes.c_void_p, _dp]),
        "orc_fmm_field": (None, [ctypes.c_void_p, _dp]),
        "orc_fmm_energy": (ctypes.c_double, [ctypes.c_void_p]),
        "orc_afmm_new": (ctypes.c_void_p, [_i64, _dp, _dp, ctypes.c_int, ctypes.c_double,
                                           ctypes.c_double, _dp]),
        "orc_afmm_free": (None, [ctypes.c_void_p]),
        "orc_afmm_run": (None, [ctypes.c_void_p]),
        "orc_afmm_field": (None, [ctypes.c_void_p, _dp]),
        "orc_afmm_energy": (ctypes.c_double, [ctypes.c_void_p]),
        "orc_afmm_ncells": (_i64, [ctypes.c_void_p]),
        "orc_afmm_cell": (None, [ctypes.c_void_p, _i64, _lp]),
        "orc_afmm_perm": (None, [ctypes.c_void_p, _lp]),
        "orc_afmm_pairs": (_i64, [ctypes.c_void_p, ctypes.c_int, _lp]),
        "orc_afmm_moments": (None, [ctypes.c_void_p, _dp]),
        "orc_afmm_locals": (None, [ctypes.c_void_p, _dp]),
        "orc_afmm_box": (None, [ctypes.c_void_p, _dp]),
        "orc_afmm_widths": (None, [ctypes.c_void_p, _dp]),
        "orc_philox4x64": (None, [_u64p, _u64p, _u64p]),
        "orc_rotate_moments": (None, [_i64, _dp, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                      _i64]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
        return _lib


class using_library:
    """Context manager: route every call of this module to another build of
    the oracle (tests plant mistakes in a copy to check that the pins catch
    them)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        _load()
        self._saved = _lib
        _lib = _bind(self.path)
        return _lib

    def __exit__(self, *exc):
        global _lib
        _lib = self._saved
        return False


def _d(a):
    return a.ctypes.data_as(_dp)


def _arr3(x, n=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if n is not None:
        a = a.reshape(n, 3)
    return a


# ---------------------------------------------------------------- indices
def nterms(order: int) -> int:
    """T(order) = number of multi-indices n with |n| <= order."""
    return _load().orc_nterms(order)


def multi_indices(order: int) -> np.ndarray:
    """The oracle's enumeration of multi-indices up to ``order`` (T x 3)."""
    T = nterms(order)
    out = np.zeros((T, 3), dtype=np.int32)
    _load().orc_multi_indices(order, out.ctypes.data_as(_ip))
    return out


def index(n) -> int:
    return _load().orc_index(int(n[0]), int(n[1]), int(n[2]))


# ---------------------------------------------------------------- primitives
def D_tensors(order: int, r) -> np.ndarray:
    """D_n(r) = d^n/d(-r)^n (1/|r|) for all |n| <= order (Eqs. Vm, Dn, Dnr)."""
    r = np.ascontiguousarray(np.asarray(r, dtype=np.float64).reshape(3))
    out = np.zeros(nterms(order))
    _load().orc_D_tensors(order, _d(r), _d(out))
    return out


def F_nnz(order: int, t: int) -> int:
    return _load().orc_F_nnz(order, t)


def p2m(p, c, pos, mom) -> np.ndarray:
    """Eq. multipolemoments about centre c."""
    pos = _arr3(pos).reshape(-1, 3)
    mom = _arr3(mom).reshape(-1, 3)
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(3))
    Q = np.zeros(nterms(p))
    _load().orc_p2m(p, _d(c), len(pos), _d(pos), _d(mom), _d(Q))
    return Q


def m2m(p, c, Qchild, Qparent=None) -> np.ndarray:
    """Eq. momentshift; c = child centre relative to the parent centre."""
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(3))
    Qc = np.ascontiguousarray(Qchild, dtype=np.float64)
    Qp = np.zeros(nterms(p)) if Qparent is None else np.array(Qparent, dtype=np.float64)
    _load().orc_m2m(p, _d(c), _d(Qc), _d(Qp))
    return Qp


def l2l(p, c, Vparent, Vchild=None) -> np.ndarray:
    """Eq. taylorshift; c = child centre relative to the parent centre."""
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(3))
    Vp = np.ascontiguousarray(Vparent, dtype=np.float64)
    Vc = np.zeros(nterms(p)) if Vchild is None else np.array(Vchild, dtype=np.float64)
    _load().orc_l2l(p, _d(c), _d(Vp), _d(Vc))
    return Vc


def m2l(p, c, Q, V=None, max_degree=None) -> np.ndarray:
    """Eq. taylorcalc; c = field-cell centre relative to the source-cell centre.
    ``max_degree`` None: square truncation; else only terms |n|+|k| <= it."""
    c = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(3))
    Q = np.ascontiguousarray(Q, dtype=np.float64)
    V = np.zeros(nterms(p)) if V is None else np.array(V, dtype=np.float64)
    if max_degree is None:
        _load().orc_m2l(p, _d(c), _d(Q), _d(V))
    else:
        _load().orc_m2l_degree(p, int(max_degree), _d(c), _d(Q), _d(V))
    return V


def l2p(p, r, V) -> np.ndarray:
    """Eq. H (with H = -grad V); r relative to the expansion centre."""
    r = np.ascontiguousarray(np.asarray(r, dtype=np.float64).reshape(3))
    V = np.ascontiguousarray(V, dtype=np.float64)
    H = np.zeros(3)
    _load().orc_l2p(p, _d(r), _d(V), _d(H))
    return H


def direct_field(pos, mom, targets=None) -> np.ndarray:
    """O(N^2) dipole field at every point (or at ``targets``), Eq. H2 as read."""
    pos = _arr3(pos).reshape(-1, 3)
    mom = _arr3(mom).reshape(-1, 3)
    n = len(pos)
    if targets is None:
        H = np.zeros((n, 3))
        _load().orc_direct_field(n, _d(pos), _d(mom), n, None, _d(H))
    else:
        t = np.ascontiguousarray(np.asarray(targets, dtype=np.int64))
        H = np.zeros((len(t), 3))
        _load().orc_direct_field(n, _d(pos), _d(mom), len(t), t.ctypes.data_as(_lp), _d(H))
    return H


def energy_from_field(mom, H) -> float:
    """E = -1/2 sum_i m_i . H_i (units of mu0/4pi)."""
    mom = _arr3(mom).reshape(-1, 3)
    H = _arr3(H).reshape(-1, 3)
    return _load().orc_energy_from_field(len(mom), _d(mom), _d(H))


def leaf_size_rule(p: int) -> float:
    """Eq. so."""
    return _load().orc_leaf_size_rule(p)


def error_estimate(p: int, alpha: float) -> float:
    """e = [alpha/(2-alpha)]^p (Sec. III, Sec. IV)."""
    return _load().orc_error_estimate(p, alpha)


def philox4x64(counter, key) -> np.ndarray:
    """Philox4x64-10 block function (Salmon et al., SC 2011)."""
    c = np.ascontiguousarray(np.asarray(counter, dtype=np.uint64).reshape(4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint64).reshape(2))
    out = np.zeros(4, dtype=np.uint64)
    _load().orc_philox4x64(c.ctypes.data_as(_u64p), k.ctypes.data_as(_u64p), out.ctypes.data_as(_u64p))
    return out


def rotate_moments(mom, seed, step, max_angle, first=0) -> np.ndarray:
    """The ensemble time step: every moment turned by a Philox-drawn random
    rotation (axis uniform on the sphere, angle uniform in [0, max_angle])."""
    m = np.array(mom, dtype=np.float64).reshape(-1, 3).copy()
    _load().orc_rotate_moments(len(m), _d(m), int(seed), int(step), float(max_angle), int(first))
    return m


def threads() -> int:
    return _load().orc_threads()


def set_threads(n: int) -> None:
    _load().orc_set_threads(n)


# ---------------------------------------------------------------- whole FMM
class OracleFMM:
    """The paper's three passes on the CPU (Appendix): tree and lists at
    construction, ``upward()`` = updateMoment, ``downward()`` = updateField."""

    def __init__(self, pos, mom, p, theta, leaf_size=0.0, box=None):
        self._lib = _load()
        self.pos = _arr3(pos).reshape(-1, 3)
        self.mom = _arr3(mom).reshape(-1, 3)
        self.n = len(self.pos)
        self.p = int(p)
        bx = None
        if box is not None:
            self._box = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(6))
            bx = _d(self._box)
        h = self._lib.orc_fmm_new(self.n, _d(self.pos), _d(self.mom), self.p, float(theta),
                                  float(leaf_size), bx)
        if not h:
            raise ValueError("oracle rejected the arguments")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_fmm_free(h)
            self._h = None

    @property
    def depth(self) -> int:
        return self._lib.orc_fmm_depth(self._h)

    @property
    def leaf_target(self) -> float:
        return self._lib.orc_fmm_leaf_target(self._h)

    def box(self) -> np.ndarray:
        out = np.zeros(6)
        self._lib.orc_fmm_box(self._h, _d(out))
        return out

    def axes(self) -> np.ndarray:
        out = np.zeros(max(self.depth, 1), dtype=np.int32)
        self._lib.orc_fmm_axes(self._h, out.ctypes.data_as(_ip))
        return out[: self.depth]

    def leaf_widths(self) -> np.ndarray:
        out = np.zeros(3)
        self._lib.orc_fmm_leaf_widths(self._h, _d(out))
        return out

    def leaf_of(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.int64)
        self._lib.orc_fmm_leaf_of(self._h, out.ctypes.data_as(_lp))
        return out

    def nonempty_leaves(self) -> int:
        return self._lib.orc_fmm_nonempty_leaves(self._h)

    def cell_center(self, c: int) -> np.ndarray:
        out = np.zeros(3)
        self._lib.orc_fmm_cell_center(self._h, int(c), _d(out))
        return out

    def far_pairs(self) -> np.ndarray:
        """(cell, partner) heap ids of every Partners entry after createPartners."""
        k = self._lib.orc_fmm_far_pairs(self._h, None)
        out = np.zeros((max(k, 1), 2), dtype=np.int64)
        self._lib.orc_fmm_far_pairs(self._h, out.ctypes.data_as(_lp))
        return out[:k]

    def near_pairs(self) -> np.ndarray:
        k = self._lib.orc_fmm_near_pairs(self._h, None)
        out = np.zeros((max(k, 1), 2), dtype=np.int64)
        self._lib.orc_fmm_near_pairs(self._h, out.ctypes.data_as(_lp))
        return out[:k]

    def set_truncation(self, max_degree=None) -> None:
        """Square truncation (None) or the total-degree bound |n|+|k| <= max_degree."""
        if self._lib.orc_fmm_set_truncation(self._h, 0 if max_degree is None else int(max_degree)):
            raise ValueError("truncation bound outside [2, 2p]")

    def upward(self) -> None:
        self._lib.orc_fmm_upward(self._h)

    def downward(self, leaf_mask=None) -> None:
        if leaf_mask is None:
            self._lib.orc_fmm_downward(self._h, None)
        else:
            m = np.ascontiguousarray(np.asarray(leaf_mask, dtype=np.uint8))
            assert len(m) == (1 << self.depth)
            self._lib.orc_fmm_downward(self._h, m.ctypes.data_as(_up))

    def moments(self) -> np.ndarray:
        T = nterms(self.p)
        out = np.zeros((1 << (self.depth + 1), T))
        self._lib.orc_fmm_moments(self._h, _d(out))
        return out

    def locals(self) -> np.ndarray:
        T = nterms(self.p)
        out = np.zeros((1 << (self.depth + 1), T))
        self._lib.orc_fmm_locals(self._h, _d(out))
        return out

    def field(self) -> np.ndarray:
        out = np.zeros((self.n, 3))
        self._lib.orc_fmm_field(self._h, _d(out))
        return out

    def energy(self) -> float:
        return self._lib.orc_fmm_energy(self._h)


def fmm_field(pos, mom, p, theta, leaf_size=0.0, box=None, leaf_mask=None, max_degree=None):
    """Run the whole oracle FMM; returns (H in input order, E, OracleFMM).
    ``max_degree``: None for the square truncation of Eq. taylorcalc, else
    the total-degree bound on |n|+|k|."""
    f = OracleFMM(pos, mom, p, theta, leaf_size, box)
    if max_degree is not None:
        f.set_truncation(max_degree)
    f.upward()
    f.downward(leaf_mask)
    return f.field(), f.energy(), f


# ---------------------------------------------------------------- adaptive tree
class OracleAFMM:
    """Adaptive-depth tree (a project extension of the paper's complete tree):
    a cell is split while it holds more than ``s`` points; lists by the
    unequal-level extension of createPartners (see the C source)."""

    def __init__(self, pos, mom, p, theta, s, box=None):
        self._lib = _load()
        self.pos = _arr3(pos).reshape(-1, 3)
        self.mom = _arr3(mom).reshape(-1, 3)
        self.n = len(self.pos)
        self.p = int(p)
        bx = None
        if box is not None:
            self._box = np.ascontiguousarray(np.asarray(box, dtype=np.float64).reshape(6))
            bx = _d(self._box)
        h = self._lib.orc_afmm_new(self.n, _d(self.pos), _d(self.mom), self.p, float(theta),
                                   float(s), bx)
        if not h:
            raise ValueError("oracle rejected the arguments")
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_afmm_free(h)
            self._h = None

    def run(self):
        self._lib.orc_afmm_run(self._h)

    def field(self) -> np.ndarray:
        out = np.zeros((self.n, 3))
        self._lib.orc_afmm_field(self._h, _d(out))
        return out

    def energy(self) -> float:
        return self._lib.orc_afmm_energy(self._h)

    def cells(self) -> np.ndarray:
        """Per cell: level, parent, child0, child1, first point, count, leaf."""
        nc = self._lib.orc_afmm_ncells(self._h)
        out = np.zeros((nc, 7), dtype=np.int64)
        row = np.zeros(7, dtype=np.int64)
        for c in range(nc):
            self._lib.orc_afmm_cell(self._h, c, row.ctypes.data_as(_lp))
            out[c] = row
        return out

    def perm(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.int64)
        self._lib.orc_afmm_perm(self._h, out.ctypes.data_as(_lp))
        return out

    def moments(self) -> np.ndarray:
        """Q of every cell (ncells x T(p), oracle multi-index order), after run()."""
        out = np.zeros((self._lib.orc_afmm_ncells(self._h), nterms(self.p)))
        self._lib.orc_afmm_moments(self._h, _d(out))
        return out

    def locals(self) -> np.ndarray:
        """V of every cell (ncells x T(p), oracle multi-index order), after run()."""
        out = np.zeros((self._lib.orc_afmm_ncells(self._h), nterms(self.p)))
        self._lib.orc_afmm_locals(self._h, _d(out))
        return out

    def box(self) -> np.ndarray:
        out = np.zeros(6)
        self._lib.orc_afmm_box(self._h, _d(out))
        return out

    def widths(self) -> np.ndarray:
        """Cell widths of every level 0..40 (41 x 3)."""
        out = np.zeros((41, 3))
        self._lib.orc_afmm_widths(self._h, _d(out))
        return out

    def pairs(self, kind: str) -> np.ndarray:
        k = {"near": 0, "far": 1}[kind]
        cnt = self._lib.orc_afmm_pairs(self._h, k, None)
        out = np.zeros((max(cnt, 1), 2), dtype=np.int64)
        self._lib.orc_afmm_pairs(self._h, k, out.ctypes.data_as(_lp))
        return out[:cnt]


def afmm_field(pos, mom, p, theta, s, box=None):
    """Run the adaptive-tree oracle; returns (H in input order, E, OracleAFMM)."""
    f = OracleAFMM(pos, mom, p, theta, s, box)
    f.run()
    return f.field(), f.energy(), f
