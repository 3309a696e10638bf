"""Thin Python binding of libccfmm (include/ccfmm.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Arrays may be NumPy arrays (host) or torch tensors (host or
CUDA, float64, contiguous); outputs are written to the array the caller
passes or to a new NumPy array.  The library is loaded on first use and a
missing ``libccfmm.so`` raises ``RuntimeError``: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libccfmm.so")
_lock = threading.Lock()
_lib = None

OK, ERR_ARG, ERR_ALLOC, ERR_CUDA, ERR_TIMEOUT, ERR_STATE = 0, -1, -2, -3, -4, -5
FP64, MIXED = 0, 1

_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_int = ctypes.c_int


class Stats(ctypes.Structure):
    _fields_ = [
        ("depth", ctypes.c_int32), ("depth_capped", ctypes.c_int32), ("p", ctypes.c_int32),
        ("precision", ctypes.c_int32), ("theta", _dbl), ("leaf_target", _dbl),
        ("box", _dbl * 6), ("leaf_width", _dbl * 3), ("n", _i64), ("nonempty_leaves", _i64),
        ("near_leaf_pairs", _i64), ("far_pairs", _i64), ("p2p_pairs", _i64),
        ("m2l_tile_entries", _i64), ("far_offsets", _i64), ("ms_build", _dbl),
        ("ms_eval", _dbl), ("ms_stage", _dbl * 8), ("ms_build_stage", _dbl * 6),
    ]

    def as_dict(self):
        d = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            d[name] = list(v) if hasattr(v, "__len__") else v
        return d


class AdaptiveStats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nsamples", ctypes.c_int32), ("p", ctypes.c_int32),
                ("theta", ctypes.c_double), ("ncells", ctypes.c_int64),
                ("nleaves", ctypes.c_int64), ("max_level", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("far_pairs", ctypes.c_int64),
                ("near_entries", ctypes.c_int64), ("near_pairs", ctypes.c_int64),
                ("d_rows", ctypes.c_int64), ("m2l_items", ctypes.c_int64),
                ("kernels_per_eval", ctypes.c_int64), ("ms_build", ctypes.c_double)]


class CCFMMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("libccfmm status %d: %s" % (status, msg))
        self.status = status


def load():
    """Load libccfmm.so; raises RuntimeError when it is missing."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libccfmm.so not found at %s: run __graft_entry__.build() "
                               "(nvcc, sm_103a) first; there is no CPU fallback" % LIB_PATH)
        lib = ctypes.CDLL(LIB_PATH)
        sig = {
            "fmm_create": (_int, [_vp, _vp, _i64, _int, _dbl, _dbl, ctypes.POINTER(_vp)]),
            "fmm_create_ex": (_int, [_vp, _vp, _i64, _int, _dbl, _dbl, _vp, _int, _vp,
                                     ctypes.POINTER(_vp)]),
            "fmm_set_positions": (_int, [_vp, _vp, _vp]),
            "fmm_set_moments": (_int, [_vp, _vp]),
            "fmm_set_truncation": (_int, [_vp, _int]),
            "fmm_get_truncation": (_int, [_vp, ctypes.POINTER(_int)]),
            "fmm_field": (_int, [_vp, _vp]),
            "fmm_field_energy": (_int, [_vp, _vp, ctypes.POINTER(_dbl)]),
            "fmm_energy": (_int, [_vp, ctypes.POINTER(_dbl)]),
            "fmm_stats": (_int, [_vp, ctypes.POINTER(Stats)]),
            "fmm_destroy": (None, [_vp]),
            "fmm_reset_stats": (_int, [_vp]),
            "ccfmm_last_error": (ctypes.c_char_p, []),
            "fmm_get_axes": (_int, [_vp, _vp]),
            "fmm_get_leaf_of": (_int, [_vp, _vp]),
            "fmm_get_pairs": (_int, [_vp, _int, _vp, _i64, ctypes.POINTER(_i64)]),
            "ccfmm_multi_indices": (_int, [_int, _vp]),
            "fmm_get_expansions": (_int, [_vp, _int, _vp]),
            "ccfmm_direct_field": (_int, [_vp, _vp, _i64, _vp, _i64, _vp, _vp]),
            "ccfmm_leaf_size_rule": (_dbl, [_int]),
            "ccfmm_kernel_launches": (_i64, []),
            "fmm_batch_create": (_int, [_vp, _vp, _vp, _int, _int, _dbl, _dbl, _int, _vp,
                                        ctypes.POINTER(_vp)]),
            "fmm_batch_create_ex": (_int, [_vp, _vp, _vp, _int, _int, _dbl, _dbl, _int, _vp,
                                           _vp, ctypes.POINTER(_vp)]),
            "fmm_batch_tuning": (_int, [_vp, ctypes.POINTER(ctypes.c_int32), _vp, _vp, _vp,
                                        ctypes.c_int32]),
            "fmm_batch_step": (_int, [_vp, ctypes.c_uint64, ctypes.c_uint64, _dbl, _vp, _vp]),
            "fmm_batch_evaluate": (_int, [_vp, _vp, _vp]),
            "fmm_batch_get_moments": (_int, [_vp, _vp]),
            "fmm_batch_set_moments": (_int, [_vp, _vp]),
            "fmm_batch_info": (_int, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
            "fmm_batch_destroy": (None, [_vp]),
            "fmm_batch_sample": (_int, [_vp, _int, ctypes.POINTER(_vp)]),
            "fmm_get_m2l_data": (_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
            "ccfmm_mlp_create": (_int, [ctypes.POINTER(_vp)]),
            "ccfmm_mlp_destroy": (None, [_vp]),
            "ccfmm_mlp_num_params": (ctypes.c_int32, []),
            "ccfmm_mlp_set_params": (_int, [_vp, _vp, _vp]),
            "ccfmm_mlp_get_params": (_int, [_vp, _vp, _vp]),
            "ccfmm_mlp_fit_norm": (_int, [_vp, _vp, _vp, _vp, _i64]),
            "ccfmm_mlp_gradient": (_int, [_vp, _vp, _vp, _vp, _i64, _vp, _vp]),
            "ccfmm_mlp_train": (_int, [_vp, _vp, _vp, _vp, _i64, _i64, ctypes.c_int32,
                                       ctypes.c_float, ctypes.c_uint64, _vp]),
            "ccfmm_mlp_predict": (_int, [_vp, _vp, _i64, _vp]),
            "ccfmm_features": (_int, [_vp, _i64, _vp]),
            "fmm_select": (_int, [_vp, _vp, _i64, _dbl, _vp, _vp, _vp, _vp]),
            "fmm_lattice_create": (_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _dbl,
                                          ctypes.c_int32, _vp, ctypes.POINTER(_vp)]),
            "fmm_lattice_field": (_int, [_vp, _vp, _vp, _vp]),
            "fmm_lattice_destroy": (None, [_vp]),
            "fmm_adaptive_create": (_int, [_vp, _vp, _vp, _int, _int, _dbl, _vp, _vp, _int, _vp,
                                           ctypes.POINTER(_vp)]),
            "fmm_adaptive_create_ex": (_int, [_vp, _vp, _vp, _int, _int, _dbl, _vp, _vp, _int,
                                              _vp, _vp, ctypes.POINTER(_vp)]),
            "fmm_adaptive_tuning": (_int, [_vp, ctypes.POINTER(ctypes.c_int32), _vp, _vp,
                                           ctypes.c_int32]),
            "fmm_adaptive_evaluate": (_int, [_vp, _vp, _vp]),
            "fmm_adaptive_step": (_int, [_vp, ctypes.c_uint64, ctypes.c_uint64, _dbl, _vp, _vp]),
            "fmm_adaptive_set_moments": (_int, [_vp, _vp]),
            "fmm_adaptive_get_moments": (_int, [_vp, _vp]),
            "fmm_adaptive_info": (_int, [_vp, ctypes.POINTER(AdaptiveStats)]),
            "fmm_adaptive_cells": (_int, [_vp, _vp]),
            "fmm_adaptive_perm": (_int, [_vp, _vp]),
            "fmm_adaptive_pairs": (_int, [_vp, _int, _vp, _i64, ctypes.POINTER(_i64)]),
            "fmm_adaptive_expansions": (_int, [_vp, _vp, _vp]),
            "fmm_adaptive_destroy": (None, [_vp]),
            "fmm_adaptive_queue": (_int, [_i64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.c_int32, _vp, ctypes.c_int32, ctypes.c_int32,
                                          _vp, _i64, ctypes.POINTER(_i64), _vp, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_int32), _vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(st):
    if st != OK:
        raise CCFMMError(st, load().ccfmm_last_error().decode(errors="replace"))


def _ptr(a, n3=None, dtype=np.float64):
    """(pointer, keepalive) for a NumPy array or torch tensor."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):  # torch tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        want = {np.float64: "torch.float64", np.int64: "torch.int64"}[dtype]
        if str(a.dtype) != want:
            raise ValueError("tensor must be %s" % want)
        if n3 is not None and a.numel() != n3:
            raise ValueError("expected %d elements, got %d" % (n3, a.numel()))
        return _vp(a.data_ptr()), a
    arr = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    if n3 is not None and arr.size != n3:
        raise ValueError("expected %d elements, got %d" % (n3, arr.size))
    return _vp(arr.ctypes.data), arr


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return _vp(stream)
    return _vp(stream.cuda_stream)


def kernel_launches() -> int:
    """Kernels the library has launched in this process."""
    return int(load().ccfmm_kernel_launches())


def leaf_size_rule(p: int) -> float:
    """Eq. so (the library's copy)."""
    return load().ccfmm_leaf_size_rule(int(p))


def multi_indices(order: int) -> np.ndarray:
    out = np.zeros(((order + 1) * (order + 2) * (order + 3) // 6, 3), dtype=np.int32)
    _check(load().ccfmm_multi_indices(int(order), _vp(out.ctypes.data)))
    return out


def direct_field(positions, moments, targets=None, out=None, stream=None):
    """FP64 GPU direct sum at ``targets`` (all dipoles when None)."""
    lib = load()
    n = len(positions) if not hasattr(positions, "shape") else positions.shape[0]
    pp, k1 = _ptr(positions, 3 * n)
    pm, k2 = _ptr(moments, 3 * n)
    if targets is None:
        pt, k3, nt = None, None, n
    else:
        pt, k3 = _ptr(targets, dtype=np.int64)
        nt = k3.numel() if hasattr(k3, "numel") else k3.size
    if out is None:
        out = np.zeros((nt, 3))
    po, k4 = _ptr(out, 3 * nt)
    _check(lib.ccfmm_direct_field(pp, pm, n, pt, nt, po, _stream_ptr(stream)))
    return out


class FMM:
    """One dipole system on the GPU (fmm_create_ex ... fmm_destroy)."""

    def __init__(self, positions, moments, p, theta, leaf_size=0.0, box=None,
                 precision="mixed", stream=None):
        lib = load()
        self._lib = lib
        n = positions.shape[0]
        self.n = int(n)
        self.p = int(p)
        pp, k1 = _ptr(positions, 3 * n)
        pm, k2 = _ptr(moments, 3 * n)
        bx, kb = (None, None) if box is None else _ptr(np.asarray(box, np.float64).reshape(6))
        prec = {"mixed": MIXED, "fp32": MIXED, "fp64": FP64}[precision]
        self._stream = stream
        h = _vp()
        _check(lib.fmm_create_ex(pp, pm, n, self.p, float(theta), float(leaf_size), bx, prec,
                                 _stream_ptr(stream), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and not getattr(self, "_borrowed", False):
            self._lib.fmm_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_positions(self, positions, moments):
        pp, k1 = _ptr(positions, 3 * self.n)
        pm, k2 = _ptr(moments, 3 * self.n)
        _check(self._lib.fmm_set_positions(self._h, pp, pm))

    def set_moments(self, moments):
        pm, k = _ptr(moments, 3 * self.n)
        _check(self._lib.fmm_set_moments(self._h, pm))

    def set_truncation(self, max_degree=None):
        """fmm_set_truncation: None for the square truncation of Eq.
        taylorcalc, else keep the terms with |n|+|k| <= max_degree."""
        _check(self._lib.fmm_set_truncation(self._h, 0 if max_degree is None else int(max_degree)))

    @property
    def max_degree(self) -> int:
        v = _int()
        _check(self._lib.fmm_get_truncation(self._h, ctypes.byref(v)))
        return int(v.value)

    def field(self, out=None):
        """H at every dipole, input order (N x 3 float64)."""
        if out is None:
            out = np.zeros((self.n, 3))
        po, k = _ptr(out, 3 * self.n)
        _check(self._lib.fmm_field(self._h, po))
        return out

    def evaluate(self):
        """Run the evaluation and keep the result on the device."""
        _check(self._lib.fmm_field(self._h, None))

    def field_energy(self, out=None):
        if out is None:
            out = np.zeros((self.n, 3))
        po, k = _ptr(out, 3 * self.n)
        e = _dbl()
        _check(self._lib.fmm_field_energy(self._h, po, ctypes.byref(e)))
        return out, e.value

    def energy(self):
        e = _dbl()
        _check(self._lib.fmm_energy(self._h, ctypes.byref(e)))
        return e.value

    def stats(self) -> dict:
        s = Stats()
        _check(self._lib.fmm_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def reset_stats(self):
        _check(self._lib.fmm_reset_stats(self._h))

    def axes(self) -> np.ndarray:
        d = self.stats()["depth"]
        out = np.zeros(max(d, 1), dtype=np.int32)
        _check(self._lib.fmm_get_axes(self._h, _vp(out.ctypes.data)))
        return out[:d]

    def leaf_of(self) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.int64)
        _check(self._lib.fmm_get_leaf_of(self._h, _vp(out.ctypes.data)))
        return out

    def pairs(self, kind: str) -> np.ndarray:
        k = {"near": 0, "far": 1}[kind]
        cnt = _i64()
        _check(self._lib.fmm_get_pairs(self._h, k, None, 0, ctypes.byref(cnt)))
        out = np.zeros((max(cnt.value, 1), 2), dtype=np.int64)
        _check(self._lib.fmm_get_pairs(self._h, k, _vp(out.ctypes.data), cnt.value,
                                       ctypes.byref(cnt)))
        return out[: cnt.value]

    def m2l_data(self):
        """(D tables, entry offset ids, entry partners, tile descriptors)."""
        sz = np.zeros(4, dtype=np.int64)
        _check(self._lib.fmm_get_m2l_data(self._h, _vp(sz.ctypes.data), None, None, None, None))
        noff, td, ne, nt = (int(x) for x in sz)
        D = np.zeros((max(noff, 1), td))
        u = np.zeros(max(ne, 1), dtype=np.int32)
        s = np.zeros((max(ne, 1), 128), dtype=np.int32)
        t = np.zeros((max(nt, 1), 8), dtype=np.int32)
        _check(self._lib.fmm_get_m2l_data(self._h, _vp(sz.ctypes.data), _vp(D.ctypes.data),
                                          _vp(u.ctypes.data), _vp(s.ctypes.data), _vp(t.ctypes.data)))
        return D[:noff], u[:ne], s[:ne], t[:nt]

    def expansions(self, kind: str) -> np.ndarray:
        """Q ("Q") or V ("V") of every cell, (2^(L+1)) x T(p), library order."""
        k = {"Q": 0, "V": 1}[kind]
        d = self.stats()["depth"]
        T = (self.p + 1) * (self.p + 2) * (self.p + 3) // 6
        out = np.zeros((1 << (d + 1), T))
        _check(self._lib.fmm_get_expansions(self._h, k, _vp(out.ctypes.data)))
        return out


class Batch:
    """An ensemble of independent samples stepped together (fmm_batch_*)."""

    def __init__(self, positions, moments, offsets, p, theta, leaf_size=0.0, precision="mixed",
                 stream=None, autotune=False, trials=3):
        lib = load()
        self._lib = lib
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        self.offsets = off
        self.ns = len(off) - 1
        self.total = int(off[-1])
        pp, k1 = _ptr(positions, 3 * self.total)
        pm, k2 = _ptr(moments, 3 * self.total)
        prec = {"mixed": MIXED, "fp32": MIXED, "fp64": FP64}[precision]
        h = _vp()
        self._p = int(p)
        opts = (ctypes.c_int32 * 2)(1 if autotune else 0, int(trials))
        _check(lib.fmm_batch_create_ex(pp, pm, _vp(off.ctypes.data), self.ns, int(p),
                                       float(theta), float(leaf_size), prec,
                                       _vp(ctypes.addressof(opts)), _stream_ptr(stream),
                                       ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fmm_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def step(self, seed, step, max_angle, H_out=None, E_out=None):
        """Rotate every moment (Philox(seed, step)) and evaluate every sample."""
        ph, k1 = _ptr(H_out, 3 * self.total) if H_out is not None else (None, None)
        pe, k2 = _ptr(E_out, self.ns) if E_out is not None else (None, None)
        _check(self._lib.fmm_batch_step(self._h, int(seed), int(step), float(max_angle), ph, pe))

    def evaluate(self, H_out=None, E_out=None):
        ph, k1 = _ptr(H_out, 3 * self.total) if H_out is not None else (None, None)
        pe, k2 = _ptr(E_out, self.ns) if E_out is not None else (None, None)
        _check(self._lib.fmm_batch_evaluate(self._h, ph, pe))

    def moments(self):
        out = np.zeros((self.total, 3))
        _check(self._lib.fmm_batch_get_moments(self._h, _vp(out.ctypes.data)))
        return out

    def set_moments(self, moments):
        pm, k = _ptr(moments, 3 * self.total)
        _check(self._lib.fmm_batch_set_moments(self._h, pm))

    def sample(self, i):
        """Borrowed FMM view of sample i (inspection only; owned by the batch)."""
        h = _vp()
        _check(self._lib.fmm_batch_sample(self._h, int(i), ctypes.byref(h)))
        f = FMM.__new__(FMM)
        f._lib = self._lib
        f._h = h
        f.n = int(self.offsets[i + 1] - self.offsets[i])
        f.p = self._p
        f._borrowed = True
        return f

    def tuning(self):
        """The autotuner's classes: list of (smallest N, leaf occupancy, M2L
        item length); empty without autotune."""
        n = ctypes.c_int32()
        _check(self._lib.fmm_batch_tuning(self._h, ctypes.byref(n), None, None, None, 0))
        k = n.value
        nmin = np.zeros(max(k, 1), np.int64)
        leaf = np.zeros(max(k, 1))
        il = np.zeros(max(k, 1), np.int32)
        _check(self._lib.fmm_batch_tuning(self._h, ctypes.byref(n), _vp(nmin.ctypes.data),
                                          _vp(leaf.ctypes.data), _vp(il.ctypes.data), k))
        return [(int(nmin[i]), float(leaf[i]), int(il[i])) for i in range(k)]

    def kernels_per_step(self):
        n, k = _i64(), _i64()
        _check(self._lib.fmm_batch_info(self._h, ctypes.byref(n), ctypes.byref(k)))
        return int(k.value)


def _f32(a, n=None):
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    if n is not None and arr.size != n:
        raise ValueError("expected %d elements, got %d" % (n, arr.size))
    return arr


def features(positions):
    """The selector's nine features of a dipole set (ccfmm_features)."""
    n = positions.shape[0]
    pp, k = _ptr(positions, 3 * n)
    out = np.zeros(9, dtype=np.float32)
    _check(load().ccfmm_features(pp, n, _vp(out.ctypes.data)))
    return out


class MLP:
    """The selector network (ccfmm_mlp_*): 12-64-64-64-2, BF16 weights."""

    def __init__(self, params=None, norm=None):
        lib = load()
        self._lib = lib
        h = _vp()
        _check(lib.ccfmm_mlp_create(ctypes.byref(h)))
        self._h = h
        self.n_params = int(lib.ccfmm_mlp_num_params())
        if params is not None or norm is not None:
            self.set_params(params, norm)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.ccfmm_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, params=None, norm=None):
        p = None if params is None else _f32(params, self.n_params)
        q = None if norm is None else _f32(norm, 28)
        _check(self._lib.ccfmm_mlp_set_params(
            self._h, None if p is None else _vp(p.ctypes.data), None if q is None else _vp(q.ctypes.data)))

    def get_params(self):
        p = np.zeros(self.n_params, dtype=np.float32)
        q = np.zeros(28, dtype=np.float32)
        _check(self._lib.ccfmm_mlp_get_params(self._h, _vp(p.ctypes.data), _vp(q.ctypes.data)))
        return p, q

    def fit_norm(self, X, T, mask):
        X, T, M = _f32(X), _f32(T), _f32(mask)
        _check(self._lib.ccfmm_mlp_fit_norm(self._h, _vp(X.ctypes.data), _vp(T.ctypes.data),
                                            _vp(M.ctypes.data), len(X)))

    def gradient(self, X, T, mask):
        X, T, M = _f32(X), _f32(T), _f32(mask)
        g = np.zeros(self.n_params, dtype=np.float32)
        loss = ctypes.c_float()
        _check(self._lib.ccfmm_mlp_gradient(self._h, _vp(X.ctypes.data), _vp(T.ctypes.data),
                                            _vp(M.ctypes.data), len(X), _vp(g.ctypes.data),
                                            ctypes.byref(loss)))
        return float(loss.value), g

    def train(self, X, T, mask, batch=256, epochs=1, lr=1e-3, seed=0):
        X, T, M = _f32(X), _f32(T), _f32(mask)
        loss = ctypes.c_float()
        _check(self._lib.ccfmm_mlp_train(self._h, _vp(X.ctypes.data), _vp(T.ctypes.data),
                                         _vp(M.ctypes.data), len(X), int(batch), int(epochs),
                                         float(lr), int(seed), ctypes.byref(loss)))
        return float(loss.value)

    def predict(self, X):
        X = _f32(X)
        Y = np.zeros((len(X), 2), dtype=np.float32)
        _check(self._lib.ccfmm_mlp_predict(self._h, _vp(X.ctypes.data), len(X), _vp(Y.ctypes.data)))
        return Y


def select(mlp, positions, target_error):
    """fmm_select: (p, theta, leaf, used_fallback) for a target RMS error."""
    n = positions.shape[0]
    pp, k = _ptr(positions, 3 * n)
    p = ctypes.c_int32()
    th = _dbl()
    lf = _dbl()
    fb = ctypes.c_int32()
    _check(load().fmm_select(None if mlp is None else mlp._h, pp, n, float(target_error),
                             ctypes.byref(p), ctypes.byref(th), ctypes.byref(lf), ctypes.byref(fb)))
    return int(p.value), float(th.value), float(lf.value), bool(fb.value)


class Lattice:
    """FFT convolution on a simple-cubic lattice (fmm_lattice_*): the
    comparator of the paper's Sec. V.  Sites are ordered as
    ``workloads.lattice`` orders them: (ix ny + iy) nz + iz."""

    def __init__(self, nx, ny=None, nz=None, spacing=1.0, precision="fp64", stream=None):
        ny = nx if ny is None else ny
        nz = nx if nz is None else nz
        self._lib = load()
        self.n = int(nx) * int(ny) * int(nz)
        prec = {"fp64": FP64, "mixed": MIXED, "fp32": MIXED}[precision]
        h = _vp()
        _check(self._lib.fmm_lattice_create(int(nx), int(ny), int(nz), float(spacing), prec,
                                            _stream_ptr(stream), ctypes.byref(h)))
        self._h = h

    def field_energy(self, moments, out=None):
        """(H, E); H is written to ``out`` (host or device) when given."""
        pm, k1 = _ptr(moments, 3 * self.n)
        if out is None:
            out = np.zeros((self.n, 3))
        po, k2 = _ptr(out, 3 * self.n)
        E = _dbl()
        _check(self._lib.fmm_lattice_field(self._h, pm, po, ctypes.byref(E)))
        return out, E.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fmm_lattice_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False

    def __del__(self):
        self.close()


class Adaptive:
    """Adaptive-depth tree (fmm_adaptive_*): one system, or an ensemble of
    independent samples (``offsets``) evaluated together.  persistent=True:
    every evaluation is one launch of the persistent step kernel (task queue
    over the stages of all samples) instead of a graph of stage kernels."""

    def __init__(self, positions, moments, p, theta, split=None, offsets=None, box=None,
                 precision="mixed", stream=None, autotune=False, trials=3, persistent=False):
        lib = load()
        self._lib = lib
        if offsets is None:
            n = int(np.asarray(positions).size // 3) if not hasattr(positions, "numel") \
                else int(positions.numel() // 3)
            offsets = [0, n]
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        self.offsets = off
        self.ns = len(off) - 1
        self.n = int(off[-1])
        pp, k1 = _ptr(positions, 3 * self.n)
        pm, k2 = _ptr(moments, 3 * self.n)
        sp = None
        if split is not None:
            sa = np.ascontiguousarray(np.broadcast_to(np.asarray(split, np.float64), (self.ns,)))
            self._split = sa
            sp = _vp(sa.ctypes.data)
        bp = None
        if box is not None:
            self._box = np.ascontiguousarray(np.asarray(box, np.float64).reshape(6))
            bp = _vp(self._box.ctypes.data)
        prec = {"mixed": MIXED, "fp32": MIXED, "fp64": FP64}[precision]
        self.p = int(p)
        h = _vp()
        opts = (ctypes.c_int32 * 3)(1 if autotune else 0, int(trials), 1 if persistent else 0)
        _check(lib.fmm_adaptive_create_ex(pp, pm, _vp(off.ctypes.data), self.ns, int(p),
                                          float(theta), sp, bp, prec,
                                          _vp(ctypes.addressof(opts)), _stream_ptr(stream),
                                          ctypes.byref(h)))
        self._h = h

    def tuning(self):
        """The autotuner's classes: list of (smallest N, split threshold)."""
        n = ctypes.c_int32()
        _check(self._lib.fmm_adaptive_tuning(self._h, ctypes.byref(n), None, None, 0))
        k = n.value
        nmin = np.zeros(max(k, 1), np.int64)
        spl = np.zeros(max(k, 1))
        _check(self._lib.fmm_adaptive_tuning(self._h, ctypes.byref(n), _vp(nmin.ctypes.data),
                                             _vp(spl.ctypes.data), k))
        return [(int(nmin[i]), float(spl[i])) for i in range(k)]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.fmm_adaptive_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _outs(self, H_out, E_out):
        # neither given: both returned as new host arrays; otherwise only the
        # given ones are written (the other is not copied out)
        if H_out is None and E_out is None:
            H_out = np.zeros((self.n, 3))
            E_out = np.zeros(self.ns)
        ph, k1 = _ptr(H_out, 3 * self.n) if H_out is not None else (None, None)
        pe, k2 = _ptr(E_out, self.ns) if E_out is not None else (None, None)
        return H_out, E_out, ph, pe, (k1, k2)

    def evaluate(self, H_out=None, E_out=None):
        """(H, E): fields in input order and the energy of every sample."""
        H_out, E_out, ph, pe, keep = self._outs(H_out, E_out)
        _check(self._lib.fmm_adaptive_evaluate(self._h, ph, pe))
        return H_out, E_out

    def step(self, seed, step, max_angle, H_out=None, E_out=None):
        """Rotate every moment (Philox(seed, step)) and evaluate."""
        H_out, E_out, ph, pe, keep = self._outs(H_out, E_out)
        _check(self._lib.fmm_adaptive_step(self._h, int(seed), int(step), float(max_angle), ph, pe))
        return H_out, E_out

    def set_moments(self, moments):
        pm, k = _ptr(moments, 3 * self.n)
        _check(self._lib.fmm_adaptive_set_moments(self._h, pm))

    def moments(self):
        out = np.zeros((self.n, 3))
        _check(self._lib.fmm_adaptive_get_moments(self._h, _vp(out.ctypes.data)))
        return out

    def stats(self) -> dict:
        st = AdaptiveStats()
        _check(self._lib.fmm_adaptive_info(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in AdaptiveStats._fields_ if k != "pad"}

    def cells(self) -> np.ndarray:
        """ncells x 8: level, parent, child0, child1, first, count, leaf, sample."""
        out = np.zeros((self.stats()["ncells"], 8), np.int64)
        _check(self._lib.fmm_adaptive_cells(self._h, _vp(out.ctypes.data)))
        return out

    def perm(self) -> np.ndarray:
        out = np.zeros(self.n, np.int64)
        _check(self._lib.fmm_adaptive_perm(self._h, _vp(out.ctypes.data)))
        return out

    def pairs(self, kind: str) -> np.ndarray:
        """(cell, partner) pairs: kind "near" or "far"."""
        k = {"near": 0, "far": 1}[kind]
        cnt = _i64()
        _check(self._lib.fmm_adaptive_pairs(self._h, k, None, 0, ctypes.byref(cnt)))
        out = np.zeros((max(cnt.value, 1), 2), np.int64)
        _check(self._lib.fmm_adaptive_pairs(self._h, k, _vp(out.ctypes.data), cnt.value,
                                            ctypes.byref(cnt)))
        return out[:cnt.value]

    def expansions(self):
        """(Q, V): ncells x (T(p) - 1) each, library multi-index order."""
        nc = self.stats()["ncells"]
        K = (self.p + 1) * (self.p + 2) * (self.p + 3) // 6 - 1
        Q = np.zeros((nc, K))
        V = np.zeros((nc, K))
        _check(self._lib.fmm_adaptive_expansions(self._h, _vp(Q.ctypes.data), _vp(V.ctypes.data)))
        return Q, V


def adaptive_queue(N, nsamples, nleaf, ncells, level_offsets, n_big, n_small):
    """The persistent step's task queue for a forest of this shape
    (fmm_adaptive_queue, host only): (tasks as an ntasks x 4 int32 array,
    tasks per phase, (dipoles per chunk, cells per tile, small-item groups
    per tile))."""
    lib = load()
    off = np.ascontiguousarray(np.asarray(level_offsets, np.int32))
    nt, nph = _i64(), ctypes.c_int32()
    args = (int(N), int(nsamples), int(nleaf), int(ncells), len(off) - 2,
            _vp(off.ctypes.data), int(n_big), int(n_small))
    _check(lib.fmm_adaptive_queue(*args, None, 0, ctypes.byref(nt), None, 0, ctypes.byref(nph),
                                  None))
    tasks = np.zeros((max(nt.value, 1), 4), np.int32)
    need = np.zeros(max(nph.value, 1), np.int32)
    tiles = np.zeros(3, np.int32)
    _check(lib.fmm_adaptive_queue(*args, _vp(tasks.ctypes.data), nt.value, ctypes.byref(nt),
                                  _vp(need.ctypes.data), nph.value, ctypes.byref(nph),
                                  _vp(tiles.ctypes.data)))
    return tasks[:nt.value], need[:nph.value], tuple(int(x) for x in tiles)
