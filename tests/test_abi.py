"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a GPU
and exports every entry point that include/ccfmm.h declares."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w \*]*?\b([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M):
            if m.group(0).lstrip().startswith(("typedef", "#")):
                continue
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    path = os.path.join(ROOT, "paper_0810_0233_gb300", "libccfmm.so")
    if not os.path.exists(path):
        if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("nvcc not available to build libccfmm.so")
        from paper_0810_0233_gb300 import build
        build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for must in ("fmm_create", "fmm_create_ex", "fmm_field", "fmm_energy", "fmm_destroy",
                 "fmm_set_moments", "fmm_set_positions", "fmm_stats", "ccfmm_last_error",
                 "ccfmm_direct_field"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points(lib):
    lib.ccfmm_leaf_size_rule.restype = ctypes.c_double
    lib.ccfmm_leaf_size_rule.argtypes = [ctypes.c_int]
    assert lib.ccfmm_leaf_size_rule(3) == 8.0
    assert abs(lib.ccfmm_leaf_size_rule(6) - 26.64) < 1e-12
    out = (ctypes.c_int32 * (3 * 84))()
    assert lib.ccfmm_multi_indices(6, out) == 0
    mi = [tuple(out[3 * t:3 * t + 3]) for t in range(84)]
    assert len(set(mi)) == 84 and mi[0] == (0, 0, 0)
    assert all(sum(a) <= sum(b) for a, b in zip(mi, mi[1:]))


def test_create_rejects_bad_arguments_without_gpu(lib):
    """Argument validation happens before any CUDA call."""
    lib.fmm_create.restype = ctypes.c_int
    lib.fmm_create.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                               ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_void_p)]
    lib.ccfmm_last_error.restype = ctypes.c_char_p
    buf = (ctypes.c_double * 6)(0, 0, 0, 1, 1, 1)
    h = ctypes.c_void_p()
    assert lib.fmm_create(buf, buf, 0, 4, 0.5, 8.0, ctypes.byref(h)) == -1
    assert lib.fmm_create(buf, buf, 2, 9, 0.5, 8.0, ctypes.byref(h)) == -1
    assert lib.fmm_create(buf, buf, 2, 4, 1.0, 8.0, ctypes.byref(h)) == -1
    assert lib.fmm_create(buf, buf, 2, 4, 0.5, 0.5, ctypes.byref(h)) == -1
    assert lib.fmm_create(None, buf, 2, 4, 0.5, 8.0, ctypes.byref(h)) == -1
    assert lib.ccfmm_last_error()
