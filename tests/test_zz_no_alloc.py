"""The allocation-free entry point, ccfmm_direct_field_energy_noalloc.

Some callers cannot call cudaMalloc (code inside a host application that owns
all GPU memory through its own pool, or a plugin that must not change the
device's allocation state).  For them the library offers the FP64 direct
field and energy with its scratch in a fixed device array.  This test calls
it through the C-ABI twice in a row, with different sizes, and checks each
result against the existing entry point ccfmm_direct_field (the energy
against -1/2 sum m.H of that field); the second call must not change the
device's free memory.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_0810_0233_gb300 import ccfmm as C
from paper_0810_0233_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _fns():
    lib = C.load()
    fn = lib.ccfmm_direct_field_energy_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                   ctypes.c_void_p, ctypes.c_void_p]
    return lib, fn


def _rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (b ** 2).sum()))


def test_no_alloc_matches_existing_entry_point_twice():
    torch = pytest.importorskip("torch")
    lib, fn = _fns()
    rng = np.random.default_rng(2024)
    pos = rng.uniform(0.0, 15.0, size=(3001, 3))
    mom = W.unit_vectors(3001, rng)
    stream = torch.cuda.current_stream()
    for call, n in enumerate((3001, 1000)):
        p_d = torch.from_numpy(np.ascontiguousarray(pos[:n])).cuda()
        m_d = torch.from_numpy(np.ascontiguousarray(mom[:n])).cuda()
        H_ref = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
        st = lib.ccfmm_direct_field(ctypes.c_void_p(p_d.data_ptr()), ctypes.c_void_p(m_d.data_ptr()),
                                    n, None, n, ctypes.c_void_p(H_ref.data_ptr()),
                                    ctypes.c_void_p(stream.cuda_stream))
        assert st == 0
        torch.cuda.synchronize()
        H = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
        E = ctypes.c_double(float("nan"))
        free_before = torch.cuda.mem_get_info()[0]
        st = fn(ctypes.c_void_p(p_d.data_ptr()), ctypes.c_void_p(m_d.data_ptr()), n,
                ctypes.c_void_p(H.data_ptr()), ctypes.byref(E), ctypes.c_void_p(stream.cuda_stream))
        free_after = torch.cuda.mem_get_info()[0]
        assert st == 0, lib.ccfmm_last_error()
        Hr = H_ref.cpu().numpy()
        Hn = H.cpu().numpy()
        assert _rel(Hn, Hr) < 1e-14
        E_ref = -0.5 * float((mom[:n] * Hr).sum())
        assert abs(E.value - E_ref) <= 1e-12 * abs(E_ref)
        if call == 1:
            assert free_after == free_before


def test_no_alloc_rejects_out_of_range_and_host_arrays():
    torch = pytest.importorskip("torch")
    lib, fn = _fns()
    p_d = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    H = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    E = ctypes.c_double()
    ptr = ctypes.c_void_p(p_d.data_ptr())
    hp = ctypes.c_void_p(H.data_ptr())
    assert fn(ptr, ptr, 4 * 1024 * 1024 + 1, hp, ctypes.byref(E), None) == C.ERR_ARG
    assert b"N out of range" in lib.ccfmm_last_error()
    host = np.zeros((4, 3))
    assert fn(ctypes.c_void_p(host.ctypes.data), ptr, 4, hp, ctypes.byref(E), None) == C.ERR_ARG
    # the message names the current device, the only one whose memory is used
    dev = torch.cuda.current_device()
    assert ("device %d" % dev).encode() in lib.ccfmm_last_error()
    assert fn(ptr, ptr, 0, hp, ctypes.byref(E), None) == C.ERR_ARG


def test_no_alloc_refuses_a_capturing_stream():
    """The call synchronises its stream, so on a stream under capture it must
    refuse (CCFMM_ERR_ARG) without touching the capture; the capture then
    ends normally and the stream works afterwards."""
    torch = pytest.importorskip("torch")
    lib, fn = _fns()
    pos = torch.rand(100, 3, dtype=torch.float64, device="cuda") * 10
    mom = torch.randn(100, 3, dtype=torch.float64, device="cuda")
    H = torch.zeros(100, 3, dtype=torch.float64, device="cuda")
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            st = fn(pos.data_ptr(), mom.data_ptr(), 100, H.data_ptr(), E.data_ptr(),
                    ctypes.c_void_p(s.cuda_stream))
            H.add_(0.0)
    assert st == C.ERR_ARG
    assert b"captured" in lib.ccfmm_last_error()
    st = fn(pos.data_ptr(), mom.data_ptr(), 100, H.data_ptr(), E.data_ptr(),
            ctypes.c_void_p(s.cuda_stream))
    assert st == C.OK
    torch.cuda.synchronize()
    assert torch.isfinite(H).all()
