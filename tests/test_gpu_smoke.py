"""The package smoke check (__graft_entry__.smoke) and the failure path of
the tensor-core M2L's bounded waits."""
import numpy as np
import pytest

import __graft_entry__ as G
from paper_0810_0233_gb300 import ccfmm as C
from paper_0810_0233_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_smoke():
    G.smoke()


def test_timed_out_wait_is_reported_and_the_handle_recovers(monkeypatch):
    """With CCFMM_TC_STALL=1 the MMA thread issues nothing, so the producers'
    waits for a free stage run out (after 2^12 polls): the kernel raises its
    time-out flag, drains its copies, frees tensor memory and returns, and
    the evaluation reports CCFMM_ERR_TIMEOUT.  The next evaluation is exact."""
    pos, mom = W.ferrofluid(20000, side=100.0 * 0.02 ** (1 / 3), seed=W.BASE_SEED + 50)
    monkeypatch.delenv("CCFMM_M2L", raising=False)
    with C.FMM(pos, mom, 6, 0.5) as f:
        H0 = f.field()
        monkeypatch.setenv("CCFMM_TC_STALL", "1")
        with pytest.raises(C.CCFMMError) as e:
            f.field()
        assert e.value.status == C.ERR_TIMEOUT, e.value
        monkeypatch.delenv("CCFMM_TC_STALL")
        H1 = f.field()
    assert np.array_equal(H0, H1)
