"""GB300-native Cartesian-coordinates FMM for point dipoles.

The compute path is the C-ABI library ``libccfmm.so`` (hand-written sm_103a
kernels, declared in ``include/ccfmm.h``); ``paper_0810_0233_gb300.ccfmm`` is
its thin Python binding.  The binding loads the library on first use and
raises if it is missing: there is no CPU fallback.
"""

__all__ = ["ccfmm", "workloads"]
