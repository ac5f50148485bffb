"""GB300-native batched evaluation of the two-machine flow-shop lower bound.

The compute path is the C-ABI library ``libfsp_gb300.so`` (hand-written
sm_103a CUDA, declared in ``include/fsp.h``); ``paper_1208_3933_gb300.fsp``
is its thin ctypes binding.  Importing this package loads nothing: the
library is opened on first use and a missing library is an error, never a
fallback.
"""

__all__ = ["fsp", "workloads"]
