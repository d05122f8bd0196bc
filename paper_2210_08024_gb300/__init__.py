"""GB300 (sm_103a) thermochemistry source step of arXiv:2210.08024.

The computation lives in libtc_gb300.so (hand-written CUDA behind the C ABI of
include/tc.h); this package is the build step (_build) and a thin ctypes binding
(tc).  Importing `paper_2210_08024_gb300.tc` fails if the library is not built.
"""
from ._build import build  # noqa: F401

__all__ = ["build"]
