"""GB300-native Hough-Transform track finder (arXiv 1507.03074).

The compute path is the CUDA library ``libht_gb300.so`` built from ``csrc/``
(hand-written sm_103a kernels behind a C ABI, declared in ``include/ht.h``).
``paper_1507_03074_gb300.ht`` is the thin ctypes binding with the same names.
Importing this package does not load the library; ``ht`` loads it on first
use and raises if it is missing.
"""
__all__ = ["synth"]
