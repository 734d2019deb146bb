"""GB300-native Fourier-seeded Gaussian-splatting mapping path (FGS-SLAM, arXiv 2503.01109).

The compute lives in ``libfgs.so`` (hand-written CUDA for sm_103a behind the C ABI
declared in ``include/fgs.h``).  :mod:`paper_2503_01109_gb300.fgs` is the thin
ctypes binding with the same entry-point names; the other modules build the
mapping step, the batched keyframe window, the autotuner and the learned prior on
top of it.  Importing this package does not load the library; the first call into
:mod:`.fgs` does, and raises if it is missing.
"""
__all__ = ["fgs", "synthetic"]
