"""FP64 CPU oracle of the FGS-SLAM mapping path (arXiv 2503.01109).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with the
CUDA library in ``paper_2503_01109_gb300`` and never imports it.

* :mod:`oracle.render` -- projection, binning, eq1 blending, its adjoint, eq15,
  eq16 and Adam, in plain C (``render_oracle.c``) driven through ctypes.
* :mod:`oracle.seed` -- the Fourier seeding of Sec. III-A (eq2-eq11) in numpy.
* :mod:`oracle.prior` -- the learned seeding prior's MLP with BF16 emulation.

Parity notes on every function live in the function's docstring.
"""
