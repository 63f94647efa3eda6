"""B300-native (sm_103a) evaluation of the multi-period AC OPF callbacks and the
condensed KKT assembly inside each interior-point iteration (arXiv 2405.14032).

The compute path is the C-ABI library ``libmpopf.so`` (hand-written CUDA for
sm_103a) declared in ``include/mpopf.h``; :mod:`paper_2405_14032_b300.mpopf`
is its thin ctypes binding.  Importing this package loads nothing; the binding
loads the library on first use and raises if it is missing.
"""
__all__ = ["synth", "mpopf"]
