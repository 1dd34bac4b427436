"""GB300-native two-level ORAS-FGMRES Helmholtz solver (arXiv 2004.06309).

The solver lives in the CUDA/C++ shared library ``libhz.so`` (C ABI declared
in ``include/hz.h``); :mod:`paper_2004_06309_gb300.hz` is a thin ctypes
binding over it and :mod:`paper_2004_06309_gb300.build` compiles it for
sm_103a.
"""
