"""Block COCG / block COCR with residual orthonormalization on GB300 (sm_103a).

The solver lives in the C-ABI shared library ``libblcoc.so`` (CUDA kernels + host
solve loop); :mod:`paper_1601_05362_gb300.blcoc` is a thin ctypes binding with the same
names.  :mod:`paper_1601_05362_gb300.problems` builds the seeded synthetic inputs.
Importing this package does not load the library; ``blcoc`` loads it on first use and
raises if it has not been built.
"""
__all__ = ["blcoc", "problems"]
