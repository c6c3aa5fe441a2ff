"""B300-native primal-dual iLQR hot path: LQ KKT solve by a parallel
associative scan over the horizon, SRBD linearisation, FP64 residual and
refinement, in-kernel line search, batched SQP and a serving loop.

The compute path lives in ``libpdilqr.so`` (CUDA for sm_103a) behind the
C ABI declared in ``include/pdilqr.h``; ``paper_2506_07823_b300.pdilqr`` is
the thin ctypes binding.  Importing this package loads nothing.
"""
