"""Column-row partitioned sparse products on GB300 (sm_103a).

The product C = A B = sum_k a_k b_k is computed by hand-written CUDA kernels
(libcrp.so, C ABI in include/crp.h); every output entry (i, j) is owned by
the hash partition (h_a(i) + h_b(j)) mod P.  This package holds the build
script and the ctypes binding (``paper_1210_0461_gb300.crp``); there is no CPU
implementation of the path.
"""
from ._build import build  # noqa: F401
