"""GB300 (sm_103a) implementation of the Adaptive Row-grouped CSR format.

CSR -> ARG-CSR conversion and SpMV y = A x (Heller & Oberhuber, Sections 3
and 4) as hand-written CUDA kernels behind the C ABI of include/argcsr.h;
this package is the thin Python binding over that ABI.
"""
from .argcsr import *  # noqa: F401,F403
from .argcsr import ArgCsrMatrix, ArgCsrServer, ArgcsrError, baseline_csr_spmv, load_library  # noqa: F401
