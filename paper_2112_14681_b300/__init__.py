"""nsamg: the solve phase of GMRES + C-AMG with Neumann-series projection and smoothers
(arXiv:2112.14681) on one NVIDIA B300.

`nsamg` is a thin ctypes binding over the C ABI declared in include/nsamg.h; every step of the
solve runs in the library's CUDA kernels. Importing this package does not load the library;
the first call does, and fails loudly if it has not been built.
"""
from . import nsamg  # noqa: F401
