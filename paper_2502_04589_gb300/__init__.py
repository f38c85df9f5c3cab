"""GB300 (sm_103a) implementation of the augmented subspace eigensolver of
Liao, Liu, Xie and Wang, "PASE: A Massively Parallel Augmented Subspace Eigensolver"
(arXiv 2502.04589).

The compute path is the C ABI in include/pase.h, implemented by libpase.so (hand-written
CUDA kernels).  `paper_2502_04589_gb300.pase` is a thin ctypes binding with the same
function names; it only marshals arguments and raises PaseError on a non-zero status.
Importing the package does not load the library; the first call does, and fails loudly
if libpase.so has not been built (there is no CPU fallback).
"""
from .pase import *  # noqa: F401,F403
