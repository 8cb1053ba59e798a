"""GB300-native ChFSI: Chebyshev Filtered Subspace Iteration for sequences
of correlated dense Hermitian eigenproblems (after arXiv 1404.4161).

The compute path is libchfsi.so (CUDA, sm_103a) behind the C ABI of
include/chfsi.h; ``solver`` wraps it for torch tensors.
"""
from .build import build, LIB  # noqa: F401
