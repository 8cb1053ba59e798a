"""FP64 CPU oracle for the ChFSI hot path -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, deliberately simple restatement of the
method of Berljafa, Wortmann and Di Napoli, "An Optimized and Scalable
Eigensolver for Sequences of Eigenvalue Problems" (arXiv 1404.4161):
Algorithm 1 (ChFSI) and Algorithm 2 (the Chebyshev filter), with
Householder QR and LAPACK's Hermitian eigensolver as library steps.

Only the test-suite, the smoke check and the benchmark's CPU-baseline
leg may import it.  The CUDA product path never imports, links or calls
anything here; the two share no code (only the seeded input generators
in ``workloads`` serve both).

Functions whose result the tests cannot pin against anything but the
method itself are marked "parity unpinned" in their docstrings.
"""
from .chfsi import (  # noqa: F401
    chebyshev_value,
    chebyshev_sigmas,
    convergence_ratio,
    splitmix64,
    lanczos_start,
    lanczos_bounds,
    chebyshev_filter,
    orthonormalize,
    rayleigh_ritz,
    residuals,
    degree_rule,
    lock_mask,
    cold_interval,
    chfsi,
    chfsi_sequence,
    chfsi_generalized,
)
from .jacobi import jacobi_eigh  # noqa: F401
from . import mlp  # noqa: F401
