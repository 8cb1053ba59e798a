"""Seeded synthetic inputs for the ChFSI hot path.

This module only *produces inputs*: Hermitian matrices with a chosen
spectrum, correlated sequences of them, and random starting blocks.  It
holds none of the eigensolver's arithmetic, so both the CPU oracle and
the CUDA path may use it without sharing any of the method.

The paper's own matrices (FLEUR/FLAPW Hamiltonians of Table 1, the
CaFe2As2 sequence of Fig. 1) are not available; these generators stand
in for them with the same kind of structure: a dense complex Hermitian
H whose low end holds a cluster of wanted eigenvalues, and a sequence
H_1, H_2, ... whose eigenvectors drift slowly from one problem to the
next (Sec. 2.2, Definitions 1 and 2).
"""
from .synthetic import (  # noqa: F401
    BASE_SEED,
    WORKLOADS,
    haar_unitary,
    two_band_spectrum,
    hermitian_from_spectrum,
    random_hermitian,
    unitary_exp,
    correlated_step,
    random_block,
    config_problem,
    config_sequence,
)
