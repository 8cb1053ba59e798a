"""The brute-force Jacobi checker against LAPACK and known spectra."""
import numpy as np
import pytest

import oracle
from workloads.synthetic import haar_unitary, hermitian_from_spectrum


@pytest.mark.parametrize("n", [1, 2, 5, 16, 33])
def test_jacobi_vs_lapack(n):
    rng = np.random.Generator(np.random.PCG64(n))
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    A = A + A.conj().T
    w, V = oracle.jacobi_eigh(A)
    assert np.allclose(w, np.linalg.eigvalsh(A), atol=1e-12 * np.abs(w).max())
    assert np.abs(V.conj().T @ V - np.eye(n)).max() < 1e-12
    assert np.abs(A @ V - V * w).max() < 1e-11 * np.abs(w).max()


def test_jacobi_known_degenerate_spectrum():
    rng = np.random.Generator(np.random.PCG64(3))
    lam = np.array([-1.0, -1.0, 0.5, 2.0, 2.0, 2.0, 7.0])
    q = haar_unitary(7, rng)
    w, _ = oracle.jacobi_eigh(hermitian_from_spectrum(lam, q))
    assert np.allclose(w, lam, atol=1e-13)
