"""Cyclic Jacobi eigensolver for small complex Hermitian matrices.

TEST INFRASTRUCTURE: a brute-force check of the Rayleigh-Ritz step's
reduced eigenproblem (Alg. 1) and of the whole-solve results on
tiny matrices, independent of LAPACK.  Each rotation first removes the
phase of a_pq and then applies the symmetric two-sided Jacobi rotation
(Golub and Van Loan, Matrix Computations, Sec. 8.5).  Pure numpy, meant
for n <= 64.
"""
from __future__ import annotations

import math

import numpy as np


def jacobi_eigh(A, tol: float = 1e-15, max_sweeps: int = 60):
    """Return (ascending eigenvalues, eigenvectors as columns)."""
    A = np.array(A, dtype=np.complex128)
    n = A.shape[0]
    V = np.eye(n, dtype=np.complex128)
    scale = max(np.linalg.norm(A), 1e-300)
    for _ in range(max_sweeps):
        off = math.sqrt(max(np.linalg.norm(A) ** 2
                            - np.sum(np.abs(np.diag(A)) ** 2), 0.0))
        if off <= tol * scale:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                b = abs(apq)
                if b <= 1e-300:
                    continue
                ph = apq / b  # a_pq = b e^{i phi}
                app, aqq = A[p, p].real, A[q, q].real
                tau = (aqq - app) / (2.0 * b)
                t = (1.0 if tau >= 0 else -1.0) / (abs(tau) + math.sqrt(1.0 + tau * tau))
                cs = 1.0 / math.sqrt(1.0 + t * t)
                sn = t * cs
                # unitary on columns (p, q):  V2 = diag(1, conj(ph)) @ [[c, s], [-s, c]]
                # i.e. new_p = c*col_p - s*conj(ph)*col_q ; new_q = s*col_p + c*conj(ph)*col_q
                cp = A[:, p].copy()
                cq = A[:, q].copy()
                A[:, p] = cs * cp - sn * np.conj(ph) * cq
                A[:, q] = sn * cp + cs * np.conj(ph) * cq
                rp = A[p, :].copy()
                rq = A[q, :].copy()
                A[p, :] = cs * rp - sn * ph * rq
                A[q, :] = sn * rp + cs * ph * rq
                A[p, q] = 0.0
                A[q, p] = 0.0
                vp = V[:, p].copy()
                vq = V[:, q].copy()
                V[:, p] = cs * vp - sn * np.conj(ph) * vq
                V[:, q] = sn * vp + cs * np.conj(ph) * vq
    w = np.real(np.diag(A))
    o = np.argsort(w, kind="stable")
    return w[o], V[:, o]
