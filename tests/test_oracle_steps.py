"""Pins for the oracle's Lanczos bounds, QR, Rayleigh-Ritz, residuals,
locking and degree rule (Alg. 1; Sec. 3.2)."""
import math
import os

import numpy as np
import pytest

import oracle
from workloads.synthetic import haar_unitary, hermitian_from_spectrum, random_block

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def known(n, seed, lo=(-3.0, -1.0), bulk=(0.0, 20.0), n_low=None):
    rng = np.random.Generator(np.random.PCG64(seed))
    n_low = n_low or max(1, n // 8)
    lam = np.sort(np.concatenate([rng.uniform(*lo, n_low), rng.uniform(*bulk, n - n_low)]))
    q = haar_unitary(n, rng)
    return hermitian_from_spectrum(lam, q), lam, q


# -------------------------- Lanczos (Alg. 1) --------------------------------
@pytest.mark.parametrize("n,seed", [(64, 1), (200, 2), (513, 3)])
def test_lanczos_bounds_enclose_spectrum(n, seed):
    H, lam, _ = known(n, seed)
    b = oracle.lanczos_bounds(H, 20, oracle.lanczos_start(n, 5))
    assert b["beta"] >= lam[-1]
    assert b["theta_min"] >= lam[0] - 1e-12
    assert b["theta_max"] <= lam[-1] + 1e-12
    assert b["beta"] - lam[-1] <= 0.3 * (lam[-1] - lam[0])  # R4 is safe but loose
    assert b["norm_h"] <= np.abs(lam).max() + 1e-12


def test_lanczos_full_krylov_space_is_exact():
    """With steps >= n the Krylov space is the whole space: the Lanczos
    Ritz values are the eigenvalues."""
    H, lam, _ = known(8, 4)
    b = oracle.lanczos_bounds(H, 20, oracle.lanczos_start(8, 1))
    assert abs(b["theta_min"] - lam[0]) < 1e-10
    assert abs(b["theta_max"] - lam[-1]) < 1e-10


# -------------------------- QR (Alg. 1) -------------------------------------
def gram_schmidt(A):
    """Brute-force modified Gram-Schmidt with positive real R diagonal."""
    A = A.copy()
    n, k = A.shape
    Q = np.zeros_like(A)
    for j in range(k):
        v = A[:, j].copy()
        for i in range(j):
            v = v - np.vdot(Q[:, i], v) * Q[:, i]
        for i in range(j):  # second pass
            v = v - np.vdot(Q[:, i], v) * Q[:, i]
        Q[:, j] = v / np.linalg.norm(v)
    return Q


def test_qr_unique_q_matches_gram_schmidt():
    Y = random_block(50, 9, 3)
    Q = oracle.orthonormalize(Y)
    assert np.allclose(Q, gram_schmidt(Y), atol=1e-12)


def test_qr_against_locked():
    L = oracle.orthonormalize(random_block(60, 5, 1))
    Y = random_block(60, 7, 2)
    Q = oracle.orthonormalize(Y, L)
    assert np.abs(Q.conj().T @ Q - np.eye(7)).max() < 1e-13
    assert np.abs(L.conj().T @ Q).max() < 1e-13
    # span([L, Q]) == span([L, Y])
    P1 = np.concatenate([L, Q], 1)
    Y2 = Y - P1 @ (P1.conj().T @ Y)
    assert np.linalg.norm(Y2) < 1e-12 * np.linalg.norm(Y)
    assert np.allclose(Q, gram_schmidt(np.concatenate([L, Y], 1))[:, 5:], atol=1e-12)


# -------------------------- Rayleigh-Ritz (Alg. 1) --------------------------
def test_rr_exact_eigenvectors_give_exact_eigenvalues():
    H, lam, q = known(40, 7)
    lam_r, Y, HY = oracle.rayleigh_ritz(H, q[:, :6])
    assert np.allclose(lam_r, lam[:6], atol=1e-12)
    r = oracle.residuals(HY, Y, lam_r, float(np.abs(lam).max()))
    assert r.max() < 1e-13


def test_rr_bounds_and_jacobi():
    H, lam, _ = known(48, 8)
    Q = oracle.orthonormalize(random_block(48, 10, 4))
    lam_r, Y, HY = oracle.rayleigh_ritz(H, Q)
    assert lam_r.min() >= lam[0] - 1e-12 and lam_r.max() <= lam[-1] + 1e-12
    assert np.all(lam_r >= lam[:10] - 1e-12)  # Courant-Fischer
    G = Q.conj().T @ H @ Q
    w, _ = oracle.jacobi_eigh(0.5 * (G + G.conj().T))
    assert np.allclose(w, lam_r, atol=1e-12)
    assert np.abs(Y.conj().T @ Y - np.eye(10)).max() < 1e-13
    assert np.allclose(HY, H @ Y, atol=1e-12)


def test_residual_hand_value():
    H = np.diag([1.0, 3.0]).astype(np.complex128)
    y = np.array([[1.0], [1.0]], dtype=np.complex128) / math.sqrt(2)
    lam = np.array([2.0])
    r = oracle.residuals(H @ y, y, lam, 3.0)
    # H y - 2 y = (-1, 1)/sqrt(2): norm 1, / ||H|| = 3
    assert abs(r[0] - 1.0 / 3.0) < 1e-15


# -------------------------- locking and degrees -----------------------------
def test_lock_mask_out_of_order():
    r = np.array([1e-11, 1e-3, 5e-11, 1e-12, 1e-12])
    m = oracle.lock_mask(r, 4, 1e-10)
    assert m.tolist() == [True, False, True, True, False]


def test_degree_rule_hand_cases():
    rows = [l.split() for l in open(os.path.join(GOLD, "degree_rule_cases.txt"))
            if l.strip() and not l.startswith("#")]
    for ritz, c, e, r, tol, dmax, want in rows:
        got = oracle.degree_rule(np.array([float(ritz)]), np.array([float(r)]),
                                 float(c), float(e), float(tol), int(dmax))
        assert int(got[0]) == int(want), (ritz, c, e, r, want, got)


def test_degree_rule_buffer_cap():
    lam = np.array([-3.0, -2.5, -1.0, -0.99])
    r = np.array([1e-3, 1e-3, 1e-3, 1e-3])
    m = oracle.degree_rule(lam, r, 1.0, 2.0, 1e-10, 36, n_wanted=2)
    # buffer columns (index >= 2) never exceed the largest wanted degree
    assert m[2:].max() <= m[:2].max()
    assert m[0] <= m[1]


def test_degree_rule_predicts_decay():
    """For an isolated wanted eigenvalue the residual after filtering with
    degree m falls like tau^m (Eq. (ratio), Eq. (resl), converging regime)."""
    n = 64
    rng = np.random.Generator(np.random.PCG64(2))
    lam = np.sort(np.concatenate([[-2.0], rng.uniform(0.0, 10.0, n - 1)]))
    q = haar_unitary(n, rng)
    H = hermitian_from_spectrum(lam, q)
    c, e = 5.0, 5.0
    y0 = q[:, :1] + 1e-2 * (q[:, 1:] @ rng.standard_normal((n - 1, 1)))
    y0 = y0 / np.linalg.norm(y0)
    tau = oracle.convergence_ratio(np.array([(lam[0] - c) / e]))[0]
    rs = []
    for m in [2, 6, 10]:
        y = oracle.chebyshev_filter(H, y0, [m], lam[0], c, e)
        y = y / np.linalg.norm(y)
        rq = np.real(np.vdot(y, H @ y))
        rs.append(np.linalg.norm(H @ y - rq * y))
    slope = math.log(rs[2] / rs[0]) / 8
    assert abs(slope - math.log(tau)) < 0.1 * abs(math.log(tau))
