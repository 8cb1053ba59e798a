"""Whole-solve pins for the oracle (Alg. 1): known spectra, brute-force
Jacobi on a tiny problem, invariants, and the qualitative claims of the
paper's experiments (warm start, Single Optimization)."""
import math

import numpy as np
import pytest

import oracle
from workloads.synthetic import (WORKLOADS, BASE_SEED, config_problem, config_sequence,
                                 haar_unitary, hermitian_from_spectrum, random_block)


def subspace_angle(X, Z):
    """Largest principal angle between span(X) and span(Z) (orthonormal)."""
    s = np.linalg.svd(X.conj().T @ Z, compute_uv=False)
    return math.acos(min(1.0, s.min()))


def check_solution(H, lam_true, res, nev, tol):
    normH = np.abs(lam_true).max()
    X, ev = res["X"], res["evals"]
    assert res["status"] == "OK"
    assert np.abs(ev[:nev] - lam_true[:nev]).max() <= 1e-12 * normH
    R = np.linalg.norm(H @ X[:, :nev] - X[:, :nev] * ev[:nev], axis=0) / normH
    assert R.max() <= tol
    assert np.abs(X.conj().T @ X - np.eye(X.shape[1])).max() < 1e-12
    assert ev.min() >= lam_true[0] - 1e-12 and ev.max() <= lam_true[-1] + 1e-12
    return R


def test_solve_config1_known_spectrum():
    cfg = WORKLOADS["single_n512"]
    H, lam = config_problem(cfg, BASE_SEED + 1000)
    X0 = random_block(cfg.n, cfg.nev + cfg.nex, BASE_SEED + 1500)
    res = oracle.chfsi(H, cfg.nev, cfg.nex, X0, cfg.tol, deg_max=cfg.deg_max)
    R = check_solution(H, lam, res, cfg.nev, cfg.tol)
    # Davis-Kahan angle against the exact invariant subspace (gap-aware)
    w, V = np.linalg.eigh(H)
    gap = lam[cfg.nev] - lam[cfg.nev - 1]
    ang = subspace_angle(res["X"][:, :cfg.nev], V[:, :cfg.nev])
    assert ang <= max(1e-9, 2 * np.linalg.norm(R) * np.abs(lam).max() / gap)


def test_solve_tiny_vs_jacobi():
    rng = np.random.Generator(np.random.PCG64(5))
    n = 40
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    H = 0.5 * (A + A.conj().T)
    w, _ = oracle.jacobi_eigh(H)
    res = oracle.chfsi(H, 4, 4, random_block(n, 8, 1), 1e-10)
    assert res["status"] == "OK"
    assert np.abs(res["evals"][:4] - w[:4]).max() <= 1e-12 * np.abs(w).max()


def test_sequence_known_spectrum_and_warm_start_gain():
    """delta = 0 keeps every problem's spectrum exact; warm starts need
    less filtering than random starts (Sec. 5.2, Fig. 2b: >2x)."""
    cfg = WORKLOADS["seq10_n4096"]
    n, nev, nex = 512, 32, 8
    Hs, lam = config_sequence(cfg, BASE_SEED + 2000, length=3, n=n, delta=0.0)
    X0 = random_block(n, nev + nex, BASE_SEED + 2500)
    out = oracle.chfsi_sequence(Hs, nev, nex, X0, 1e-10)
    for H, res in zip(Hs, out):
        check_solution(H, lam, res, nev, 1e-10)
    cold = oracle.chfsi(Hs[2], nev, nex, X0, 1e-10)
    warm = out[2]
    assert warm["filter_col_degrees"] * 1.5 < cold["filter_col_degrees"]
    assert warm["loops"] < cold["loops"]


def test_single_optimization_saves_work():
    """Per-vector degrees need fewer matrix-vector products than one
    uniform degree for the same tolerance (Sec. 5.2, Fig. 5a)."""
    cfg = WORKLOADS["single_n512"]
    H, lam = config_problem(cfg, BASE_SEED + 1000)
    X0 = random_block(cfg.n, 48, BASE_SEED + 1500)
    opt = oracle.chfsi(H, 32, 16, X0, 1e-10)

    def uniform(ritz, resid, c, e, tol, dmax, n_wanted=None):
        m = oracle.degree_rule(ritz, resid, c, e, tol, dmax, n_wanted=n_wanted)
        return np.full_like(m, m[:n_wanted].max() if n_wanted else m.max())

    uni = oracle.chfsi(H, 32, 16, X0, 1e-10, degree_fn=uniform)
    assert uni["status"] == "OK" and opt["status"] == "OK"
    assert opt["filter_col_degrees"] < uni["filter_col_degrees"]


def test_bad_sizes():
    H = np.eye(10, dtype=np.complex128)
    with pytest.raises(ValueError):
        oracle.chfsi(H, 4, 0, random_block(10, 4, 1), 1e-10)
    with pytest.raises(ValueError):
        oracle.chfsi(H, 8, 4, random_block(10, 12, 1), 1e-10)


def generalized_known(n, seed, lo=(-2.0, -1.0), bulk=(0.0, 10.0), n_low=None):
    """A = L V diag(lam) V^H L^H with B = L L^H Hermitian positive definite
    (eigenvalues in [0.5, 3]) and V Haar unitary: A c = lam B c has exactly
    the eigenvalues lam, eigenvectors C = L^-H V."""
    from workloads.synthetic import haar_unitary
    rng = np.random.Generator(np.random.PCG64(seed))
    n_low = n_low or max(1, n // 8)
    lam = np.sort(np.concatenate([rng.uniform(*lo, n_low), rng.uniform(*bulk, n - n_low)]))
    qb = haar_unitary(n, rng)
    B = (qb * rng.uniform(0.5, 3.0, n)[None, :]) @ qb.conj().T
    B = 0.5 * (B + B.conj().T)
    L = np.linalg.cholesky(B)
    V = haar_unitary(n, rng)
    A = L @ ((V * lam[None, :]) @ V.conj().T) @ L.conj().T
    A = 0.5 * (A + A.conj().T)
    return A, B, lam


def test_generalized_known_spectrum_and_lapack():
    """Sec. 3: the reduction to standard form, ChFSI, the back-transform.
    Pinned against the exact generalized spectrum and LAPACK's zhegvd
    (scipy.linalg.eigh(A, B)); the eigenvectors are B-orthonormal and
    satisfy A c = lam B c."""
    import scipy.linalg as sla
    from workloads.synthetic import random_block
    n, nev, nex = 160, 12, 6
    A, B, lam = generalized_known(n, 31)
    res = oracle.chfsi_generalized(A, B, nev, nex, random_block(n, nev + nex, 32), 1e-10)
    assert res["status"] == "OK"
    ev = res["evals"][:nev]
    w = sla.eigh(A, B, eigvals_only=True)
    scale = np.abs(lam).max()
    assert np.abs(ev - lam[:nev]).max() <= 1e-12 * scale
    assert np.abs(ev - w[:nev]).max() <= 1e-12 * scale
    C = res["C"][:, :nev]
    assert np.abs(C.conj().T @ B @ C - np.eye(nev)).max() < 1e-12
    R = np.linalg.norm(A @ C - (B @ C) * ev[None, :], axis=0)
    assert R.max() <= 1e-10 * (np.linalg.norm(A, 2) + scale * np.linalg.norm(B, 2))
