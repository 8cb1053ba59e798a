"""Pins for the oracle's Chebyshev filter (Alg. 2) against the closed
form Y_m = Q diag(C_m(t)/C_m(gamma_hat)) Q^H Y0 on matrices with a known
spectrum, and the convergence-rate bound of Eq. (ratio)."""
import math

import numpy as np
import pytest

import oracle
from workloads.synthetic import haar_unitary, hermitian_from_spectrum, random_block


def known(n, seed, lo=(-2.0, -1.0), bulk=(0.0, 10.0), n_low=None):
    rng = np.random.Generator(np.random.PCG64(seed))
    n_low = n_low or max(1, n // 8)
    lam = np.sort(np.concatenate([rng.uniform(*lo, n_low), rng.uniform(*bulk, n - n_low)]))
    q = haar_unitary(n, rng)
    return hermitian_from_spectrum(lam, q), lam, q


def closed_form(lam, q, Y0, degrees, lam1, c, e):
    t = (lam - c) / e
    g = (lam1 - c) / e
    out = np.empty_like(Y0)
    coef = q.conj().T @ Y0
    for j, m in enumerate(degrees):
        f = oracle.chebyshev_value(int(m), t) / oracle.chebyshev_value(int(m), np.array([g]))[0]
        out[:, j] = q @ (f * coef[:, j])
    return out


@pytest.mark.parametrize("degrees", [
    [1, 1, 2, 3, 5, 5, 5, 8, 13, 20, 36],
    [7] * 6,
    [1],
    [2, 36],
    list(range(1, 25)),
])
def test_filter_closed_form(degrees):
    H, lam, q = known(72, 11)
    Y0 = random_block(72, len(degrees), 5)
    alpha, beta = 0.4, 10.2
    c, e = 0.5 * (alpha + beta), 0.5 * (beta - alpha)
    got = oracle.chebyshev_filter(H, Y0, degrees, lam[0], c, e)
    ref = closed_form(lam, q, Y0, degrees, lam[0], c, e)
    err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err.max() < 1e-12


def test_filter_empty_block():
    H, lam, _ = known(16, 1)
    Y0 = np.zeros((16, 0), dtype=np.complex128)
    assert oracle.chebyshev_filter(H, Y0, [], lam[0], 5.0, 4.0).shape == (16, 0)


def test_filter_rejects_unsorted():
    H, lam, _ = known(16, 1)
    with pytest.raises(ValueError):
        oracle.chebyshev_filter(H, random_block(16, 2, 1), [3, 2], lam[0], 5.0, 4.0)


def test_planted_recurrence_mistake_is_caught(monkeypatch):
    """Alg. 2 as printed (second term with Y_i instead of Y_{i-1}) must
    fail the closed-form pin; this shows the pin sees reading R1."""
    H, lam, q = known(40, 3)
    Y0 = random_block(40, 3, 2)
    deg = [4, 6, 9]
    c, e = 5.3, 4.9

    def printed(H, Y0, degrees, lam1, c, e):
        m = np.asarray(degrees)
        s1 = e / (lam1 - c)
        sig = s1
        yp, yc = Y0, s1 * (H @ Y0 - c * Y0) / e
        out = np.empty_like(Y0)
        s = int(np.searchsorted(m, 1, side="right"))
        out[:, :s] = yc[:, :s]
        for i in range(1, int(m[-1])):
            sn = 1.0 / (2.0 / s1 - sig)
            yn = yc.copy()
            yn[:, s:] = 2 * sn * (H @ yc[:, s:] - c * yc[:, s:]) / e - sn * sig * yc[:, s:]
            yp, yc, sig = yc, yn, sn
            s2 = int(np.searchsorted(m, i + 1, side="right"))
            out[:, s:s2] = yc[:, s:s2]
            s = s2
        return out

    ref = closed_form(lam, q, Y0, deg, lam[0], c, e)
    bad = printed(H, Y0, deg, lam[0], c, e)
    good = oracle.chebyshev_filter(H, Y0, deg, lam[0], c, e)
    assert np.linalg.norm(good - ref) / np.linalg.norm(ref) < 1e-12
    assert np.linalg.norm(bad - ref) / np.linalg.norm(ref) > 1e-3


def test_filter_rate_bound():
    """Eq. (ratio): a component outside [alpha, beta] is kept, the ones
    inside shrink at least like 1/|C_m(gamma_hat)| ~ 2 tau^m."""
    n = 48
    rng = np.random.Generator(np.random.PCG64(9))
    lam = np.sort(np.concatenate([[-2.0], rng.uniform(0.0, 10.0, n - 1)]))
    q = haar_unitary(n, rng)
    H = hermitian_from_spectrum(lam, q)
    alpha, beta = 0.0, 10.0
    c, e = 5.0, 5.0
    y0 = q @ np.ones((n, 1), dtype=np.complex128)  # equal weight on every eigenvector
    g = (lam[0] - c) / e
    tau = oracle.convergence_ratio(np.array([g]))[0]
    prev = None
    for m in [4, 8, 12, 16]:
        y = oracle.chebyshev_filter(H, y0, [m], lam[0], c, e)
        coef = q.conj().T @ y[:, 0]
        assert abs(coef[0] - 1.0) < 1e-10  # wanted component normalised to 1
        unwanted = np.abs(coef[1:]).max()
        bound = 1.0 / abs(oracle.chebyshev_value(m, np.array([g]))[0])
        assert unwanted <= bound * (1 + 1e-9)
        assert bound <= 2 * tau ** m * (1 + 1e-12)
        if prev is not None:
            slope = math.log(bound / prev) / 4
            assert abs(slope - math.log(tau)) < 0.02
        prev = bound
