"""Pins for the oracle's Chebyshev scalars (Sec. 3.2, Eqs. (polydef),
(ratio), (3term)) and the counter-based generator."""
import math
import os

import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def cheb_lib(m, t):
    c = np.zeros(m + 1)
    c[m] = 1.0
    return npcheb.chebval(t, c)


@pytest.mark.parametrize("m", [0, 1, 2, 3, 7, 20, 36])
def test_chebyshev_value_matches_power_series(m):
    t = np.concatenate([np.linspace(-1, 1, 41), [-3.0, -1.7, -1.01, 1.01, 1.3, 2.5]])
    got = oracle.chebyshev_value(m, t)
    ref = cheb_lib(m, t)
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-12)


def test_chebyshev_growth_formula():
    # C_m(t) = (|rho|^m + |rho|^-m)/2 up to sign(t)^m for |t| > 1
    for t in [-2.5, -1.2, 1.05, 3.0]:
        rho = abs(t) + math.sqrt(t * t - 1)
        for m in [1, 5, 17]:
            v = oracle.chebyshev_value(m, np.array([t]))[0]
            assert math.isclose(abs(v), 0.5 * (rho ** m + rho ** -m), rel_tol=1e-12)


def test_sigmas_are_ratios_of_chebyshev_values():
    g = -1.37
    s = oracle.chebyshev_sigmas(12, g)
    for i in range(1, 13):
        assert math.isclose(s[i - 1], cheb_lib(i - 1, g) / cheb_lib(i, g), rel_tol=1e-12)


def test_convergence_ratio():
    t = np.array([-3.0, -1.5, -1.0, 0.0, 0.7, 1.0, 2.0])
    tau = oracle.convergence_ratio(t)
    for ti, ta in zip(t, tau):
        if abs(ti) <= 1:
            assert ta == 1.0
        else:
            # both roots t +- sqrt(t^2-1) have product 1; tau is the smaller
            r1, r2 = abs(ti + math.sqrt(ti * ti - 1)), abs(ti - math.sqrt(ti * ti - 1))
            assert math.isclose(ta, min(r1, r2), rel_tol=1e-14)
            assert math.isclose(-math.log(ta), math.acosh(abs(ti)), rel_tol=1e-12)


def test_splitmix64_published_vector():
    want = [int(l, 16) for l in open(os.path.join(GOLD, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    got = [int(x) for x in oracle.splitmix64(0, 3)]
    assert got == want


def test_lanczos_start_uniform():
    v = oracle.lanczos_start(20000, 7)
    assert v.shape == (20000,)
    for part in (v.real, v.imag):
        assert part.min() >= -1 and part.max() < 1
        assert abs(part.mean()) < 0.02 and abs(part.var() - 1 / 3) < 0.01
