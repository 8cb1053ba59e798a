"""GPU parity of every FP64 step of the hot path against the CPU oracle,
through the C ABI.  Tolerances follow from FP64 rounding (n * u * growth):
1e-12 relative for the filter and the factorisations, 1e-12 * ||H|| for
eigenvalues, bit-exact for integer degrees."""
import numpy as np
import pytest
import torch

import oracle
from paper_1404_4161_gb300 import _lib as L
from paper_1404_4161_gb300.solver import Chfsi
from tests.gpu_util import DEV, colrel, from_dev_cm, known_problem, to_dev_cm
from workloads.synthetic import random_block

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1404_4161_gb300.build import build
    build()
    s = Chfsi()
    yield s
    s.close()


@pytest.mark.parametrize("n,seed", [(64, 1), (333, 2), (1000, 3)])
def test_lanczos_parity(ctx, n, seed):
    H, lam, _ = known_problem(n, seed)
    got = ctx.lanczos(to_dev_cm(H), 20, 77)
    ref = oracle.lanczos_bounds(H, 20, oracle.lanczos_start(n, 77))
    for key in ["beta", "theta_min", "theta_max", "norm_h"]:
        assert abs(got[key] - ref[key]) <= 1e-10 * abs(ref["norm_h"]), key
    assert got["beta"] >= lam[-1]


def _gue(n, seed):
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    return (g + g.conj().T) / (2.0 * np.sqrt(2.0 * n))


@pytest.mark.parametrize("n", [2049, 4096, 5000])
def test_lanczos_parity_segments(ctx, n):
    """Sizes where the persistent Lanczos kernel splits each column into
    several mat-vec segments with a ragged last one and the last CTA owns
    fewer indices than the others; the result is also bitwise reproducible
    (fixed-order reductions)."""
    H = _gue(n, n)
    Hd = to_dev_cm(H)
    got = ctx.lanczos(Hd, 20, 5)
    again = ctx.lanczos(Hd, 20, 5)
    ref = oracle.lanczos_bounds(H, 20, oracle.lanczos_start(n, 5))
    for key in ["beta", "theta_min", "theta_max", "norm_h"]:
        assert abs(got[key] - ref[key]) <= 1e-10 * abs(ref["norm_h"]), key
        assert got[key] == again[key], key


def test_lanczos_small_n_breakdown(ctx):
    H, lam, _ = known_problem(8, 4)
    got = ctx.lanczos(to_dev_cm(H), 20, 1)
    assert abs(got["theta_min"] - lam[0]) < 1e-9 and abs(got["theta_max"] - lam[-1]) < 1e-9


@pytest.mark.parametrize("n,degrees", [
    (200, [1, 1, 2, 3, 3, 5, 8, 8, 8, 13, 20, 36] + [36] * 25),   # ragged tail, 37 cols
    (513, list(range(1, 66))),                                  # every degree distinct
    (96, [6]),                                                  # single column
    (130, [1] * 33),                                            # degree 1 only
])
def test_filter_fp64_parity(ctx, n, degrees):
    H, lam, q = known_problem(n, n)
    Y0 = random_block(n, len(degrees), n + 1)
    alpha, beta = 0.3, 10.5
    c, e = 0.5 * (alpha + beta), 0.5 * (beta - alpha)
    ref = oracle.chebyshev_filter(H, Y0, degrees, lam[0], c, e)
    got = from_dev_cm(ctx.filter(to_dev_cm(H), to_dev_cm(Y0), degrees, lam[0], c, e))
    assert colrel(got, ref) < 1e-12


def test_filter_rejects_bad_degrees(ctx):
    H, lam, _ = known_problem(40, 1)
    Y0 = to_dev_cm(random_block(40, 3, 1))
    with pytest.raises(L.ChfsiError) as ei:
        ctx.filter(to_dev_cm(H), Y0, [3, 2, 4], lam[0], 5.0, 4.0)
    assert ei.value.code == L.EINVAL


@pytest.mark.parametrize("n,k,nl", [(300, 40, 0), (300, 40, 10), (1111, 65, 33), (64, 1, 5),
                                    (2000, 320, 0), (1500, 333, 17), (4000, 1000, 0)])
def test_orthonormalize_parity(ctx, n, k, nl):
    Lk = oracle.orthonormalize(random_block(n, nl, 3)) if nl else None
    Y = random_block(n, k, 4)
    ref = oracle.orthonormalize(Y, Lk)
    Yc = to_dev_cm(Y)
    ctx.orthonormalize(Yc, to_dev_cm(Lk) if nl else None)
    got = from_dev_cm(Yc)
    assert colrel(got, ref) < 1e-11
    assert np.abs(got.conj().T @ got - np.eye(k)).max() < 1e-13


def test_orthonormalize_ill_conditioned_against_locked(ctx):
    """An ill-conditioned block next to a locked one: what the projection
    leaves along L is amplified by 1/sigma_min in the first Cholesky pass
    and removed by the projection after it, so L^H Q stays at rounding."""
    n, k, nl, cond = 3000, 100, 40, 1e6
    Lk = oracle.orthonormalize(random_block(n, nl, 91))
    Y = random_block(n, k, 92) @ np.diag(np.logspace(0, -np.log10(cond), k)) @ random_block(k, k, 93)
    ref = oracle.orthonormalize(Y, Lk)
    Yc = to_dev_cm(Y)
    ctx.orthonormalize(Yc, to_dev_cm(Lk))
    got = from_dev_cm(Yc)
    assert np.abs(got.conj().T @ got - np.eye(k)).max() < 1e-13
    assert np.abs(Lk.conj().T @ got).max() < 1e-14 * np.sqrt(k) * 3
    span_diff = np.linalg.norm(got @ (got.conj().T @ ref) - ref)
    assert span_diff < 1e3 * 1.1e-16 * cond * np.sqrt(k)


@pytest.mark.parametrize("cond,k", [(1e9, 24), (1e11, 24), (1e11, 100)])
def test_orthonormalize_ill_conditioned(ctx, cond, k):
    """Columns almost dependent (Gram matrix not numerically positive
    definite, so the shifted CholQR pass runs): the result is orthonormal
    and spans the same space as Householder QR, to the u * cond(Y) to which
    that span is defined at all."""
    n = 400 if k <= 24 else 600
    base = random_block(n, k, 9)
    Y = base @ np.diag(np.logspace(0, -np.log10(cond), k)) @ random_block(k, k, 10)
    ref = oracle.orthonormalize(Y)
    Yc = to_dev_cm(Y)
    ctx.orthonormalize(Yc)
    got = from_dev_cm(Yc)
    assert np.abs(got.conj().T @ got - np.eye(k)).max() < 1e-12
    span_diff = np.linalg.norm(got @ (got.conj().T @ ref) - ref)
    assert span_diff < 1e3 * 1.1e-16 * cond


@pytest.mark.parametrize("n,k", [(256, 24), (700, 97)])
def test_rayleigh_ritz_parity(ctx, n, k):
    H, lam, q = known_problem(n, 5 + n)
    Q = oracle.orthonormalize(random_block(n, k, 6))
    lr, Yr, HYr = oracle.rayleigh_ritz(H, Q)
    ev, Y, HY = ctx.rayleigh_ritz(to_dev_cm(H), to_dev_cm(Q))
    ev = ev.cpu().numpy()
    Y, HY = from_dev_cm(Y), from_dev_cm(HY)
    normH = np.abs(lam).max()
    assert np.abs(ev - lr).max() <= 1e-12 * normH
    # eigenvectors are unique up to a phase for simple Ritz values
    ov = np.abs(np.sum(Y.conj() * Yr, axis=0))
    gaps = np.minimum(np.diff(lr, prepend=-np.inf), np.diff(lr, append=np.inf))
    ok = gaps > 1e-6 * normH
    assert np.all(ov[ok] > 1 - 1e-10)
    assert np.allclose(HY, H @ Y, atol=1e-11 * normH)
    r_gpu = ctx.residuals(to_dev_cm(HY), to_dev_cm(Y), torch.from_numpy(ev).to(DEV), normH)
    r_ref = oracle.residuals(HY, Y, ev, normH)
    assert np.allclose(r_gpu.cpu().numpy(), r_ref, rtol=1e-12, atol=1e-16)


def test_degrees_bit_exact(ctx):
    rng = np.random.Generator(np.random.PCG64(11))
    k = 700
    ritz = np.sort(rng.uniform(-3.0, 1.0, k))
    resid = 10.0 ** rng.uniform(-11, -1, k)
    c, e, tol = 2.0, 2.5, 1e-10
    for n_wanted in [0, 350, 700]:
        ref = oracle.degree_rule(ritz, resid, c, e, tol, 36, n_wanted=n_wanted or None)
        got = ctx.degrees(torch.from_numpy(ritz).to(DEV), torch.from_numpy(resid).to(DEV),
                          c, e, tol, n_wanted).cpu().numpy()
        assert np.array_equal(got, ref)
