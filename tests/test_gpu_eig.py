"""The k x k Hermitian eigensolve of Rayleigh-Ritz (Alg. 1) with the
tensor-core engine: refinement on FP64-accurate products from the identity
(nearly diagonal Rayleigh quotients) or from FP32 eigenvectors (dense ones),
with exact Jacobi rotations for clusters of close eigenvalues.

Driven through chfsi_rayleigh_ritz with n = k and Q = I, so that the
Rayleigh quotient G is H itself and the Ritz pairs are H's eigenpairs.
The definition-level oracle is numpy's eigh (LAPACK zheevd): eigenvalues
to 1e-12 ||H||; every eigenvector's residual to 1e-12 ||H||; orthonormal
to 1e-13 k; clusters of close eigenvalues (gap below 1e-6 ||H||), whose
single vectors are not determined to FP64 accuracy, are compared as
subspaces (largest principal angle)."""
import numpy as np
import pytest
import scipy.linalg
import torch

from paper_1404_4161_gb300 import _lib as L
from paper_1404_4161_gb300.solver import Chfsi
from tests.gpu_util import DEV, from_dev_cm, to_dev_cm
from workloads.synthetic import haar_unitary, two_band_spectrum

pytestmark = pytest.mark.gpu


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def eig_gpu(H):
    k = H.shape[0]
    s = Chfsi(f64_gemm=L.GEMM_OZAKI)
    Q = np.eye(k, dtype=np.complex128)
    ev, Y, HY = s.rayleigh_ritz(to_dev_cm(H), to_dev_cm(Q))
    s.close()
    return ev.cpu().numpy(), from_dev_cm(Y), from_dev_cm(HY)


def check(H, ev, Y, HY, lam_exact=None):
    k = H.shape[0]
    lr, Vr = np.linalg.eigh(H)
    normH = np.abs(lr).max()
    assert np.all(np.diff(ev) >= 0), "ascending"
    assert np.abs(ev - lr).max() <= 1e-12 * normH
    if lam_exact is not None:
        assert np.abs(ev - np.sort(lam_exact)).max() <= 1e-12 * normH
    assert np.abs(Y.conj().T @ Y - np.eye(k)).max() <= 1e-13 * k
    r = np.linalg.norm(H @ Y - Y * ev[None, :], axis=0) / normH
    assert r.max() <= 1e-12, r.max()
    assert np.linalg.norm(HY - H @ Y, axis=0).max() / normH <= 1e-12
    # clusters: consecutive eigenvalues closer than 1e-6 ||H||, as subspaces
    bounds = np.flatnonzero(np.diff(lr) > 1e-6 * normH) + 1
    worst = 0.0
    for idx in np.split(np.arange(k), bounds):
        sv = np.linalg.svd(Vr[:, idx].conj().T @ Y[:, idx], compute_uv=False)
        worst = max(worst, float(np.arccos(min(1.0, sv.min()))))
    # the gap to the next cluster is >= 1e-6 ||H||: angle <= ||R|| / gap
    assert worst <= 1e-5, worst
    return r.max(), worst


@pytest.mark.parametrize("k", [48, 320, 640, 1000])
def test_dense_clustered(k):
    """Dense Hermitian with a clustered low band (random gaps down to ~1e-6):
    the FP32 start, then refinement and the cluster rotations."""
    rng = _rng(900 + k)
    lam = two_band_spectrum(k, (9 * k) // 10, (-5.0, -1.0), (0.0, 40.0), rng)
    q = haar_unitary(k, rng)
    H = (q * lam[None, :]) @ q.conj().T
    H = 0.5 * (H + H.conj().T)
    ev, Y, HY = eig_gpu(H)
    r, ang = check(H, ev, Y, HY, lam)
    print(f"dense k={k}: max resid {r:.2e}, worst cluster angle {ang:.2e}, "
          f"min gap {np.diff(lam).min():.2e}")


@pytest.mark.parametrize("k", [48, 320, 640])
def test_nearly_diagonal_with_close_pairs(k):
    """G = U^H diag(lam) U with U = exp(i 1e-3 A) (a warm Rayleigh quotient),
    lam with pairs 1e-9 and 3e-7 apart, a triple and an exactly degenerate
    quadruple: the identity start, cluster rotations and refinement."""
    rng = _rng(700 + k)
    lam = np.sort(rng.uniform(-3.0, 20.0, k))
    lam[10] = lam[9] + 1e-9
    lam[30] = lam[29] + 3e-7
    lam[31] = lam[29] + 5e-7
    lam[40:44] = lam[40]
    lam = np.sort(lam)
    A = rng.standard_normal((k, k)) + 1j * rng.standard_normal((k, k))
    A = (A + A.conj().T) / (2 * np.sqrt(2 * k))
    U = scipy.linalg.expm(1j * 1e-3 * A)
    H = U.conj().T @ np.diag(lam) @ U
    H = 0.5 * (H + H.conj().T)
    ev, Y, HY = eig_gpu(H)
    r, ang = check(H, ev, Y, HY, lam)
    print(f"nearly diagonal k={k}: max resid {r:.2e}, worst cluster angle {ang:.2e}")


def test_diagonal_and_tiny():
    """Already diagonal (converged at once, W = I), and k = 1."""
    lam = np.linspace(-2.0, 3.0, 64)
    H = np.diag(lam).astype(np.complex128)
    ev, Y, HY = eig_gpu(H)
    # the diagonal passes through two products of the tensor-core engine
    assert np.abs(ev - lam).max() <= 1e-14 * 3.0
    assert np.abs(Y - np.eye(64)).max() == 0.0
    ev1, Y1, _ = eig_gpu(np.array([[2.5 + 0j]]))
    assert ev1[0] == 2.5 and abs(abs(Y1[0, 0]) - 1.0) < 1e-15


@pytest.mark.parametrize("k", [200, 640])
def test_dense_large_degenerate_clusters(k):
    """Dense Hermitian with a 40-fold exactly degenerate eigenvalue (more
    than one 32-column Jacobi block) and a 12-fold cluster spread over 1e-10:
    the FP32 start spans each cluster's invariant subspace, the refinement
    must still reach FP64 accuracy (clusters compared as subspaces)."""
    rng = _rng(1300 + k)
    lam = np.sort(rng.uniform(-3.0, 20.0, k))
    lam[20:60] = -1.0
    lam[100:112] = 7.5 + 1e-10 * np.arange(12)
    lam = np.sort(lam)
    q = haar_unitary(k, rng)
    H = (q * lam[None, :]) @ q.conj().T
    H = 0.5 * (H + H.conj().T)
    ev, Y, HY = eig_gpu(H)
    r, ang = check(H, ev, Y, HY, lam)
    print(f"degenerate clusters k={k}: max resid {r:.2e}, worst cluster angle {ang:.2e}")
