"""FP64-accurate complex GEMM on the tensor cores (Ozaki scheme) against
FP64 references, through chfsi_zgemm, and whole solves that use it.

Bound: each operand is scaled per row (A) or per column (B) by a power of
two s >= max|x| and represented to 2^-49 by seven 7-bit slices; the
dropped slice pairs add ~2^-50.  A product term a b is therefore off by at
most ~2^-48 s_row s_col, and an entry of C by at most K 2^-48 s_row s_col
(worst case, equal signs); the tests check that bound per entry and a
typical-size relative Frobenius bound (2^-49 times the ratios of the
scales to the rms entry sizes, times 4)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1404_4161_gb300 import _lib as L
from paper_1404_4161_gb300.solver import Chfsi, colmajor
from tests.gpu_util import DEV, from_dev_cm, known_problem, to_dev_cm
from workloads.synthetic import BASE_SEED, WORKLOADS, config_problem, config_sequence, random_block

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1404_4161_gb300.build import build
    build()
    s = Chfsi()
    yield s
    s.close()


def pow2ceil(x):
    return 2.0 ** np.ceil(np.log2(np.maximum(x, 1e-300)))


def check(got, ref, A_rows, B_cols, K):
    """A_rows: the (sliced) left factor as rows (m x K complex), B_cols:
    K x n.  Per entry: the worst-case bound.  Frobenius: each term's error
    is ~2^-42 s_row s_col with random sign, so relative to C it is about
    2^-42 times the ratio of the scales to the rms entry sizes; the test
    allows 4x that."""
    mag_a = np.maximum(np.abs(A_rows.real), np.abs(A_rows.imag))
    mag_b = np.maximum(np.abs(B_cols.real), np.abs(B_cols.imag))
    sa = pow2ceil(mag_a.max(axis=1))
    sb = pow2ceil(mag_b.max(axis=0))
    lim = 2 * K * 2.0 ** -48 * np.outer(sa, sb)
    err = np.abs(got - ref)
    assert np.all(err <= lim), float(np.max(err / lim))
    ra = np.max(sa / np.sqrt(np.mean(np.abs(A_rows) ** 2, axis=1)))
    rb = np.max(sb / np.sqrt(np.mean(np.abs(B_cols) ** 2, axis=0)))
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel < 4 * 2.0 ** -49 * ra * rb, (rel, ra, rb)
    return rel


@pytest.mark.parametrize("n,k", [(1000, 97), (4096, 320), (257, 1)])
def test_hq_shape(ctx, n, k):
    H, lam, _ = known_problem(n, 40 + n)
    Q = random_block(n, k, 41 + n)
    got = from_dev_cm(ctx.zgemm(1, to_dev_cm(H), to_dev_cm(Q), n, k, n))
    ref = H @ Q
    rel = check(got, ref, H.conj().T, Q, 2 * n)
    print(f"H^H Q (general entry) n={n} k={k} rel {rel:.2e}")


@pytest.mark.parametrize("n,k", [(1000, 97), (4096, 320)])
def test_rayleigh_ritz_with_shifted_hq(ctx, n, k):
    """The Rayleigh-Ritz entry computes H Q as (H - mu I) Q + mu Q on the
    tensor cores: Ritz values against the FP64 oracle to 1e-12 ||H||."""
    H, lam, _ = known_problem(n, 60 + n)
    Q = oracle.orthonormalize(random_block(n, k, 61 + n))
    s = Chfsi(f64_gemm=L.GEMM_OZAKI)
    ev, Y, HY = s.rayleigh_ritz(to_dev_cm(H), to_dev_cm(Q))
    s.close()
    lr, Yr, HYr = oracle.rayleigh_ritz(H, Q)
    normH = np.abs(lam).max()
    assert np.abs(ev.cpu().numpy() - lr).max() <= 1e-12 * normH
    HY = from_dev_cm(HY)
    Y = from_dev_cm(Y)
    rel = np.linalg.norm(HY - H @ Y) / np.linalg.norm(H @ Y)
    print(f"RR shifted HQ n={n} rel {rel:.2e}")
    assert rel < 1e-13


@pytest.mark.parametrize("n,k1,k2", [(4096, 320, 320), (1500, 93, 117)])
def test_gram_shape_split_k(ctx, n, k1, k2):
    L_ = oracle.orthonormalize(random_block(n, k1, 3))
    R = random_block(n, k2, 4)
    got = from_dev_cm(ctx.zgemm(1, to_dev_cm(L_), to_dev_cm(R), k1, k2, n))
    ref = L_.conj().T @ R
    check(got, ref, L_.conj().T, R, 2 * n)


def test_update_shape_alpha_beta(ctx):
    n, k1, k2 = 2000, 64, 80
    S = random_block(n, k1, 5)
    W = random_block(k1, k2, 6)
    C0 = random_block(n, k2, 7)
    Cc = to_dev_cm(C0)
    ctx.zgemm(0, to_dev_cm(S), to_dev_cm(W), n, k2, k1, alpha=-1.0, beta=1.0, C_cm=Cc)
    got = from_dev_cm(Cc)
    ref = C0 - S @ W
    rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert rel < 1e-12


@pytest.mark.parametrize("n,k,nl,cond", [(2000, 320, 0, 1.0), (1500, 333, 17, 1.0),
                                         (3000, 100, 40, 1e5), (400, 24, 0, 1e11)])
def test_orthonormalize_fp32_first_pass_polar(n, k, nl, cond):
    """With the tensor-core FP64 engine the QR step runs its first Cholesky
    pass in FP32 and a polar correction (binomial series) after it, falling
    back to FP64 CholQR2 / shifted CholQR3 when the FP32 pass breaks down
    (cond 1e11).  The result spans what Householder QR spans (to u * cond,
    the accuracy to which that span is defined) and is orthonormal and
    orthogonal to the locked block to FP64 rounding."""
    Lk = oracle.orthonormalize(random_block(n, nl, 81)) if nl else None
    base = random_block(n, k, 82)
    Y = base @ np.diag(np.logspace(0, -np.log10(cond), k)) @ random_block(k, k, 83)
    ref = oracle.orthonormalize(Y, Lk)
    s = Chfsi(f64_gemm=L.GEMM_OZAKI)
    Yc = to_dev_cm(Y)
    s.orthonormalize(Yc, to_dev_cm(Lk) if nl else None)
    s.close()
    got = from_dev_cm(Yc)
    assert np.abs(got.conj().T @ got - np.eye(k)).max() < 1e-13
    if nl:
        # the projection leaves L^H Y at the products' accuracy (~1e-15
        # relative per entry); the two passes multiply it by ||W|| ~
        # 1 / sigma_min(Y) (about 2 here) and mix k columns: ~sqrt(k) * 1e-14
        assert np.abs(Lk.conj().T @ got).max() < 1e-14 * np.sqrt(k) * 3
    span_diff = np.linalg.norm(got @ (got.conj().T @ ref) - ref)
    assert span_diff < max(1e-12, 1e3 * 1.1e-16 * cond) * np.sqrt(k)


def test_dfma_engine_same_entry(ctx):
    n, k = 300, 40
    H, lam, _ = known_problem(n, 9)
    Q = random_block(n, k, 10)
    got = from_dev_cm(ctx.zgemm(1, to_dev_cm(H), to_dev_cm(Q), n, k, n, engine=L.GEMM_FP64))
    assert np.linalg.norm(got - H @ Q) / np.linalg.norm(H @ Q) < 1e-14


def test_solve_with_tensor_core_fp64_products():
    from paper_1404_4161_gb300.build import build
    build()
    cfg = WORKLOADS["single_n512"]
    H, lam = config_problem(cfg, BASE_SEED + 1000)
    X0 = random_block(cfg.n, cfg.nev + cfg.nex, BASE_SEED + 1500)
    s = Chfsi(precision=L.PREC_TC, f64_gemm=L.GEMM_OZAKI)
    Xc = to_dev_cm(X0)
    ev, st, rc = s.solve(to_dev_cm(H), cfg.nev, cfg.nex, Xc, cfg.tol)
    assert rc == L.OK
    ev = ev.cpu().numpy()
    X = from_dev_cm(Xc)
    normH = np.abs(lam).max()
    assert np.abs(ev[:cfg.nev] - lam[:cfg.nev]).max() <= 1e-12 * normH
    R = np.linalg.norm(H @ X[:, :cfg.nev] - X[:, :cfg.nev] * ev[:cfg.nev], axis=0) / normH
    assert R.max() <= 1e-10
    # X^H X = I to 1e-13 k (the Gram and R^-1 products carry ~1e-12)
    assert np.abs(X.conj().T @ X - np.eye(X.shape[1])).max() < 1e-13 * X.shape[1]
    # a correlated sequence with the exact spectrum kept (delta = 0)
    cfg2 = WORKLOADS["seq10_n4096"]
    n, nev, nex = 1024, 64, 16
    Hs, lam2 = config_sequence(cfg2, BASE_SEED + 2000, length=3, n=n, delta=0.0)
    Xc = to_dev_cm(random_block(n, nev + nex, BASE_SEED + 2500))
    ev2, sts, rc = s.solve_sequence([to_dev_cm(h) for h in Hs], nev, nex, Xc, 1e-10)
    s.close()
    assert rc == L.OK
    ev2 = ev2.cpu().numpy()
    for l in range(3):
        assert np.abs(ev2[l, :nev] - lam2[:nev]).max() <= 1e-12 * np.abs(lam2).max()
    X = from_dev_cm(Xc)
    R = np.linalg.norm(Hs[-1] @ X[:, :nev] - X[:, :nev] * ev2[-1, :nev], axis=0) / np.abs(lam2).max()
    assert R.max() <= 1e-10
    print("loops", [t["loops"] for t in sts])


@pytest.mark.parametrize("n,k", [(700, 48), (2048, 320)])
def test_rayleigh_ritz_mixed_eigensolver(ctx, n, k):
    """With the tensor-core engine the k x k eigensolve is a refinement on
    FP64-accurate products (here from the identity: Q is close to
    eigenvectors, so the Rayleigh quotient is nearly diagonal): Ritz values
    to 1e-12 ||H||, Ritz vectors orthonormal to 1e-13 k, residual block
    consistent."""
    H, lam, q = known_problem(n, 80 + n)
    Q = oracle.orthonormalize(q[:, :k] + 1e-3 * random_block(n, k, 81 + n))
    s = Chfsi(f64_gemm=L.GEMM_OZAKI)
    ev, Y, HY = s.rayleigh_ritz(to_dev_cm(H), to_dev_cm(Q))
    s.close()
    lr, Yr, HYr = oracle.rayleigh_ritz(H, Q)
    normH = np.abs(lam).max()
    ev = ev.cpu().numpy()
    assert np.abs(ev - lr).max() <= 1e-12 * normH
    Y = from_dev_cm(Y)
    assert np.abs(Y.conj().T @ Y - np.eye(k)).max() < 1e-13 * k
    r_gpu = np.linalg.norm(H @ Y - Y * ev[None, :], axis=0) / normH
    r_ref = np.linalg.norm(H @ Yr - Yr * lr[None, :], axis=0) / normH
    assert np.all(r_gpu <= r_ref * (1 + 1e-9) + 1e-13)


def test_sequence_warm_rayleigh_ritz():
    """opts.warm_rr: a Rayleigh-Ritz step on each warm start before the
    first filter (degrees and the refinement form from the first loop):
    same eigenpairs, no more loops than without it."""
    from paper_1404_4161_gb300.build import build
    build()
    cfg2 = WORKLOADS["seq10_n4096"]
    n, nev, nex = 1024, 64, 16
    Hs, lam2 = config_sequence(cfg2, BASE_SEED + 2200, length=4, n=n, delta=0.0)
    loops = {}
    for wr in (0, 1):
        s = Chfsi(precision=L.PREC_TC, f64_gemm=L.GEMM_OZAKI, warm_rr=wr, warm_resid=0)
        Xc = to_dev_cm(random_block(n, nev + nex, BASE_SEED + 2600))
        ev, sts, rc = s.solve_sequence([to_dev_cm(h) for h in Hs], nev, nex, Xc, 1e-10)
        s.close()
        assert rc == L.OK
        ev = ev.cpu().numpy()
        for l in range(4):
            assert np.abs(ev[l, :nev] - lam2[:nev]).max() <= 1e-12 * np.abs(lam2).max()
        X = from_dev_cm(Xc)
        R = np.linalg.norm(Hs[-1] @ X[:, :nev] - X[:, :nev] * ev[-1, :nev], axis=0)
        assert R.max() / np.abs(lam2).max() <= 1e-10
        loops[wr] = [t["loops"] for t in sts]
    print("loops without / with warm RR", loops)
    assert sum(loops[1][1:]) <= sum(loops[0][1:])


def test_sequence_warm_residual_start():
    """opts.warm_resid: on each warm start the residuals of the starting block
    on the new H (one product, no reduced eigensolve) give the first loop
    per-vector degrees and the refinement form: same eigenpairs, no more
    loops than the uniform first-loop degree."""
    from paper_1404_4161_gb300.build import build
    build()
    cfg2 = WORKLOADS["seq10_n4096"]
    n, nev, nex = 1024, 64, 16
    Hs, lam2 = config_sequence(cfg2, BASE_SEED + 2200, length=4, n=n, delta=0.0)
    loops = {}
    for wr in (0, 1):
        s = Chfsi(precision=L.PREC_TC, f64_gemm=L.GEMM_OZAKI, warm_resid=wr)
        Xc = to_dev_cm(random_block(n, nev + nex, BASE_SEED + 2600))
        ev, sts, rc = s.solve_sequence([to_dev_cm(h) for h in Hs], nev, nex, Xc, 1e-10)
        s.close()
        assert rc == L.OK
        ev = ev.cpu().numpy()
        for l in range(4):
            assert np.abs(ev[l, :nev] - lam2[:nev]).max() <= 1e-12 * np.abs(lam2).max()
        X = from_dev_cm(Xc)
        R = np.linalg.norm(Hs[-1] @ X[:, :nev] - X[:, :nev] * ev[-1, :nev], axis=0)
        assert R.max() / np.abs(lam2).max() <= 1e-10
        assert np.abs(X.conj().T @ X - np.eye(nev + nex)).max() < 1e-12
        loops[wr] = [t["loops"] for t in sts]
    print("loops with uniform / residual-based first-loop degrees", loops)
    assert sum(loops[1][1:]) <= sum(loops[0][1:])
