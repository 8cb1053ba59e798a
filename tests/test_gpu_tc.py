"""Parity of the split-precision tensor-core filter (BF16x3, and BF16x6
with three pieces) with the oracle's Alg. 2, through the C ABI.

Tolerances follow from the arithmetic.  A BF16x3 product keeps about 16
bits (the dropped lo*lo term and the rounding of lo are both ~2^-16 of
|x||y|), accumulated in FP32.  Each of the m steps adds an error of about
2^-16 ||Hs|| ||Y_i|| (Hs = (H - cI)/e) which the later steps do not
amplify relative to the normalised output, so a column filtered to
degree m is off by at most ~ m * 2^-16 * max(1, ||H - cI||/e) relative;
the tests allow 4x that.  In the refinement form the same error applies
to D, whose size is that of the residual block, so the bound is scaled by
max_j ||R_j|| / ||Y_j psi_j||."""
import numpy as np
import pytest
import torch

import oracle
from paper_1404_4161_gb300 import _lib as L
from paper_1404_4161_gb300.solver import Chfsi
from tests.gpu_util import DEV, colrel, from_dev_cm, known_problem, to_dev_cm
from workloads.synthetic import BASE_SEED, WORKLOADS, config_problem, config_sequence, random_block

pytestmark = pytest.mark.gpu
U16 = 2.0 ** -16


@pytest.fixture(scope="module")
def ctx():
    from paper_1404_4161_gb300.build import build
    build()
    s = Chfsi()
    yield s
    s.close()


def bound(degrees, lam, c, e):
    hs = max(abs(lam[0] - c), abs(lam[-1] - c)) / e
    return 4.0 * max(degrees) * U16 * max(1.0, hs)


@pytest.mark.parametrize("n,degrees", [
    (256, [1, 2, 3, 5, 8, 8, 13, 20]),
    (777, [1] * 5 + [4] * 40 + [9] * 30 + [17] * 20 + [30]),   # ragged M, N and K tails
    (1024, list(range(1, 161))),                                # 160 columns, all degrees
    (130, [36] * 3),
])
def test_tc_filter_plain(ctx, n, degrees):
    H, lam, _ = known_problem(n, 100 + n)
    Y0 = random_block(n, len(degrees), 200 + n)
    alpha, beta = 0.4, 10.3
    c, e = 0.5 * (alpha + beta), 0.5 * (beta - alpha)
    ref = oracle.chebyshev_filter(H, Y0, degrees, lam[0], c, e)
    got = from_dev_cm(ctx.filter(to_dev_cm(H), to_dev_cm(Y0), degrees, lam[0], c, e,
                                 precision=L.PREC_MIXED))
    err = colrel(got, ref)
    print(f"n={n} k={len(degrees)} max col rel err {err:.3e} bound {bound(degrees, lam, c, e):.3e}")
    assert err < bound(degrees, lam, c, e)


@pytest.mark.parametrize("n,k,noise", [(512, 40, 1e-3), (1000, 97, 1e-6)])
def test_tc_filter_refine(ctx, n, k, noise):
    H, lam, q = known_problem(n, 300 + n)
    Q = oracle.orthonormalize(q[:, :k] + noise * random_block(n, k, 7))
    ritz, Y, HY = oracle.rayleigh_ritz(H, Q)
    R = HY - Y * ritz[None, :]
    degrees = np.sort(np.random.Generator(np.random.PCG64(k)).integers(1, 30, k))
    alpha, beta = float(lam[k + 5]), 10.3
    c, e = 0.5 * (alpha + beta), 0.5 * (beta - alpha)
    ref = oracle.chebyshev_filter(H, Y, degrees, lam[0], c, e)
    got = from_dev_cm(ctx.filter_refine(to_dev_cm(H), to_dev_cm(Y), to_dev_cm(R),
                                        torch.from_numpy(ritz).to(DEV), degrees, lam[0], c, e))
    # The split precision applies to the products H D_i of every step: with
    # the normalised recurrence no injected error grows beyond its size,
    # so column j is off by at most ~ 2 ||Hs|| 2^-16 sum_i ||D_i,j||
    # (the test allows 2x that); the D_i come from an FP64 run of the same
    # recurrence.
    from tests.test_refine_identity import defect_filter
    sums = []
    ref2 = defect_filter(H, Y, ritz, degrees, lam[0], c, e, norms=sums)
    assert colrel(ref2, ref) < 1e-9  # two FP64 evaluations, different order
    hs = max(1.0, max(abs(lam[0] - c), abs(lam[-1] - c)) / e)
    lim = 4.0 * hs * U16 * sums[0] + 1e-13 * np.linalg.norm(ref, axis=0)
    err = np.linalg.norm(got - ref, axis=0)
    ratio = float(np.max(err / lim))
    plain_scale = float(np.median(sums[0] / np.linalg.norm(ref, axis=0)))
    print(f"refine n={n} k={k} max err/bound {ratio:.3f}, "
          f"median sum||D_i||/||Y'|| {plain_scale:.2e}, max col rel err {colrel(got, ref):.2e}")
    assert ratio < 1.0


@pytest.mark.parametrize("n,degrees", [
    (777, [1] * 5 + [4] * 40 + [9] * 30 + [17] * 20 + [30]),
    (1024, list(range(1, 161))),
])
def test_tc_filter_six_products(n, degrees):
    """Three bf16 pieces per operand (6 products): the split error drops to
    ~2^-23 and what is left is the bias of the tensor cores' FP32
    accumulation within one K chunk (about 96 accumulates rounding toward
    zero, ~1.5e-6 relative per product); the bound is m 2^-19 ||Hs|| (4x
    margin), and the result must be at least 2x closer to the oracle than
    the 3-product split (whose ~2^-16 split error dominates)."""
    H, lam, _ = known_problem(n, 100 + n)
    Y0 = random_block(n, len(degrees), 200 + n)
    alpha, beta = 0.4, 10.3
    c, e = 0.5 * (alpha + beta), 0.5 * (beta - alpha)
    ref = oracle.chebyshev_filter(H, Y0, degrees, lam[0], c, e)
    errs = {}
    for split in (L.SPLIT_BF16X3, L.SPLIT_BF16X6):
        s = Chfsi(split=split)
        got = from_dev_cm(s.filter(to_dev_cm(H), to_dev_cm(Y0), degrees, lam[0], c, e,
                                   precision=L.PREC_MIXED))
        s.close()
        errs[split] = colrel(got, ref)
    hs = max(abs(lam[0] - c), abs(lam[-1] - c)) / e
    lim = 4.0 * max(degrees) * 2.0 ** -19 * max(1.0, hs)
    print(f"n={n}: 3 products {errs[L.SPLIT_BF16X3]:.2e}, 6 products {errs[L.SPLIT_BF16X6]:.2e}"
          f" (bound {lim:.2e})")
    assert errs[L.SPLIT_BF16X6] < lim
    assert errs[L.SPLIT_BF16X6] * 2 < errs[L.SPLIT_BF16X3]


def check(H, lam, X, ev, nev, tol=1e-10):
    normH = np.abs(lam).max()
    assert np.abs(ev[:nev] - lam[:nev]).max() <= 1e-12 * normH
    R = np.linalg.norm(H @ X[:, :nev] - X[:, :nev] * ev[:nev], axis=0) / normH
    assert R.max() <= tol
    assert np.abs(X.conj().T @ X - np.eye(X.shape[1])).max() < 1e-12


@pytest.mark.parametrize("prec", [L.PREC_TC, L.PREC_MIXED])
def test_solve_config1_tensor_core(prec):
    from paper_1404_4161_gb300.build import build
    build()
    cfg = WORKLOADS["single_n512"]
    H, lam = config_problem(cfg, BASE_SEED + 1000)
    X0 = random_block(cfg.n, cfg.nev + cfg.nex, BASE_SEED + 1500)
    s = Chfsi(precision=prec)
    Xc = to_dev_cm(X0)
    ev, st, rc = s.solve(to_dev_cm(H), cfg.nev, cfg.nex, Xc, cfg.tol)
    s.close()
    assert rc == L.OK, st
    print(prec, st["loops"], st["loops_lowp"], st["col_degrees"], st["col_degrees_lowp"])
    check(H, lam, from_dev_cm(Xc), ev.cpu().numpy(), cfg.nev)
    assert st["loops_lowp"] >= 1


def test_sequence_tensor_core_known_spectrum():
    cfg = WORKLOADS["seq10_n4096"]
    n, nev, nex = 768, 48, 12
    Hs, lam = config_sequence(cfg, BASE_SEED + 2000, length=3, n=n, delta=0.0)
    X0 = random_block(n, nev + nex, BASE_SEED + 2500)
    s = Chfsi(precision=L.PREC_TC)
    Xc = to_dev_cm(X0)
    ev, sts, rc = s.solve_sequence([to_dev_cm(h) for h in Hs], nev, nex, Xc, 1e-10)
    s.close()
    assert rc == L.OK
    ev = ev.cpu().numpy()
    for l, st in enumerate(sts):
        assert st["status"] == L.OK and st["loops_lowp"] == st["loops"]
        assert np.abs(ev[l, :nev] - lam[:nev]).max() <= 1e-12 * np.abs(lam).max()
    check(Hs[-1], lam, from_dev_cm(Xc), ev[-1], nev)


def test_autotuned_tiling_gives_identical_results():
    """The filter's autotuner only changes which CTA computes which tile:
    with and without it the output is bit-identical, and the table lists
    the tuned shape (n, k rounded up to 32, 2 pieces) with a candidate
    tiling."""
    n, k = 1000, 97
    H, lam, _ = known_problem(n, 4242)
    Y0 = random_block(n, k, 4243)
    degrees = sorted(np.random.Generator(np.random.PCG64(5)).integers(1, 12, k))
    c, e = 5.35, 4.95
    outs = {}
    for tune in (0, 1):
        s = Chfsi(autotune=tune, split=L.SPLIT_BF16X3)
        outs[tune] = s.filter(to_dev_cm(H), to_dev_cm(Y0), degrees, lam[0], c, e,
                              precision=L.PREC_MIXED).cpu().numpy()
        table = s.autotune_table()
        s.close()
        if tune:
            assert len(table) == 1
            t = table[0]
            assert (t["n"], t["k_bucket"], t["pieces"]) == (n, 128, 2)
            assert t["block_width"] in (64, 96, 128, 160, 192, 224, 256) and t["group"] in (1, 2, 4)
        else:
            assert table == []
    assert np.array_equal(outs[0], outs[1])
