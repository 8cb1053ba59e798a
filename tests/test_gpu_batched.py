"""The batched persistent filter (one cooperative launch for many problems
of uneven size) against the single-problem tensor-core filter and the
oracle's Alg. 2.  Same split arithmetic and the same K order per output
element, so the batched result matches the single-problem one to FP32
rounding of the epilogue (1e-6 relative); against the oracle the BF16x3
bound of the plain filter applies."""
import numpy as np
import pytest

import oracle
from paper_1404_4161_gb300 import _lib as L
from paper_1404_4161_gb300.solver import Chfsi
from tests.gpu_util import DEV, colrel, from_dev_cm, known_problem, to_dev_cm
from workloads.synthetic import random_block

pytestmark = pytest.mark.gpu
U16 = 2.0 ** -16


@pytest.fixture(scope="module")
def ctx():
    from paper_1404_4161_gb300.build import build
    build()
    s = Chfsi()
    yield s
    s.close()


def make_jobs(specs, seed0):
    jobs, refs = [], []
    for i, (n, degrees) in enumerate(specs):
        H, lam, _ = known_problem(n, seed0 + i)
        Y0 = random_block(n, len(degrees), seed0 + 100 + i)
        alpha, beta = 0.3 + 0.1 * i, 10.4
        c, e = 0.5 * (alpha + beta), 0.5 * (beta - alpha)
        jobs.append((to_dev_cm(H), to_dev_cm(Y0), degrees, lam[0], c, e))
        refs.append((H, Y0, degrees, lam, c, e))
    return jobs, refs


def test_batched_matches_single_and_oracle(ctx):
    rng = np.random.Generator(np.random.PCG64(5))
    specs = [
        (300, [1, 2, 3, 5, 8, 13, 21, 30]),
        (517, sorted(rng.integers(1, 25, 61).tolist())),
        (1000, sorted(rng.integers(3, 36, 130).tolist())),
        (130, [36, 36]),
        (777, sorted(rng.integers(1, 12, 40).tolist())),
    ]
    jobs, refs = make_jobs(specs, 700)
    outs = ctx.filter_batched(jobs)
    for (Hc, Y0c, degrees, lam1, c, e), out, (H, Y0, deg, lam, c_, e_) in zip(jobs, outs, refs):
        single = from_dev_cm(ctx.filter(Hc, Y0c, degrees, lam1, c, e, precision=L.PREC_MIXED))
        got = from_dev_cm(out)
        assert colrel(got, single) < 1e-6
        ref = oracle.chebyshev_filter(H, Y0, deg, lam1, c, e)
        hs = max(abs(lam[0] - c), abs(lam[-1] - c)) / e
        assert colrel(got, ref) < 4.0 * max(deg) * U16 * max(1.0, hs)


def test_batched_twice_and_many_problems(ctx):
    """64 small problems (k-point style) in one launch, twice in a row
    (counters and buffers are reset between launches)."""
    rng = np.random.Generator(np.random.PCG64(9))
    specs = []
    for i in range(64):
        n = int(rng.integers(96, 400))
        k = max(1, n // 16)
        specs.append((n, sorted(rng.integers(1, 16, k).tolist())))
    jobs, refs = make_jobs(specs, 2000)
    for _ in range(2):
        outs = ctx.filter_batched(jobs)
        for (Hc, Y0c, degrees, lam1, c, e), out in zip(jobs[::9], outs[::9]):
            single = from_dev_cm(ctx.filter(Hc, Y0c, degrees, lam1, c, e,
                                            precision=L.PREC_MIXED))
            assert colrel(from_dev_cm(out), single) < 1e-6


def test_solve_batched_sequences():
    """Six independent correlated sequences of uneven size (delta = 0, so
    every step has its problem's known spectrum), two steps, solved in
    lockstep with one batched filter launch per loop."""
    from paper_1404_4161_gb300.build import build
    from workloads.synthetic import BASE_SEED, WORKLOADS, config_sequence
    build()
    cfg = WORKLOADS["batched64"]
    sizes = [(320, 20, 5), (448, 28, 7), (512, 32, 8), (600, 37, 9), (384, 24, 6), (700, 43, 10)]
    seqs, ref = [], []
    for i, (n, nev, nex) in enumerate(sizes):
        Hs, lam = config_sequence(cfg, BASE_SEED + 4000 + i, length=2, n=n, eps=1e-3, delta=0.0)
        X0 = random_block(n, nev + nex, BASE_SEED + 4500 + i)
        seqs.append(([to_dev_cm(h) for h in Hs], nev, nex, to_dev_cm(X0)))
        ref.append((Hs, lam, nev))
    s = Chfsi(precision=L.PREC_TC)
    evs, stats, rc, _ = s.solve_batched(seqs, 1e-10)
    s.close()
    assert rc == L.OK
    for (Hcs, nev, nex, Xc), ev, (Hs, lam, nev_) in zip(seqs, evs, ref):
        ev = ev.cpu().numpy()
        normH = np.abs(lam).max()
        for l in range(2):
            assert np.abs(ev[l, :nev] - lam[:nev]).max() <= 1e-12 * normH
        X = from_dev_cm(Xc)
        R = np.linalg.norm(Hs[-1] @ X[:, :nev] - X[:, :nev] * ev[-1, :nev], axis=0) / normH
        assert R.max() <= 1e-10
    for l in range(2):
        for st in stats[l]:
            assert st["status"] == L.OK and st["loops_lowp"] == st["loops"]


def test_solve_batched_in_windows_equals_one_call():
    """Three steps of four sequences solved in one call, or as one step and
    then two more that start warm from the first call's Ritz blocks and
    lambda_1, lambda_k (the problems' warm fields): the same eigenvalues,
    bit for bit."""
    from paper_1404_4161_gb300.build import build
    from workloads.synthetic import BASE_SEED, WORKLOADS, circulant_window
    build()
    cfg = WORKLOADS["batched64"]
    sizes = [640, 768, 512, 896]
    runs = {}
    for mode in ("one", "windows"):
        s = Chfsi(precision=L.PREC_TC)
        seqs, Xs = [], []
        hs_all = []
        for i, n in enumerate(sizes):
            hs, lam = circulant_window(cfg, BASE_SEED + 6000 + i, 0, 3, n, device=DEV)
            hs_all.append([h.t().contiguous() for h in hs])
            nev = n // 16
            nex = nev // 4
            Xs.append(to_dev_cm(random_block(n, nev + nex, BASE_SEED + 6100 + i)))
        if mode == "one":
            seqs = [(hs_all[i], n // 16, (n // 16) // 4, Xs[i]) for i, n in enumerate(sizes)]
            evs, _, rc, _ = s.solve_batched(seqs, 1e-10)
            assert rc == L.OK
            runs[mode] = [e.cpu().numpy() for e in evs]
        else:
            seqs = [(hs_all[i][:1], n // 16, (n // 16) // 4, Xs[i]) for i, n in enumerate(sizes)]
            ev1, _, rc, warm = s.solve_batched(seqs, 1e-10)
            assert rc == L.OK
            seqs = [(hs_all[i][1:], n // 16, (n // 16) // 4, Xs[i]) for i, n in enumerate(sizes)]
            ev2, _, rc, _ = s.solve_batched(seqs, 1e-10, warm=warm)
            assert rc == L.OK
            runs[mode] = [np.vstack([a.cpu().numpy(), b.cpu().numpy()]) for a, b in zip(ev1, ev2)]
        s.close()
    for a, b in zip(runs["one"], runs["windows"]):
        assert np.array_equal(a, b)
