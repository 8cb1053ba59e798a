"""Whole solves on the GPU (FP64 path) against the known spectrum and the
oracle: eigenvalues to 1e-12 ||H||, residuals <= 1e-10 ||H||, subspace
angles per the gap-aware Davis-Kahan bound, loop counts against the
oracle's."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_1404_4161_gb300 import _lib as L
from paper_1404_4161_gb300.solver import Chfsi
from tests.gpu_util import DEV, from_dev_cm, known_problem, to_dev_cm
from workloads.synthetic import (BASE_SEED, WORKLOADS, config_problem, config_sequence,
                                 random_block)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1404_4161_gb300.build import build
    build()
    s = Chfsi()
    yield s
    s.close()


def angle(X, Z):
    s = np.linalg.svd(X.conj().T @ Z, compute_uv=False)
    return math.acos(min(1.0, s.min()))


def check(H, lam, X, ev, nev, tol=1e-10):
    normH = np.abs(lam).max()
    assert np.abs(ev[:nev] - lam[:nev]).max() <= 1e-12 * normH
    R = np.linalg.norm(H @ X[:, :nev] - X[:, :nev] * ev[:nev], axis=0) / normH
    assert R.max() <= tol
    assert np.abs(X.conj().T @ X - np.eye(X.shape[1])).max() < 1e-12
    return R


def test_solve_config1(ctx):
    cfg = WORKLOADS["single_n512"]
    H, lam = config_problem(cfg, BASE_SEED + 1000)
    X0 = random_block(cfg.n, cfg.nev + cfg.nex, BASE_SEED + 1500)
    ref = oracle.chfsi(H, cfg.nev, cfg.nex, X0, cfg.tol)
    Xc = to_dev_cm(X0)
    ev, st, rc = ctx.solve(to_dev_cm(H), cfg.nev, cfg.nex, Xc, cfg.tol)
    assert rc == L.OK
    ev = ev.cpu().numpy()
    X = from_dev_cm(Xc)
    R = check(H, lam, X, ev, cfg.nev)
    assert np.abs(ev[:cfg.nev] - ref["evals"][:cfg.nev]).max() <= 1e-12 * np.abs(lam).max()
    assert abs(st["loops"] - ref["loops"]) <= 1
    w, V = np.linalg.eigh(H)
    gap = lam[cfg.nev] - lam[cfg.nev - 1]
    assert angle(X[:, :cfg.nev], V[:, :cfg.nev]) <= max(1e-9, 2 * np.linalg.norm(R) * np.abs(lam).max() / gap)
    assert angle(X[:, :cfg.nev], ref["X"][:, :cfg.nev]) <= max(1e-9, 4 * np.linalg.norm(R) * np.abs(lam).max() / gap)


def test_sequence_known_spectrum(ctx):
    cfg = WORKLOADS["seq10_n4096"]
    n, nev, nex = 512, 32, 8
    Hs, lam = config_sequence(cfg, BASE_SEED + 2000, length=3, n=n, delta=0.0)
    X0 = random_block(n, nev + nex, BASE_SEED + 2500)
    ref = oracle.chfsi_sequence(Hs, nev, nex, X0, 1e-10)
    Xc = to_dev_cm(X0)
    ev, sts, rc = ctx.solve_sequence([to_dev_cm(h) for h in Hs], nev, nex, Xc, 1e-10)
    assert rc == L.OK
    ev = ev.cpu().numpy()
    for l, (H, st) in enumerate(zip(Hs, sts)):
        assert st["status"] == L.OK
        assert np.abs(ev[l, :nev] - lam[:nev]).max() <= 1e-12 * np.abs(lam).max()
        assert abs(st["loops"] - ref[l]["loops"]) <= 1
    check(Hs[-1], lam, from_dev_cm(Xc), ev[-1], nev)
    assert sts[2]["col_degrees"] < sts[0]["col_degrees"]


def test_sequence_host_buffers_match_device(ctx):
    cfg = WORKLOADS["seq10_n4096"]
    n, nev, nex = 384, 16, 8
    Hs, lam = config_sequence(cfg, BASE_SEED + 2100, length=2, n=n)
    X0 = random_block(n, nev + nex, BASE_SEED + 2600)
    Xc = to_dev_cm(X0)
    ev_d, _, _ = ctx.solve_sequence([to_dev_cm(h) for h in Hs], nev, nex, Xc, 1e-10)
    Xh = torch.from_numpy(np.ascontiguousarray(X0.T)).pin_memory()
    Hh = [torch.from_numpy(np.ascontiguousarray(h.T)).pin_memory() for h in Hs]
    ev_h, _, rc = ctx.solve_sequence_host(Hh, nev, nex, Xh, 1e-10)
    assert rc == L.OK
    assert np.array_equal(ev_h.numpy(), ev_d.cpu().numpy())
    assert np.array_equal(Xh.numpy(), Xc.cpu().numpy())


def test_invalid_and_nan_inputs(ctx):
    H, lam, _ = known_problem(64, 3)
    Xc = to_dev_cm(random_block(64, 8, 1))
    with pytest.raises(L.ChfsiError) as ei:
        ctx.solve(to_dev_cm(H), 8, 0, Xc, 1e-10)
    assert ei.value.code == L.EINVAL
    X0 = random_block(64, 8, 1)
    X0[3, 2] = np.nan
    with pytest.raises(L.ChfsiError) as ei:
        ctx.solve(to_dev_cm(H), 4, 4, to_dev_cm(X0), 1e-10)
    assert ei.value.code in (L.ENAN, L.EBREAKDOWN)


def test_max_loops_reports_enoconv(ctx):
    H, lam, _ = known_problem(200, 6)
    ctx.set_opts(max_loops=1)
    try:
        Xc = to_dev_cm(random_block(200, 24, 2))
        ev, st, rc = ctx.solve(to_dev_cm(H), 16, 8, Xc, 1e-10)
        assert rc == L.ENOCONV and st["loops"] == 1
        X = from_dev_cm(Xc)
        assert np.abs(X.conj().T @ X - np.eye(24)).max() < 1e-12
    finally:
        ctx.set_opts(max_loops=50)
