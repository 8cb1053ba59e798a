"""The degree MLP on the GPU: forward and gradient parity with the FP64
oracle (oracle/mlp.py), the Adam update, and an A/B test of the trained
network against the analytic degree rule on a correlated sequence.

Tolerances: the kernels round weights and activations to FP16 (unit
roundoff 2^-11 ~ 4.9e-4) and accumulate in FP32.  Against the oracle run
on the FP16-rounded weights the remaining difference comes from rounding
the activations (64-term sums, two layers), about 64 * 2^-11 * |W||h| in
the worst case; the tests allow 2e-2 on outputs of size O(1) and 5e-2
relative on each gradient tensor."""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_1404_4161_gb300 import _lib as L
from paper_1404_4161_gb300 import learned
from paper_1404_4161_gb300.solver import Chfsi, colmajor
from tests.gpu_util import DEV, from_dev_cm, to_dev_cm
from workloads.synthetic import BASE_SEED, WORKLOADS, config_sequence, random_block

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1404_4161_gb300.build import build
    build()
    s = Chfsi()
    yield s
    s.close()


def fp16_params(p):
    return {k: v.astype(np.float16).astype(np.float64) for k, v in p.items()}


def data(B, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    x = rng.standard_normal((B, omlp.N_FEAT)) * np.array([2.0, 0.4, 1.0, 2.0, 1.0])
    t = rng.uniform(0.1, 1.2, B)
    return x, t


def test_forward_parity(ctx):
    p = omlp.init_params(11)
    for k in p:
        p[k] = p[k] + 0.05 * np.random.Generator(np.random.PCG64(3)).standard_normal(p[k].shape)
    ctx.mlp_set_params(learned.flatten(p))
    x, _ = data(777, 5)
    x16 = x.astype(np.float16).astype(np.float64)
    y = ctx.mlp_forward(torch.from_numpy(x.astype(np.float32)).to(DEV)).cpu().numpy()
    ref, _ = omlp.forward(fp16_params(p), x16)
    assert np.abs(y - ref).max() < 2e-2


def test_gradient_and_adam_parity(ctx):
    p = omlp.init_params(12)
    for k in p:
        p[k] = p[k] + 0.05 * np.random.Generator(np.random.PCG64(4)).standard_normal(p[k].shape)
    flat0 = learned.flatten(p)
    ctx.mlp_set_params(flat0)
    x, t = data(1500, 6)
    xd = torch.from_numpy(x.astype(np.float32)).to(DEV)
    td = torch.from_numpy(t.astype(np.float32)).to(DEV)
    loss, g = ctx.mlp_train_step(xd, td, 1e-3)
    pe = fp16_params(p)
    loss_ref, g_ref = omlp.loss_and_grads(pe, x.astype(np.float16).astype(np.float64), t)
    assert abs(loss - loss_ref) <= 2e-2 * max(loss_ref, 1e-3)
    gd = learned.unflatten(g.cpu().numpy())
    for k in g_ref:
        rel = np.linalg.norm(gd[k] - g_ref[k]) / max(np.linalg.norm(g_ref[k]), 1e-12)
        assert rel < 5e-2, (k, rel)
    # Adam (Kingma and Ba, Alg. 1) applied to the GPU's own gradient
    p32 = learned.unflatten(flat0.numpy())
    omlp.adam_step(p32, {k: gd[k] for k in gd}, {}, lr=1e-3)
    got = learned.unflatten(ctx.mlp_get_params().numpy())
    for k in p32:
        assert np.allclose(got[k], p32[k], rtol=1e-5, atol=1e-6), k


def test_training_reduces_loss(ctx):
    x, t = data(2000, 8)
    y = np.tanh(0.5 * x[:, 0]) * 0.3 + 0.6  # a smooth target in the label range
    xd = torch.from_numpy(x.astype(np.float32)).to(DEV)
    yd = torch.from_numpy(y.astype(np.float32)).to(DEV)
    losses = learned.train(ctx, xd, yd, steps=400, lr=3e-3)
    assert losses[-1] < 0.05 * losses[0]


def test_learned_degrees_ab():
    """Train on traces of problems 1-10 of a 30-problem correlated
    sequence (n = 1024), then compare the learned degrees with the analytic
    rule (a) on random-start solves of problems 11, 20 and 30 and (b) on the
    warm-started continuation 11-30.  Both must reach the tolerance.  The
    learned degrees must save outer loops on the random starts (each loop
    costs an FP64 Rayleigh-Ritz and QR) and must not add a loop over the
    continuation; loops and times are printed."""
    from paper_1404_4161_gb300.build import build
    build()
    cfg = WORKLOADS["seq30_n8192"]
    n, nev, nex = 1024, 64, 16
    Hs, lam = config_sequence(cfg, BASE_SEED + 5000, length=30, n=n)
    Hc = [to_dev_cm(h) for h in Hs]
    X0 = random_block(n, nev + nex, BASE_SEED + 5500)
    tol = 1e-10
    s = Chfsi(precision=L.PREC_TC)
    s.trace_enable(200000)
    Xc = to_dev_cm(X0)
    ev, sts, rc = s.solve_sequence(Hc[:10], nev, nex, Xc, tol)
    assert rc == L.OK
    x, y = learned.dataset(s)
    assert x.shape[0] > 200
    losses = learned.train(s, x, y, steps=3000, lr=2e-3)
    assert losses[-1] < 0.25 * losses[0]
    s.trace_enable(0)
    X10 = Xc.clone()

    def run(model, which):
        s.set_opts(degree_model=model)
        if which == "cold":
            loops = ms = 0
            for l in (10, 19, 29):
                s.set_opts(step0=l)
                Xr = to_dev_cm(random_block(n, nev + nex, BASE_SEED + 5600 + l))
                ev_, st_, rc_ = s.solve(Hc[l], nev, nex, Xr, tol)
                assert rc_ == L.OK
                loops += st_["loops"]
                ms += st_["ms_total"]
            return loops, ms, None, None
        s.set_opts(step0=10)
        Xw = X10.clone()
        ev_, st_, rc_ = s.solve_sequence(Hc[10:], nev, nex, Xw, tol)
        assert rc_ == L.OK
        return sum(t["loops"] for t in st_), sum(t["ms_total"] for t in st_), Xw, ev_

    ca, cta, _, _ = run(L.DEG_ANALYTIC, "cold")
    cm, ctm, _, _ = run(L.DEG_MLP, "cold")
    wa, wta, _, _ = run(L.DEG_ANALYTIC, "warm")
    wm, wtm, Xm, evm = run(L.DEG_MLP, "warm")
    s.close()
    print(f"random starts: analytic {ca} loops {cta:.0f} ms | learned {cm} loops {ctm:.0f} ms; "
          f"warm 11-30: analytic {wa} loops {wta:.0f} ms | learned {wm} loops {wtm:.0f} ms")
    X = from_dev_cm(Xm)
    e_last = evm.cpu().numpy()[-1]
    H = Hs[-1]
    w = np.linalg.eigvalsh(H)
    normH = np.abs(w).max()
    R = np.linalg.norm(H @ X[:, :nev] - X[:, :nev] * e_last[:nev], axis=0) / normH
    assert R.max() <= tol
    assert np.abs(e_last[:nev] - w[:nev]).max() <= 1e-12 * normH
    # The gain is on random starts (fewer outer loops, each one an FP64
    # Rayleigh-Ritz and QR); on the warm continuation both converge in the
    # same number of loops (the analytic rule already lands the residuals
    # just below tol), so the learned degrees may not add a loop there.
    assert cm < ca
    assert wm <= wa
