"""Degree-predictor MLP: FP64 reference forward, backward and Adam step.

TEST INFRASTRUCTURE: checks the CUDA training and inference kernels.
The network replaces the decay rate inside the Single Optimization rule
of Sec. 3.2 (the paper has no such network).

Why a decay rate: the rule m_i = ln(Res_i/tol)/ln|rho_i| assumes that the
residual of vector i falls like |rho_i|^-m.  Eq. (resl) also has terms
from the other wanted components, and for the lowest Ritz values (large
|t|) the residual is held back by their slower-decaying neighbours, so the
realised decay per degree is far below acosh|t_i|.  The network learns the
ratio y = kappa_realised / acosh|t_i| from the solver's own traces; the
degree then follows in closed form:
    m_i = ceil(ln(max(r_i, tol)/tol) / (acosh|t_i| * y_i)) + extra,
clamped to [4, 60] (60 when |t_i| <= 1).

Architecture: x (F) -> tanh(W1 x + b1) (H) -> tanh(W2 h1 + b2) (H) ->
y = W3 h2 + b3 (1).  Loss: 0.5 * mean((y - target)^2).  Adam follows
Kingma and Ba, ICLR 2015, Algorithm 1.

Features of one active column (``features``):
  x0 = clip(t, -8, 8),  t = (lam - c)/e   (Ritz value in the filter frame)
  x1 = log10(r) / 10                      (residual)
  x2 = acosh(max(|t|, 1))                 (analytic decay per degree)
  x3 = clip((gamma - c)/e, -8, 8)         (filter bounds: lower end)
  x4 = min(step, 9) / 10                  (index in the sequence, saturating:
                                           a network trained on the first ten
                                           problems sees every later one as
                                           the tenth instead of extrapolating)

Label (``decay_label``): with r_b the residual when degree m was chosen and
r_a the residual after filtering with it, y = clip(ln(r_b/r_a) / m /
acosh|t|, 0.02, 1.5).  Pairs that converged (r_a <= tol) give a lower
bound of the true ratio, which biases the fit toward larger degrees.
Parity unpinned for the label and the degree map (not in the paper).
"""
from __future__ import annotations

import math

import numpy as np

N_FEAT = 5
STEP_CAP = 9
HIDDEN = 64
DEG_LO, DEG_HI, DEG_SCALE = 4, 60, 60.0


def init_params(seed: int, n_feat: int = N_FEAT, hidden: int = HIDDEN) -> dict:
    """Glorot-uniform weights, zero biases."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def glorot(o, i):
        lim = math.sqrt(6.0 / (i + o))
        return rng.uniform(-lim, lim, size=(o, i))

    return {"W1": glorot(hidden, n_feat), "b1": np.zeros(hidden),
            "W2": glorot(hidden, hidden), "b2": np.zeros(hidden),
            "W3": glorot(1, hidden), "b3": np.zeros(1)}


def features(ritz, resid, c, e, gamma, step):
    t = (np.asarray(ritz, dtype=np.float64) - c) / e
    r = np.maximum(np.asarray(resid, dtype=np.float64), 1e-300)
    x = np.empty((t.size, N_FEAT))
    x[:, 0] = np.clip(t, -8.0, 8.0)
    x[:, 1] = np.log10(r) / 10.0
    x[:, 2] = np.arccosh(np.maximum(np.abs(t), 1.0))
    x[:, 3] = np.clip((gamma - c) / e, -8.0, 8.0)
    x[:, 4] = min(step, STEP_CAP) / 10.0
    return x


Y_LO, Y_HI = 0.02, 1.5


def decay_label(ritz, r_before, r_after, m_used, c, e):
    t = np.abs((np.asarray(ritz, dtype=np.float64) - c) / e)
    kan = np.arccosh(np.maximum(t, 1.0 + 1e-12))
    rb = np.asarray(r_before, dtype=np.float64)
    ra = np.maximum(np.asarray(r_after, dtype=np.float64), 1e-300)
    kre = np.log(rb / ra) / np.asarray(m_used, dtype=np.float64)
    return np.clip(kre / kan, Y_LO, Y_HI)


def degrees_from_prediction(y, ritz, resid, c, e, tol, extra=2):
    """Closed-form degree from the predicted decay ratio y."""
    t = np.abs((np.asarray(ritz, dtype=np.float64) - c) / e)
    kan = np.arccosh(np.maximum(t, 1.0 + 1e-12))
    yy = np.clip(np.asarray(y, dtype=np.float64), Y_LO, Y_HI)
    r = np.maximum(np.asarray(resid, dtype=np.float64), tol)
    m = np.ceil(np.log(r / tol) / (kan * yy)) + extra
    m = np.where(t > 1.0, m, DEG_HI)
    return np.clip(m, DEG_LO, DEG_HI).astype(np.int64)


def forward(p: dict, x):
    z1 = x @ p["W1"].T + p["b1"]
    h1 = np.tanh(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.tanh(z2)
    y = h2 @ p["W3"].T + p["b3"]
    return y[:, 0], {"x": x, "h1": h1, "h2": h2}


def loss_and_grads(p: dict, x, target):
    """0.5 * mean((y - target)^2) and its gradient (backpropagation)."""
    y, cache = forward(p, x)
    B = x.shape[0]
    d = (y - target) / B
    loss = 0.5 * float(np.mean((y - target) ** 2))
    h1, h2 = cache["h1"], cache["h2"]
    g = {"W3": d[None, :] @ h2, "b3": np.array([d.sum()])}
    dh2 = d[:, None] * p["W3"]
    dz2 = dh2 * (1.0 - h2 ** 2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2 @ p["W2"]
    dz1 = dh1 * (1.0 - h1 ** 2)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(axis=0)
    return loss, g


def adam_step(p: dict, g: dict, state: dict, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, Algorithm 1), in place on p."""
    t = state.get("t", 0) + 1
    state["t"] = t
    for kname in p:
        mo = state.setdefault("m_" + kname, np.zeros_like(p[kname]))
        ve = state.setdefault("v_" + kname, np.zeros_like(p[kname]))
        mo[...] = b1 * mo + (1 - b1) * g[kname]
        ve[...] = b2 * ve + (1 - b2) * g[kname] ** 2
        mh = mo / (1 - b1 ** t)
        vh = ve / (1 - b2 ** t)
        p[kname] = p[kname] - lr * mh / (np.sqrt(vh) + eps)
    return p
