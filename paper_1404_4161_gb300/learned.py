"""Training driver of the degree MLP (marshalling only).

The solver records traces on the device (chfsi_trace_enable); this module
turns them into a training set (chfsi_trace_dataset, labels computed in
the library's kernel) and runs full-batch Adam steps through the
library's forward, backward and optimiser kernels (chfsi_mlp_train_step).

Parameter layout of the flat vector (CHFSI_MLP_NPARAM floats):
W1[64][5], b1[64], W2[64][64], b2[64], W3[64], b3[1].
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _lib as L

N_FEAT, HIDDEN = 5, 64


def glorot_init(seed: int) -> torch.Tensor:
    """Glorot-uniform weights, zero biases, flat float32 (host)."""
    rng = np.random.Generator(np.random.PCG64(seed))

    def u(o, i):
        lim = math.sqrt(6.0 / (i + o))
        return rng.uniform(-lim, lim, size=(o, i))

    parts = [u(HIDDEN, N_FEAT).ravel(), np.zeros(HIDDEN), u(HIDDEN, HIDDEN).ravel(),
             np.zeros(HIDDEN), u(1, HIDDEN).ravel(), np.zeros(1)]
    flat = np.concatenate(parts).astype(np.float32)
    assert flat.size == L.MLP_NPARAM
    return torch.from_numpy(flat)


def unflatten(flat) -> dict:
    f = np.asarray(flat, dtype=np.float64)
    o = 0
    out = {}
    for name, shape in [("W1", (HIDDEN, N_FEAT)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)),
                        ("b2", (HIDDEN,)), ("W3", (1, HIDDEN)), ("b3", (1,))]:
        size = int(np.prod(shape))
        out[name] = f[o:o + size].reshape(shape)
        o += size
    return out


def flatten(p: dict) -> torch.Tensor:
    return torch.from_numpy(np.concatenate(
        [np.asarray(p[k]).ravel() for k in ["W1", "b1", "W2", "b2", "W3", "b3"]]).astype(np.float32))


def dataset(solver, max_rows: int = 1 << 20):
    """(x, y) device tensors from the solver's recorded traces."""
    dev = torch.device("cuda", torch.cuda.current_device())
    x = torch.empty((max_rows, N_FEAT), dtype=torch.float32, device=dev)
    y = torch.empty(max_rows, dtype=torch.float32, device=dev)
    nrows = C.c_int()
    solver._check(solver.lib.chfsi_trace_dataset(solver.ctx, C.c_void_p(x.data_ptr()),
                                                 C.c_void_p(y.data_ptr()), max_rows,
                                                 C.byref(nrows)))
    n = nrows.value
    return x[:n].contiguous(), y[:n].contiguous()


def train(solver, x, y, steps: int = 2000, lr: float = 2e-3, seed: int = 1):
    """Full-batch Adam on (x, y) from a Glorot start; returns the losses."""
    solver.mlp_set_params(glorot_init(seed))
    losses = []
    for _ in range(steps):
        loss, _ = solver.mlp_train_step(x, y, lr)
        losses.append(loss)
    return losses
