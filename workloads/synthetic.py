"""Synthetic dense Hermitian eigenproblems and correlated sequences.

Recipe (all seeded; numpy PCG64 draws the random numbers, the dense
algebra runs in complex128 on the CPU with numpy or, for large n, on a
torch device):

* Q: Haar-random unitary, QR of a complex Ginibre matrix with the
  phases of diag(R) folded back into Q (Mezzadri, Notices AMS 54, 2007).
* spectrum: ``n_low`` eigenvalues uniform in ``low``, the rest uniform in
  ``bulk``, sorted ascending.
* H = Q diag(lam) Q^H, then Hermitianised as (H + H^H)/2.
* correlated step: H_{l+1} = U H_l U^H + delta * diag(d), U = exp(i eps A),
  A = (G + G^H) / (2 sqrt(2n)) with G complex Ginibre (unit-variance
  entries, so ||A||_2 is about 2), d ~ N(0, 1); exp by its Taylor series
  to order 8 (||eps A|| ~ 2e-3 makes the truncation below 1e-25).
* starting block X0: complex Gaussian, entries (a + ib)/sqrt(2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 14044161


@dataclass(frozen=True)
class Config:
    """One workload: sizes, spectrum layout and sequence parameters."""
    name: str
    n: int
    nev: int
    nex: int
    n_low: int
    low: tuple
    bulk: tuple
    length: int = 1
    eps: float = 0.0
    delta: float = 0.0
    tol: float = 1e-10
    deg_max: int = 36
    extra: dict = field(default_factory=dict)


# The five workloads of the hot path.  n_low follows the stated split
# (40 for the n=512 problem, 300 for the n=4096 sequence) and otherwise
# nev + nex//2.
WORKLOADS = {
    "single_n512": Config("single_n512", 512, 32, 16, 40, (-2.0, -1.0), (0.0, 10.0)),
    "seq10_n4096": Config("seq10_n4096", 4096, 256, 64, 300, (-3.0, -1.0), (0.0, 20.0),
              length=10, eps=1e-3, delta=1e-4),
    "seq20_n13000": Config("seq20_n13000", 13000, 800, 200, 900, (-5.0, -1.0), (0.0, 40.0),
              length=20, eps=1e-3, delta=1e-4),
    "batched64": Config("batched64", 0, 0, 0, 0, (-3.0, -1.0), (0.0, 20.0),
              length=10, eps=1e-3, delta=1e-4,
              extra={"problems": 64, "n_range": (1500, 6000)}),
    "seq30_n8192": Config("seq30_n8192", 8192, 512, 128, 576, (-3.0, -1.0), (0.0, 20.0),
              length=30, eps=1e-3, delta=1e-4),
}


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def ginibre(n: int, m: int, rng: np.random.Generator) -> np.ndarray:
    """Complex Gaussian n x m matrix with unit-variance entries."""
    g = rng.standard_normal((n, m)) + 1j * rng.standard_normal((n, m))
    return g / math.sqrt(2.0)


def haar_unitary(n: int, rng: np.random.Generator, device=None):
    """Haar-distributed n x n unitary (numpy array, or torch tensor on
    ``device`` when one is given)."""
    z = ginibre(n, n, rng)
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    q = q * (d / np.abs(d))[None, :]
    if device is None:
        return q
    import torch
    return torch.from_numpy(q).to(device)


def two_band_spectrum(n: int, n_low: int, low, bulk, rng) -> np.ndarray:
    """n eigenvalues: n_low uniform in ``low``, the rest uniform in ``bulk``."""
    lo = rng.uniform(low[0], low[1], size=n_low)
    hi = rng.uniform(bulk[0], bulk[1], size=n - n_low)
    return np.sort(np.concatenate([lo, hi]))


def hermitian_from_spectrum(lam, q):
    """H = Q diag(lam) Q^H, exactly Hermitian after (H + H^H)/2.  Works on
    numpy arrays and on torch tensors."""
    if isinstance(q, np.ndarray):
        h = (q * np.asarray(lam)[None, :]) @ q.conj().T
        return 0.5 * (h + h.conj().T)
    import torch
    lam_t = torch.as_tensor(np.asarray(lam), dtype=torch.float64, device=q.device)
    h = (q * lam_t.unsqueeze(0)) @ q.conj().T
    return 0.5 * (h + h.conj().T)


def random_hermitian(n: int, rng, device=None):
    """A = (G + G^H) / (2 sqrt(2n)), G complex Ginibre: ||A||_2 ~ 2."""
    g = ginibre(n, n, rng)
    a = (g + g.conj().T) / (2.0 * math.sqrt(2.0 * n))
    if device is None:
        return a
    import torch
    return torch.from_numpy(a).to(device)


def unitary_exp(a, eps: float, order: int = 8):
    """U = exp(i eps A) by the Taylor series to ``order`` (Horner form)."""
    if isinstance(a, np.ndarray):
        eye = np.eye(a.shape[0], dtype=np.complex128)
    else:
        import torch
        eye = torch.eye(a.shape[0], dtype=torch.complex128, device=a.device)
    x = 1j * eps * a
    u = eye.copy() if isinstance(a, np.ndarray) else eye.clone()
    for j in range(order, 0, -1):
        u = eye + (x @ u) / j
    return u


def correlated_step(h, rng, eps: float, delta: float):
    """H' = U H U^H + delta * diag(d), Hermitianised."""
    n = h.shape[0]
    dev = None if isinstance(h, np.ndarray) else h.device
    a = random_hermitian(n, rng, device=dev)
    u = unitary_exp(a, eps)
    d = rng.standard_normal(n)
    if dev is None:
        h2 = u @ h @ u.conj().T
        h2 = h2 + delta * np.diag(d)
        return 0.5 * (h2 + h2.conj().T)
    import torch
    h2 = u @ h @ u.conj().T
    h2 = h2 + delta * torch.diag(torch.from_numpy(d).to(dev).to(torch.complex128))
    return 0.5 * (h2 + h2.conj().T)


def random_block(n: int, k: int, seed: int, device=None):
    """Complex Gaussian starting block X0 (n x k), column-major friendly."""
    x = ginibre(n, k, _rng(seed))
    if device is None:
        return x
    import torch
    return torch.from_numpy(x).to(device)


def config_problem(cfg: Config, seed: int, n: int | None = None, device=None):
    """First problem of a workload: (H, lam) with H = Q diag(lam) Q^H.

    ``n`` overrides the size (the spectrum layout scales with it)."""
    n = cfg.n if n is None else n
    rng = _rng(seed)
    if cfg.n == 0:  # per-problem sizes (batched): nev = n/16, nex = nev/4
        nev = max(1, n // 16)
        n_low = nev + max(1, nev // 4) // 2
    elif n == cfg.n:
        n_low = cfg.n_low
    else:
        n_low = max(1, int(round(cfg.n_low * n / cfg.n)))
    lam = two_band_spectrum(n, n_low, cfg.low, cfg.bulk, rng)
    q = haar_unitary(n, rng, device=device)
    return hermitian_from_spectrum(lam, q), lam


def config_sequence(cfg: Config, seed: int, length: int | None = None,
                    n: int | None = None, eps: float | None = None,
                    delta: float | None = None, device=None):
    """Correlated sequence H_1..H_N (Definitions 1 and 2 of Sec. 2.2).

    Returns (list of H, lam of H_1).  With delta = 0 every H_l has exactly
    the spectrum lam (U is unitary to ~1e-25), which pins sequence
    results against a known spectrum."""
    length = cfg.length if length is None else length
    eps = cfg.eps if eps is None else eps
    delta = cfg.delta if delta is None else delta
    h, lam = config_problem(cfg, seed, n=n, device=device)
    rng = _rng(seed + 7)
    hs = [h]
    for _ in range(length - 1):
        hs.append(correlated_step(hs[-1], rng, eps, delta))
    return hs, lam


def circulant_sequence(cfg: Config, seed: int, length: int = 2, eps: float | None = None,
                       device=None):
    """A cheap correlated sequence with an exactly known spectrum at the full
    sizes, where a Haar eigenbasis would cost minutes of FP64 matmuls.

    H_1 = D C D^H: C the Hermitian circulant whose eigenvalues are the
    workload's spectrum lam (first column = FFT of lam / n; eigenvectors the
    Fourier modes, dense and delocalised), D a diagonal of random phases.
    H_{l+1} = E_l H_l E_l^H with E_l = diag(exp(i eps theta)), theta ~ N(0, 1):
    same spectrum, eigenvectors turned by ~eps.  Returns (list of H as torch
    complex128 tensors on ``device``, lam ascending)."""
    import torch
    eps = cfg.eps if eps is None else eps
    n = cfg.n
    rng = _rng(seed)
    lam = two_band_spectrum(n, cfg.n_low, cfg.low, cfg.bulk, rng)
    perm = rng.permutation(n)  # spread the wanted eigenvalues over the Fourier modes
    col = np.fft.ifft(lam[perm])  # C[r, s] = col[(r - s) mod n]
    phase = np.exp(2j * np.pi * rng.uniform(size=n))
    col_t = torch.from_numpy(col).to(device)
    idx = (torch.arange(n, device=device).unsqueeze(1) - torch.arange(n, device=device).unsqueeze(0)) % n
    h = col_t[idx]
    del idx
    d = torch.from_numpy(phase).to(device)
    h = d.unsqueeze(1) * h * d.conj().unsqueeze(0)
    h = 0.5 * (h + h.conj().T)
    hs = [h]
    for _ in range(length - 1):
        e = torch.from_numpy(np.exp(1j * eps * rng.standard_normal(n))).to(device)
        h = e.unsqueeze(1) * hs[-1] * e.conj().unsqueeze(0)
        hs.append(0.5 * (h + h.conj().T))
    return hs, lam


def circulant_window(cfg: Config, seed: int, first: int, count: int, n: int, device=None,
                     eps: float | None = None):
    """Problems first .. first + count - 1 of a correlated circulant
    sequence of size n, made directly (each step is one elementwise pass,
    so a window of a long sequence costs no more than the window):

    H_l = Phi_l C Phi_l^H, Hermitianised, with C the Hermitian circulant of
    the workload's spectrum (two bands; n_low = nev + nex/2 with nev = n/16,
    nex = nev/4 for the per-problem-size workloads) and Phi_l =
    diag(phi_0 prod_{i<=l} exp(i eps theta_i)), theta_i ~ N(0, 1): every H_l
    has the spectrum lam exactly, eigenvectors turned by ~eps per step.
    Returns (list of H as torch complex128 tensors on ``device``, lam)."""
    import torch
    eps = cfg.eps if eps is None else eps
    rng = _rng(seed)
    if cfg.n == 0:
        nev = max(1, n // 16)
        n_low = nev + max(1, nev // 4) // 2
    else:
        n_low = cfg.n_low if n == cfg.n else max(1, int(round(cfg.n_low * n / cfg.n)))
    lam = two_band_spectrum(n, n_low, cfg.low, cfg.bulk, rng)
    perm = rng.permutation(n)
    col = np.fft.ifft(lam[perm])
    phi = np.exp(2j * np.pi * rng.uniform(size=n))
    col_t = torch.from_numpy(col).to(device)
    idx = (torch.arange(n, device=device).unsqueeze(1) - torch.arange(n, device=device).unsqueeze(0)) % n
    c = col_t[idx]
    del idx
    out = []
    for l in range(first + count):
        if l > 0:
            phi = phi * np.exp(1j * eps * rng.standard_normal(n))
        if l >= first:
            d = torch.from_numpy(phi).to(device)
            h = d.unsqueeze(1) * c * d.conj().unsqueeze(0)
            out.append(0.5 * (h + h.conj().T))
    del c
    return out, lam
