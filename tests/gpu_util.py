"""Helpers shared by the GPU parity tests (layout conversion, problem
construction).  They hold none of the method's arithmetic."""
import numpy as np
import torch

from workloads.synthetic import haar_unitary, hermitian_from_spectrum, random_block

DEV = torch.device("cuda:0") if torch.cuda.is_available() else None


def to_dev_cm(a: np.ndarray) -> torch.Tensor:
    """numpy (rows, cols) -> device tensor holding it column-major."""
    return torch.from_numpy(np.ascontiguousarray(a.T)).to(DEV)


def from_dev_cm(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().T.copy()


def known_problem(n, seed, lo=(-2.0, -1.0), bulk=(0.0, 10.0), n_low=None):
    rng = np.random.Generator(np.random.PCG64(seed))
    n_low = n_low or max(1, n // 8)
    lam = np.sort(np.concatenate([rng.uniform(*lo, n_low), rng.uniform(*bulk, n - n_low)]))
    q = haar_unitary(n, rng)
    return hermitian_from_spectrum(lam, q), lam, q


def colrel(a, b):
    """Largest column-wise relative difference ||a_j - b_j|| / ||b_j||."""
    return float((np.linalg.norm(a - b, axis=0) / np.maximum(np.linalg.norm(b, axis=0), 1e-300)).max())
