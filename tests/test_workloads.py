"""The input generators (CPU): the spectra they promise are the spectra
of the matrices they build, which is what the known-spectrum GPU tests
rely on."""
import dataclasses

import numpy as np
import torch

from workloads.synthetic import WORKLOADS, circulant_sequence, config_sequence


def test_circulant_sequence_has_the_stated_spectrum():
    cfg = dataclasses.replace(WORKLOADS["seq20_n13000"], n=300, n_low=40)
    hs, lam = circulant_sequence(cfg, 11, length=3, device="cpu")
    assert len(hs) == 3 and np.all(np.diff(lam) >= 0)
    normH = np.abs(lam).max()
    prev = None
    for h in hs:
        H = h.numpy()
        assert np.abs(H - H.conj().T).max() == 0.0
        assert np.abs(np.linalg.eigvalsh(H) - lam).max() <= 1e-13 * normH
        # dense, delocalised eigenvectors (no near-diagonal structure)
        w, V = np.linalg.eigh(H)
        assert np.abs(V[:, :10]).max() < 0.5
        if prev is not None:
            # the next problem is close to the previous one but not equal
            d = np.linalg.norm(H - prev) / np.linalg.norm(prev)
            assert 1e-5 < d < 1e-1
        prev = H


def test_config_sequence_keeps_spectrum_without_diagonal_term():
    cfg = WORKLOADS["single_n512"]
    hs, lam = config_sequence(cfg, 5, length=2, n=128, delta=0.0)
    for H in hs:
        assert np.abs(np.linalg.eigvalsh(H) - lam).max() <= 1e-12 * np.abs(lam).max()
