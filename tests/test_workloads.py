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


def test_circulant_window_has_the_spectrum_and_matches_its_windows():
    """A window of the direct circulant sequence is Hermitian with exactly the
    workload's spectrum, and problem l is the same whichever window holds it."""
    import torch
    from workloads.synthetic import WORKLOADS, circulant_window
    cfg = WORKLOADS["batched64"]
    hs, lam = circulant_window(cfg, 77, 0, 3, 96)
    hs2, lam2 = circulant_window(cfg, 77, 2, 1, 96)
    assert np.array_equal(lam, lam2)
    assert torch.equal(hs[2], hs2[0])
    for h in hs:
        a = h.numpy()
        assert np.abs(a - a.conj().T).max() == 0.0
        assert np.abs(np.linalg.eigvalsh(a) - lam).max() < 1e-12 * np.abs(lam).max()
    nev = 96 // 16
    assert (lam < 0).sum() == nev + max(1, nev // 4) // 2
