"""Whole solves at the full sizes of the n = 8192 and n = 13000 sequence
workloads (nev + nex = 640 and 1000), in the launch configuration the bench
times (tensor-core filter, tensor-core FP64 products), on a two-problem
sequence with an exactly known spectrum (circulant construction, see
``workloads.synthetic.circulant_sequence``).  The oracle cannot run at these
sizes; the checks are the properties that hold at any size: eigenvalues
against the known spectrum to 1e-12 ||H||, residuals <= 1e-10 ||H||, an
orthonormal block."""
import numpy as np
import pytest
import torch

from paper_1404_4161_gb300 import _lib as L
from paper_1404_4161_gb300.solver import Chfsi, colmajor
from tests.gpu_util import DEV
from workloads.synthetic import BASE_SEED, WORKLOADS, circulant_sequence, random_block

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["seq30_n8192", "seq20_n13000"])
def test_full_size_sequence_known_spectrum(name):
    from paper_1404_4161_gb300.build import build
    build()
    cfg = WORKLOADS[name]
    n, nev, nex = cfg.n, cfg.nev, cfg.nex
    k = nev + nex
    hs, lam = circulant_sequence(cfg, BASE_SEED + 7000, length=2, device=DEV)
    Hc = [colmajor(h) for h in hs]
    del hs
    Xc = colmajor(torch.from_numpy(random_block(n, k, BASE_SEED + 7500)).to(DEV))
    # correctness at full size, not loop counts: the n = 13000 warm solve
    # needed 50 loops (the products' error sits close to the 1e-10 target)
    s = Chfsi(precision=L.PREC_TC, f64_gemm=L.GEMM_OZAKI, max_loops=150)
    ev, sts, rc = s.solve_sequence(Hc, nev, nex, Xc, cfg.tol)
    s.close()
    assert rc == L.OK
    normH = float(np.abs(lam).max())
    ev = ev.cpu().numpy()
    for l, st in enumerate(sts):
        assert st["status"] == L.OK
        err = np.abs(ev[l, :nev] - lam[:nev]).max()
        print(f"{name} problem {l}: loops {st['loops']}, max |lambda - exact| {err:.2e}")
        assert err <= 1e-12 * normH
    H = Hc[-1].t()  # H Hermitian: the transpose of its column-major copy
    X = Xc.t()      # n x k
    R = torch.linalg.vector_norm(H @ X[:, :nev] - X[:, :nev] * torch.from_numpy(ev[-1, :nev]).to(DEV),
                                 dim=0) / normH
    assert float(R.max()) <= cfg.tol
    G = X.conj().T @ X
    assert float((G - torch.eye(k, dtype=G.dtype, device=DEV)).abs().max()) < 1e-12
