"""Generalized problems A c = lam B c (Sec. 3: the reduction to standard
form before Alg. 1) through chfsi_solve_generalized, against the exact
generalized spectrum, the oracle's chfsi_generalized and LAPACK's zhegvd;
B-orthonormal eigenvectors, generalized residuals; a two-problem sequence
whose second problem starts from the first one's standard-form Ritz
vectors, as the paper's sequences do."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_1404_4161_gb300 import _lib as L
from paper_1404_4161_gb300.solver import Chfsi
from tests.gpu_util import from_dev_cm, to_dev_cm
from tests.test_oracle_solve import generalized_known
from workloads.synthetic import random_block

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("engine", [L.GEMM_FP64, L.GEMM_OZAKI])
def test_generalized_known_spectrum(engine):
    from paper_1404_4161_gb300.build import build
    build()
    n, nev, nex = 512, 32, 16
    A, B, lam = generalized_known(n, 77, n_low=40)
    X0 = random_block(n, nev + nex, 78)
    prec = L.PREC_FP64 if engine == L.GEMM_FP64 else L.PREC_TC
    s = Chfsi(precision=prec, f64_gemm=engine)
    Xc = to_dev_cm(X0)
    ev, Cc, st, rc = s.solve_generalized(to_dev_cm(A), to_dev_cm(B), nev, nex, Xc, 1e-10)
    assert rc == L.OK
    ev = ev.cpu().numpy()
    scale = np.abs(lam).max()
    assert np.abs(ev[:nev] - lam[:nev]).max() <= 1e-12 * scale
    w = sla.eigh(A, B, eigvals_only=True)
    assert np.abs(ev[:nev] - w[:nev]).max() <= 1e-12 * scale
    ref = oracle.chfsi_generalized(A, B, nev, nex, X0, 1e-10)
    assert np.abs(ev[:nev] - ref["evals"][:nev]).max() <= 1e-12 * scale
    Cm = from_dev_cm(Cc)[:, :nev]
    assert np.abs(Cm.conj().T @ B @ Cm - np.eye(nev)).max() < 1e-11
    R = np.linalg.norm(A @ Cm - (B @ Cm) * ev[None, :nev], axis=0)
    assert R.max() <= 1e-10 * (np.linalg.norm(A, 2) + scale * np.linalg.norm(B, 2))
    # warm second problem: same pair perturbed (A + 1e-4 diag), start from Y
    A2 = A + 1e-4 * np.diag(np.random.Generator(np.random.PCG64(79)).standard_normal(n))
    ev2, Cc2, st2, rc2 = s.solve_generalized(to_dev_cm(A2), to_dev_cm(B), nev, nex, Xc, 1e-10,
                                             warm=(float(ev[0]), float(ev[-1])))
    s.close()
    assert rc2 == L.OK and st2["loops"] < st["loops"]
    w2 = sla.eigh(A2, B, eigvals_only=True)
    assert np.abs(ev2.cpu().numpy()[:nev] - w2[:nev]).max() <= 1e-12 * scale
    print(f"engine {engine}: loops cold {st['loops']}, warm {st2['loops']}")


def test_generalized_rejects_indefinite_b():
    from paper_1404_4161_gb300.build import build
    build()
    n = 64
    A, B, lam = generalized_known(n, 5)
    B = B - 10.0 * np.eye(n)  # indefinite
    s = Chfsi()
    ev, Cc, st, rc = s.solve_generalized(to_dev_cm(A), to_dev_cm(B), 4, 4,
                                         to_dev_cm(random_block(n, 8, 6)), 1e-10,
                                         allow=(L.EBREAKDOWN,))
    s.close()
    assert rc == L.EBREAKDOWN
