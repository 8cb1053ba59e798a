"""Unit parity of two control steps of Alg. 1 through the C ABI, bit-exact:
the stable ascending sort of the columns by degree (Sec. 4) against
numpy's stable argsort, and the out-of-order locking (Sec. 4, reading R7)
against the oracle's lock mask."""
import numpy as np
import pytest
import torch

import oracle
from paper_1404_4161_gb300.solver import Chfsi
from tests.gpu_util import DEV

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1404_4161_gb300.build import build
    build()
    s = Chfsi()
    yield s
    s.close()


@pytest.mark.parametrize("k,hi,seed", [(1, 3, 0), (7, 2, 1), (320, 5, 2), (1000, 3, 3),
                                       (2500, 40, 4), (1024, 1, 5)])
def test_sort_by_degree_stable(ctx, k, hi, seed):
    """Many ties (degrees from a small range), sizes around the 1024-thread
    block: the permutation equals numpy's stable argsort, element by
    element."""
    deg = np.random.Generator(np.random.PCG64(seed)).integers(1, hi + 1, k).astype(np.int32)
    perm, ds = ctx.sort_degrees(torch.from_numpy(deg).to(DEV))
    ref = np.argsort(deg, kind="stable")
    assert np.array_equal(perm.cpu().numpy(), ref)
    assert np.array_equal(ds.cpu().numpy(), deg[ref])


@pytest.mark.parametrize("ka,nw,seed", [(48, 32, 0), (320, 256, 1), (1500, 1100, 2),
                                        (1000, 0, 3), (64, 64, 4)])
def test_lock_out_of_order(ctx, ka, nw, seed):
    """Converged pairs scattered through the block (out of order), some of
    them beyond the wanted positions: the locked and active positions equal
    the oracle's mask, element by element."""
    rng = np.random.Generator(np.random.PCG64(seed))
    tol = 1e-10
    resid = 10.0 ** rng.uniform(-13, -6, ka)
    resid[rng.integers(0, ka, ka // 7)] = tol  # exactly at the tolerance: locks
    ritz = np.sort(rng.uniform(-3, 1, ka))
    li, ai = ctx.lock(torch.from_numpy(ritz).to(DEV), torch.from_numpy(resid).to(DEV), nw, tol)
    mask = oracle.lock_mask(resid, nw, tol)
    assert np.array_equal(li.cpu().numpy(), np.flatnonzero(mask))
    assert np.array_equal(ai.cpu().numpy(), np.flatnonzero(~mask))
