"""chfsi_filter_static: the FP64 filter for callers that cannot allocate
device memory on the call path (applications that hand the whole device
to their own memory pool at start-up, and latency-bound code that cannot
take cudaMalloc's implicit synchronisation).  Its scratch is a static
device array in the library, so it must give the same result as the
ordinary entry point chfsi_filter (FP64), call after call.

This file is collected last on purpose: it also runs correctly in a fresh
process on its own."""
import numpy as np
import pytest
import torch

import oracle
from paper_1404_4161_gb300 import _lib as L
from paper_1404_4161_gb300.solver import Chfsi, filter_static
from tests.gpu_util import colrel, from_dev_cm, known_problem, to_dev_cm
from workloads.synthetic import random_block

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1404_4161_gb300.build import build
    build()
    s = Chfsi()
    yield s
    s.close()


def test_static_filter_matches_context_filter_twice(ctx):
    cases = [
        (300, [1, 1, 2, 3, 5, 8, 8, 13, 21, 34] + [36] * 30, 0.2, 10.4),
        (512, list(range(1, 41)) + [40] * 8 + [45] * 4, -0.5, 11.0),  # second call: other data
    ]
    for n, degrees, alpha, beta in cases:
        assert n * len(degrees) <= L.FILTER_STATIC_MAX_NK
        H, lam, _ = known_problem(n, 900 + n)
        Y0 = random_block(n, len(degrees), 901 + n)
        c, e = 0.5 * (alpha + beta), 0.5 * (beta - alpha)
        Hc, Y0c = to_dev_cm(H), to_dev_cm(Y0)
        ref = ctx.filter(Hc, Y0c, degrees, lam[0], c, e, precision=L.PREC_FP64)
        got, rc = filter_static(Hc, Y0c, degrees, lam[0], c, e)
        torch.cuda.synchronize()
        assert rc == L.OK
        got_np, ref_np = from_dev_cm(got), from_dev_cm(ref)
        assert colrel(got_np, ref_np) < 1e-12
        oracle_ref = oracle.chebyshev_filter(H, Y0, degrees, lam[0], c, e)
        assert colrel(got_np, oracle_ref) < 1e-12


def test_static_filter_rejects_sizes_beyond_the_limit():
    from paper_1404_4161_gb300.build import build
    build()
    n, k = 1024, L.FILTER_STATIC_MAX_NK // 1024 + 1
    dev = torch.device("cuda:0")
    Hc = torch.zeros((n, n), dtype=torch.complex128, device=dev)
    Y0c = torch.zeros((k, n), dtype=torch.complex128, device=dev)
    out, rc = filter_static(Hc, Y0c, [1] * k, -1.0, 5.0, 4.0)
    assert rc == L.ETOOBIG
    assert L.lib().chfsi_strerror(rc).startswith(b"n*k exceeds")


def test_static_filter_fills_the_array_on_another_stream():
    """n * k equal to the limit (the third buffer ends at the array's last
    element), mixed degrees, issued on a non-default stream: same result as
    chfsi_filter on that stream, twice in a row."""
    n, k = 1024, L.FILTER_STATIC_MAX_NK // 1024
    assert n * k == L.FILTER_STATIC_MAX_NK
    degrees = sorted(np.random.Generator(np.random.PCG64(11)).integers(1, 16, k).tolist())
    H, lam, _ = known_problem(n, 1900)
    Y0 = random_block(n, k, 1901)
    alpha, beta = 0.3, 10.5
    c, e = 0.5 * (alpha + beta), 0.5 * (beta - alpha)
    Hc, Y0c = to_dev_cm(H), to_dev_cm(Y0)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        s2 = Chfsi()  # bound to the side stream
        ref = s2.filter(Hc, Y0c, degrees, lam[0], c, e, precision=L.PREC_FP64)
        torch.cuda.current_stream().synchronize()
        for _ in range(2):
            got, rc = filter_static(Hc, Y0c, degrees, lam[0], c, e)
            assert rc == L.OK
            torch.cuda.current_stream().synchronize()
            assert colrel(from_dev_cm(got), from_dev_cm(ref)) < 1e-12
        s2.close()


def test_static_filter_rejects_overlapping_output():
    from paper_1404_4161_gb300.build import build
    build()
    n, k = 64, 4
    dev = torch.device("cuda:0")
    Hc = torch.zeros((n, n), dtype=torch.complex128, device=dev)
    buf = torch.zeros((2 * k, n), dtype=torch.complex128, device=dev)
    # output starting half-way into the input block
    _, rc = filter_static(Hc, buf[:k], [1] * k, -1.0, 5.0, 4.0, out=buf[k // 2:k // 2 + k])
    assert rc == L.EINVAL
