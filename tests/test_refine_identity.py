"""CPU check of the refinement ("defect") form used by the tensor-core
filter: for Ritz pairs (Y, Lambda) and R = HY - Y Lambda, the filter of
Alg. 2 satisfies p_m(H) Y = Y psi_m(Lambda) + D_m with D_0 = 0, D_1 = a_0 R,
D_{i+1} = a_i (H D_i - c D_i) + b_i D_{i-1} + a_i psi_i(Lambda) R.
This pins the algebra the CUDA path relies on against the oracle filter."""
import numpy as np

import oracle
from workloads.synthetic import haar_unitary, hermitian_from_spectrum, random_block


def defect_filter(H, Y, lam, degrees, lam1, c, e, norms=None):
    """FP64 refinement-form filter; if ``norms`` is a list it receives, per
    column, sum over the steps taken of ||D_i|| (i = 1 .. m_j - 1)."""
    n, k = Y.shape
    R = H @ Y - Y * lam[None, :]
    m = np.asarray(degrees)
    mk = int(m[-1])
    s1 = e / (lam1 - c)
    a = [s1 / e]
    b = [0.0]
    sig = s1
    for i in range(1, mk):
        sn = 1.0 / (2.0 / s1 - sig)
        a.append(2 * sn / e)
        b.append(-sn * sig)
        sig = sn
    psi = [np.ones(k), a[0] * (lam - c)]
    for i in range(1, mk):
        psi.append(a[i] * (lam - c) * psi[i] + b[i] * psi[i - 1])
    D_prev = np.zeros_like(Y)
    D = a[0] * R
    out = np.empty_like(Y)
    acc = np.zeros(k)
    for j in range(k):
        if m[j] == 1:
            out[:, j] = Y[:, j] * psi[1][j] + D[:, j]
    for i in range(1, mk):
        acc += np.where(m > i, np.linalg.norm(D, axis=0), 0.0)
        D_next = a[i] * (H @ D - c * D) + b[i] * D_prev + a[i] * psi[i][None, :] * R
        D_prev, D = D, D_next
        for j in range(k):
            if m[j] == i + 1:
                out[:, j] = Y[:, j] * psi[i + 1][j] + D[:, j]
    if norms is not None:
        norms.append(acc)
    return out


def test_defect_form_equals_alg2():
    rng = np.random.Generator(np.random.PCG64(3))
    n = 80
    lam_true = np.sort(np.concatenate([rng.uniform(-2, -1, 10), rng.uniform(0, 10, n - 10)]))
    q = haar_unitary(n, rng)
    H = hermitian_from_spectrum(lam_true, q)
    Q = oracle.orthonormalize(q[:, :12] + 1e-3 * random_block(n, 12, 5))
    lam, Y, _ = oracle.rayleigh_ritz(H, Q)
    deg = np.array([1, 2, 2, 3, 5, 8, 8, 13, 20, 20, 30, 36])
    c, e = 5.2, 4.9
    ref = oracle.chebyshev_filter(H, Y, deg, lam_true[0], c, e)
    got = defect_filter(H, Y, lam, deg, lam_true[0], c, e)
    err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert err.max() < 1e-11
