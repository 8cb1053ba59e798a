"""Plain FP64 ChFSI (Algorithm 1) with the Chebyshev filter (Algorithm 2).

TEST INFRASTRUCTURE: imported only by tests, the smoke check and the
benchmark's CPU baseline.  Every function cites the passage of the paper
(arXiv 1404.4161, Sec. 3) that it follows.  Readings of passages that are
garbled, ambiguous or silent are stated where they are used:

R1  Alg. 2 writes the second term of the three-term update with Y_i; the
    recurrence of Eq. (3term) needs Y_{i-1}.  Y_{i-1} is used.
R2  Alg. 2 indexes columns "s:n" and uses I_N; the columns are 1..k and
    the identity is I_n.  s is the first column (in ascending-degree
    order) whose degree exceeds the step just taken.
R3  The paper's block has nev columns and takes alpha = lambda_{nev+1}.
    Here the block has nev + nex columns; alpha is the largest Ritz value
    of the active block.  With no previous Ritz values (random start),
    gamma = smallest Lanczos Ritz value and alpha = gamma + (beta -
    gamma) * (nev + nex) / n.
R4  The Lanczos upper bound is theta_max + ||f|| (largest Ritz value of
    the Lanczos tridiagonal plus the norm of the last residual vector).
R5  Degree rule: the paper's "m_i >~ ln(Res/tol)/ln|rho_i|" is read as
    m_i = ceil(ln(r_i / tol) / acosh|t_i|) + deg_extra (deg_extra = 1,
    one degree of margin on the "at least about"), t_i = (lam_i - c)/e,
    clamped to [deg_min, deg_max]; |t_i| <= 1 gives deg_max.
    Columns outside the wanted set (the nex buffer) are capped at the
    largest degree of the wanted columns.
R6  Residuals are ||H y - lam y||_2 / ||H||_est with ||H||_est =
    max(|theta_max|, |theta_min|), the extreme Lanczos Ritz values; both
    lie inside the spectrum, so ||H||_est <= ||H||_2 and a residual that
    passes here also passes against the exact norm.
R7  Out-of-order locking: an active pair is locked when its residual is
    <= tol and its position in the ascending active block is below
    nev - n_locked.
"""
from __future__ import annotations

import math

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


# ----------------------------------------------------------------------
# Chebyshev polynomials (Sec. 3.2, Definition of C_m, Eq. (polydef))
# ----------------------------------------------------------------------
def chebyshev_value(m: int, t):
    """C_m(t) = cos(m acos t) on [-1, 1] and cosh(m acosh|t|) sign(t)^m
    outside it (Eq. (polydef) and the cos form below it)."""
    t = np.asarray(t, dtype=np.float64)
    out = np.empty_like(t)
    inside = np.abs(t) <= 1.0
    out[inside] = np.cos(m * np.arccos(t[inside]))
    ti = t[~inside]
    out[~inside] = np.cosh(m * np.arccosh(np.abs(ti))) * np.sign(ti) ** m
    return out


def chebyshev_sigmas(m: int, gamma_hat: float) -> np.ndarray:
    """sigma_1..sigma_m of Alg. 2: sigma_1 = 1/gamma_hat after the shift
    and scale to (H - cI)/e, sigma_{i+1} = 1 / (2/sigma_1 - sigma_i)."""
    s = np.empty(m)
    s[0] = 1.0 / gamma_hat
    for i in range(1, m):
        s[i] = 1.0 / (2.0 / s[0] - s[i - 1])
    return s


def convergence_ratio(t):
    """tau = |rho|^{-1} of Eq. (ratio): the smaller of |t +- sqrt(t^2-1)|
    for |t| > 1, i.e. |t| - sqrt(t^2 - 1); 1 inside [-1, 1]."""
    t = np.abs(np.asarray(t, dtype=np.float64))
    out = np.ones_like(t)
    o = t > 1.0
    out[o] = t[o] - np.sqrt(t[o] ** 2 - 1.0)
    return out


# ----------------------------------------------------------------------
# Counter-based generator for the Lanczos start vector
# ----------------------------------------------------------------------
def splitmix64(seed: int, count: int) -> np.ndarray:
    """SplitMix64 outputs 0..count-1 for ``seed`` (Steele, Lea, Flood,
    OOPSLA 2014): state_t = seed + (t+1)*0x9E3779B97F4A7C15, then the
    published 64-bit finaliser."""
    with np.errstate(over="ignore"):
        t = np.arange(1, count + 1, dtype=np.uint64)
        z = np.uint64(seed) + t * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def lanczos_start(n: int, seed: int) -> np.ndarray:
    """Start vector v0 (unnormalised): entry j = u(2j) + i u(2j+1), with
    u(t) = 2 * (splitmix64_t >> 11) * 2^-53 - 1 uniform in [-1, 1)."""
    z = splitmix64(seed, 2 * n)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53) * 2.0 - 1.0
    return u[0::2] + 1j * u[1::2]


# ----------------------------------------------------------------------
# Alg. 1: Lanczos estimate of the spectral bounds
# ----------------------------------------------------------------------
def lanczos_bounds(H: np.ndarray, steps: int, v0: np.ndarray) -> dict:
    """A few Lanczos steps (Alg. 1, Sec. 3.1 and footnote of
    Sec. 3.2) with full reorthogonalisation (classical Gram-Schmidt,
    applied twice).  Returns beta = theta_max + ||f|| (reading R4), the
    smallest Ritz value theta_min and ||H||_est (R6)."""
    n = H.shape[0]
    s = min(steps, n)
    V = np.zeros((n, s + 1), dtype=np.complex128)
    V[:, 0] = v0 / np.linalg.norm(v0)
    a = np.zeros(s)
    b = np.zeros(s)
    used = s
    for j in range(s):
        w = H @ V[:, j]
        a[j] = np.real(np.vdot(V[:, j], w))
        w = w - a[j] * V[:, j]
        if j > 0:
            w = w - b[j - 1] * V[:, j - 1]
        for _ in range(2):
            w = w - V[:, : j + 1] @ (V[:, : j + 1].conj().T @ w)
        b[j] = np.linalg.norm(w)
        if b[j] <= 1e-14 * max(abs(a[j]), 1.0):
            used = j + 1
            break
        V[:, j + 1] = w / b[j]
    T = np.diag(a[:used]) + np.diag(b[: used - 1], 1) + np.diag(b[: used - 1], -1)
    theta = np.linalg.eigvalsh(T)
    beta = theta[-1] + b[used - 1]
    return {
        "beta": float(beta),
        "theta_min": float(theta[0]),
        "theta_max": float(theta[-1]),
        "f_norm": float(b[used - 1]),
        "norm_h": float(max(abs(theta[-1]), abs(theta[0]))),
        "steps": used,
    }


def cold_interval(bounds: dict, n: int, k: int) -> tuple:
    """(alpha, gamma) when no previous Ritz values exist (reading R3).
    Parity unpinned: the paper gives no rule for this case."""
    gamma = bounds["theta_min"]
    alpha = gamma + (bounds["beta"] - gamma) * k / n
    return alpha, gamma


# ----------------------------------------------------------------------
# Alg. 2: the Chebyshev filter with per-column degrees
# ----------------------------------------------------------------------
def chebyshev_filter(H, Y0, degrees, lam1: float, c: float, e: float):
    """Alg. 2 with readings R1 and R2.

    Y0's columns are sorted by ascending degree (m_j >= 1).  Each column j
    of the result equals C_{m_j}(Hs) Y0_j / C_{m_j}(gamma_hat), Hs =
    (H - cI)/e, gamma_hat = (lam1 - c)/e.  The shift and scale are
    applied to each product rather than to H, so H is left untouched."""
    m = np.asarray(degrees, dtype=np.int64)
    k = Y0.shape[1]
    if k == 0:
        return Y0.copy()
    if np.any(m < 1) or np.any(np.diff(m) < 0):
        raise ValueError("degrees must be >= 1 and ascending")

    def hs(Y):  # (H - cI)/e applied to a block
        return (H @ Y - c * Y) / e

    sigma1 = e / (lam1 - c)
    sigma = sigma1
    y_prev = Y0
    y_cur = sigma1 * hs(Y0)  # first degree: Y_1
    out = np.empty_like(Y0)
    s = int(np.searchsorted(m, 1, side="right"))  # first column with m_j > 1
    out[:, :s] = y_cur[:, :s]
    for i in range(1, int(m[-1])):  # builds Y_{i+1}
        sigma_next = 1.0 / (2.0 / sigma1 - sigma)
        y_next = y_cur.copy()  # finished columns carried over
        y_next[:, s:] = (2.0 * sigma_next * hs(y_cur[:, s:])
                         - sigma_next * sigma * y_prev[:, s:])  # reading R1
        y_prev, y_cur, sigma = y_cur, y_next, sigma_next
        s_new = int(np.searchsorted(m, i + 1, side="right"))  # columns finished at degree i+1
        out[:, s:s_new] = y_cur[:, s:s_new]
        s = s_new
    return out


# ----------------------------------------------------------------------
# Alg. 1, QR step: orthonormalise [Y_locked, Y] (Householder QR)
# ----------------------------------------------------------------------
def orthonormalize(Y, locked=None):
    """Householder QR (LAPACK zgeqrf via numpy) of [locked, Y], as in
    Alg. 1 (QR step) and Sec. 3.1.  Returns the columns of Q that belong to
    Y, with phases fixed so that the corresponding diagonal of R is real
    and positive (which makes Q unique)."""
    nl = 0 if locked is None else locked.shape[1]
    A = Y if nl == 0 else np.concatenate([locked, Y], axis=1)
    Q, R = np.linalg.qr(A)
    d = np.diag(R)[nl:]
    ph = d / np.abs(d)
    return Q[:, nl:] * ph[None, :]


# ----------------------------------------------------------------------
# Alg. 1: Rayleigh-Ritz
# ----------------------------------------------------------------------
def rayleigh_ritz(H, Q):
    """G = Q^H H Q (Hermitianised), G W = W Lambda by LAPACK's Hermitian
    eigensolver (ascending), Y = Q W; also returns H Y = (H Q) W
    (Alg. 1, Sec. 3.1)."""
    HQ = H @ Q
    G = Q.conj().T @ HQ
    G = 0.5 * (G + G.conj().T)
    lam, W = np.linalg.eigh(G)
    return lam, Q @ W, HQ @ W


def residuals(HY, Y, lam, norm_h: float):
    """r_j = ||H y_j - lam_j y_j||_2 / ||H||_est (Sec. 3.1, reading R6)."""
    return np.linalg.norm(HY - Y * lam[None, :], axis=0) / norm_h


# ----------------------------------------------------------------------
# Alg. 1: locking and degree optimisation
# ----------------------------------------------------------------------
def lock_mask(resid, n_wanted_left: int, tol: float):
    """Pairs to lock (reading R7): residual <= tol and ascending position
    below nev - n_locked; convergence may be out of order (Sec. 4)."""
    r = np.asarray(resid)
    return (np.arange(r.size) < n_wanted_left) & (r <= tol)


def degree_rule(ritz, resid, c: float, e: float, tol: float, deg_max: int,
                n_wanted: int | None = None, deg_min: int = 1, deg_extra: int = 1):
    """Single Optimization (Sec. 3.2, the inequality after Eq. (resl)):
    m_i >= ln(Res_i / tol) / ln|rho_i|, ln|rho_i| = acosh|t_i|, t_i =
    (lam_i - c)/e (Eq. (ratio)).  Reading R5 for rounding, clamps and the
    buffer columns beyond ``n_wanted``."""
    lam = np.asarray(ritz, dtype=np.float64)
    r = np.asarray(resid, dtype=np.float64)
    t = np.abs((lam - c) / e)
    m = np.full(lam.size, deg_max, dtype=np.int64)
    out = t > 1.0
    with np.errstate(divide="ignore"):
        ratio = np.log(r[out] / tol) / np.arccosh(t[out])
    m[out] = np.ceil(ratio).astype(np.int64) + deg_extra if ratio.size else m[out]
    m = np.clip(m, deg_min, deg_max)
    if n_wanted is not None and 0 < n_wanted < m.size:
        m[n_wanted:] = np.minimum(m[n_wanted:], m[:n_wanted].max())
    return m


# ----------------------------------------------------------------------
# Alg. 1: ChFSI on one problem
# ----------------------------------------------------------------------
def chfsi(H, nev: int, nex: int, X0, tol: float, *, deg: int | None = None,
          deg_max: int = 36, lanczos_steps: int = 20, max_loops: int = 50,
          seed: int = 1, warm: tuple | None = None, degree_fn=None,
          trace: list | None = None) -> dict:
    """Alg. 1 for one Hermitian H (n x n), block of nev + nex columns.

    warm = (lam_1, lam_k) of the previous problem in a sequence (Alg. 1
    Require line) or None for a random start (reading R3).  ``degree_fn``
    may replace the degree rule (same arguments as ``degree_rule``).
    ``trace`` (a list) receives one dict per loop."""
    n = H.shape[0]
    k = nev + nex
    if nex < 1 or nev < 1 or k > n or X0.shape != (n, k):
        raise ValueError("bad sizes")
    bnd = lanczos_bounds(H, lanczos_steps, lanczos_start(n, seed))
    beta, norm_h = bnd["beta"], bnd["norm_h"]
    if warm is None:
        alpha, gamma = cold_interval(bnd, n, k)
        deg0 = 20 if deg is None else deg
    else:
        gamma, alpha = float(warm[0]), float(warm[1])
        deg0 = 8 if deg is None else deg
    rule = degree_rule if degree_fn is None else degree_fn

    Y = np.array(X0, dtype=np.complex128)
    lockY = np.zeros((n, 0), dtype=np.complex128)
    lockL = np.zeros(0)
    lockR = np.zeros(0)
    m = np.full(k, deg0, dtype=np.int64)
    lam = np.zeros(k)
    r = np.ones(k)
    col_deg = 0
    loops = 0
    status = "ENOCONV"
    while loops < max_loops:
        loops += 1
        c, e = 0.5 * (alpha + beta), 0.5 * (beta - alpha)
        order = np.argsort(m, kind="stable")  # Sec. 4: ascending degrees
        Yf = chebyshev_filter(H, Y[:, order], m[order], gamma, c, e)
        col_deg += int(m.sum())
        Q = orthonormalize(Yf, lockY if lockY.shape[1] else None)
        lam, Y, HY = rayleigh_ritz(H, Q)
        r = residuals(HY, Y, lam, norm_h)
        n_left = nev - lockY.shape[1]
        lk = lock_mask(r, n_left, tol)
        if trace is not None:
            trace.append({"loop": loops, "c": c, "e": e, "gamma": gamma,
                          "alpha": alpha, "beta": beta, "degrees": m.copy(),
                          "ritz": lam.copy(), "resid": r.copy(),
                          "n_locked": lockY.shape[1], "locked_now": int(lk.sum())})
        lockY = np.concatenate([lockY, Y[:, lk]], axis=1)
        lockL = np.concatenate([lockL, lam[lk]])
        lockR = np.concatenate([lockR, r[lk]])
        Y, lam, r = Y[:, ~lk], lam[~lk], r[~lk]
        gamma = min(gamma, float(lam[0]) if lam.size else gamma,
                    float(lockL.min()) if lockL.size else gamma)
        if lockY.shape[1] >= nev:
            status = "OK"
            break
        alpha = float(lam[-1])  # R3: largest Ritz value of the active block
        c, e = 0.5 * (alpha + beta), 0.5 * (beta - alpha)
        m = rule(lam, r, c, e, tol, deg_max, n_wanted=nev - lockY.shape[1])
    srt = np.argsort(lockL, kind="stable")
    X = np.concatenate([lockY[:, srt], Y], axis=1)
    evals = np.concatenate([lockL[srt], lam])
    resid = np.concatenate([lockR[srt], r])
    return {"evals": evals, "X": X, "resid": resid, "loops": loops,
            "filter_col_degrees": col_deg, "status": status,
            "n_locked": int(lockY.shape[1]), "beta": beta, "norm_h": norm_h,
            "lanczos": bnd}


def chfsi_sequence(Hs, nev: int, nex: int, X0, tol: float, **kw) -> list:
    """Solve a sequence (Definition 1): problem l+1 starts from problem
    l's nev + nex Ritz vectors, with gamma = lam_1 and alpha = lam_k of
    problem l (Alg. 1 Require line; Sec. 2.2 warm start)."""
    out = []
    X = X0
    warm = None
    for H in Hs:
        res = chfsi(H, nev, nex, X, tol, warm=warm, **kw)
        out.append(res)
        X = res["X"]
        warm = (res["evals"][0], res["evals"][-1])
    return out


# ----------------------------------------------------------------------
# Sec. 3 (the problem statement before Alg. 1): generalized problems
# ----------------------------------------------------------------------
def chfsi_generalized(A, B, nev: int, nex: int, X0, tol: float, **kw) -> dict:
    """A c = lambda B c with A Hermitian and B Hermitian positive definite:
    the input of Alg. 1 is the reduction to standard form H = L^-1 A L^-H,
    B = L L^H (Cholesky), whose eigenvectors Y give c = L^-H Y.  X0 is a
    starting block of H (in a sequence, the previous problem's Y).
    Returns chfsi's dict plus "C" = L^-H X (B-orthonormal)."""
    import scipy.linalg as sla
    L = np.linalg.cholesky(np.asarray(B, dtype=np.complex128))
    T = sla.solve_triangular(L, np.asarray(A, dtype=np.complex128), lower=True)  # L^-1 A
    H = sla.solve_triangular(L, T.conj().T, lower=True).conj().T                  # T L^-H
    H = 0.5 * (H + H.conj().T)
    res = chfsi(H, nev, nex, X0, tol, **kw)
    res["C"] = sla.solve_triangular(L.conj().T, res["X"], lower=False)            # L^-H Y
    res["H"] = H
    return res
