"""Torch-facing wrapper of the C ABI (argument marshalling only).

Layout: the library takes complex128 column-major matrices.  A torch
tensor ``A`` of shape (rows, cols) is passed as ``A.t().contiguous()``
(whose row-major memory is A's column-major memory) and read back with
``.t()``.  Every call runs on torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L
from ._lib import ChfsiError, Opts, Stats  # noqa: F401


def colmajor(a: torch.Tensor) -> torch.Tensor:
    """Contiguous (cols, rows) tensor holding ``a`` column-major."""
    return a.t().contiguous()


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


class Chfsi:
    """One library context bound to the current device and stream."""

    def __init__(self, **opts):
        self.lib = L.lib()
        self.opts = L.default_opts(**opts)
        self.ctx = C.c_void_p()
        stream = torch.cuda.current_stream().cuda_stream
        rc = self.lib.chfsi_init(C.byref(self.ctx), C.byref(self.opts), C.c_void_p(stream))
        if rc != L.OK:
            raise ChfsiError(rc, self.lib.chfsi_strerror(rc).decode())

    def close(self):
        if self.ctx:
            self.lib.chfsi_free(self.ctx)
            self.ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, allow=()):
        if rc != L.OK and rc not in allow:
            raise ChfsiError(rc, self.lib.chfsi_last_error(self.ctx).decode())
        return rc

    def set_opts(self, **over):
        for k, v in over.items():
            setattr(self.opts, k, v)
        self._check(self.lib.chfsi_set_opts(self.ctx, C.byref(self.opts)))

    # -- whole solves -------------------------------------------------
    def solve(self, Hc, nev, nex, Xc, tol, warm=None, allow=(L.ENOCONV,)):
        """Hc: colmajor(H) (n, n); Xc: colmajor(X0) (k, n), overwritten."""
        n = Hc.shape[0]
        k = nev + nex
        ev = torch.empty(k, dtype=torch.float64, device=Hc.device)
        st = Stats()
        w = (C.c_double * 2)(*warm) if warm is not None else None
        rc = self.lib.chfsi_solve(self.ctx, _ptr(Hc), n, nev, nex, _ptr(Xc), tol, _ptr(ev),
                                  C.cast(w, C.c_void_p) if w is not None else None,
                                  C.byref(st))
        self._check(rc, allow)
        return ev, st.as_dict(), rc

    def solve_generalized(self, Ac, Bc, nev, nex, Xc, tol, warm=None, allow=(L.ENOCONV,)):
        """A c = lam B c: Ac, Bc colmajor (n, n); Xc colmajor starting block of
        the standard form, overwritten with its Ritz vectors.  Returns
        (evals, C colmajor (k, n), stats, rc)."""
        n = Ac.shape[0]
        k = nev + nex
        ev = torch.empty(k, dtype=torch.float64, device=Ac.device)
        Cc = torch.empty_like(Xc)
        st = Stats()
        w = (C.c_double * 2)(*warm) if warm is not None else None
        rc = self.lib.chfsi_solve_generalized(self.ctx, _ptr(Ac), _ptr(Bc), n, nev, nex, _ptr(Xc),
                                              _ptr(Cc), tol, _ptr(ev),
                                              C.cast(w, C.c_void_p) if w is not None else None,
                                              C.byref(st))
        self._check(rc, allow)
        return ev, Cc, st.as_dict(), rc

    def solve_sequence(self, Hcs, nev, nex, Xc, tol, allow=(L.ENOCONV,)):
        N = len(Hcs)
        n = Hcs[0].shape[0]
        k = nev + nex
        ptrs = (C.c_void_p * N)(*[h.data_ptr() for h in Hcs])
        ev = torch.empty((N, k), dtype=torch.float64, device=Xc.device)
        st = (Stats * N)()
        rc = self.lib.chfsi_solve_sequence(self.ctx, C.cast(ptrs, C.c_void_p), N, n, nev, nex,
                                           _ptr(Xc), tol, _ptr(ev), C.cast(st, C.c_void_p))
        self._check(rc, allow)
        return ev, [s.as_dict() for s in st], rc

    def solve_sequence_host(self, Hcs_host, nev, nex, Xc_host, tol, allow=(L.ENOCONV,)):
        """All buffers on the host (ideally pinned); copies happen inside."""
        N = len(Hcs_host)
        n = Hcs_host[0].shape[0]
        k = nev + nex
        ptrs = (C.c_void_p * N)(*[h.data_ptr() for h in Hcs_host])
        ev = torch.empty((N, k), dtype=torch.float64).pin_memory()
        st = (Stats * N)()
        rc = self.lib.chfsi_solve_sequence_host(self.ctx, C.cast(ptrs, C.c_void_p), N, n, nev,
                                                nex, _ptr(Xc_host), tol, _ptr(ev),
                                                C.cast(st, C.c_void_p))
        self._check(rc, allow)
        return ev, [s.as_dict() for s in st], rc

    def solve_batched(self, seqs, tol, allow=(L.ENOCONV,), warm=None):
        """seqs: list of (list of Hc per step, nev, nex, Xc); all sequences
        have the same number of steps.  warm: None (random starts) or one
        (lam_1, lam_k) pair per sequence of the step that produced Xc.
        Returns (evals per problem, stats [step][problem], rc, warm pairs of
        the last step)."""
        P = len(seqs)
        steps = len(seqs[0][0])
        probs = (L.Problem * P)()
        keep, evs = [], []
        for p, (Hcs, nev, nex, Xc) in enumerate(seqs):
            ptrs = (C.c_void_p * steps)(*[h.data_ptr() for h in Hcs])
            keep.append(ptrs)
            ev = torch.empty((steps, nev + nex), dtype=torch.float64, device=Xc.device)
            evs.append(ev)
            w = warm[p] if warm is not None else (0.0, 0.0)
            probs[p] = L.Problem(C.cast(ptrs, C.c_void_p), Hcs[0].shape[0], nev, nex,
                                 Xc.data_ptr(), ev.data_ptr(), 1 if warm is not None else 0,
                                 float(w[0]), float(w[1]))
        st = (Stats * (P * steps))()
        rc = self.lib.chfsi_solve_batched(self.ctx, P, C.cast(probs, C.c_void_p), steps, tol,
                                          C.cast(st, C.c_void_p))
        self._check(rc, allow)
        stats = [[st[l * P + p].as_dict() for p in range(P)] for l in range(steps)]
        last = [(probs[p].lam_lo, probs[p].lam_hi) for p in range(P)]
        return evs, stats, rc, last

    # -- single steps -------------------------------------------------
    def lanczos(self, Hc, steps, seed):
        out = (C.c_double * 4)()
        self._check(self.lib.chfsi_lanczos(self.ctx, _ptr(Hc), Hc.shape[0], steps, seed,
                                           C.cast(out, C.c_void_p)))
        return {"beta": out[0], "theta_min": out[1], "theta_max": out[2], "norm_h": out[3]}

    def filter(self, Hc, Y0c, degrees, lam1, c, e, precision=L.PREC_FP64):
        k, n = Y0c.shape
        out = torch.empty_like(Y0c)
        d = (C.c_int * max(k, 1))(*[int(x) for x in degrees])
        self._check(self.lib.chfsi_filter(self.ctx, _ptr(Hc), n, k, _ptr(Y0c),
                                          C.cast(d, C.c_void_p), lam1, c, e, _ptr(out),
                                          precision))
        return out

    def filter_batched(self, jobs):
        """jobs: list of (Hc, Y0c, degrees, lam1, c, e); one launch for all."""
        items = (L.FilterItem * max(len(jobs), 1))()
        outs, keep = [], []
        for i, (Hc, Y0c, degrees, lam1, c, e) in enumerate(jobs):
            k, n = Y0c.shape
            out = torch.empty_like(Y0c)
            d = (C.c_int * max(k, 1))(*[int(x) for x in degrees])
            keep.append(d)
            items[i] = L.FilterItem(Hc.data_ptr(), n, k, Y0c.data_ptr(), d, lam1, c, e,
                                    out.data_ptr())
            outs.append(out)
        self._check(self.lib.chfsi_filter_batched(self.ctx, len(jobs), C.cast(items, C.c_void_p)))
        return outs

    def filter_refine(self, Hc, Yc, Rc, ritz, degrees, lam1, c, e):
        k, n = Yc.shape
        out = torch.empty_like(Yc)
        d = (C.c_int * max(k, 1))(*[int(x) for x in degrees])
        self._check(self.lib.chfsi_filter_refine(self.ctx, _ptr(Hc), n, k, _ptr(Yc), _ptr(Rc),
                                                 _ptr(ritz), C.cast(d, C.c_void_p), lam1, c, e,
                                                 _ptr(out)))
        return out

    def zgemm(self, op_a, A_cm, B_cm, m, n, k, alpha=1.0, beta=0.0, C_cm=None, engine=L.GEMM_OZAKI):
        """Column-major operands as colmajor() tensors: A_cm (cols, rows) etc."""
        if C_cm is None:
            C_cm = torch.zeros((n, m), dtype=torch.complex128, device=A_cm.device)
        self._check(self.lib.chfsi_zgemm(self.ctx, op_a, m, n, k, alpha, _ptr(A_cm),
                                         A_cm.shape[1], _ptr(B_cm), B_cm.shape[1], beta,
                                         _ptr(C_cm), C_cm.shape[1], engine))
        return C_cm

    def orthonormalize(self, Yc, Lc=None):
        k, n = Yc.shape
        nl = 0 if Lc is None else Lc.shape[0]
        self._check(self.lib.chfsi_orthonormalize(self.ctx, n, nl, _ptr(Lc), k, _ptr(Yc)))
        return Yc

    def rayleigh_ritz(self, Hc, Qc):
        k, n = Qc.shape
        Y = torch.empty_like(Qc)
        HY = torch.empty_like(Qc)
        ev = torch.empty(k, dtype=torch.float64, device=Qc.device)
        self._check(self.lib.chfsi_rayleigh_ritz(self.ctx, _ptr(Hc), n, k, _ptr(Qc), _ptr(Y),
                                                 _ptr(HY), _ptr(ev)))
        return ev, Y, HY

    def residuals(self, HYc, Yc, evals, norm_h):
        k, n = Yc.shape
        r = torch.empty(k, dtype=torch.float64, device=Yc.device)
        self._check(self.lib.chfsi_residuals(self.ctx, n, k, _ptr(HYc), _ptr(Yc), _ptr(evals),
                                             norm_h, _ptr(r)))
        return r

    def degrees(self, ritz, resid, c, e, tol, n_wanted):
        k = ritz.shape[0]
        d = torch.empty(k, dtype=torch.int32, device=ritz.device)
        self._check(self.lib.chfsi_degrees(self.ctx, k, _ptr(ritz), _ptr(resid), c, e, tol,
                                           n_wanted, _ptr(d)))
        return d

    def sort_degrees(self, deg):
        """deg: int32 device tensor -> (perm, deg_sorted)."""
        k = deg.shape[0]
        perm = torch.empty_like(deg)
        ds = torch.empty_like(deg)
        self._check(self.lib.chfsi_sort_degrees(self.ctx, k, _ptr(deg), _ptr(perm), _ptr(ds)))
        return perm, ds

    def lock(self, ritz, resid, n_wanted_left, tol):
        """-> (locked positions, active positions) as int32 device tensors."""
        ka = ritz.shape[0]
        li = torch.empty(ka, dtype=torch.int32, device=ritz.device)
        ai = torch.empty(ka, dtype=torch.int32, device=ritz.device)
        cnt = (C.c_int * 2)()
        self._check(self.lib.chfsi_lock(self.ctx, ka, _ptr(ritz), _ptr(resid), n_wanted_left,
                                        tol, _ptr(li), _ptr(ai), C.cast(cnt, C.c_void_p)))
        return li[:cnt[0]], ai[:cnt[1]]

    def autotune_table(self):
        """Tilings chosen by the filter's autotuner: list of dicts."""
        cnt = C.c_int()
        self._check(self.lib.chfsi_autotune_table(self.ctx, 0, None, C.byref(cnt)))
        n = cnt.value
        buf = (C.c_int * max(6 * n, 1))()
        self._check(self.lib.chfsi_autotune_table(self.ctx, n, C.cast(buf, C.c_void_p),
                                                  C.byref(cnt)))
        keys = ["n", "k_bucket", "pieces", "block_width", "group", "us"]
        return [dict(zip(keys, buf[6 * i:6 * i + 6])) for i in range(n)]

    # -- traces and MLP ------------------------------------------------
    def trace_enable(self, capacity_rows):
        self._check(self.lib.chfsi_trace_enable(self.ctx, int(capacity_rows)))

    def mlp_set_params(self, flat):
        f = flat.detach().to(torch.float32).contiguous().cpu()
        self._check(self.lib.chfsi_mlp_set_params(self.ctx, _ptr(f)))

    def mlp_get_params(self):
        f = torch.empty(L.MLP_NPARAM, dtype=torch.float32)
        self._check(self.lib.chfsi_mlp_get_params(self.ctx, _ptr(f)))
        return f

    def mlp_forward(self, x):
        y = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        self._check(self.lib.chfsi_mlp_forward(self.ctx, x.shape[0], _ptr(x), _ptr(y)))
        return y

    def mlp_train_step(self, x, target, lr):
        g = torch.empty(L.MLP_NPARAM, dtype=torch.float32, device=x.device)
        loss = C.c_float()
        self._check(self.lib.chfsi_mlp_train_step(self.ctx, x.shape[0], _ptr(x), _ptr(target),
                                                  lr, _ptr(g), C.byref(loss)))
        return float(loss.value), g


def filter_static(Hc, Y0c, degrees, lam1, c, e, out=None):
    """chfsi_filter_static on torch's current stream: the FP64 filter with
    its scratch in the library's static device array (no allocation by
    the library; ``out`` may be passed in to avoid one by torch).
    Returns (out, return code)."""
    lib = L.lib()
    k, n = Y0c.shape
    if out is None:
        out = torch.empty_like(Y0c)
    d = (C.c_int * max(k, 1))(*[int(x) for x in degrees])
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.chfsi_filter_static(_ptr(Hc), n, k, _ptr(Y0c), C.cast(d, C.c_void_p), lam1, c, e,
                                 _ptr(out), C.c_void_p(stream))
    return out, rc
