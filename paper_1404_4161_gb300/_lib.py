"""ctypes binding of libchfsi.so (the C ABI declared in include/chfsi.h).

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  Importing this module fails loudly when the library has not
been built; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

OK, EINVAL, ENOMEM, ENOCONV, EBREAKDOWN, ENAN, ETIMEOUT, ECUDA, ENOTSUP, ETOOBIG = range(10)
FILTER_STATIC_MAX_NK = 262144
PREC_FP64, PREC_MIXED, PREC_TC = 0, 1, 2
SPLIT_BF16X3, SPLIT_BF16X6, SPLIT_ADAPTIVE = 0, 1, 2
DEG_ANALYTIC, DEG_MLP = 0, 1
GEMM_FP64, GEMM_OZAKI = 0, 1
MLP_NPARAM = 64 * 5 + 64 + 64 * 64 + 64 + 64 + 1


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("split", C.c_int), ("degree_model", C.c_int),
                ("deg_cold", C.c_int), ("deg_warm", C.c_int), ("deg_min", C.c_int),
                ("deg_max", C.c_int), ("deg_extra", C.c_int), ("lanczos_steps", C.c_int),
                ("max_loops", C.c_int), ("switch_tol", C.c_double), ("seed", C.c_ulonglong),
                ("profile", C.c_int), ("mlp_extra", C.c_int), ("step0", C.c_int),
                ("f64_gemm", C.c_int), ("warm_rr", C.c_int), ("warm_resid", C.c_int),
                ("autotune", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("status", C.c_int), ("loops", C.c_int), ("loops_lowp", C.c_int),
                ("n_locked", C.c_int), ("col_degrees", C.c_longlong),
                ("col_degrees_lowp", C.c_longlong), ("beta", C.c_double),
                ("norm_h", C.c_double), ("max_resid", C.c_double), ("ms_total", C.c_double),
                ("ms_lanczos", C.c_double), ("ms_filter", C.c_double), ("ms_qr", C.c_double),
                ("ms_rr", C.c_double), ("ms_resid", C.c_double), ("ms_lock", C.c_double),
                ("filter_flops", C.c_double), ("filter_launches", C.c_longlong),
                ("launches", C.c_longlong), ("k_f64_ms", C.c_double), ("k_f64_flops", C.c_double),
                ("k_f64_launches", C.c_longlong), ("k_tc_ms", C.c_double),
                ("k_tc_flops", C.c_double), ("k_tc_launches", C.c_longlong),
                ("k_solver_ms", C.c_double), ("k_solver_calls", C.c_longlong),
                ("loops_mlp", C.c_int), ("mlp_fallback", C.c_int),
                ("k_f64_exec_flops", C.c_double), ("k_cholinv_ms", C.c_double),
                ("k_lanczos_ms", C.c_double), ("k_slice_ms", C.c_double),
                ("k_eigctl_ms", C.c_double), ("k_tc_exec_flops", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class FilterItem(C.Structure):
    _fields_ = [("H", C.c_void_p), ("n", C.c_int), ("k", C.c_int), ("Y0", C.c_void_p),
                ("degrees_host", C.POINTER(C.c_int)), ("lam1", C.c_double), ("c", C.c_double),
                ("e", C.c_double), ("Y", C.c_void_p)]


class Problem(C.Structure):
    _fields_ = [("H_host", C.c_void_p), ("n", C.c_int), ("nev", C.c_int), ("nex", C.c_int),
                ("X", C.c_void_p), ("evals", C.c_void_p), ("warm", C.c_int),
                ("lam_lo", C.c_double), ("lam_hi", C.c_double)]


class ChfsiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"chfsi error {code}: {msg}")
        self.code = code


_lib = None

_P = C.c_void_p
_SIGS = {
    "chfsi_default_opts": (None, [C.POINTER(Opts)]),
    "chfsi_init": (C.c_int, [C.POINTER(C.c_void_p), C.POINTER(Opts), _P]),
    "chfsi_set_opts": (C.c_int, [_P, C.POINTER(Opts)]),
    "chfsi_free": (None, [_P]),
    "chfsi_strerror": (C.c_char_p, [C.c_int]),
    "chfsi_last_error": (C.c_char_p, [_P]),
    "chfsi_solve": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, _P, C.c_double, _P, _P,
                              C.POINTER(Stats)]),
    "chfsi_solve_generalized": (C.c_int, [_P, _P, _P, C.c_int, C.c_int, C.c_int, _P, _P,
                                          C.c_double, _P, _P, C.POINTER(Stats)]),
    "chfsi_solve_sequence": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, _P,
                                       C.c_double, _P, _P]),
    "chfsi_solve_sequence_host": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_int, C.c_int, _P,
                                            C.c_double, _P, _P]),
    "chfsi_solve_batched": (C.c_int, [_P, C.c_int, _P, C.c_int, C.c_double, _P]),
    "chfsi_lanczos": (C.c_int, [_P, _P, C.c_int, C.c_int, C.c_ulonglong, _P]),
    "chfsi_autotune_table": (C.c_int, [_P, C.c_int, _P, C.POINTER(C.c_int)]),
    "chfsi_sort_degrees": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "chfsi_lock": (C.c_int, [_P, C.c_int, _P, _P, C.c_int, C.c_double, _P, _P, _P]),
    "chfsi_filter": (C.c_int, [_P, _P, C.c_int, C.c_int, _P, _P, C.c_double, C.c_double,
                               C.c_double, _P, C.c_int]),
    "chfsi_filter_batched": (C.c_int, [_P, C.c_int, _P]),
    "chfsi_filter_refine": (C.c_int, [_P, _P, C.c_int, C.c_int, _P, _P, _P, _P, C.c_double,
                                      C.c_double, C.c_double, _P]),
    "chfsi_zgemm": (C.c_int, [_P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, _P, C.c_int,
                              _P, C.c_int, C.c_double, _P, C.c_int, C.c_int]),
    "chfsi_orthonormalize": (C.c_int, [_P, C.c_int, C.c_int, _P, C.c_int, _P]),
    "chfsi_rayleigh_ritz": (C.c_int, [_P, _P, C.c_int, C.c_int, _P, _P, _P, _P]),
    "chfsi_residuals": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, _P, C.c_double, _P]),
    "chfsi_degrees": (C.c_int, [_P, C.c_int, _P, _P, C.c_double, C.c_double, C.c_double,
                                C.c_int, _P]),
    "chfsi_filter_static": (C.c_int, [_P, C.c_int, C.c_int, _P, _P, C.c_double, C.c_double,
                                      C.c_double, _P, _P]),
    "chfsi_trace_enable": (C.c_int, [_P, C.c_int]),
    "chfsi_trace_dataset": (C.c_int, [_P, _P, _P, C.c_int, C.POINTER(C.c_int)]),
    "chfsi_mlp_set_params": (C.c_int, [_P, _P]),
    "chfsi_mlp_get_params": (C.c_int, [_P, _P]),
    "chfsi_mlp_forward": (C.c_int, [_P, C.c_int, _P, _P]),
    "chfsi_mlp_train_step": (C.c_int, [_P, C.c_int, _P, _P, C.c_float, _P, _P]),
}


def lib():
    """The loaded library (ctypes.CDLL); raises if it is not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise ImportError(f"{LIB} is missing: build it with paper_1404_4161_gb300.build.build()")
        h = C.CDLL(LIB)
        for name, (res, args) in _SIGS.items():
            f = getattr(h, name)
            f.restype = res
            f.argtypes = args
        _lib = h
    return _lib


def exported_names():
    return list(_SIGS)


def default_opts(**over) -> Opts:
    o = Opts()
    lib().chfsi_default_opts(C.byref(o))
    for k, v in over.items():
        setattr(o, k, v)
    return o
