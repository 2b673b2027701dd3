"""ctypes binding of include/sign.h (argument marshalling only).

Every step of the solve runs in the CUDA library; if the library is missing
this module raises instead of computing anything itself.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsign_gb300.so")

SIGN_OK, SIGN_EINVAL, SIGN_ENOMEM, SIGN_ENOTCONV, SIGN_EDIVERGED, SIGN_ECUDA, SIGN_ETIMEOUT, \
    SIGN_ESTATE, SIGN_EAGAIN = range(9)
SIGN_FILTER_NONE, SIGN_FILTER_EXACT, SIGN_FILTER_BOUND = 0, 1, 2
SIGN_PREC_FP64, SIGN_PREC_MIXED = 0, 1
STATUS_NAMES = ["SIGN_OK", "SIGN_EINVAL", "SIGN_ENOMEM", "SIGN_ENOTCONV", "SIGN_EDIVERGED",
                "SIGN_ECUDA", "SIGN_ETIMEOUT", "SIGN_ESTATE", "SIGN_EAGAIN"]


class sign_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("filter", C.c_int), ("c4", C.c_double),
                ("switch_resid", C.c_double), ("max_iter", C.c_int), ("prec", C.c_int),
                ("fp32_until", C.c_double), ("dense_frac", C.c_double), ("scale_1norm", C.c_int),
                ("div_limit", C.c_double), ("dense64_min_n", C.c_int), ("fp32_band", C.c_int),
                ("filter_t", C.c_int), ("budget_norm", C.c_int), ("method", C.c_int),
                ("band_min_eff", C.c_double), ("group_margin", C.c_double),
                ("pair_rows", C.c_int)]


class sign_tune_report(C.Structure):
    _fields_ = [("timed", C.c_int), ("cached", C.c_int), ("ms_base", C.c_double),
                ("ms_best", C.c_double)]


class sign_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("status", C.c_int), ("resid", C.c_double),
                ("nnz_final", C.c_int64), ("cap", C.c_int), ("count", C.c_int),
                ("nnz_x", C.POINTER(C.c_int64)), ("nnz_t", C.POINTER(C.c_int64)),
                ("resid_k", C.POINTER(C.c_double)), ("xnorm_k", C.POINTER(C.c_double)),
                ("beta_k", C.POINTER(C.c_double)), ("tau_k", C.POINTER(C.c_double)),
                ("fnorm_k", C.POINTER(C.c_double)), ("nnz_bar", C.POINTER(C.c_int64)),
                ("prec_k", C.POINTER(C.c_int)), ("mults_t", C.POINTER(C.c_double)),
                ("mults_bar", C.POINTER(C.c_double)), ("nnz_that", C.POINTER(C.c_int64))]


class sign_server_opts(C.Structure):
    _fields_ = [("solve", sign_opts), ("mem_budget", C.c_double), ("max_active", C.c_int),
                ("max_queue", C.c_int), ("lanes", C.c_int), ("max_wait_s", C.c_double)]


class sign_request_times(C.Structure):
    _fields_ = [("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("footprint", C.c_double), ("lane", C.c_int)]


class sign_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("refused", C.c_int64), ("admitted", C.c_int64),
                ("completed", C.c_int64), ("queued", C.c_int64), ("active", C.c_int64),
                ("max_active_seen", C.c_int64), ("rounds", C.c_int64), ("reserved", C.c_double)]


class sign_prof_entry(C.Structure):
    _fields_ = [("name", C.c_char * 32), ("launches", C.c_int64), ("ms", C.c_double),
                ("flops", C.c_double), ("bytes", C.c_double)]


sign_t = C.c_void_p
_P64, _P32, _PD = C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_double)

# name -> (restype, argtypes); every function declared in include/sign.h
SIGNATURES = {
    "sign_default_opts": (None, [C.POINTER(sign_opts)]),
    "sign_create": (C.c_int, [C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int,
                              C.c_void_p, C.POINTER(sign_t)]),
    "sign_create_batch": (C.c_int, [C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                    C.POINTER(C.c_void_p), C.POINTER(C.c_void_p),
                                    C.POINTER(C.c_void_p), C.c_int, C.c_void_p,
                                    C.POINTER(sign_t)]),
    "sign_get_csr_batch": (C.c_int, [C.c_int, C.POINTER(sign_t), C.POINTER(C.c_void_p),
                                     C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int]),
    "sign_trim_memory": (C.c_int, []),
    "sign_solve": (C.c_int, [sign_t, C.POINTER(sign_opts), C.POINTER(sign_info)]),
    "sign_solve_batch": (C.c_int, [C.POINTER(sign_t), C.c_int, C.POINTER(sign_opts),
                                   C.POINTER(sign_info)]),
    "sign_result_nnz_batch": (C.c_int, [C.c_int, C.POINTER(sign_t), C.POINTER(C.c_int64)]),
    "sign_destroy_batch": (None, [C.POINTER(sign_t), C.c_int]),
    "sign_tune_batch": (C.c_int, [C.POINTER(sign_t), C.c_int, C.POINTER(sign_opts), C.c_int,
                                  C.c_int, C.POINTER(sign_opts), C.POINTER(sign_tune_report)]),
    "sign_get_csr": (C.c_int, [sign_t, C.POINTER(C.c_int64), C.c_void_p, C.c_void_p, C.c_void_p,
                               C.c_int]),
    "sign_destroy": (None, [sign_t]),
    "sign_last_error": (C.c_char_p, []),
    "sign_threshold_exact": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_int, C.c_void_p,
                                       C.POINTER(C.c_double)]),
    "sign_threshold_exact_noalloc": (C.c_int, [C.c_void_p, C.c_int64, C.c_double, C.c_void_p,
                                               C.POINTER(C.c_double)]),
    "sign_dense_product": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p,
                                     C.c_int, C.c_void_p, C.c_int, C.c_void_p]),
    "sign_dense_product_f64": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                         C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p]),
    "sign_footprint_bytes": (C.c_double, [C.c_int64, C.c_int64, C.c_double, C.c_double,
                                          C.c_int64]),
    "sign_server_default_opts": (None, [C.POINTER(sign_server_opts)]),
    "sign_server_create": (C.c_int, [C.POINTER(sign_server_opts), C.POINTER(C.c_void_p)]),
    "sign_server_submit": (C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p,
                                     C.c_void_p, C.c_int, C.POINTER(C.c_uint64)]),
    "sign_server_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int, C.POINTER(sign_info),
                                   C.POINTER(sign_request_times)]),
    "sign_server_take": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.POINTER(sign_t)]),
    "sign_server_get_stats": (C.c_int, [C.c_void_p, C.POINTER(sign_server_stats)]),
    "sign_server_destroy": (None, [C.c_void_p]),
    "sign_kernel_launches": (C.c_int64, []),
    "sign_prof_enable": (C.c_int, [C.c_int]),
    "sign_prof_read": (C.c_int, [C.c_void_p, C.c_int]),
    "sign_prof_reset": (None, []),
    "sign_fma_probe": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                 C.POINTER(C.c_double)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return load().sign_last_error().decode()


class SignError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < 9 else status}: "
                         f"{last_error()}")


def default_opts(**kw) -> sign_opts:
    o = sign_opts()
    load().sign_default_opts(C.byref(o))
    for k, v in kw.items():
        if k == "filter" and isinstance(v, str):
            v = {"none": 0, "exact": 1, "bound": 2}[v]
        if k == "prec" and isinstance(v, str):
            v = {"fp64": 0, "mixed": 1}[v]
        if k == "method" and isinstance(v, str):
            v = {"nsf": 0, "nmf": 1}[v]
        setattr(o, k, v)
    return o


def prof_read() -> dict:
    """Per-kernel-class timings accumulated since the last reset."""
    L = load()
    n = L.sign_prof_read(None, 0)
    arr = (sign_prof_entry * n)()
    n = L.sign_prof_read(C.cast(arr, C.c_void_p), n)
    return {e.name.decode(): {"launches": e.launches, "ms": e.ms, "flops": e.flops,
                              "bytes": e.bytes} for e in arr[:n]}
