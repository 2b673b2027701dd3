"""CPU oracle for the filtered Newton-Schulz sign iteration (TEST INFRASTRUCTURE).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg import this package. The library's compute path never does, and the two
share no code: the oracle is plain C (``oracle.c``) compiled with
contraction off, wrapped here with ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")

FILTER_NONE, FILTER_EXACT, FILTER_BOUND = 0, 1, 2
OK, EINVAL, ENOMEM, ENOTCONV, EDIVERGED = 0, 1, 2, 3, 4
_FILTERS = {"none": FILTER_NONE, "exact": FILTER_EXACT, "bound": FILTER_BOUND}


def build(force: bool = False) -> str:
    """Compiles liboracle.so with gcc (no GPU needed)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
            os.path.getmtime(src), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-Wall", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("filter", C.c_int), ("c4", C.c_double),
                ("switch_resid", C.c_double), ("max_iter", C.c_int), ("mixed", C.c_int),
                ("fp32_until", C.c_double), ("scale_1norm", C.c_int), ("div_limit", C.c_double),
                ("filter_t", C.c_int), ("budget_norm", C.c_int)]


class _Trace(C.Structure):
    _fields_ = [("cap", C.c_int), ("count", C.c_int),
                ("nnz_x", C.POINTER(C.c_int64)), ("nnz_t", C.POINTER(C.c_int64)),
                ("resid", C.POINTER(C.c_double)), ("xnorm", C.POINTER(C.c_double)),
                ("beta", C.POINTER(C.c_double)), ("tau", C.POINTER(C.c_double)),
                ("fnorm", C.POINTER(C.c_double)), ("nnz_bar", C.POINTER(C.c_int64)),
                ("prec", C.POINTER(C.c_int)), ("nnz_that", C.POINTER(C.c_int64))]


_lib = None
_P64, _P32, _PD, _PF = (C.POINTER(C.c_int64), C.POINTER(C.c_int32), C.POINTER(C.c_double),
                        C.POINTER(C.c_float))


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        L.oracle_free.argtypes = [C.c_void_p]
        L.oracle_onenorm.restype = C.c_double
        L.oracle_onenorm.argtypes = [C.c_int64, _P64, _P32, _PD]
        L.oracle_spgemm.argtypes = [C.c_int64, _P64, _P32, _PD, _P64, _P32, _PD,
                                    C.POINTER(_P64), C.POINTER(_P32), C.POINTER(_PD)]
        L.oracle_spgemm_f32.argtypes = [C.c_int64, _P64, _P32, _PF, _P64, _P32, _PF,
                                        C.POINTER(_P64), C.POINTER(_P32), C.POINTER(_PF)]
        L.oracle_resid_rms.restype = C.c_double
        L.oracle_resid_rms.argtypes = [C.c_int64, _P64, _P32, _PD]
        L.oracle_fro_rms.restype = C.c_double
        L.oracle_fro_rms.argtypes = [C.c_int64, _P64, _PD]
        L.oracle_ns_update.argtypes = [C.c_int64, _P64, _P32, _PD, _P64, _P32, _PD,
                                       C.POINTER(_P64), C.POINTER(_P32), C.POINTER(_PD)]
        L.oracle_filter.argtypes = [C.c_int64, _P64, _P32, _PD, C.c_int, C.c_double,
                                    C.POINTER(_P64), C.POINTER(_P32), C.POINTER(_PD),
                                    _PD, _PD]
        L.oracle_budget.restype = C.c_double
        L.oracle_budget.argtypes = [C.c_double] * 5
        L.oracle_nsf.argtypes = [C.c_int64, _P64, _P32, _PD, C.POINTER(_Opts), C.POINTER(_Trace),
                                 C.POINTER(C.c_int), _PD, C.POINTER(_P64), C.POINTER(_P32),
                                 C.POINTER(_PD)]
        L.oracle_nmf.argtypes = L.oracle_nsf.argtypes
        L.oracle_nm_dense.argtypes = [C.c_int64, _PD, C.c_double, C.c_int, _PD,
                                      C.POINTER(C.c_int), _PD]
        L.oracle_norm2_est.restype = C.c_double
        L.oracle_norm2_est.argtypes = [C.c_int64, _P64, _P32, _PD, C.c_int]
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _csr_args(rowptr, col, val, dtype=np.float64):
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=dtype)
    return rowptr, col, val


def _take(n, rp, cp, vp, vdtype):
    L = lib()
    rowptr = np.ctypeslib.as_array(rp, shape=(n + 1,)).copy()
    nnz = int(rowptr[-1])
    col = np.ctypeslib.as_array(cp, shape=(max(nnz, 1),))[:nnz].copy()
    val = np.ctypeslib.as_array(vp, shape=(max(nnz, 1),))[:nnz].copy().astype(vdtype, copy=False)
    for p in (rp, cp, vp):
        L.oracle_free(C.cast(p, C.c_void_p))
    return rowptr, col, val


def onenorm(n, rowptr, col, val) -> float:
    rowptr, col, val = _csr_args(rowptr, col, val)
    return lib().oracle_onenorm(n, _p(rowptr, _P64), _p(col, _P32), _p(val, _PD))


def spgemm(n, a, b, f32: bool = False):
    """C = A B with the oracle's Gustavson product; a, b are (rowptr, col, val)."""
    dt = np.float32 if f32 else np.float64
    ar, ac, av = _csr_args(*a, dtype=dt)
    br, bc, bv = _csr_args(*b, dtype=dt)
    rp, cp = _P64(), _P32()
    if f32:
        vp = _PF()
        rc = lib().oracle_spgemm_f32(n, _p(ar, _P64), _p(ac, _P32), _p(av, _PF), _p(br, _P64),
                                     _p(bc, _P32), _p(bv, _PF), C.byref(rp), C.byref(cp), C.byref(vp))
    else:
        vp = _PD()
        rc = lib().oracle_spgemm(n, _p(ar, _P64), _p(ac, _P32), _p(av, _PD), _p(br, _P64),
                                 _p(bc, _P32), _p(bv, _PD), C.byref(rp), C.byref(cp), C.byref(vp))
    if rc:
        raise MemoryError("oracle_spgemm")
    return _take(n, rp, cp, vp, dt)


def resid_rms(n, rowptr, col, val) -> float:
    rowptr, col, val = _csr_args(rowptr, col, val)
    return lib().oracle_resid_rms(n, _p(rowptr, _P64), _p(col, _P32), _p(val, _PD))


def fro_rms(n, rowptr, val) -> float:
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    val = np.ascontiguousarray(val, dtype=np.float64)
    return lib().oracle_fro_rms(n, _p(rowptr, _P64), _p(val, _PD))


def ns_update(n, x, t):
    xr, xc, xv = _csr_args(*x)
    tr, tc, tv = _csr_args(*t)
    rp, cp, vp = _P64(), _P32(), _PD()
    rc = lib().oracle_ns_update(n, _p(xr, _P64), _p(xc, _P32), _p(xv, _PD), _p(tr, _P64),
                                _p(tc, _P32), _p(tv, _PD), C.byref(rp), C.byref(cp), C.byref(vp))
    if rc:
        raise MemoryError("oracle_ns_update")
    return _take(n, rp, cp, vp, np.float64)


def filter_csr(n, x, mode, b):
    """Returns ((rowptr, col, val), tau, fnorm) for filter mode 'none'|'exact'|'bound'."""
    xr, xc, xv = _csr_args(*x)
    rp, cp, vp = _P64(), _P32(), _PD()
    tau, fn = C.c_double(), C.c_double()
    rc = lib().oracle_filter(n, _p(xr, _P64), _p(xc, _P32), _p(xv, _PD), _FILTERS.get(mode, mode),
                             float(b), C.byref(rp), C.byref(cp), C.byref(vp), C.byref(tau),
                             C.byref(fn))
    if rc:
        raise RuntimeError(f"oracle_filter rc={rc}")
    return _take(n, rp, cp, vp, np.float64), tau.value, fn.value


def budget(r, x, c4=1e-4, tol_stage=1e-8, switch_resid=1e-6) -> float:
    return lib().oracle_budget(r, x, c4, tol_stage, switch_resid)


@dataclass
class Result:
    status: int
    iters: int
    resid: float
    rowptr: np.ndarray
    col: np.ndarray
    val: np.ndarray
    trace: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self, n: int) -> np.ndarray:
        d = np.zeros((n, n))
        rows = np.repeat(np.arange(n), np.diff(self.rowptr))
        d[rows, self.col] = self.val
        return d


def _trace(trace_cap):
    arrs = {k: np.zeros(trace_cap, dtype=t) for k, t in
            [("nnz_x", np.int64), ("nnz_t", np.int64), ("resid", np.float64),
             ("xnorm", np.float64), ("beta", np.float64), ("tau", np.float64),
             ("fnorm", np.float64), ("nnz_bar", np.int64), ("prec", np.int32),
             ("nnz_that", np.int64)]}
    tr = _Trace(trace_cap, 0, _p(arrs["nnz_x"], _P64), _p(arrs["nnz_t"], _P64),
                _p(arrs["resid"], _PD), _p(arrs["xnorm"], _PD), _p(arrs["beta"], _PD),
                _p(arrs["tau"], _PD), _p(arrs["fnorm"], _PD), _p(arrs["nnz_bar"], _P64),
                _p(arrs["prec"], C.POINTER(C.c_int)), _p(arrs["nnz_that"], _P64))
    return arrs, tr


def norm2_est(n, rowptr, col, val, steps=8) -> float:
    """The oracle's power-iteration estimate of ||X||_2 (budget_norm variant)."""
    rowptr, col, val = _csr_args(rowptr, col, val)
    return lib().oracle_norm2_est(n, _p(rowptr, _P64), _p(col, _P32), _p(val, _PD), steps)


def nsf(a, tol=1e-8, filter="exact", c4=1e-4, switch_resid=1e-6, max_iter=100, mixed=False,
        fp32_until=1e-4, scale_1norm=True, div_limit=1e6, trace_cap=256, filter_t=False,
        budget_norm="rms") -> Result:
    """Runs the oracle's NSF (filter='none' is plain Newton-Schulz) on a CSR input.
    Variants: filter_t=True filters T = X^2 with the same budget before the
    update; budget_norm='2' takes ||X||_2 (power iteration) in Eq. (1.18)."""
    n = a.n
    rowptr, col, val = _csr_args(a.rowptr, a.col, a.val)
    o = _Opts(tol, _FILTERS[filter], c4, switch_resid, max_iter, int(mixed), fp32_until,
              int(scale_1norm), div_limit, int(bool(filter_t)), int(budget_norm == "2"))
    arrs, tr = _trace(trace_cap)
    it, r = C.c_int(), C.c_double()
    rp, cp, vp = _P64(), _P32(), _PD()
    rc = lib().oracle_nsf(n, _p(rowptr, _P64), _p(col, _P32), _p(val, _PD), C.byref(o),
                          C.byref(tr), C.byref(it), C.byref(r), C.byref(rp), C.byref(cp),
                          C.byref(vp))
    if rc in (EINVAL, ENOMEM):
        raise RuntimeError(f"oracle_nsf rc={rc}")
    srp, scol, sval = _take(n, rp, cp, vp, np.float64)
    trace = {k: v[:tr.count].copy() for k, v in arrs.items()}
    return Result(rc, it.value, r.value, srp, scol, sval, trace)


def _nsf_worker(job):
    a, kw = job
    return nsf(a, **kw)


def nsf_many(mats, processes=None, **kw) -> list:
    """nsf(a, **kw) for every matrix, spread over a pool of spawned processes
    (spawn, so that callers that already use CUDA stay safe); results in order."""
    import multiprocessing as mp
    build()
    procs = max(1, min(len(mats), processes or (os.cpu_count() or 1)))
    if procs == 1:
        return [nsf(a, **kw) for a in mats]
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_nsf_worker, [(a, kw) for a in mats], chunksize=1)


def nmf(a, tol=1e-12, filter="exact", c4=1e-4, switch_resid=1e-6, max_iter=100, div_limit=1e6,
        trace_cap=256) -> Result:
    """Runs the oracle's NMF (Alg. 3.1.1; filter='none' is Newton's method) on a
    CSR input: X1 = A, dense inverse, filter budget c4*tol, then Eq. (1.13)."""
    n = a.n
    rowptr, col, val = _csr_args(a.rowptr, a.col, a.val)
    o = _Opts(tol, _FILTERS[filter], c4, switch_resid, max_iter, 0, 0.0, 0, div_limit, 0, 0)
    arrs, tr = _trace(trace_cap)
    it, r = C.c_int(), C.c_double()
    rp, cp, vp = _P64(), _P32(), _PD()
    rc = lib().oracle_nmf(n, _p(rowptr, _P64), _p(col, _P32), _p(val, _PD), C.byref(o),
                          C.byref(tr), C.byref(it), C.byref(r), C.byref(rp), C.byref(cp),
                          C.byref(vp))
    if rc in (EINVAL, ENOMEM):
        raise RuntimeError(f"oracle_nmf rc={rc}")
    srp, scol, sval = _take(n, rp, cp, vp, np.float64)
    trace = {k: v[:tr.count].copy() for k, v in arrs.items()}
    return Result(rc, it.value, r.value, srp, scol, sval, trace)


def nm_dense(a: np.ndarray, tol=1e-12, max_iter=100):
    """Newton's method X <- (X + X^-1)/2 from X0 = A (dense). Returns (S, iters, resid, status)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    n = a.shape[0]
    s = np.empty_like(a)
    it, r = C.c_int(), C.c_double()
    rc = lib().oracle_nm_dense(n, _p(a, _PD), tol, max_iter, _p(s, _PD), C.byref(it), C.byref(r))
    if rc == ENOMEM:
        raise MemoryError("oracle_nm_dense")
    return s, it.value, r.value, rc
