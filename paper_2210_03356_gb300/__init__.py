"""GB300-native filtered Newton-Schulz sign solver (arXiv 2210.03356, Alg. 3.2.1).

Python binding of the C ABI in include/sign.h. The functions here only move
arguments across the ABI; every step of a solve runs in the CUDA library
``libsign_gb300.so`` (built in-tree by ``build.build()``).

    import paper_2210_03356_gb300 as sg
    res = sg.solve(csr, tol=1e-8, filter="exact")        # host numpy CSR in
    res.rowptr, res.col, res.val, res.iters, res.trace    # host numpy CSR out

Inputs are objects with ``n``, ``rowptr`` (int64), ``col`` (int32) and ``val``
(float64): numpy arrays (copied host to device) or CUDA torch tensors (copied
device to device).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np

from . import _native as N
from ._native import (SIGN_EAGAIN, SIGN_ECUDA, SIGN_EDIVERGED, SIGN_EINVAL, SIGN_ENOMEM,
                      SIGN_ENOTCONV, SIGN_ESTATE, SIGN_ETIMEOUT, SIGN_OK, SignError, default_opts,
                      last_error, load, prof_read)

__all__ = ["solve", "solve_batch", "Handle", "Batch", "Result", "Server", "default_opts", "load",
           "last_error", "prof_read", "kernel_launches", "prof_enable", "prof_reset", "trim_memory",
           "SignError", "SIGN_OK", "SIGN_EINVAL", "SIGN_ENOMEM", "SIGN_ENOTCONV", "SIGN_EDIVERGED",
           "SIGN_ECUDA", "SIGN_ETIMEOUT", "SIGN_ESTATE", "SIGN_EAGAIN"]

_TRACE = [("nnz_x", np.int64), ("nnz_t", np.int64), ("resid_k", np.float64),
          ("xnorm_k", np.float64), ("beta_k", np.float64), ("tau_k", np.float64),
          ("fnorm_k", np.float64), ("nnz_bar", np.int64), ("prec_k", np.int32),
          ("mults_t", np.float64), ("mults_bar", np.float64), ("nnz_that", np.int64)]


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(x.is_cuda)


def _ptr(x):
    if _is_torch_cuda(x) or hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    return x.ctypes.data_as(C.c_void_p)


def _addr(x) -> int:
    """The address of a torch tensor's or numpy array's data, as an int (for
    filling pointer arrays of a batch without one ctypes object per array)."""
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.__array_interface__["data"][0]


def current_stream():
    """The torch current CUDA stream handle, or None (legacy default stream)."""
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return None


@dataclass
class Result:
    status: int
    iters: int
    resid: float
    rowptr: object
    col: object
    val: object
    trace: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])


class _Info:
    """A sign_info with numpy-owned trace arrays (none when cap == 0)."""

    def __init__(self, cap: int):
        self.s = N.sign_info()
        self.s.cap = cap
        self.arrays = {}
        if cap > 0:
            self.arrays = {k: np.zeros(cap, dtype=t) for k, t in _TRACE}
            for k, t in _TRACE:
                setattr(self.s, k,
                        self.arrays[k].ctypes.data_as(C.POINTER(np.ctypeslib.as_ctypes_type(t))))

    def trace(self, s=None) -> dict:
        c = (s if s is not None else self.s).count
        return {k: v[:c].copy() for k, v in self.arrays.items()}


class Handle:
    """One matrix on the device (sign_create / sign_destroy)."""

    def __init__(self, a, stream=None):
        L = load()
        self.n = int(a.n)
        on_dev = _is_torch_cuda(a.val)
        if not on_dev:
            self._keep = (np.ascontiguousarray(a.rowptr, dtype=np.int64),
                          np.ascontiguousarray(a.col, dtype=np.int32),
                          np.ascontiguousarray(a.val, dtype=np.float64))
        else:
            self._keep = (a.rowptr.contiguous(), a.col.contiguous(), a.val.contiguous())
        rp, col, val = self._keep
        nnz = int(rp[-1])
        self.stream = stream if stream is not None else current_stream()
        h = N.sign_t()
        st = L.sign_create(self.n, nnz, _ptr(rp), _ptr(col), _ptr(val), int(on_dev), self.stream,
                           C.byref(h))
        if st != SIGN_OK:
            raise SignError(st, "sign_create")
        self.h = h
        self._keep = None

    @classmethod
    def _adopt(cls, h, n, stream):
        """Wraps a handle that sign_create_batch made."""
        self = cls.__new__(cls)
        self.n, self.stream, self.h, self._keep = int(n), stream, h, None
        return self

    def close(self):
        if getattr(self, "h", None):
            load().sign_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def result_nnz(self) -> int:
        """Stored entries of the result (sign_get_csr with no arrays)."""
        nnz = C.c_int64()
        st = load().sign_get_csr(self.h, C.byref(nnz), None, None, None, 0)
        if st != SIGN_OK:
            raise SignError(st, "sign_get_csr")
        return nnz.value

    def result(self, device=False, out=None):
        """sign_get_csr: host numpy arrays, or CUDA torch tensors if device=True.

        out = (rowptr, col, val) reads into caller-owned host arrays instead
        (numpy views, e.g. of pinned memory, reused across solves); they must
        hold n + 1 and result_nnz() entries. Returns views of them.
        """
        L = load()
        nnz = C.c_int64()
        st = L.sign_get_csr(self.h, C.byref(nnz), None, None, None, 0)
        if st != SIGN_OK:
            raise SignError(st, "sign_get_csr")
        if out is not None:
            rp, col, val = out
            if (rp.dtype != np.int64 or col.dtype != np.int32 or val.dtype != np.float64 or
                    rp.size < self.n + 1 or col.size < nnz.value or val.size < nnz.value or
                    not (rp.flags.c_contiguous and col.flags.c_contiguous and
                         val.flags.c_contiguous)):
                raise ValueError("out arrays: need contiguous int64[n+1], int32[nnz], "
                                 "float64[nnz]")
            st = L.sign_get_csr(self.h, C.byref(nnz), _ptr(rp), _ptr(col), _ptr(val), 0)
            if st != SIGN_OK:
                raise SignError(st, "sign_get_csr")
            return rp[:self.n + 1], col[:nnz.value], val[:nnz.value]
        if device:
            import torch
            rp = torch.empty(self.n + 1, dtype=torch.int64, device="cuda")
            col = torch.empty(max(nnz.value, 1), dtype=torch.int32, device="cuda")
            val = torch.empty(max(nnz.value, 1), dtype=torch.float64, device="cuda")
            st = L.sign_get_csr(self.h, C.byref(nnz), _ptr(rp), _ptr(col), _ptr(val), 1)
            col, val = col[:nnz.value], val[:nnz.value]
        else:
            rp = np.empty(self.n + 1, dtype=np.int64)
            col = np.empty(max(nnz.value, 1), dtype=np.int32)
            val = np.empty(max(nnz.value, 1), dtype=np.float64)
            st = L.sign_get_csr(self.h, C.byref(nnz), _ptr(rp), _ptr(col), _ptr(val), 0)
            col, val = col[:nnz.value], val[:nnz.value]
        if st != SIGN_OK:
            raise SignError(st, "sign_get_csr")
        return rp, col, val


def _opts(opts, kw):
    if opts is None:
        return default_opts(**kw)
    for k, v in kw.items():
        setattr(opts, k, v)
    return opts


def solve(a, opts=None, trace_cap: int = 256, device_out: bool = False, stream=None,
          **kw) -> Result:
    """sign_create + sign_solve + sign_get_csr for one matrix."""
    o = _opts(opts, kw)
    with Handle(a, stream) as h:
        info = _Info(trace_cap)
        st = load().sign_solve(h.h, C.byref(o), C.byref(info.s))
        if st not in (SIGN_OK, SIGN_ENOTCONV, SIGN_EDIVERGED):
            raise SignError(st, "sign_solve")
        rp, col, val = h.result(device=device_out)
        return Result(info.s.status, info.s.iters, info.s.resid, rp, col, val, info.trace())


def solve_batch(mats, opts=None, trace_cap: int = 256, device_out: bool = False, stream=None,
                **kw) -> list[Result]:
    """sign_solve_batch: all matrices in the same kernel launches, one result each."""
    o = _opts(opts, kw)
    hs = Batch(mats, stream).handles
    try:
        arr = (N.sign_t * len(hs))(*[h.h for h in hs])
        infos = [_Info(trace_cap) for _ in hs]
        iarr = (N.sign_info * len(hs))(*[i.s for i in infos])
        st = load().sign_solve_batch(arr, len(hs), C.byref(o), iarr)
        if st != SIGN_OK:
            raise SignError(st, "sign_solve_batch")
        out = []
        for h, i, s in zip(hs, infos, iarr):  # iarr holds the filled copies of the structs
            rp, col, val = h.result(device=device_out)
            out.append(Result(s.status, s.iters, s.resid, rp, col, val, i.trace(s)))
        return out
    finally:
        for h in hs:
            h.close()


def trim_memory() -> None:
    """sign_trim_memory: kept device blocks and unused pool memory back to the device."""
    st = load().sign_trim_memory()
    if st != SIGN_OK:
        raise SignError(st, "sign_trim_memory")


def threshold_exact(values, b: float, stream=None) -> float:
    """sign_threshold_exact on a numpy array (host) or CUDA torch tensor."""
    on_dev = _is_torch_cuda(values)
    if not on_dev:
        values = np.ascontiguousarray(values, dtype=np.float64)
    tau = C.c_double()
    st = load().sign_threshold_exact(_ptr(values), int(values.shape[0]), float(b), int(on_dev),
                                     stream if stream is not None else current_stream(),
                                     C.byref(tau))
    if st != SIGN_OK:
        raise SignError(st, "sign_threshold_exact")
    return tau.value


def dense_product(a, b, out=None, stream=None):
    """sign_dense_product for CUDA torch float32 matrices (row-major)."""
    import torch
    M, K = a.shape
    K2, N = b.shape
    assert K == K2 and a.dtype == b.dtype == torch.float32 and a.is_cuda and b.is_cuda
    if out is None:
        out = torch.empty(M, N, dtype=torch.float32, device=a.device)
    st = load().sign_dense_product(M, N, K, _ptr(a), a.stride(0), _ptr(b), b.stride(0), _ptr(out),
                                   out.stride(0),
                                   stream if stream is not None else current_stream())
    if st != SIGN_OK:
        raise SignError(st, "sign_dense_product")
    return out


def dense_product_f64(a, b, out=None, stream=None):
    """sign_dense_product_f64 for CUDA torch float64 matrices (row-major)."""
    import torch
    M, K = a.shape
    K2, N = b.shape
    assert K == K2 and a.dtype == b.dtype == torch.float64 and a.is_cuda and b.is_cuda
    if out is None:
        out = torch.empty(M, N, dtype=torch.float64, device=a.device)
    st = load().sign_dense_product_f64(M, N, K, _ptr(a), a.stride(0), _ptr(b), b.stride(0),
                                       _ptr(out), out.stride(0),
                                       stream if stream is not None else current_stream())
    if st != SIGN_OK:
        raise SignError(st, "sign_dense_product_f64")
    return out


def kernel_launches() -> int:
    return int(load().sign_kernel_launches())


def prof_enable(on: bool = True) -> bool:
    return bool(load().sign_prof_enable(int(on)))


def prof_reset() -> None:
    load().sign_prof_reset()


class Batch:
    """Device-resident matrices solved together with sign_solve_batch.

    The handles are created once (inputs copied to the device); every call of
    solve() runs the whole batch again from those inputs.
    """

    def __init__(self, mats, stream=None):
        mats = list(mats)
        if not mats:
            raise ValueError("empty batch")
        L = load()
        stream = stream if stream is not None else current_stream()
        on_dev = [_is_torch_cuda(a.val) for a in mats]
        if any(on_dev) and not all(on_dev):
            raise ValueError("a batch is all on the host or all on the device")
        if on_dev[0]:
            keep = [(a.rowptr.contiguous(), a.col.contiguous(), a.val.contiguous()) for a in mats]
        else:
            keep = [(np.ascontiguousarray(a.rowptr, dtype=np.int64),
                     np.ascontiguousarray(a.col, dtype=np.int32),
                     np.ascontiguousarray(a.val, dtype=np.float64)) for a in mats]
        k = len(mats)
        ns = (C.c_int64 * k)(*[int(a.n) for a in mats])
        nnzs = (C.c_int64 * k)(*[int(rp[-1]) for rp, _, _ in keep])
        rps = (C.c_void_p * k)(*[_addr(t[0]) for t in keep])
        cols = (C.c_void_p * k)(*[_addr(t[1]) for t in keep])
        vals = (C.c_void_p * k)(*[_addr(t[2]) for t in keep])
        out = (N.sign_t * k)()
        st = L.sign_create_batch(k, ns, nnzs, rps, cols, vals, int(on_dev[0]), stream, out)
        if st != SIGN_OK:
            raise SignError(st, "sign_create_batch")
        self.handles = [Handle._adopt(out[i], ns[i], stream) for i in range(k)]
        self.arr = (N.sign_t * k)(*[h.h for h in self.handles])
        self.infos = None

    def solve(self, opts, trace_cap: int = 0) -> list:
        """Runs sign_solve_batch; returns per-matrix (status, iters, resid)."""
        if self.infos is None or self.infos[2] != trace_cap:
            infos = [_Info(trace_cap) for _ in self.handles]
            iarr = (N.sign_info * len(infos))(*[i.s for i in infos])
            self.infos = (infos, iarr, trace_cap)
        infos, iarr, _ = self.infos
        st = load().sign_solve_batch(self.arr, len(self.handles), C.byref(opts), iarr)
        if st != SIGN_OK:
            raise SignError(st, "sign_solve_batch")
        return [(s.status, s.iters, s.resid) for s in iarr]

    def tune(self, opts, reps: int = 1, force: bool = False):
        """sign_tune_batch: the fastest schedule for this batch (timed, or from
        the cache). Returns (opts with the chosen schedule, report dict)."""
        best = N.sign_opts()
        rep = N.sign_tune_report()
        st = load().sign_tune_batch(self.arr, len(self.handles), C.byref(opts), int(reps),
                                    int(force), C.byref(best), C.byref(rep))
        if st != SIGN_OK:
            raise SignError(st, "sign_tune_batch")
        return best, {"timed": rep.timed, "cached": bool(rep.cached), "ms_base": rep.ms_base,
                      "ms_best": rep.ms_best, "band_min_eff": best.band_min_eff,
                      "group_margin": best.group_margin, "pair_rows": best.pair_rows}

    def traces(self) -> list:
        """The per-iteration records of the last solve(trace_cap > 0), one dict per matrix."""
        if self.infos is None:
            return []
        infos, iarr, _ = self.infos
        return [i.trace(s) for i, s in zip(infos, iarr)]

    def results(self, outs) -> list:
        """sign_get_csr_batch: every result at once into caller-owned host arrays.

        outs holds one (rowptr, col, val) per handle (numpy views, e.g. of
        pinned memory, reused across solves), sized from result_nnz(); the
        copies are queued together and waited for once. Returns views.
        """
        if len(outs) != len(self.handles):
            raise ValueError("one (rowptr, col, val) per handle")
        views = []
        for h, nnz, (rp, col, val) in zip(self.handles, self.result_nnz(), outs):
            if (rp.dtype != np.int64 or col.dtype != np.int32 or val.dtype != np.float64 or
                    rp.size < h.n + 1 or col.size < nnz or val.size < nnz or
                    not (rp.flags.c_contiguous and col.flags.c_contiguous and
                         val.flags.c_contiguous)):
                raise ValueError("out arrays: need contiguous int64[n+1], int32[nnz], "
                                 "float64[nnz]")
            views.append((rp[:h.n + 1], col[:nnz], val[:nnz]))
        k = len(outs)
        rps = (C.c_void_p * k)(*[_addr(o[0]) for o in outs])
        cols = (C.c_void_p * k)(*[_addr(o[1]) for o in outs])
        vals = (C.c_void_p * k)(*[_addr(o[2]) for o in outs])
        st = load().sign_get_csr_batch(k, self.arr, rps, cols, vals, 0)
        if st != SIGN_OK:
            raise SignError(st, "sign_get_csr_batch")
        return views

    def result_nnz(self) -> list:
        """sign_result_nnz_batch: the stored entries of every result."""
        k = len(self.handles)
        out = (C.c_int64 * k)()
        st = load().sign_result_nnz_batch(k, self.arr, out)
        if st != SIGN_OK:
            raise SignError(st, "sign_result_nnz_batch")
        return list(out)

    def close(self):
        """sign_destroy_batch: one wait per stream, then every handle freed."""
        live = [h for h in self.handles if getattr(h, "h", None)]
        if live:
            arr = (N.sign_t * len(live))(*[h.h for h in live])
            load().sign_destroy_batch(arr, len(live))
            for h in live:
                h.h = None


class Server:
    """A continuous-batching request loop on the GPU (sign_server_*).

    submit() copies a matrix in and returns a ticket; the library's worker
    thread admits it at a round boundary when its predicted footprint fits
    the budget, solves it beside the requests already in flight, and poll()
    reports it finished; take() reads its result.
    """

    def __init__(self, opts=None, mem_budget: float = 120e9, max_active: int = 1024,
                 max_queue: int = 65536, lanes: int = 2, max_wait_s: float = 0.0, **kw):
        L = load()
        so = N.sign_server_opts()
        L.sign_server_default_opts(C.byref(so))
        if opts is not None:
            so.solve = opts
        if kw:
            so.solve = _opts(so.solve, {k: ({"none": 0, "exact": 1, "bound": 2}[v]
                                             if k == "filter" and isinstance(v, str) else
                                             {"fp64": 0, "mixed": 1}[v]
                                             if k == "prec" and isinstance(v, str) else v)
                                        for k, v in kw.items()})
        so.mem_budget, so.max_active, so.max_queue = float(mem_budget), int(max_active), int(max_queue)
        so.lanes = int(lanes)
        so.max_wait_s = float(max_wait_s)
        self.opts = so
        self.h = C.c_void_p()
        st = L.sign_server_create(C.byref(so), C.byref(self.h))
        if st != SIGN_OK:
            raise SignError(st, "sign_server_create")
        self._n = {}

    def submit(self, a) -> int:
        """Queues matrix a (host numpy or CUDA torch CSR); raises SignError if refused
        (status SIGN_EAGAIN when its predicted wait exceeds max_wait_s)."""
        on_dev = _is_torch_cuda(a.val)
        if on_dev:
            keep = (a.rowptr.contiguous(), a.col.contiguous(), a.val.contiguous())
        else:
            keep = (np.ascontiguousarray(a.rowptr, dtype=np.int64),
                    np.ascontiguousarray(a.col, dtype=np.int32),
                    np.ascontiguousarray(a.val, dtype=np.float64))
        rp, col, val = keep
        t = C.c_uint64()
        st = load().sign_server_submit(self.h, int(a.n), int(rp[-1]), _ptr(rp), _ptr(col), _ptr(val),
                                       int(on_dev), C.byref(t))
        if st != SIGN_OK:
            raise SignError(st, "sign_server_submit")
        self._n[t.value] = int(a.n)
        return t.value

    def poll(self, ticket: int, wait_ms: int = 0):
        """None while pending; else a dict with the outcome and the request's times."""
        info, times = N.sign_info(), N.sign_request_times()
        st = load().sign_server_poll(self.h, ticket, int(wait_ms), C.byref(info), C.byref(times))
        if st == SIGN_EAGAIN:
            return None
        if st != SIGN_OK:
            raise SignError(st, "sign_server_poll")
        return {"status": info.status, "iters": info.iters, "resid": info.resid,
                "nnz_final": info.nnz_final, "t_submit": times.t_submit,
                "t_admit": times.t_admit, "t_done": times.t_done, "footprint": times.footprint,
                "lane": times.lane}

    def take(self, ticket: int, device: bool = False):
        """The finished request's result CSR (rowptr, col, val); forgets the ticket."""
        h = N.sign_t()
        stream = current_stream()
        st = load().sign_server_take(self.h, ticket, stream, C.byref(h))
        if st != SIGN_OK:
            raise SignError(st, "sign_server_take")
        hd = Handle.__new__(Handle)
        hd.h, hd.n, hd.stream = h, self._n.pop(ticket), stream
        try:
            return hd.result(device=device)
        finally:
            hd.close()

    def stats(self) -> dict:
        s = N.sign_server_stats()
        st = load().sign_server_get_stats(self.h, C.byref(s))
        if st != SIGN_OK:
            raise SignError(st, "sign_server_get_stats")
        return {k: getattr(s, k) for k, _ in N.sign_server_stats._fields_}

    def close(self):
        if getattr(self, "h", None):
            load().sign_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def footprint_bytes(n: int, nnz: int, delta: float, rho: float, bw: int) -> float:
    """sign_footprint_bytes: the server's admission model (host arithmetic)."""
    return float(load().sign_footprint_bytes(int(n), int(nnz), float(delta), float(rho), int(bw)))
