"""sign_threshold_exact_noalloc, the threshold entry point for callers that
cannot allocate device memory (their own pool already holds the GPU, or their
loop cannot afford cudaMalloc's device-wide synchronization).

It must give the same threshold as the allocating sign_threshold_exact on the
same device values, on consecutive calls that reuse its static scratch, and
the threshold of the oracle's EXACT filter; at its full capacity and on an
empty input too; it must refuse inputs larger than its fixed capacity and
take no device memory. This file is collected last so that a failure here
leaves every other test already run; it also passes on its own in a fresh
process.
"""
import ctypes as C
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_03356_gb300 as sg
    from paper_2210_03356_gb300 import build
    build.build()
    return sg.load()


def _values(seed, n):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(n) * 10.0 ** rng.uniform(-13, 0, n)
    v[rng.integers(0, n, n // 100)] = 0.0
    ties = rng.integers(0, n, n // 50)
    v[ties] = np.sign(v[ties]) * 2.5e-9
    return v


def _both(lib, dev, n, b):
    import torch
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    t_alloc, t_none = C.c_double(), C.c_double()
    st = lib.sign_threshold_exact(C.c_void_p(dev.data_ptr()), n, b, 1, stream, C.byref(t_alloc))
    assert st == 0, lib.sign_last_error()
    st = lib.sign_threshold_exact_noalloc(C.c_void_p(dev.data_ptr()), n, b, stream, C.byref(t_none))
    assert st == 0, lib.sign_last_error()
    return t_alloc.value, t_none.value


def test_noalloc_threshold_matches_allocating_entry_point(lib):
    import torch
    # two calls in a row on different inputs: the second must not see the first's scratch
    for seed, n, b in [(11, 700_000, 3e-7), (12, 90_000, 1e-9)]:
        dev = torch.from_numpy(_values(seed, n)).cuda()
        t_alloc, t_none = _both(lib, dev, n, b)
        # the threshold is one of the input magnitudes (or +inf): exact equality
        assert t_none == t_alloc, (seed, t_none, t_alloc)
        assert np.isfinite(t_none) and t_none > 0.0


def _tau_oracle(vals, b):
    """tau of the oracle's EXACT filter for an array (one CSR row per value)."""
    import oracle
    n = len(vals)
    rp = np.arange(n + 1, dtype=np.int64)
    _, tau, _ = oracle.filter_csr(n, (rp, np.zeros(n, np.int32), vals), "exact", b)
    return tau


def test_noalloc_threshold_matches_the_oracle(lib):
    import torch
    v = _values(13, 300_000)
    dev = torch.from_numpy(v).cuda()
    for b in (1e-9, 3e-7, 1e-3):
        t_alloc, t_none = _both(lib, dev, v.size, b)
        assert t_none == t_alloc == _tau_oracle(v, b), (b, t_none, t_alloc)


def test_noalloc_threshold_at_capacity_with_ties_and_empty(lib):
    """nnz = SIGN_NOALLOC_MAX_NNZ with few distinct magnitudes, so the select
    keeps many candidates in its fixed scratch; and nnz = 0 (tau = +inf)."""
    import torch
    limit = 1 << 20
    rng = np.random.default_rng(21)
    mags = 10.0 ** rng.uniform(-12, -2, 40)
    v = rng.choice(mags, limit) * np.where(rng.random(limit) < 0.5, -1.0, 1.0)
    dev = torch.from_numpy(v).cuda()
    srt = np.sort(np.abs(v))
    # budgets that end inside big tie groups (and one that keeps everything)
    for b in (math.sqrt(np.sum(srt[: limit // 3] ** 2)), math.sqrt(np.sum(srt[: limit // 2] ** 2)),
              1e9):
        t_alloc, t_none = _both(lib, dev, limit, b)
        assert t_none == t_alloc == _tau_oracle(v, b), (b, t_none, t_alloc)
    empty = torch.zeros(1, dtype=torch.float64, device="cuda")
    out = C.c_double()
    st = lib.sign_threshold_exact_noalloc(C.c_void_p(empty.data_ptr()), 0, 1.0,
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream),
                                          C.byref(out))
    assert st == 0 and out.value == math.inf


def test_noalloc_threshold_takes_no_device_memory(lib):
    """After the library's cached memory is handed back, repeated calls leave
    the device's free memory exactly as it was."""
    import torch
    v = torch.from_numpy(_values(14, 500_000)).cuda()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = C.c_double()
    assert lib.sign_threshold_exact_noalloc(C.c_void_p(v.data_ptr()), v.numel(), 1e-6, stream,
                                            C.byref(out)) == 0
    assert lib.sign_trim_memory() == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for b in (1e-9, 1e-6, 1e-3):
        assert lib.sign_threshold_exact_noalloc(C.c_void_p(v.data_ptr()), v.numel(), b, stream,
                                                C.byref(out)) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_threshold_edge_values_and_limit(lib):
    import torch
    dev = torch.tensor([1e-3, -1e-3, 2e-3, 5.0], dtype=torch.float64, device="cuda")
    for b in (0.0, 1e-3, 2.5e-3, 1e3):
        t_alloc, t_none = _both(lib, dev, 4, b)
        assert t_none == t_alloc
    # more values than the static scratch holds: refused with a message
    limit = 1 << 20
    big = torch.zeros(limit + 1, dtype=torch.float64, device="cuda")
    out = C.c_double()
    st = lib.sign_threshold_exact_noalloc(C.c_void_p(big.data_ptr()), limit + 1, 1.0,
                                          C.c_void_p(torch.cuda.current_stream().cuda_stream),
                                          C.byref(out))
    assert st == 1 and "SIGN_NOALLOC_MAX_NNZ" in lib.sign_last_error().decode()
