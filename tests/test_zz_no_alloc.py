"""sign_threshold_exact_noalloc, the threshold entry point for callers that
cannot allocate device memory (their own pool already holds the GPU, or their
loop cannot afford cudaMalloc's device-wide synchronization).

It must give the same threshold as the allocating sign_threshold_exact on the
same device values, on consecutive calls that reuse its static scratch, and
refuse inputs larger than its fixed capacity. This file is collected last so
that a failure here leaves every other test already run; it also passes on
its own in a fresh process.
"""
import ctypes as C

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
