"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Both sides accumulate every product in ascending k with one fused
multiply-add, so the iterates are expected to agree bit for bit; the
contract checked everywhere is the FP64 tolerance
||S_gpu - S_ref||_F / ||S_ref||_F <= 1e-10 at equal iteration count, plus
identical sparsity patterns and per-iteration nnz. These tests pin the
sparse path: dense_frac = 2 keeps every matrix off the dense tensor-core
path, whose rounding differs (tests/test_gpu_dense.py checks it within the
tolerance).
"""
import ctypes as C
import math

import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-10


@pytest.fixture(scope="module")
def sg():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_03356_gb300 as sg
    from paper_2210_03356_gb300 import build
    build.build()
    sg.load()
    return sg


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def assert_parity(res, ref, tol=TOL_F64, bitwise=True, trace=True):
    assert res.status == ref.status, (res.status, ref.status)
    assert res.iters == ref.iters, (res.iters, ref.iters)
    assert np.array_equal(res.rowptr, ref.rowptr)
    assert np.array_equal(res.col, ref.col)
    assert _rel(res.val, ref.val) <= tol
    if bitwise:
        assert np.array_equal(res.val, ref.val)
    if trace:
        t, o = res.trace, ref.trace
        assert np.array_equal(t["nnz_x"], o["nnz_x"])
        assert np.array_equal(t["nnz_t"], o["nnz_t"])
        assert np.array_equal(t["prec_k"], o["prec"])
        np.testing.assert_allclose(t["resid_k"], o["resid"], rtol=1e-9, atol=1e-15)
        np.testing.assert_allclose(t["tau_k"], o["tau"], rtol=1e-12)
        np.testing.assert_allclose(t["fnorm_k"], o["fnorm"], rtol=1e-8, atol=1e-300)
    assert abs(res.resid - ref.resid) <= 1e-9 * max(ref.resid, 1e-300) + 1e-16


# ---------------------------------------------------------------- tridiagonal n = 2000
@pytest.mark.parametrize("mode", ["exact", "bound"])
def test_tridiagonal_2000(sg, orc, mode):
    a = w.tridiagonal()
    res = sg.solve(a, tol=1e-8, filter=mode, dense_frac=2.0)
    ref = orc.nsf(a, tol=1e-8, filter=mode)
    assert res.status == sg.SIGN_OK
    assert_parity(res, ref)


def test_tridiagonal_tight_tol_adaptive_budget(sg, orc):
    """tol 1e-12 reaches the Eq. (1.18) phase (r < 1e-6)."""
    a = w.tridiagonal(1200)
    res = sg.solve(a, tol=1e-12, filter="exact", dense_frac=2.0)
    ref = orc.nsf(a, tol=1e-12, filter="exact")
    assert_parity(res, ref)
    assert np.any(res.trace["resid_k"] < 1e-6) and np.any(res.trace["beta_k"] < 1e-16)


def test_unfiltered_ns_dense_fill(sg, orc):
    """filter NONE: plain NS; rows fill in past 1024 columns (CTA kernels)."""
    a = w.tridiagonal(1500)
    res = sg.solve(a, tol=1e-8, filter="none", dense_frac=2.0)
    ref = orc.nsf(a, tol=1e-8, filter="none")
    assert_parity(res, ref)
    assert res.nnz > 0.9 * a.n * a.n


def test_mixed_precision_matches_mixed_oracle(sg, orc):
    a = w.tridiagonal()
    res = sg.solve(a, tol=1e-8, filter="exact", prec=1, dense_frac=2.0)
    ref = orc.nsf(a, tol=1e-8, filter="exact", mixed=True)
    assert_parity(res, ref)
    assert res.trace["prec_k"][0] == 32 and res.trace["prec_k"][-1] == 64
    ref64 = orc.nsf(a, tol=1e-8, filter="exact")
    d = ref64.to_dense(a.n) - res_dense(res, a.n)
    assert np.linalg.norm(d) / np.linalg.norm(ref64.to_dense(a.n)) < 1e-6


def _with_explicit_zeros(a, b):
    """a with every other entry of its outermost diagonals stored as +0 or -0."""
    rows = np.repeat(np.arange(a.n), np.diff(a.rowptr))
    val = a.val.copy()
    edge = np.abs(a.col - rows) == b
    key = np.minimum(rows, a.col)[edge]      # the same sign for (i, j) and (j, i)
    val[np.flatnonzero(edge)[key % 2 == 0]] = np.where(key[key % 2 == 0] % 4 == 0, -0.0, 0.0)
    return w.CSR(a.n, a.rowptr, a.col, val)


@pytest.mark.parametrize("filt,max_iter", [("none", 1), ("none", 3), ("exact", 100)])
def test_explicit_zeros_keep_pattern_and_signs(sg, orc, filt, max_iter):
    """Products that are all +-0 still create their entry, with the value +0.

    Explicit zeros on the outermost diagonals make some entries of X X and
    X T reachable only through a zero factor; the FP32 accumulators mark
    untouched slots with -0, so these entries test that marking. Signs of
    zeros are compared bit for bit.
    """
    a = _with_explicit_zeros(w.banded(400, 5, w.BASE_SEED + 77), 5)
    assert np.signbit(a.val[a.val == 0]).any() and (~np.signbit(a.val[a.val == 0])).any()
    res = sg.solve(a, tol=1e-8, filter=filt, prec=1, max_iter=max_iter, dense_frac=2.0)
    ref = orc.nsf(a, tol=1e-8, filter=filt, mixed=True, max_iter=max_iter)
    assert_parity(res, ref)
    assert np.array_equal(res.val.view(np.uint64), ref.val.view(np.uint64))
    if filt == "none" and max_iter == 1:
        assert (ref.val == 0).any()  # the case arises: entries whose products were all zero


def res_dense(res, n):
    d = np.zeros((n, n))
    d[np.repeat(np.arange(n), np.diff(res.rowptr)), res.col] = res.val
    return d


def test_deterministic_runs(sg):
    a = w.tridiagonal()
    r1 = sg.solve(a, tol=1e-8, filter="exact", dense_frac=2.0)
    r2 = sg.solve(a, tol=1e-8, filter="exact", dense_frac=2.0)
    assert np.array_equal(r1.val, r2.val) and np.array_equal(r1.col, r2.col)


# ---------------------------------------------------------------- wide rows
@pytest.mark.parametrize("m,dim", [(24, 2), (8, 3)])
def test_shifted_laplacians(sg, orc, m, dim):
    a = w.laplacian(m, dim)
    res = sg.solve(a, tol=1e-8, filter="exact", max_iter=200, dense_frac=2.0)
    ref = orc.nsf(a, tol=1e-8, filter="exact", max_iter=200)
    assert_parity(res, ref)
    assert res.status == sg.SIGN_OK


def _two_scale(n, far, seed):
    rng = np.random.default_rng(seed)
    i = np.arange(n)
    d = np.where(rng.random(n) < 0.5, -1.0, 1.0) * (1.5 + 0.5 * rng.random(n))
    rows, cols, vals = [i], [i], [d]
    for off, scale in ((1, 0.2), (far, 0.15)):
        j = np.arange(n - off)
        v = scale * rng.uniform(-1, 1, n - off)
        rows += [j, j + off]
        cols += [j + off, j]
        vals += [v, v]
    return w.csr_from_coo(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))


def test_multichunk_rows(sg, orc):
    """Rows whose column range spans several shared-memory chunks."""
    a = _two_scale(30000, 10000, 5)
    res = sg.solve(a, tol=1e-8, filter="exact", dense_frac=2.0)
    ref = orc.nsf(a, tol=1e-8, filter="exact")
    assert_parity(res, ref)


# ---------------------------------------------------------------- the paper's Sec. 4.2 matrix
def test_ode_block_unscaled_nonsymmetric(sg, orc):
    a = w.ode_block(400)
    res = sg.solve(a, tol=1e-12, filter="exact", scale_1norm=0, dense_frac=2.0)
    ref = orc.nsf(a, tol=1e-12, filter="exact", scale_1norm=False)
    assert_parity(res, ref)


def test_nonsymmetric_onenorm_scaling(sg, orc):
    a = w.ode_block(300)
    res = sg.solve(a, tol=1e-10, filter="bound", dense_frac=2.0)
    ref = orc.nsf(a, tol=1e-10, filter="bound")
    assert_parity(res, ref)


# ---------------------------------------------------------------- batches
def test_batch_matches_lone_solves_and_oracle(sg, orc):
    shapes = w.banded_batch_shapes(24, nmin=200, nmax=1500)
    mats = [w.banded(n, b, s) for n, b, s in shapes]
    out = sg.solve_batch(mats, tol=1e-8, filter="exact", dense_frac=2.0)
    for a, res in zip(mats, out):
        ref = orc.nsf(a, tol=1e-8, filter="exact")
        assert_parity(res, ref)
    for a, res in list(zip(mats, out))[:4]:
        alone = sg.solve(a, tol=1e-8, filter="exact", dense_frac=2.0)
        assert np.array_equal(alone.val, res.val) and alone.iters == res.iters


def test_batch_mixed_precision_moves_per_matrix(sg, orc):
    shapes = w.banded_batch_shapes(12, nmin=200, nmax=900)
    mats = [w.banded(n, b, s) for n, b, s in shapes]
    # sparse FP32 products only (dense_frac > 1): bit-for-bit with the oracle
    out = sg.solve_batch(mats, tol=1e-8, filter="exact", prec=1, dense_frac=2.0)
    for a, res in zip(mats, out):
        ref = orc.nsf(a, tol=1e-8, filter="exact", mixed=True)
        assert_parity(res, ref)


def test_batch_full_512_sampled(sg, orc):
    """The 512-matrix banded batch in one call; sampled matrices vs the oracle."""
    shapes = w.banded_batch_shapes()
    mats = [w.banded(n, b, s) for n, b, s in shapes]
    out = sg.solve_batch(mats, tol=1e-8, filter="exact", prec=1, dense_frac=2.0)
    assert all(r.status == sg.SIGN_OK for r in out)
    order = np.argsort([n * (b + 1) for n, b, _ in shapes])
    sample = [int(order[-1]), int(order[len(order) // 2]), int(order[0]), 7]
    for i in sample:
        ref = orc.nsf(mats[i], tol=1e-8, filter="exact", mixed=True)
        assert_parity(out[i], ref)
    # every result is an involution to the requested tolerance
    assert max(r.resid for r in out) <= 1e-8


def _dense_records(res, n, o):
    """Records of a result whose round ran the dense tensor-core path, by the
    solver's rule: a filter on, n <= 32768 and nnz(X_k) >= dense_frac n^2, and
    in the FP64 stage also n >= dense64_min_n."""
    t = res.trace
    dense = (t["nnz_x"] >= o.dense_frac * n * n) & (n <= 32768) & (o.filter != 0)
    return dense & ((t["prec_k"] == 32) | (n >= o.dense64_min_n))


def test_batch_full_512_bench_options(sg, orc):
    """The benchmark's own configuration, all options at their defaults
    (dense_frac 0.25, dense64_min_n 1024; mixed, EXACT, tol 1e-8): the full
    batch of 512 in one call. Every member that took the dense tensor-core
    path is compared with the oracle's mixed run within the dense path's
    1e-5 (relative Frobenius; its products round differently), and a spread
    of the others, which stay on the sparse path, bit for bit."""
    shapes = w.banded_batch_shapes()
    mats = [w.banded(n, b, s) for n, b, s in shapes]
    o = sg.default_opts(tol=1e-8, filter="exact", prec="mixed")
    assert o.dense_frac == 0.25 and o.dense64_min_n == 1024
    sg.prof_reset()
    sg.prof_enable(True)
    out = sg.solve_batch(mats, opts=o)
    sg.prof_enable(False)
    prof = sg.prof_read()
    assert all(r.status == sg.SIGN_OK for r in out)
    assert max(r.resid for r in out) <= 1e-8
    assert prof.get("dense_tf32x3", {}).get("launches", 0) > 0  # the dense path ran
    dense = [i for i, (a, r) in enumerate(zip(mats, out)) if _dense_records(r, a.n, o).any()]
    assert dense, "no member met the dense path's rule"
    order = [i for i in np.argsort([n * (b + 1) for n, b, _ in shapes]) if i not in dense]
    sparse = [int(order[j]) for j in np.linspace(0, len(order) - 1, 12).astype(int)]
    refs = orc.nsf_many([mats[i] for i in dense + sparse], tol=1e-8, filter="exact", mixed=True)
    for i, ref in zip(dense, refs[:len(dense)]):
        n = mats[i].n
        err = _rel(res_dense(out[i], n), ref.to_dense(n))
        assert err <= 1e-5, (i, n, err)
    for i, ref in zip(sparse, refs[len(dense):]):
        assert not _dense_records(out[i], mats[i].n, o).any()
        assert_parity(out[i], ref)


# ---------------------------------------------------------------- device pointers
def test_device_pointers_in_and_out(sg, orc):
    import torch
    a = w.tridiagonal(800)
    class T:  # CSR of CUDA tensors
        n = a.n
        rowptr = torch.from_numpy(a.rowptr).cuda()
        col = torch.from_numpy(a.col).cuda()
        val = torch.from_numpy(a.val).cuda()
    res = sg.solve(T, tol=1e-8, filter="exact", device_out=True, dense_frac=2.0)
    ref = orc.nsf(a, tol=1e-8, filter="exact")
    assert res.val.is_cuda
    assert np.array_equal(res.val.cpu().numpy(), ref.val)
    assert np.array_equal(res.col.cpu().numpy(), ref.col)


# ---------------------------------------------------------------- edge cases
def test_edge_cases(sg, orc):
    one = w.csr_from_dense(np.array([[-3.0]]))
    r = sg.solve(one, tol=1e-14, dense_frac=2.0)
    assert r.status == sg.SIGN_OK and r.val[0] == -1.0 and r.iters == 0
    # singular (empty row): never converges
    sing = w.csr_from_dense(np.diag([1.0, 0.0, -2.0]))
    r = sg.solve(sing, tol=1e-12, max_iter=30, dense_frac=2.0)
    ref = orc.nsf(sing, tol=1e-12, max_iter=30)
    assert r.status == sg.SIGN_ENOTCONV and r.iters == 30
    assert_parity(r, ref)
    # unscaled 3I leaves the region of convergence
    big = w.csr_from_dense(3.0 * np.eye(4))
    r = sg.solve(big, scale_1norm=0, filter="none", dense_frac=2.0)
    assert r.status == sg.SIGN_EDIVERGED == orc.nsf(big, scale_1norm=False, filter="none").status
    # max_iter = 0: the scaled input comes back with its residual
    a = w.tridiagonal(300)
    r = sg.solve(a, max_iter=0, dense_frac=2.0)
    ref = orc.nsf(a, max_iter=0)
    assert r.status == sg.SIGN_ENOTCONV and r.iters == 0
    assert_parity(r, ref)


def test_invalid_inputs_rejected(sg):
    from paper_2210_03356_gb300 import Handle, SignError
    bad = w.CSR(2, np.array([0, 2, 3], np.int64), np.array([1, 0, 1], np.int32), np.ones(3))
    with pytest.raises(SignError) as e:
        Handle(bad)
    assert e.value.status == sg.SIGN_EINVAL
    nan = w.CSR(2, np.array([0, 1, 2], np.int64), np.array([0, 1], np.int32),
                np.array([1.0, np.nan]))
    with pytest.raises(SignError):
        Handle(nan)
    out_of_range = w.CSR(2, np.array([0, 1, 2], np.int64), np.array([0, 2], np.int32), np.ones(2))
    with pytest.raises(SignError):
        Handle(out_of_range)
    z = w.CSR(3, np.array([0, 0, 0, 0], np.int64), np.zeros(0, np.int32), np.zeros(0))
    with pytest.raises(SignError) as e:
        sg.solve(z, dense_frac=2.0)
    assert e.value.status == sg.SIGN_EINVAL
    with pytest.raises(SignError):
        sg.solve(w.tridiagonal(10), filter=7)


def test_create_batch_names_the_bad_matrix_and_reads_into_caller_buffers(sg):
    import torch
    from paper_2210_03356_gb300 import Batch, SignError
    good = [w.tridiagonal(300), w.banded(500, 3, 11)]
    bad = w.CSR(2, np.array([0, 2, 3], np.int64), np.array([1, 0, 1], np.int32), np.ones(3))
    with pytest.raises(SignError) as e:
        Batch(good + [bad] + good)
    assert e.value.status == sg.SIGN_EINVAL and "matrix 2" in str(e.value)
    class T:  # the same CSR as CUDA tensors
        n = good[0].n
        rowptr = torch.from_numpy(good[0].rowptr).cuda()
        col = torch.from_numpy(good[0].col).cuda()
        val = torch.from_numpy(good[0].val).cuda()
    with pytest.raises(ValueError):
        Batch([good[0], T])
    opts = sg.default_opts(tol=1e-8, dense_frac=2.0)
    for mats in (good, [T, T]):
        b = Batch(mats)
        try:
            b.solve(opts)
            h = b.handles[0]
            rp, col, val = h.result()
            nnz = h.result_nnz()
            assert nnz == col.size
            pin = (torch.empty(h.n + 1, dtype=torch.int64, pin_memory=True).numpy(),
                   torch.empty(nnz + 5, dtype=torch.int32, pin_memory=True).numpy(),
                   torch.empty(nnz + 5, dtype=torch.float64, pin_memory=True).numpy())
            rp2, col2, val2 = h.result(out=pin)
            assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
            assert np.array_equal(val, val2)
            with pytest.raises(ValueError):
                h.result(out=(pin[0], pin[1][:nnz - 1], pin[2]))
            outs = [(np.empty(x.n + 1, np.int64), np.empty(x.result_nnz() + 3, np.int32),
                     np.empty(x.result_nnz() + 3, np.float64)) for x in b.handles]
            for x, (rp3, col3, val3) in zip(b.handles, b.results(outs)):
                r1, c1, v1 = x.result()
                assert np.array_equal(r1, rp3) and np.array_equal(c1, col3)
                assert np.array_equal(v1, val3)
        finally:
            b.close()
    # results before any solve: refused, naming the handle
    b = Batch(good)
    try:
        outs = [(np.empty(x.n + 1, np.int64), np.empty(1, np.int32), np.empty(1, np.float64))
                for x in b.handles]
        with pytest.raises(SignError) as e:
            b.results(outs)
        assert e.value.status == sg.SIGN_ESTATE
    finally:
        b.close()


def test_batch_transfers_pinned_device_and_pageable(sg):
    """sign_create_batch and sign_get_csr_batch take one gather kernel when
    every array is pinned host or device memory, and one copy per array
    otherwise: the handles and results must be the same either way, and a
    malformed matrix read through the gather must still be named."""
    import torch
    from paper_2210_03356_gb300 import Batch, SignError
    shapes = w.banded_batch_shapes(12, nmin=200, nmax=2500)
    mats = [w.banded(n, b, s) for n, b, s in shapes] + [w.tridiagonal(777)]

    def pinned(a):
        t = [torch.from_numpy(x).pin_memory() for x in (a.rowptr, a.col, a.val)]
        return type("P", (), {"n": a.n, "rowptr": t[0].numpy(), "col": t[1].numpy(),
                              "val": t[2].numpy(), "_keep": t})

    def on_dev(a):
        return type("D", (), {"n": a.n, "rowptr": torch.from_numpy(a.rowptr).cuda(),
                              "col": torch.from_numpy(a.col).cuda(),
                              "val": torch.from_numpy(a.val).cuda()})

    opts = sg.default_opts(tol=1e-8, filter="exact", prec="mixed", dense_frac=2.0)
    ref = None
    for make in (lambda a: a, pinned, on_dev,
                 lambda a: pinned(a) if a.n % 2 else a):  # pinned and pageable mixed
        b = Batch([make(a) for a in mats])
        try:
            b.solve(opts)
            nnz = [h.result_nnz() for h in b.handles]
            assert b.result_nnz() == nnz
            pin = [tuple(torch.empty(k, dtype=d, pin_memory=True).numpy()
                         for k, d in ((h.n + 1, torch.int64), (z, torch.int32),
                                      (z, torch.float64)))
                   for h, z in zip(b.handles, nnz)]
            page = [(np.empty(h.n + 1, np.int64), np.empty(z, np.int32), np.empty(z, np.float64))
                    for h, z in zip(b.handles, nnz)]
            got_pin = [tuple(x.copy() for x in r) for r in b.results(pin)]
            got_page = b.results(page)
            for (r1, c1, v1), (r2, c2, v2) in zip(got_pin, got_page):
                assert np.array_equal(r1, r2) and np.array_equal(c1, c2)
                assert np.array_equal(v1.view(np.uint64), v2.view(np.uint64))
            if ref is None:
                ref = got_pin
            for (r1, c1, v1), (r2, c2, v2) in zip(got_pin, ref):
                assert np.array_equal(r1, r2) and np.array_equal(c1, c2)
                assert np.array_equal(v1.view(np.uint64), v2.view(np.uint64))
        finally:
            b.close()
    bad = w.CSR(3, np.array([0, 1, 3, 4], np.int64), np.array([0, 2, 1, 2], np.int32),
                np.array([1.0, 2.0, np.nan, 1.0]))
    with pytest.raises(SignError) as e:
        Batch([pinned(a) for a in mats[:3]] + [pinned(bad)])
    assert e.value.status == sg.SIGN_EINVAL and "matrix 3" in str(e.value)


def test_trim_memory_between_solves(sg):
    """Kept blocks and pool memory handed back; the next solve is unchanged."""
    mats = [w.banded(n, b, s) for n, b, s in w.banded_batch_shapes(6, nmin=200, nmax=900)]
    first = sg.solve_batch(mats, tol=1e-8, filter="exact", prec=1, dense_frac=2.0)
    sg.trim_memory()
    again = sg.solve_batch(mats, tol=1e-8, filter="exact", prec=1, dense_frac=2.0)
    for r1, r2 in zip(first, again):
        assert np.array_equal(r1.col, r2.col) and np.array_equal(r1.val, r2.val)


# ---------------------------------------------------------------- threshold select (step a5)
def _tau_ref(orc, vals, b):
    """tau of the oracle's EXACT filter for an array (laid out as one CSR row per value)."""
    n = len(vals)
    rp = np.arange(n + 1, dtype=np.int64)
    col = np.zeros(n, np.int32)
    _, tau, _ = orc.filter_csr(n, (rp, col, vals), "exact", b)
    return tau


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_threshold_exact_matches_oracle(sg, orc, seed):
    rng = np.random.default_rng(seed)
    n = 200_000
    vals = rng.standard_normal(n) * 10.0 ** rng.uniform(-14, 0, n)
    vals[rng.integers(0, n, 500)] = 0.0
    ties = rng.integers(0, n, 3000)
    vals[ties] = np.sign(vals[ties]) * 3.0e-9  # a tie group near the crossing
    for b in [0.0, 1e-12, 1e-9, 2e-7, 1e-4, 1.0, 1e6]:
        t_gpu = sg.threshold_exact(vals, b)
        t_ref = _tau_ref(orc, vals, b)
        assert t_gpu == t_ref, (b, t_gpu, t_ref)


def test_threshold_exact_edge_cases(sg, orc):
    assert sg.threshold_exact(np.zeros(0), 1.0) == math.inf
    assert sg.threshold_exact(np.zeros(5), 1.0) == math.inf
    v = np.array([1e-3, -1e-3, 2e-3, 5.0])
    for b in (0.0, 1e-3, 1.5e-3, 2.5e-3, 1e3):
        assert sg.threshold_exact(v, b) == _tau_ref(orc, v, b)
    with pytest.raises(Exception):
        sg.threshold_exact(v, -1.0)


def test_threshold_exact_boundary(sg, orc):
    """Squares that add up to exactly b^2 fit the budget (Alg. 3.2.1 step 4:
    dropped while the sum stays within it); one more tips it over. Every
    square here is exact in FP64, so the oracle's sums are exact too."""
    cases = [
        ([0.5] * 4 + [2.0], 1.0),          # 4 x 0.25 = 1 = b^2: all fit
        ([0.5] * 5 + [2.0], 1.0),          # 1.25 > 1: the 0.5 group is kept
        ([0.375] * 4 + [1.0], 0.75),       # 4 x 0.140625 = 0.5625 = b^2
        ([0.375] * 4 + [2.0 ** -20, 1.0], 0.75),  # the same plus a small square
        ([0.25] * 16 + [0.25 + 2.0 ** -54], 1.0),  # 16 x 1/16 = 1, then just above
        ([3.0 * 2.0 ** -1060] * 3, 2.0 ** -1055),  # subnormal values and budget
        ([1e-300] * 7 + [1e300], 3e-300),
    ]
    for v, b in cases:
        v = np.array(v, dtype=np.float64)
        for w in (v, -v[::-1]):
            assert sg.threshold_exact(w, b) == _tau_ref(orc, w, b), (v, b)
