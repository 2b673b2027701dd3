"""The FP32 band-tile products against the row-wise FP32 products and the
oracle's mixed run, bit for bit: every stored product enters its output in
ascending k with one fused multiply-add from +0, and the staged zeros of the
band's holes leave the sums unchanged, so the values and the patterns are
the same as the row-wise kernels' and the oracle's."""
import numpy as np
import pytest

import workloads as w

pytestmark = pytest.mark.gpu


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


def _same(r1, r2):
    assert r1.status == r2.status and r1.iters == r2.iters
    assert np.array_equal(r1.rowptr, r2.rowptr) and np.array_equal(r1.col, r2.col)
    assert np.array_equal(r1.val.view(np.uint64), r2.val.view(np.uint64))
    for k in ("nnz_x", "nnz_t", "nnz_bar", "tau_k"):
        assert np.array_equal(r1.trace[k], r2.trace[k]), k


def _with_explicit_zeros(a, b):
    rows = np.repeat(np.arange(a.n), np.diff(a.rowptr))
    val = a.val.copy()
    edge = np.abs(a.col - rows) == b
    key = np.minimum(rows, a.col)[edge]
    val[np.flatnonzero(edge)[key % 2 == 0]] = np.where(key[key % 2 == 0] % 4 == 0, -0.0, 0.0)
    return w.CSR(a.n, a.rowptr, a.col, val)


CASES = {
    "banded_b3": lambda: w.banded(1000, 3, w.BASE_SEED + 901),
    "banded_b10": lambda: w.banded(2500, 10, w.BASE_SEED + 902),
    "tridiagonal": lambda: w.tridiagonal(1700),
    "laplacian2d_m24": lambda: w.laplacian(24, 2),
    "zeros_b5": lambda: _with_explicit_zeros(w.banded(400, 5, w.BASE_SEED + 77), 5),
    "spd_random": lambda: w.spd_random(600, 0.01, seed=w.BASE_SEED + 903),
}


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("filt", ["exact", "bound", "none"])
def test_band_tiles_match_rowwise_and_oracle(sg, orc, name, filt):
    a = CASES[name]()
    kw = dict(tol=1e-8, filter=filt, prec="mixed", dense_frac=2.0, max_iter=100 if filt != "none" else 4)
    sg.prof_reset()
    sg.prof_enable(True)
    on = sg.solve(a, fp32_band=1, **kw)
    sg.prof_enable(False)
    ran = sg.prof_read().get("band_layout", {}).get("launches", 0)
    off = sg.solve(a, fp32_band=0, **kw)
    _same(on, off)
    ref = orc.nsf(a, tol=1e-8, filter=filt, mixed=True, max_iter=kw["max_iter"])
    assert on.iters == ref.iters and np.array_equal(on.col, ref.col)
    assert np.array_equal(on.val.view(np.uint64), ref.val.view(np.uint64))
    assert np.array_equal(on.trace["nnz_t"], ref.trace["nnz_t"])
    if name.startswith("banded") or name == "tridiagonal":
        assert ran > 0  # band tiles were taken


def test_band_tiles_in_a_batch(sg, orc):
    """A batch of banded matrices of mixed widths: band tiles and row-wise rows
    side by side in the same launches, every member equal to its lone solve
    without band tiles."""
    shapes = w.banded_batch_shapes(20, nmin=200, nmax=3000)
    mats = [w.banded(n, b, s) for n, b, s in shapes]
    kw = dict(tol=1e-8, filter="exact", prec="mixed", dense_frac=2.0)
    on = sg.solve_batch(mats, fp32_band=1, **kw)
    off = sg.solve_batch(mats, fp32_band=0, **kw)
    for r1, r2 in zip(on, off):
        _same(r1, r2)
    for i in (0, 7, 19):
        ref = orc.nsf(mats[i], tol=1e-8, filter="exact", mixed=True)
        assert np.array_equal(on[i].val.view(np.uint64), ref.val.view(np.uint64))
