"""The two variants of the readings on the GPU against the oracle's, bit for
bit: T = X^2 filtered with the same budget before the update (filter_t) and
the 2-norm of X, estimated by power steps, in the budget of Eq. (1.18)
(budget_norm). The sparse path keeps one fused multiply-add per product in
ascending k, so the iterates, patterns and thresholds are the oracle's."""
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


def _parity(res, ref):
    assert res.status == ref.status and res.iters == ref.iters
    assert np.array_equal(res.rowptr, ref.rowptr) and np.array_equal(res.col, ref.col)
    assert np.array_equal(res.val, ref.val)
    t, o = res.trace, ref.trace
    for k, ko in (("nnz_x", "nnz_x"), ("nnz_t", "nnz_t"), ("nnz_that", "nnz_that"),
                  ("prec_k", "prec")):
        assert np.array_equal(t[k], o[ko]), k
    np.testing.assert_allclose(t["beta_k"], o["beta"], rtol=1e-12, atol=0)
    np.testing.assert_allclose(t["tau_k"], o["tau"], rtol=1e-12)


CASES = [
    ("tridiagonal", lambda: w.tridiagonal(1200), 1e-12, "fp64"),
    ("banded", lambda: w.banded(900, 6, w.BASE_SEED + 911), 1e-12, "fp64"),
    ("banded_mixed", lambda: w.banded(1500, 4, w.BASE_SEED + 912), 1e-8, "mixed"),
]


@pytest.mark.parametrize("name,make,tol,prec", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("filt", ["exact", "bound"])
def test_filtered_t_matches_oracle(sg, orc, name, make, tol, prec, filt):
    a = make()
    res = sg.solve(a, tol=tol, filter=filt, prec=prec, filter_t=1)
    ref = orc.nsf(a, tol=tol, filter=filt, mixed=prec == "mixed", filter_t=True)
    _parity(res, ref)
    assert np.any(res.trace["nnz_that"] < res.trace["nnz_t"])  # T was filtered


@pytest.mark.parametrize("name,make,tol,prec", CASES, ids=[c[0] for c in CASES])
def test_budget_norm_matches_oracle(sg, orc, name, make, tol, prec):
    a = make()
    res = sg.solve(a, tol=tol, filter="exact", prec=prec, budget_norm=1)
    ref = orc.nsf(a, tol=tol, filter="exact", mixed=prec == "mixed", budget_norm="2")
    _parity(res, ref)


def test_both_variants_in_a_batch(sg, orc):
    shapes = w.banded_batch_shapes(10, nmin=200, nmax=1500)
    mats = [w.banded(n, b, s) for n, b, s in shapes]
    out = sg.solve_batch(mats, tol=1e-12, filter="exact", prec="fp64", filter_t=1, budget_norm=1)
    for i in (0, 4, 9):
        ref = orc.nsf(mats[i], tol=1e-12, filter="exact", filter_t=True, budget_norm="2")
        _parity(out[i], ref)
