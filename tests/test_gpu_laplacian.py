"""The shifted 2-D and 3-D Dirichlet Laplacians at the largest sizes the
dense path serves (n = 4096), against the closed-form sign from the sine
eigenbasis: S = V sign(Lambda - sigma) V^T with V = kron of the 1-D bases,
evaluated at 10^4 seeded entries (an O(m^dim) sum each), and the trace
n_plus - n_minus counted from the closed-form spectrum."""
import numpy as np
import pytest

import workloads as w
from workloads import closed_form

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


def _entries(res, n, p, pp):
    return closed_form.csr_entries(res.rowptr, res.col, res.val, p, pp)


@pytest.mark.parametrize("dim,m,prec,bound", [(2, 64, "fp64", 1e-7), (2, 64, "mixed", 1e-5),
                                              (3, 16, "fp64", 1e-7), (3, 16, "mixed", 1e-5)])
def test_laplacian_sign_against_closed_form(sg, dim, m, prec, bound):
    a = w.laplacian(m, dim)
    n = a.n
    sg.prof_reset()
    sg.prof_enable(True)
    res = sg.solve(a, tol=1e-8, filter="exact", prec=prec, max_iter=200)
    sg.prof_enable(False)
    prof = sg.prof_read()
    assert res.status == sg.SIGN_OK and res.resid <= 1e-8
    # the filled-in iterate ran on the dense paths
    assert prof.get("dense_f64_slices", {}).get("launches", 0) > 0
    if prec == "mixed":
        assert prof.get("dense_tf32x3", {}).get("launches", 0) > 0
    rng = np.random.default_rng(dim * 1000 + m)
    p = rng.integers(0, n, 10000)
    pp = np.where(rng.random(10000) < 0.5, p + rng.integers(-3 * m, 3 * m, 10000),
                  rng.integers(0, n, 10000)) % n  # near and far entries
    ref = closed_form.laplacian_sign_entries(m, dim, p, pp)
    got = _entries(res, n, p, pp)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= bound
    # trace = n_plus - n_minus of the closed-form spectrum
    lam = w.laplacian_eigs(m, dim)
    want = int(np.sum(np.sign(lam - w.laplacian_shift(m, dim))))
    diag = _entries(res, n, np.arange(n), np.arange(n))
    assert round(diag.sum()) == want
