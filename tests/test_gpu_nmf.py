"""NMF (Alg. 3.1.1) on the GPU against the oracle's NMF, bit for bit: the
check's sparse product, the dense inverse (LU with partial pivoting and the
column solves in the oracle's operation order), Xbar = (X + X^-1)/2, the
budget of Eq. (1.13) and the EXACT filter. With filter NONE it is Newton's
method (Eq. 1.1). Also Sec. 4.1's first filter-error test (Fig. 4.1.1, NM
against NMF on sprand-like matrices) and Sec. 4.2's block matrix against its
closed form."""
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
    for k, ko in (("nnz_x", "nnz_x"), ("nnz_t", "nnz_t"), ("nnz_bar", "nnz_bar")):
        assert np.array_equal(t[k], o[ko]), k
    np.testing.assert_allclose(t["resid_k"], o["resid"], rtol=1e-9, atol=1e-15)
    np.testing.assert_allclose(t["beta_k"], o["beta"], rtol=1e-9, atol=0)
    # EXACT selects tau among the entries (exact); BOUND computes it from b,
    # whose residual factor may differ in the last bit
    np.testing.assert_allclose(t["tau_k"], o["tau"], rtol=1e-12, atol=0)


@pytest.mark.parametrize("n,filt", [(300, "exact"), (800, "exact"), (500, "bound"), (400, "none")])
def test_nmf_matches_oracle(sg, orc, n, filt):
    a = w.sprand_like(n, 0.01, seed=w.BASE_SEED + 8100 + n)
    res = sg.solve(a, tol=1e-12, filter=filt, method="nmf")
    ref = orc.nmf(a, tol=1e-12, filter=filt)
    assert ref.status == orc.OK
    _parity(res, ref)


def test_newton_matches_dense_newton(sg, orc):
    """filter NONE: Newton's method, against the oracle's dense NM."""
    a = w.sprand_like(250, 0.01, seed=w.BASE_SEED + 8200)
    res = sg.solve(a, tol=1e-12, filter="none", method="nmf")
    S, iters, resid, st = orc.nm_dense(a.to_dense(), tol=1e-12)
    D = np.zeros((a.n, a.n))
    D[np.repeat(np.arange(a.n), np.diff(res.rowptr)), res.col] = res.val
    assert res.status == sg.SIGN_OK and res.iters == iters
    assert np.linalg.norm(D - S) / np.linalg.norm(S) < 1e-12


def test_nmf_ode_block_against_closed_form(sg, orc):
    """Sec. 4.2's [[0, B], [I, 0]] by NMF, within the paper's AE of Eq. (1.26)."""
    from workloads import closed_form
    nb = 200
    a = w.ode_block(nb)
    res = sg.solve(a, tol=1e-12, filter="exact", method="nmf")
    ref = orc.nmf(a, tol=1e-12, filter="exact")
    _parity(res, ref)
    D = np.zeros((a.n, a.n))
    D[np.repeat(np.arange(a.n), np.diff(res.rowptr)), res.col] = res.val
    assert np.abs(D - closed_form.ode_block_sign(nb)).max() < 1e-12


def test_nmf_batch_and_singular_and_options(sg, orc):
    mats = [w.sprand_like(n, 0.01, seed=w.BASE_SEED + 8300 + n) for n in (200, 350, 500)]
    sing = w.csr_from_dense(np.diag([1.0, 0.0, -2.0]))
    out = sg.solve_batch(mats + [sing], tol=1e-12, filter="exact", method="nmf")
    for a, r in zip(mats, out):
        _parity(r, orc.nmf(a, tol=1e-12, filter="exact"))
    r, ref = out[-1], orc.nmf(sing, tol=1e-12, filter="exact")
    assert r.status == sg.SIGN_EDIVERGED == ref.status and r.iters == ref.iters == 0
    assert np.array_equal(r.val, sing.val)  # the iterate X_1 = A is the result
    with pytest.raises(sg.SignError) as e:
        sg.solve(mats[0], tol=1e-12, method="nmf", prec="mixed")
    assert e.value.status == sg.SIGN_EINVAL


def test_fig_4_1_1_nm_vs_nmf(sg):
    """Sec. 4.1's first test: NM and NMF (EXACT) to tol 1e-12 on sprand-like
    matrices; the filtered and unfiltered iterates stay within tol."""
    import bench

    def gpu_solve(a, filt, max_iter):
        r = sg.solve(a, tol=1e-12, filter=filt, method="nmf", max_iter=max_iter)
        return r.status, r.iters, r.rowptr, r.col, r.val

    runs = bench.filter_error_leg(
        gpu_solve, [500], seeds=2,
        make=lambda n, s: w.sprand_like(n, 0.01, seed=w.BASE_SEED + 8000 + 10 * n + s))
    for run in runs:
        assert run["ns_status"] == sg.SIGN_OK and run["iters"] >= 3
        assert max(run["dX"]) < 1e-12 and max(run["dR"]) < 1e-12, run
