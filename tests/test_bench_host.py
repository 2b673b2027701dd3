"""Host-side helpers of bench.py, checked without a GPU."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


@pytest.mark.parametrize("nb", [1, 7, 30])
def test_ode_closed_form_is_the_sign_of_the_block_matrix(nb):
    """Eq. (1.26) from B's sine eigenbasis agrees with scipy's signm of the
    dense block matrix, and is an involution commuting with it."""
    linalg = pytest.importorskip("scipy.linalg")
    import workloads as w
    from workloads import closed_form
    a = w.ode_block(nb)
    A = np.zeros((a.n, a.n))
    A[np.repeat(np.arange(a.n), np.diff(a.rowptr)), a.col] = a.val
    S = closed_form.ode_block_sign(nb)
    assert np.allclose(S @ S, np.eye(a.n), atol=1e-13)
    assert np.allclose(S @ A, A @ S, atol=1e-13)
    assert np.allclose(S, np.real(linalg.signm(A)), atol=1e-10)


def test_filter_error_leg_on_the_oracle(oracle_lib):
    """bench.py's Fig. 4.1.2 leg driven by the oracle on a small SPD matrix:
    the filtered and unfiltered iterates stay within tol = 1e-12 of each other
    at every iteration, as Sec. 4.1 reports."""
    import bench

    def solve(a, filt, max_iter):
        r = oracle_lib.nsf(a, tol=1e-12, filter=filt, max_iter=max_iter)
        return r.status, r.iters, r.rowptr, r.col, r.val

    (res,) = bench.filter_error_leg(solve, [150], seeds=1)
    assert res["ns_status"] == 0 and res["iters"] >= 8
    assert len(res["dX"]) == len(res["dR"]) == res["iters"]
    assert res["max_dX"] < 1e-12 and res["max_dR"] < 1e-12
    assert res["resid"][-1] <= 1e-12 < res["resid"][0]


def test_step_hbm_roofline():
    """The step-level HBM figure sums the classes' algorithmic bytes per step
    and divides by the step time; classes without byte counts add nothing."""
    import bench
    prof = {"numeric_square_f64": {"launches": 25, "ms": 200.0, "flops": 1e12, "bytes": 30e9},
            "filter": {"launches": 60, "ms": 50.0, "flops": 0.0, "bytes": 10e9},
            "bounds": {"launches": 130, "ms": 49.0, "flops": 0.0, "bytes": 0.0}}
    h = bench.step_hbm(prof, 5, 200.0, 8000.0)
    assert h["algorithmic_bytes_per_step"] == 8e9
    assert abs(h["achieved_gbs"] - 40.0) < 1e-9 and abs(h["frac"] - 0.005) < 1e-12
    assert h["covers"] == ["filter", "numeric_square_f64"] and h["peak_gbs"] == 8000.0


@pytest.mark.parametrize("dim,m", [(2, 6), (3, 4)])
def test_laplacian_closed_form_entries_match_eigh(dim, m):
    """The closed-form entries of sign(L - sigma I) agree with the sign from a
    dense eigendecomposition of the shifted Laplacian."""
    import workloads as w
    from workloads import closed_form
    a = w.laplacian(m, dim)
    d = a.to_dense()
    ev, v = np.linalg.eigh(d)
    S = (v * np.sign(ev)) @ v.T
    rng = np.random.default_rng(3)
    p, pp = rng.integers(0, a.n, 200), rng.integers(0, a.n, 200)
    assert np.allclose(closed_form.laplacian_sign_entries(m, dim, p, pp), S[p, pp], atol=1e-12)
    rp = np.arange(a.n + 1) * a.n
    col = np.tile(np.arange(a.n, dtype=np.int32), a.n)
    assert np.array_equal(closed_form.csr_entries(rp, col, S.ravel(), p, pp), S[p, pp])
