"""Sec. 4.1's filter-error test (Fig. 4.1.2) on the GPU: random sparse SPD
matrices of density 1% (the stand-in for sprandsym(n, 0.01, 1)), NS and NSF
(EXACT) in FP64 to tol 1e-12. After every update k the filtered and
unfiltered iterates differ by dX_k = Xhat_k - X_k and their residuals by
dR_k = Rhat_k - R_k (RMS-Frobenius); the paper shows both below tol at every
k, which is what Eq. (1.22) and Thm 3.2.1 predict."""
import pytest

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


def test_fig_4_1_2_filtered_and_unfiltered_iterates_stay_within_tol(sg):
    import bench

    def gpu_solve(a, filt, max_iter):
        r = sg.solve(a, tol=1e-12, filter=filt, prec="fp64", max_iter=max_iter)
        return r.status, r.iters, r.rowptr, r.col, r.val

    runs = bench.filter_error_leg(gpu_solve, [500], seeds=2)
    for run in runs:
        assert run["ns_status"] == sg.SIGN_OK and run["iters"] >= 5
        assert max(run["dX"]) < 1e-12 and max(run["dR"]) < 1e-12, run
