"""The dense tensor-core product (split TF32 on tcgen05) against an FP64
reference: it must keep about FP32 accuracy, far below what a single TF32
pass (10-bit mantissa) would give."""
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


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (128, 128, 128), (256, 384, 160),
                                   (200, 300, 100), (1000, 516, 260), (64, 4, 12),
                                   (4096, 2048, 64), (3000, 1284, 36), (4096, 4096, 4096)])
def test_dense_product_matches_fp64(sg, M, N, K):
    import torch
    g = torch.Generator(device="cuda").manual_seed(M * 7 + N * 3 + K)
    a = torch.randn(M, K, device="cuda", generator=g, dtype=torch.float32)
    b = torch.randn(K, N, device="cuda", generator=g, dtype=torch.float32)
    c = sg.dense_product(a, b)
    torch.cuda.synchronize()
    ref = a.double() @ b.double()
    scale = (a.double().abs() @ b.double().abs())
    err = ((c.double() - ref).abs() / scale.clamp_min(1e-30)).max().item()
    # FP32 level: rounding of random-sign FP32 sums grows like sqrt(K) u (u = 2^-24),
    # plus the split's dropped lo*lo term (< 2^-22); one TF32 pass would give ~1e-3
    tol = 2.0 ** -24 * (8 + 4 * K ** 0.5)
    assert err < tol, (err, tol)


def test_dense_product_exact_zeros_and_identity(sg):
    import torch
    n = 256
    x = torch.zeros(n, n, device="cuda")
    x[:100, :100] = torch.randn(100, 100, device="cuda")
    eye = torch.eye(n, device="cuda")
    c = sg.dense_product(x, eye)
    # hi * 1 is exact; lo * 1 keeps the 10-bit TF32 part of lo (|lo| <= 2^-11 |x|)
    assert ((c - x).abs() <= x.abs() * 2.0 ** -20).all()
    c2 = sg.dense_product(x, x)
    assert torch.count_nonzero(c2[100:, :]) == 0 and torch.count_nonzero(c2[:, 100:]) == 0


def test_dense_product_rejects_misaligned(sg):
    import torch
    a = torch.randn(8, 6, device="cuda")
    b = torch.randn(6, 8, device="cuda")
    with pytest.raises(Exception):
        sg.dense_product(a, b)  # K = 6 is not a multiple of 4


# ---------------------------------------------------------------- the dense path in the solver
def _dense(res, n):
    import numpy as np
    d = np.zeros((n, n))
    d[np.repeat(np.arange(n), np.diff(res.rowptr)), res.col] = res.val
    return d


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _dense_launches(sg):
    return sg.prof_read().get("dense_tf32x3", {}).get("launches", 0)


@pytest.mark.parametrize("case", ["banded", "laplacian"])
def test_solver_dense_path_matches_oracle(sg, orc, case):
    """Matrices whose FP32 iterate fills in take the tensor-core path; the
    result agrees with the oracle's mixed run to FP32-stage accuracy and is an
    involution to the requested tolerance."""
    import numpy as np
    import workloads as w
    a = w.banded(300, 10, 1234) if case == "banded" else w.laplacian(18, 2)
    sg.prof_reset()
    sg.prof_enable(True)
    res = sg.solve(a, tol=1e-8, filter="exact", prec=1, dense_frac=0.25, max_iter=200)
    sg.prof_enable(False)
    assert _dense_launches(sg) > 0
    assert res.status == sg.SIGN_OK and res.resid <= 1e-8
    ref = orc.nsf(a, tol=1e-8, filter="exact", mixed=True, max_iter=200)
    ref64 = orc.nsf(a, tol=1e-8, filter="exact", max_iter=200)
    S, R, R64 = _dense(res, a.n), ref.to_dense(a.n), ref64.to_dense(a.n)
    assert np.linalg.norm(S - R) / np.linalg.norm(R) < 1e-5
    assert np.linalg.norm(S - R64) / np.linalg.norm(R64) < 1e-5
    assert np.linalg.norm(S @ S - np.eye(a.n)) / np.sqrt(a.n) < 1e-7


def test_solver_dense_and_sparse_in_one_batch(sg, orc):
    import numpy as np
    import workloads as w
    mats = [w.banded(260, 9, 77), w.tridiagonal(900), w.banded(1500, 3, 78), w.banded(220, 8, 79)]
    out = sg.solve_batch(mats, tol=1e-8, filter="exact", prec=1, dense_frac=0.25)
    for a, res in zip(mats, out):
        assert res.status == sg.SIGN_OK and res.resid <= 1e-8
        ref = orc.nsf(a, tol=1e-8, filter="exact", mixed=True)
        S, R = _dense(res, a.n), ref.to_dense(a.n)
        assert np.linalg.norm(S - R) / np.linalg.norm(R) < 1e-5
    # the sparse members are untouched by the dense path: bit for bit
    ref = orc.nsf(mats[1], tol=1e-8, filter="exact", mixed=True)
    assert np.array_equal(out[1].val, ref.val)


# ---------------------------------------------------------------- the dense path of the FP64 stage
def _f64_launches(sg):
    return sg.prof_read().get("dense_f64_slices", {}).get("launches", 0)


def _rel(S, R):
    import numpy as np
    return np.linalg.norm(S - R) / np.linalg.norm(R)


@pytest.mark.parametrize("case", ["banded", "laplacian2d", "laplacian3d"])
def test_fp64_dense_path_within_fp64_tolerance(sg, orc, case):
    """FP64 solves whose iterate fills in run both products as exact-slice
    tensor-core GEMMs; the result stays within the FP64 bound 1e-10 of the
    oracle's FP64 run, at the same iteration count."""
    import workloads as w
    a = {"banded": w.banded(300, 10, 1234), "laplacian2d": w.laplacian(18, 2),
         "laplacian3d": w.laplacian(7, 3)}[case]
    tol = 1e-8
    sg.prof_reset()
    sg.prof_enable(True)
    res = sg.solve(a, tol=tol, filter="exact", dense_frac=0.25, dense64_min_n=1, max_iter=200)
    sg.prof_enable(False)
    assert _f64_launches(sg) > 0
    ref = orc.nsf(a, tol=tol, filter="exact", max_iter=200)
    assert res.status == ref.status == sg.SIGN_OK
    assert res.iters == ref.iters
    assert _rel(_dense(res, a.n), ref.to_dense(a.n)) <= 1e-10


def test_fp64_dense_and_sparse_in_one_batch_equal_lone_solves(sg, orc):
    """Dense-path results do not depend on the batch: each equals its lone
    solve bit for bit, and stays within 1e-10 of the oracle."""
    import numpy as np
    import workloads as w
    mats = [w.banded(260, 9, 77), w.tridiagonal(900), w.laplacian(16, 2), w.banded(220, 8, 79)]
    out = sg.solve_batch(mats, tol=1e-8, filter="exact", dense_frac=0.25, dense64_min_n=1)
    for a, res in zip(mats, out):
        alone = sg.solve(a, tol=1e-8, filter="exact", dense_frac=0.25, dense64_min_n=1)
        assert np.array_equal(res.val, alone.val) and np.array_equal(res.col, alone.col)
        ref = orc.nsf(a, tol=1e-8, filter="exact")
        assert res.iters == ref.iters
        assert _rel(_dense(res, a.n), ref.to_dense(a.n)) <= 1e-10
    # the sparse member is untouched by the dense path: bit for bit with the oracle
    ref = orc.nsf(mats[1], tol=1e-8, filter="exact")
    assert np.array_equal(out[1].val, ref.val)
