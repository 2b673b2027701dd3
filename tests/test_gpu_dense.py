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
                                   (200, 300, 100), (1000, 516, 260), (64, 4, 12)])
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
    assert err < 2e-6, err  # FP32-level; one TF32 pass would be ~1e-3


def test_dense_product_exact_zeros_and_identity(sg):
    import torch
    n = 256
    x = torch.zeros(n, n, device="cuda")
    x[:100, :100] = torch.randn(100, 100, device="cuda")
    eye = torch.eye(n, device="cuda")
    c = sg.dense_product(x, eye)
    assert torch.equal(c, x)  # hi*1 + lo*1 reproduces x exactly
    c2 = sg.dense_product(x, x)
    assert torch.count_nonzero(c2[100:, :]) == 0 and torch.count_nonzero(c2[:, 100:]) == 0


def test_dense_product_rejects_misaligned(sg):
    import torch
    a = torch.randn(8, 6, device="cuda")
    b = torch.randn(6, 8, device="cuda")
    with pytest.raises(Exception):
        sg.dense_product(a, b)  # K = 6 is not a multiple of 4
