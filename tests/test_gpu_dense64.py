"""The FP64 dense product from exact BF16 digit slices on the tensor cores:
its error against exact products stays within the bound the splitting gives,
2^-41 (K/4096) 2^(e_i + f_j), and integer digit sums at the 2^24 limit are
exact."""
from fractions import Fraction

import numpy as np
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


def _scales(a, b):
    """2^e_i > max |row i of a|, 2^f_j > max |column j of b| (as in the splitting)."""
    ea = np.frexp(np.abs(a).max(axis=1))[1].astype(float)
    fb = np.frexp(np.abs(b).max(axis=0))[1].astype(float)
    return np.exp2(ea)[:, None] * np.exp2(fb)[None, :]


def _mats(rng, m, n, k):
    # entries spread over many binades, and a few zero rows / columns
    a = rng.standard_normal((m, k)) * np.exp2(rng.integers(-30, 4, (m, 1)))
    b = rng.standard_normal((k, n)) * np.exp2(rng.integers(-30, 4, (1, n)))
    a *= np.exp2(rng.integers(-8, 1, (m, k)))
    a[rng.integers(0, m)] = 0.0
    b[:, rng.integers(0, n)] = 0.0
    return a, b


@pytest.mark.parametrize("m,n,k", [(128, 256, 64), (300, 130, 257), (257, 514, 1000),
                                   (64, 2, 3)])
def test_matches_exact_product(sg, m, n, k):
    import torch
    rng = np.random.default_rng(m * 131 + n * 7 + k)
    a, b = _mats(rng, m, n, k)
    c = sg.dense_product_f64(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    exact = (a.astype(np.longdouble) @ b.astype(np.longdouble))  # quad on AArch64, 80-bit on x86
    err = np.abs(c.astype(np.longdouble) - exact).astype(np.float64)
    bound = 2.0 ** -41 * max(1.0, k / 4096) * _scales(a, b)
    assert (err <= bound).all(), float((err / bound).max())
    # and it is as close as an FP64 product: far below the bound in practice
    fp64 = np.abs((a @ b).astype(np.longdouble) - exact).astype(np.float64)
    assert err.max() <= 4 * fp64.max() + 2.0 ** -60 * _scales(a, b).max()


def test_full_size_sampled_entries_exact(sg):
    import torch
    rng = np.random.default_rng(5)
    n = 4096
    a = rng.uniform(-1, 1, (n, n))
    b = rng.uniform(-1, 1, (n, n))
    c = sg.dense_product_f64(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    sc = _scales(a, b)
    for i, j in zip(rng.integers(0, n, 24), rng.integers(0, n, 24)):
        exact = sum(Fraction(x) * Fraction(y) for x, y in zip(a[i], b[:, j]))
        assert abs(Fraction(c[i, j]) - exact) <= Fraction(2.0 ** -41) * Fraction(sc[i, j])


def test_digit_sums_at_the_fp32_limit_are_exact(sg):
    """Every entry 1 - 2^-53: the leading digits are all 64, so with K = 4096
    the leading pair's integer sums reach 4096 * 64 * 64 = 2^24 exactly."""
    import torch
    k = 4096
    x = 1.0 - 2.0 ** -53
    a = np.full((128, k), x)
    b = np.full((k, 256), x)
    b[:, 1::2] *= -1.0
    c = sg.dense_product_f64(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    exact = float(k * Fraction(x) * Fraction(x))
    assert np.all(c[:, 0::2] == exact) and np.all(c[:, 1::2] == -exact)


def test_k_beyond_one_exact_block(sg):
    """K = 9000 runs as three exact blocks of at most 4096, added in FP64."""
    import torch
    rng = np.random.default_rng(9)
    m, n, k = 200, 300, 9000
    a = rng.uniform(-1, 1, (m, k))
    b = rng.uniform(-1, 1, (k, n))
    c = sg.dense_product_f64(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    sc = _scales(a, b)
    for i, j in zip(rng.integers(0, m, 12), rng.integers(0, n, 12)):
        exact = sum(Fraction(x) * Fraction(y) for x, y in zip(a[i], b[:, j]))
        assert abs(Fraction(c[i, j]) - exact) <= Fraction(2.0 ** -41 * k / 4096) * Fraction(sc[i, j])


def test_rejects_bad_shapes(sg):
    import torch
    a = torch.zeros(8, 16, dtype=torch.float64, device="cuda")
    b = torch.zeros(16, 7, dtype=torch.float64, device="cuda")
    with pytest.raises(sg.SignError):
        sg.dense_product_f64(a, b)  # N odd
