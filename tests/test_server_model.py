"""The server's admission model (sign_footprint_bytes, host arithmetic only):
its closed form on chosen statistics, and which synthetic workloads a 120 GB
budget admits. Runs without a GPU."""
import numpy as np
import pytest

import workloads as w


@pytest.fixture(scope="module")
def sg():
    import paper_2210_03356_gb300 as sg
    from paper_2210_03356_gb300 import build
    build.build()
    sg.load()
    return sg


def _stats(a):
    """Gershgorin gap, row-sum bound and half-bandwidth of a host CSR."""
    rows = np.repeat(np.arange(a.n), np.diff(a.rowptr))
    mag = np.abs(a.val)
    diag = np.zeros(a.n)
    on = rows == a.col
    diag[rows[on]] = mag[on]
    rowsum = np.bincount(rows, weights=mag, minlength=a.n)
    gap = 2 * diag - rowsum
    delta = gap.min() if (gap > 0).all() else 0.0
    return delta, rowsum.max(), int(np.abs(rows - a.col).max())


def test_footprint_closed_form(sg):
    # no Gershgorin gap: the dense bound, with the dense path's blocks
    assert sg.footprint_bytes(65536, 326656, 0.0, 8.0, 256) == 176.0 * 65536 ** 2 + 24 * 326656
    assert sg.footprint_bytes(100, 400, -1.0, 8.0, 3) == 176.0 * 100 * 100 + 24 * 400
    # 1.5 (rho/delta)(2 bw + 1) = 1.5 * 12 * 21 = 378 entries per row
    assert sg.footprint_bytes(8000, 160000, 0.25, 3.0, 10) == 96.0 * 8000 * 378 + 24 * 160000
    # at least 32 per row: 1.5 * 5 * 3 = 22.5 -> 32
    assert sg.footprint_bytes(2000, 5998, 0.5, 2.5, 1) == 96.0 * 2000 * 32 + 24 * 5998
    # at most n per row (and then dense)
    assert sg.footprint_bytes(100, 300, 0.01, 2.0, 10) == 176.0 * 100 * 100 + 24 * 300
    # a predicted quarter of the row already takes the dense path: 1.5 * 4 * 21 = 126 >= 500/4
    assert sg.footprint_bytes(500, 1000, 0.5, 2.0, 10) == 96.0 * 500 * 126 + 80.0 * 500 ** 2 + 24 * 1000


def test_budget_admits_the_sparse_workloads_and_refuses_the_3d_laplacian(sg):
    budget = 120e9
    big = w.laplacian(64, 3)           # 64^3 = 262,144 rows
    delta, rho, bw = _stats(big)
    assert delta == 0.0                # no Gershgorin gap: predicted dense
    assert sg.footprint_bytes(big.n, big.rowptr[-1], delta, rho, bw) > budget
    lap2 = w.laplacian(256, 2)         # 65,536 rows: dense prediction exceeds 120 GB too
    assert sg.footprint_bytes(lap2.n, lap2.rowptr[-1], *_stats(lap2)) > budget
    for a in (w.tridiagonal(), w.banded(8000, 10, 7), w.banded(2000, 1, 8), w.laplacian(32, 2)):
        fp = sg.footprint_bytes(a.n, a.rowptr[-1], *_stats(a))
        assert fp < 1e9, (a.n, fp)     # a small slice of the budget
