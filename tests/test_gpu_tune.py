"""Schedules and their tuner (sign_tune_batch).

A schedule only moves rows between kernels: band tiles or row-wise FP32
products (band_min_eff), 32-, 16- or 8-lane FP64 groups (group_margin), one
or two FP32 rows per warp (pair_rows). Every kernel adds a product's terms in
ascending k with one fused multiply-add from +0, so every schedule must give
the results of the default one bit for bit, and the tuner only picks the
fastest among them. The residual and norm sums of a check are reduced in an
order that depends on the kernel, so their records agree to rounding."""
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


def _mats():
    shapes = w.banded_batch_shapes(24, nmin=200, nmax=3000)
    mats = [w.banded(n, b, s) for n, b, s in shapes]
    mats += [w.laplacian(20, 2), w.tridiagonal(2500)]
    return mats


KW = dict(tol=1e-8, filter="exact", prec="mixed", dense_frac=2.0)

SCHEDULES = [
    dict(band_min_eff=0.0),     # every eligible 16-row group as a band tile
    dict(band_min_eff=1e9),     # no band tile
    dict(group_margin=-1.0),    # every FP64 row on 32 lanes
    dict(group_margin=0.3),
    dict(group_margin=0.0),
    dict(pair_rows=0),
]


def _results(b):
    outs = []
    for h in b.handles:
        rp, col, val = h.result()
        outs.append((rp.copy(), col.copy(), val.view(np.uint64).copy()))
    return outs


def _same(r1, r2):
    for (p1, c1, v1), (p2, c2, v2) in zip(r1, r2):
        assert np.array_equal(p1, p2) and np.array_equal(c1, c2) and np.array_equal(v1, v2)


def test_every_schedule_gives_the_same_results(sg):
    b = sg.Batch(_mats())
    o = sg.default_opts(**KW)
    st0 = b.solve(o, trace_cap=64)
    assert all(s[0] == sg.SIGN_OK for s in st0)
    tr0 = b.traces()
    ref = _results(b)
    for sch in SCHEDULES:
        st = b.solve(sg.default_opts(**KW, **sch), trace_cap=64)
        assert [x[:2] for x in st] == [x[:2] for x in st0], sch  # status, iterations
        np.testing.assert_allclose([x[2] for x in st], [x[2] for x in st0], rtol=1e-12, atol=0)
        _same(_results(b), ref)
        for t0, t1 in zip(tr0, b.traces()):
            for k in ("nnz_x", "nnz_t", "nnz_bar", "tau_k", "mults_t"):
                assert np.array_equal(t0[k], t1[k]), (sch, k)
            for k in ("resid_k", "xnorm_k", "fnorm_k", "beta_k"):
                np.testing.assert_allclose(t1[k], t0[k], rtol=1e-12, atol=0, err_msg=str(sch))


def test_tuner_picks_a_candidate_and_caches_it(sg):
    b = sg.Batch(_mats())
    o = sg.default_opts(**KW)
    b.solve(o)
    ref = _results(b)
    best, rep = b.tune(o, reps=1, force=True)
    assert rep["timed"] >= 1 and not rep["cached"]
    assert 0.0 < rep["ms_best"] <= rep["ms_base"]
    assert rep["band_min_eff"] in (0.02, 0.04, 0.08, 0.16, 0.32)
    assert rep["group_margin"] in (-1.0, 0.0, 0.05, 0.15)
    assert rep["pair_rows"] in (0, 1)
    # every field outside the schedule is the base's
    for name, _ in type(o)._fields_:
        if name not in ("band_min_eff", "group_margin", "pair_rows"):
            assert getattr(best, name) == getattr(o, name), name
    _same(_results(b), ref)  # the handles hold the last solve's (equal) results
    best2, rep2 = b.tune(o)
    assert rep2["cached"] and rep2["timed"] == 0
    assert (best2.band_min_eff, best2.group_margin, best2.pair_rows) == \
        (best.band_min_eff, best.group_margin, best.pair_rows)
    b.solve(best2)
    _same(_results(b), ref)


def test_tuner_rejects_bad_arguments(sg):
    b = sg.Batch([w.tridiagonal(300)])
    with pytest.raises(sg.SignError):
        b.tune(sg.default_opts(**KW), reps=0)
    with pytest.raises(sg.SignError):
        b.tune(sg.default_opts(**KW, band_min_eff=-1.0))
