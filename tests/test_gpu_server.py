"""The continuous-batching server on the GPU: requests submitted while others
are in flight come out bit-identical to lone solves with the same options;
the footprint budget gates admission; refusals and bad inputs report."""
import threading
import time

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


def _mix(seed, count):
    """Requests drawn from the tridiagonal, banded and shifted-Laplacian generators."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        kind = i % 4
        if kind == 0:
            out.append(w.tridiagonal(int(rng.integers(1000, 4000)), seed=seed * 100 + i))
        elif kind == 1:
            out.append(w.banded(int(rng.integers(200, 3000)), int(rng.integers(1, 11)),
                                seed * 100 + i))
        elif kind == 2:
            out.append(w.laplacian(int(rng.integers(12, 25)), 2))
        else:
            out.append(w.laplacian(int(rng.integers(6, 10)), 3))
    return out


def _same(res, rp, col, val):
    assert np.array_equal(res.rowptr, rp)
    assert np.array_equal(res.col, col)
    assert np.array_equal(res.val, val)


@pytest.mark.parametrize("lanes", [1, 2])
def test_results_in_the_mix_equal_lone_solves(sg, lanes):
    mats = _mix(3, 16)
    with sg.Server(tol=1e-8, filter="exact", prec="mixed", lanes=lanes) as srv:
        tickets = []

        def feed():  # arrivals spread over the first rounds of the earlier requests
            for a in mats:
                tickets.append(srv.submit(a))
                time.sleep(0.002)

        th = threading.Thread(target=feed)
        th.start()
        th.join()
        done = {}
        for t in tickets:
            r = None
            while r is None:
                r = srv.poll(t, wait_ms=1000)
            done[t] = r
        outs = {t: srv.take(t) for t in tickets}
        st = srv.stats()
    assert st["completed"] == len(mats) == st["admitted"] and st["refused"] == 0
    assert st["max_active_seen"] > 1  # requests did share rounds
    for a, t in zip(mats, tickets):
        lone = sg.solve(a, tol=1e-8, filter="exact", prec=1)
        assert done[t]["status"] == lone.status == sg.SIGN_OK
        assert done[t]["iters"] == lone.iters
        _same(lone, *outs[t])
        tm = done[t]
        assert tm["t_submit"] <= tm["t_admit"] <= tm["t_done"]
        # shifted Laplacians have no Gershgorin gap: predicted dense, second lane
        assert tm["lane"] == (1 if lanes == 2 and a.name.startswith("laplacian") else 0)


def test_budget_admits_one_request_at_a_time(sg):
    mats = [w.banded(1500, 4, 40 + i) for i in range(4)]
    with sg.Server(tol=1e-8, filter="exact", prec="mixed") as probe:
        t = probe.submit(mats[0])
        fp = probe.poll(t, wait_ms=60000)["footprint"]
    # room for one of these requests at a time
    with sg.Server(tol=1e-8, filter="exact", prec="mixed", mem_budget=1.5 * fp) as srv:
        tickets = [srv.submit(a) for a in mats]
        res = [srv.poll(t, wait_ms=60000) for t in tickets]
        outs = [srv.take(t) for t in tickets]
        st = srv.stats()
    assert st["max_active_seen"] == 1 and st["completed"] == 4
    for a, r, o in zip(mats, res, outs):
        assert r["status"] == sg.SIGN_OK
        _same(sg.solve(a, tol=1e-8, filter="exact", prec=1), *o)
    # first come, first served: each admitted once the one before it was done
    for prev, nxt in zip(res, res[1:]):
        assert nxt["t_admit"] >= prev["t_done"]


def test_refusals_and_invalid_requests(sg):
    with sg.Server(tol=1e-8, filter="exact", prec="mixed") as srv:
        # predicted dense: 96 n^2 bytes for n = 262,144 exceeds 120 GB
        with pytest.raises(sg.SignError) as e:
            srv.submit(w.laplacian(64, 3))
        assert e.value.status == sg.SIGN_ENOMEM and "mem_budget" in str(e.value)
        # malformed CSR: refused at submission
        bad = w.tridiagonal(100)
        bad.col = bad.col.copy()
        bad.col[5], bad.col[6] = bad.col[6], bad.col[5]
        with pytest.raises(sg.SignError) as e:
            srv.submit(bad)
        assert e.value.status == sg.SIGN_EINVAL
        # zero matrix: admitted, then stops with SIGN_EINVAL (no finite nonzero 1-norm)
        z = w.csr_from_coo(50, np.arange(50), np.arange(50), np.zeros(50))
        t = srv.submit(z)
        r = srv.poll(t, wait_ms=60000)
        assert r["status"] == sg.SIGN_EINVAL and r["nnz_final"] == 0
        with pytest.raises(sg.SignError):
            srv.take(t)  # no result to read
        # a good request after the failures still works
        a = w.banded(800, 3, 9)
        t = srv.submit(a)
        assert srv.poll(t, wait_ms=60000)["status"] == sg.SIGN_OK
        _same(sg.solve(a, tol=1e-8, filter="exact", prec=1), *srv.take(t))
        with pytest.raises(sg.SignError):
            srv.poll(t)  # taken: the ticket is forgotten
        st = srv.stats()
    # the malformed matrix failed validation before admission: not counted
    assert st["submitted"] == 3 and st["refused"] == 1 and st["completed"] == 2


def test_latency_target_refuses_with_eagain(sg):
    """max_wait_s: once a lane has a completion rate (8 completions), a
    submission whose predicted wait (queued ahead / rate) exceeds the target
    is refused with SIGN_EAGAIN; what is admitted still solves as alone."""
    with pytest.raises(sg.SignError):
        sg.Server(max_wait_s=-1.0)
    mats = [w.banded(int(n), 4, 50 + i) for i, n in enumerate(np.linspace(600, 1400, 24))]
    with sg.Server(tol=1e-8, filter="exact", prec="mixed", lanes=1, max_active=4,
                   max_wait_s=1e-4) as srv:
        first = [srv.submit(a) for a in mats[:10]]  # no rate yet: never refused
        for t in first:
            assert srv.poll(t, wait_ms=60000)["status"] == sg.SIGN_OK
        taken, refused = [], 0
        for a in mats * 8:  # a burst: at most 4 on the GPU, the rest queues
            try:
                taken.append((srv.submit(a), a))
            except sg.SignError as e:
                assert e.status == sg.SIGN_EAGAIN and "max_wait_s" in str(e)
                refused += 1
        assert refused > 0 and taken
        for t, a in taken[:6]:
            assert srv.poll(t, wait_ms=60000)["status"] == sg.SIGN_OK
            _same(sg.solve(a, tol=1e-8, filter="exact", prec=1), *srv.take(t))
        st = srv.stats()
    assert st["refused"] == refused


def test_trim_after_a_destroyed_server(sg):
    """Blocks freed on this thread for a server's upload stream outlive the
    stream; trimming afterwards must not use it, and solving still works."""
    mats = _mix(5, 4)
    with sg.Server(tol=1e-8, filter="exact", prec="mixed") as srv:
        tickets = [srv.submit(a) for a in mats]
        for t in tickets:
            while srv.poll(t, wait_ms=1000) is None:
                pass
        outs = [srv.take(t) for t in tickets]
    del outs
    sg.trim_memory()
    lone = sg.solve(mats[0], tol=1e-8, filter="exact", prec=1)
    assert lone.status == sg.SIGN_OK
    sg.trim_memory()
