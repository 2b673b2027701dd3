"""Pins for the CPU oracle: every test checks it against something other than
itself (exact rational arithmetic, closed forms, eigendecompositions, the
paper's lemmas and theorems, or values the paper prints)."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import workloads as w

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_csr(n, density, seed, symmetric=False, spread=False):
    """Random sparse matrix with empty rows allowed (numpy RNG, test-local)."""
    rng = np.random.default_rng(seed)
    d = (rng.random((n, n)) < density) * rng.uniform(-1, 1, (n, n))
    if spread:
        d *= 10.0 ** rng.integers(-12, 3, (n, n))
    if symmetric:
        d = np.triu(d) + np.triu(d, 1).T
    return w.csr_from_dense(d), d


def _dense(n, rp, col, val):
    d = np.zeros((n, n))
    rows = np.repeat(np.arange(n), np.diff(rp))
    d[rows, col] = val
    return d


def _sign_eig(d):
    ev, v = np.linalg.eigh(d)
    return (v * np.sign(ev)) @ v.T


# --------------------------------------------------------------------------
# generators
# --------------------------------------------------------------------------
def test_generators_are_seeded_and_shaped():
    a, b = w.tridiagonal(), w.tridiagonal()
    assert a.n == 2000 and a.nnz == 5998
    assert np.array_equal(a.val, b.val)
    d = a.to_dense()
    assert np.allclose(d, d.T)
    # Gershgorin: |d_i| >= 1, off-diagonal row sums <= 0.6, so |lambda| >= 0.4
    assert np.min(np.abs(np.linalg.eigvalsh(d))) >= 0.4
    L = w.laplacian2d(256)
    assert L.n == 65536 and L.nnz == 326656
    # sigma: midpoint of 4 and the nearest distinct eigenvalue above 4
    lam_plus = 4.0 - 2.0 * math.cos(127 * math.pi / 257) - 2.0 * math.cos(131 * math.pi / 257)
    ev = w.laplacian_eigs(256, 2)
    above = ev[ev > 4.0 + 1e-12].min()
    assert abs(above - 4.000448257653280) < 1e-12
    assert abs(w.laplacian_shift(256, 2) - (4.0 + (above - 4.0) / 2)) < 1e-15
    assert lam_plus > 4.0
    assert w.laplacian_shift(64, 3) == 6.0
    L3 = w.laplacian3d(64)
    assert L3.n == 262144 and L3.nnz == 1810432


def test_banded_batch_rows_and_symmetry():
    shapes = w.banded_batch_shapes()
    assert len(shapes) == 512
    assert all(200 <= n <= 8000 and 1 <= b <= 10 for n, b, _ in shapes)
    for n, b, s in shapes[:6]:
        m = w.banded(n, b, s)
        d = m.to_dense()
        assert np.allclose(d, d.T)
        off = np.abs(d).sum(1) - np.abs(np.diag(d))
        assert off.max() <= 0.8 + 1e-12
        assert np.all(np.abs(np.diag(d)) >= 1.0)


# --------------------------------------------------------------------------
# 1-norm (initial scale, step a1)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_onenorm_matches_exact_rational(oracle_lib, seed):
    a, d = _rand_csr(40, 0.2, seed, spread=True)
    exact = max(sum(Fraction(float(abs(x))) for x in d[:, j]) for j in range(40))
    got = oracle_lib.onenorm(a.n, a.rowptr, a.col, a.val)
    assert abs(Fraction(got) - exact) <= exact * Fraction(4, 2 ** 52)
    # the plain sum of a column in any order agrees to rounding
    assert abs(got - np.abs(d).sum(0).max()) <= 1e-14 * got


def test_onenorm_nonsymmetric_uses_columns(oracle_lib):
    d = np.array([[1.0, 5.0], [0.0, 1.0]])
    a = w.csr_from_dense(d)
    assert oracle_lib.onenorm(2, a.rowptr, a.col, a.val) == 6.0  # column 1, not row 0 (=6 too)
    d = np.array([[1.0, 0.0], [7.0, 1.0]])
    a = w.csr_from_dense(d)
    assert oracle_lib.onenorm(2, a.rowptr, a.col, a.val) == 8.0


# --------------------------------------------------------------------------
# sparse product (steps a2, a3)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("seed", [4, 5])
def test_spgemm_matches_dense_and_symbolic_pattern(oracle_lib, seed):
    n = 60
    a, da = _rand_csr(n, 0.08, seed)
    b, db = _rand_csr(n, 0.08, seed + 100)
    rp, col, val = oracle_lib.spgemm(n, (a.rowptr, a.col, a.val), (b.rowptr, b.col, b.val))
    got = _dense(n, rp, col, val)
    assert np.allclose(got, da @ db, rtol=1e-14, atol=1e-15)
    pattern = ((da != 0).astype(int) @ (db != 0).astype(int)) > 0
    mine = np.zeros((n, n), bool)
    mine[np.repeat(np.arange(n), np.diff(rp)), col] = True
    assert np.array_equal(pattern, mine)
    for i in range(n):  # ascending, no duplicates
        assert np.all(np.diff(col[rp[i]:rp[i + 1]]) > 0)


def test_spgemm_keeps_exact_cancellation(oracle_lib):
    # row 0 of A = [1, 1], B rows k=0: (0, 2.0), k=1: (0, -2.0) -> C[0,0] = 0 kept
    A = w.csr_from_dense(np.array([[1.0, 1.0], [0.0, 1.0]]))
    B = w.csr_from_dense(np.array([[2.0, 0.0], [-2.0, 3.0]]))
    rp, col, val = oracle_lib.spgemm(2, (A.rowptr, A.col, A.val), (B.rowptr, B.col, B.val))
    assert list(rp) == [0, 2, 4]
    assert list(col) == [0, 1, 0, 1] and val[0] == 0.0 and val[1] == 3.0


def test_spgemm_f32_matches_float_products(oracle_lib):
    n = 50
    a, da = _rand_csr(n, 0.1, 7)
    rp, col, val = oracle_lib.spgemm(n, (a.rowptr, a.col, a.val.astype(np.float32)),
                                     (a.rowptr, a.col, a.val.astype(np.float32)), f32=True)
    assert val.dtype == np.float32
    ref = da.astype(np.float32).astype(np.float64) @ da.astype(np.float32).astype(np.float64)
    assert np.allclose(_dense(n, rp, col, val), ref, rtol=1e-5, atol=1e-6)


# --------------------------------------------------------------------------
# residual and norms (steps a2, a4)
# --------------------------------------------------------------------------
def test_resid_rms_includes_missing_diagonal(oracle_lib):
    n = 30
    a, d = _rand_csr(n, 0.1, 9)
    assert np.any(np.diag(d) == 0)
    got = oracle_lib.resid_rms(n, a.rowptr, a.col, a.val)
    assert abs(got - np.linalg.norm(d - np.eye(n)) / math.sqrt(n)) < 1e-15
    assert abs(oracle_lib.fro_rms(n, a.rowptr, a.val) - np.linalg.norm(d) / math.sqrt(n)) < 1e-15


# --------------------------------------------------------------------------
# Newton-Schulz update, Lemma 2.1.1 (Eq. 1.3) and diagonal closed form
# --------------------------------------------------------------------------
@pytest.mark.parametrize("k", [0, 1, 3])
def test_ns_update_obeys_lemma_2_1_1(oracle_lib, k):
    a = w.banded(120, 4, 11)
    x = oracle_lib.nsf(a, tol=0.0, filter="none", max_iter=k)
    n = a.n
    X = (x.rowptr, x.col, x.val)
    T = oracle_lib.spgemm(n, X, X)
    Xb = oracle_lib.ns_update(n, X, T)
    xd, xbd = _dense(n, *X), _dense(n, *Xb)
    R = np.eye(n) - xd @ xd
    R1 = np.eye(n) - xbd @ xbd
    pred = 0.75 * R @ R + 0.25 * R @ R @ R
    assert np.linalg.norm(R1 - pred) <= 1e-13 * max(1.0, np.linalg.norm(R))
    # the update really is X(3I - X^2)/2
    assert np.allclose(xbd, 0.5 * xd @ (3 * np.eye(n) - xd @ xd), rtol=0, atol=1e-14)


def _csr_of(d):
    n = d.shape[0]
    rows, cols = np.nonzero(d)
    rp = np.zeros(n + 1, np.int64)
    np.add.at(rp, rows + 1, 1)
    return np.cumsum(rp), cols.astype(np.int32), d[rows, cols]


def test_ns_step_keeps_the_anticommuting_part_of_an_error(oracle_lib):
    """Near S = sign(A) one step X(3I - X^2)/2 maps S + E to S + (E - S E S)/2
    + O(|E|^2): a perturbation commuting with S is removed, one anticommuting
    with S passes unchanged. An FP64 finish therefore cannot remove the
    anticommuting part of the FP32 stage's rounding error."""
    n = 40
    a = w.banded(n, 3, 5)
    A = _dense(n, a.rowptr, a.col, a.val)
    S = _sign_eig(A)
    Pp, Pm = (np.eye(n) + S) / 2, (np.eye(n) - S) / 2
    rng = np.random.default_rng(0)
    B = rng.standard_normal((n, n)) * 1e-6
    Ec = Pp @ B @ Pp + Pm @ B @ Pm      # commutes with S
    Ea = Pp @ B @ Pm + Pm @ B @ Pp      # anticommutes with S
    assert np.linalg.norm(S @ Ec - Ec @ S) < 1e-15 and np.linalg.norm(S @ Ea + Ea @ S) < 1e-15

    def step(X):
        Xc = _csr_of(X)
        return _dense(n, *oracle_lib.ns_update(n, Xc, oracle_lib.spgemm(n, Xc, Xc)))

    e2 = np.linalg.norm(B) ** 2
    assert np.linalg.norm(step(S + Ec) - S) <= 10 * e2                 # removed
    assert np.linalg.norm(step(S + Ea) - (S + Ea)) <= 10 * e2          # kept
    assert np.linalg.norm(Ea) > 1e3 * 10 * e2                          # and the test can tell


def test_diagonal_follows_scalar_map_exactly(oracle_lib):
    vals = np.array([0.3, -0.05, 2.0, -1.0, 0.9, -0.6])
    n = len(vals)
    a = w.csr_from_dense(np.diag(vals))
    norm = Fraction(float(np.abs(vals).max()))
    for k in (1, 4, 9):
        r = oracle_lib.nsf(a, tol=0.0, filter="none", max_iter=k)
        assert r.status == oracle_lib.ENOTCONV and r.iters == k
        for i in range(n):
            x = Fraction(float(vals[i])) / norm
            for _ in range(k):
                x = x * (3 - x * x) / 2
            got = _dense(n, r.rowptr, r.col, r.val)[i, i]
            assert abs(Fraction(got) - x) <= abs(x) * Fraction(8 * (k + 1), 2 ** 52) + Fraction(1, 2 ** 80)
    r = oracle_lib.nsf(a, tol=1e-14, filter="exact")
    assert r.status == oracle_lib.OK
    assert np.allclose(_dense(n, r.rowptr, r.col, r.val), np.diag(np.sign(vals)), atol=1e-14)


# --------------------------------------------------------------------------
# converged result: brute force and invariants
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mode", ["none", "exact", "bound"])
def test_tridiagonal_500_matches_eigendecomposition(oracle_lib, mode):
    a = w.tridiagonal(500)
    r = oracle_lib.nsf(a, tol=1e-12, filter=mode)
    assert r.status == oracle_lib.OK
    S = _dense(a.n, r.rowptr, r.col, r.val)
    ref = _sign_eig(a.to_dense())
    assert np.linalg.norm(S - ref) / np.linalg.norm(ref) < 1e-10
    d = a.to_dense()
    assert np.linalg.norm(S @ d - d @ S) / np.linalg.norm(d) < 1e-10  # SA = AS
    assert np.linalg.norm(S - S.T) / np.linalg.norm(S) < 1e-12
    ev = np.linalg.eigvalsh(d)
    assert round(np.trace(S)) == int((ev > 0).sum() - (ev < 0).sum())  # trace = n+ - n-
    assert np.linalg.norm(S @ S - np.eye(a.n)) / math.sqrt(a.n) < 1e-11


def test_tridiagonal_2000_matches_eigendecomposition(oracle_lib):
    """The tridiagonal workload at its full size (n = 2000, tol 1e-8, EXACT)
    against the dense eigendecomposition; the filtered iterate stays a small
    fraction of n^2 (the unfiltered one fills to about a quarter)."""
    a = w.tridiagonal()
    d = a.to_dense()
    ref = _sign_eig(d)
    r = oracle_lib.nsf(a, tol=1e-8, filter="exact")
    assert r.status == oracle_lib.OK and r.resid <= 1e-8
    S = _dense(a.n, r.rowptr, r.col, r.val)
    assert np.linalg.norm(S - ref) / np.linalg.norm(ref) < 1e-9
    assert np.linalg.norm(S @ d - d @ S) / np.linalg.norm(d) < 1e-9
    assert r.trace["nnz_x"].max() < 0.02 * a.n * a.n


def test_spd_gives_identity(oracle_lib):
    a = w.spd_random(300, 0.01)
    r = oracle_lib.nsf(a, tol=1e-12, filter="exact")
    assert r.status == oracle_lib.OK
    assert np.allclose(_dense(a.n, r.rowptr, r.col, r.val), np.eye(a.n), atol=1e-11)


def test_banded_filtered_matches_eig(oracle_lib):
    for n, b, s in [(300, 7, 21), (450, 2, 22)]:
        a = w.banded(n, b, s)
        r = oracle_lib.nsf(a, tol=1e-10, filter="exact")
        assert r.status == oracle_lib.OK
        S = _dense(n, r.rowptr, r.col, r.val)
        ref = _sign_eig(a.to_dense())
        assert np.linalg.norm(S - ref) / np.linalg.norm(ref) < 1e-9
        assert r.nnz < n * n  # the filter really dropped something


@pytest.mark.parametrize("dim,m", [(1, 300), (2, 14)])
def test_shifted_laplacian_closed_form(oracle_lib, dim, m):
    """sign(L - sigma I) from the sine eigenbasis of the Dirichlet Laplacian."""
    a = w.laplacian(m, dim)
    sigma = w.laplacian_shift(m, dim)
    h = math.pi / (m + 1)
    q = np.sqrt(2.0 / (m + 1)) * np.sin(np.outer(np.arange(1, m + 1), np.arange(1, m + 1)) * h)
    lam1 = 2 - 2 * np.cos(np.arange(1, m + 1) * h)
    if dim == 1:
        V, lam = q, lam1
    else:
        V = np.kron(q, q)  # index x + m*y  <->  kron(q_y, q_x)
        lam = (lam1[None, :] + lam1[:, None]).ravel()
    ref = (V * np.sign(lam - sigma)) @ V.T
    r = oracle_lib.nsf(a, tol=1e-12, filter="exact", max_iter=200)
    assert r.status == oracle_lib.OK
    S = _dense(a.n, r.rowptr, r.col, r.val)
    assert np.linalg.norm(S - ref) / np.linalg.norm(ref) < 1e-9
    assert round(np.trace(S)) == int(np.sum(np.sign(lam - sigma)))


# --------------------------------------------------------------------------
# the paper's Sec. 4.2 workload: closed form, Newton's method, Table 4.2.1
# --------------------------------------------------------------------------
def _ode_closed_form(n, lam=1.0 / 16):
    j = np.arange(1, n + 1)
    q = np.sqrt(2.0 / (n + 1)) * np.sin(np.outer(j, j) * math.pi / (n + 1))
    mu = 1 - 2 * lam + 2 * lam * np.cos(j * math.pi / (n + 1))
    bh = (q * np.sqrt(mu)) @ q.T
    bmh = (q / np.sqrt(mu)) @ q.T
    z = np.zeros((n, n))
    return np.block([[z, bh], [bmh, z]])


def test_ode_block_closed_form_ns_and_nm(oracle_lib):
    n = 60
    a = w.ode_block(n)
    ref = _ode_closed_form(n)
    r = oracle_lib.nsf(a, tol=1e-12, filter="exact", scale_1norm=False)
    assert r.status == oracle_lib.OK
    S = _dense(a.n, r.rowptr, r.col, r.val)
    assert np.linalg.norm(S - ref) / np.linalg.norm(ref) < 1e-11
    Snm, it, res, st = oracle_lib.nm_dense(a.to_dense(), tol=1e-12)
    assert st == oracle_lib.OK and it < 20
    assert np.linalg.norm(Snm - ref) / np.linalg.norm(ref) < 1e-11


def test_nm_matches_eig_on_symmetric(oracle_lib):
    a = w.tridiagonal(150)
    d = a.to_dense()
    S, it, res, st = oracle_lib.nm_dense(d, tol=1e-12)
    assert st == oracle_lib.OK
    assert np.linalg.norm(S - _sign_eig(d)) / math.sqrt(150) < 1e-12


def test_table_4_2_1_ae_not_worse_than_paper(oracle_lib):
    """AE = ||X_NS - X_NSF|| stays at or below the values the paper prints."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table_4_2_1.txt"))
            if l.strip() and not l.startswith("#")]
    paper_ae = {int(r[0]): float(r[2]) for r in rows}
    for nb in (250, 500):  # n read as the order of the block matrix, then of B
        a = w.ode_block(nb)
        r0 = oracle_lib.nsf(a, tol=1e-12, filter="none", scale_1norm=False)
        r1 = oracle_lib.nsf(a, tol=1e-12, filter="exact", scale_1norm=False)
        assert r0.status == r1.status == oracle_lib.OK
        ae = np.linalg.norm(r0.to_dense(a.n) - r1.to_dense(a.n))
        assert ae <= paper_ae[500]
        assert r1.nnz < r0.nnz


# --------------------------------------------------------------------------
# Newton's method with filtering, Alg. 3.1.1
# --------------------------------------------------------------------------
def _dense_of(a):
    d = np.zeros((a.n, a.n))
    d[np.repeat(np.arange(a.n), np.diff(a.rowptr)), a.col] = a.val
    return d


@pytest.mark.parametrize("which", ["ode", "banded"])
def test_nmf_without_filter_is_newton(oracle_lib, which):
    """With no filter, NMF is Newton's method: bit for bit the dense NM."""
    a = w.ode_block(60) if which == "ode" else w.banded(90, 3, 4)
    r = oracle_lib.nmf(a, tol=1e-12, filter="none")
    s, iters, resid, st = oracle_lib.nm_dense(_dense_of(a), tol=1e-12)
    assert r.status == st == oracle_lib.OK and r.iters == iters
    assert np.array_equal(r.to_dense(a.n), s)


def test_nmf_table_4_2_1_ae_not_worse_than_paper(oracle_lib):
    """AE = ||X_NM - X_NMF|| at or below the paper's NMF column, and the
    filtered result at the closed form (Eq. 1.26)."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "table_4_2_1.txt"))
            if l.strip() and not l.startswith("#")]
    paper_ae = {int(r[0]): float(r[5]) for r in rows}
    a = w.ode_block(250)  # n = 500 read as the order of the block matrix
    r0 = oracle_lib.nmf(a, tol=1e-12, filter="none")
    r1 = oracle_lib.nmf(a, tol=1e-12, filter="exact")
    assert r0.status == r1.status == oracle_lib.OK
    assert np.linalg.norm(r0.to_dense(a.n) - r1.to_dense(a.n)) <= paper_ae[500]
    assert r1.nnz < r0.nnz // 10
    lam = 1.0 / 16
    nb = 250
    j = np.arange(1, nb + 1)
    h = np.pi / (nb + 1)
    V = np.sqrt(2.0 / (nb + 1)) * np.sin(np.outer(j, j) * h)
    mu = 7.0 / 8.0 + 2.0 * lam * np.cos(j * h)
    S = np.zeros((2 * nb, 2 * nb))
    S[:nb, nb:] = (V * np.sqrt(mu)) @ V.T
    S[nb:, :nb] = (V / np.sqrt(mu)) @ V.T
    assert np.abs(r1.to_dense(a.n) - S).max() <= 1e-13


def test_nmf_matches_eig_on_symmetric(oracle_lib):
    a = w.banded(200, 4, 9)
    r = oracle_lib.nmf(a, tol=1e-12, filter="exact")
    S = _sign_eig(_dense_of(a))
    assert r.status == oracle_lib.OK
    assert np.linalg.norm(r.to_dense(a.n) - S) / np.linalg.norm(S) <= 1e-12


def test_newton_with_one_step_inverse_is_newton_schulz(oracle_lib):
    """Newton's update (X + X^-1)/2 with X^-1 replaced by one Newton-Schulz
    inverse step from Y0 = X, Y1 = X(2I - X X), is the NS update X(3I - X^2)/2:
    the oracle's NS update reproduces it to rounding. (A GPU NMF built on an
    iterative inverse is therefore the NS family again, one order per
    extra inner step.)"""
    a = w.banded(80, 3, 2)
    x = oracle_lib.nsf(a, tol=0.0, filter="none", max_iter=3)  # r well below 1
    n = a.n
    X = _dense(n, x.rowptr, x.col, x.val)
    Y1 = X @ (2 * np.eye(n) - X @ X)
    newton_one_step = 0.5 * (X + Y1)
    Xc = (x.rowptr, x.col, x.val)
    ns = _dense(n, *oracle_lib.ns_update(n, Xc, oracle_lib.spgemm(n, Xc, Xc)))
    assert np.abs(newton_one_step - ns).max() <= 1e-14
    # and the exact inverse differs from it at second order in R = I - X^2
    R = np.eye(n) - X @ X
    exact = 0.5 * (X + np.linalg.inv(X))
    assert np.linalg.norm(exact - ns) <= 2 * np.linalg.norm(R) ** 2 * np.linalg.norm(X)
    assert np.linalg.norm(exact - ns) >= 1e-3 * np.linalg.norm(R) ** 2


def test_nmf_theorem_3_1_2(oracle_lib):
    """Once the budget of Eq. (1.13) is in force, ||dR_k|| <= 4 ||R_k|| with
    dR_k = Rhat_k - R_k between NMF and Newton's method (Thm 3.1.2). The
    adaptive phase starts early here (switch at 1e-2) to give it several steps."""
    a = w.ode_block(60)
    A = _dense_of(a)
    full = oracle_lib.nmf(a, tol=1e-12, filter="exact", switch_resid=1e-2)
    assert full.status == oracle_lib.OK
    adaptive = [k for k in range(full.iters) if full.trace["resid"][k] < 1e-2]
    assert len(adaptive) >= 2
    checked = 0
    for k in range(1, full.iters + 1):
        if k - 1 not in adaptive:
            continue  # X_k was not formed under Eq. (1.13)
        # the same runs stopped after k updates (only the last k converges)
        xh = oracle_lib.nmf(a, tol=1e-12, filter="exact", switch_resid=1e-2, max_iter=k)
        xn, _, _, _ = oracle_lib.nm_dense(A, tol=1e-12, max_iter=k)
        Rh = np.eye(a.n) - xh.to_dense(a.n) @ xh.to_dense(a.n)
        R = np.eye(a.n) - xn @ xn
        assert np.linalg.norm(Rh - R) <= 4 * np.linalg.norm(R) + 1e-15
        checked += 1
    assert checked >= 2


# --------------------------------------------------------------------------
# filters (steps a4-a6)
# --------------------------------------------------------------------------
def _brute_exact(vals, b):
    """Largest threshold v (a magnitude, or inf) with sum_{|x|<v} x^2 <= b^2, exactly."""
    mags = sorted({abs(float(x)) for x in vals})
    b2 = Fraction(b) ** 2
    best = 0.0
    for v in mags + [math.inf]:
        s = sum((Fraction(float(x)) ** 2 for x in vals if abs(x) < v), Fraction(0))
        if s <= b2:
            best = v
    return best


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_filter_exact_brute_force_with_ties(oracle_lib, seed):
    rng = np.random.default_rng(seed)
    n = 12
    d = rng.uniform(-1, 1, (n, n)) * (rng.random((n, n)) < 0.5) * 10.0 ** rng.integers(-6, 0, (n, n))
    # plant ties and exact zeros
    d[0, :4] = 1e-3
    d[1, :3] = -1e-3
    d[2, 2] = 0.0
    a = w.csr_from_dense(d)
    a.val[:3] = 0.0  # explicit stored zeros
    vals = a.val.copy()
    for b in [0.0, 1e-7, 1e-4, 1.5e-3, 2.2e-3, 1e-1, 1e3]:
        (rp, col, val), tau, fn = oracle_lib.filter_csr(n, (a.rowptr, a.col, a.val), "exact", b)
        assert tau == _brute_exact(vals, b)
        kept = np.abs(vals) >= tau
        assert rp[-1] == kept.sum()
        dropped = vals[~kept]
        assert fn <= b * (1 + 1e-15)
        assert abs(fn - math.sqrt(float(np.sum(dropped ** 2)))) <= 1e-15 * max(fn, 1e-300)
        # ties are never split
        assert not (set(np.abs(vals[kept])) & set(np.abs(dropped)))
        assert np.all(vals[kept] != 0.0)


def test_filter_bound_formula(oracle_lib):
    a, d = _rand_csr(40, 0.3, 5, spread=True)
    a.val[5] = 0.0
    b = 1e-3
    (rp, col, val), tau, fn = oracle_lib.filter_csr(40, (a.rowptr, a.col, a.val), "bound", b)
    assert tau == b / math.sqrt(a.nnz)
    keep = (np.abs(a.val) >= tau) & (a.val != 0)
    assert rp[-1] == keep.sum() and fn <= b
    (rp, col, val), tau, fn = oracle_lib.filter_csr(40, (a.rowptr, a.col, a.val), "none", b)
    assert rp[-1] == a.nnz and tau == 0.0 and fn == 0.0


def test_budget_phases(oracle_lib):
    assert oracle_lib.budget(0.5, 1.0, 1e-4, 1e-8, 1e-6) == 1e-4 * 1e-8
    assert oracle_lib.budget(1e-6, 1.0, 1e-4, 1e-8, 1e-6) == 1e-4 * 1e-8
    r, x = 1e-7, 0.9
    got = oracle_lib.budget(r, x, 1e-4, 1e-8, 1e-6)
    assert 0 < got < r * r  # Eq. (1.18) is of order r^2
    # the budget shrinks with the residual and with ||X||
    assert oracle_lib.budget(r / 2, x, 1e-4, 1e-8, 1e-6) < got
    assert oracle_lib.budget(r, 2 * x, 1e-4, 1e-8, 1e-6) < got
    # at ||X|| = 1 (a symmetric involution) Eq. (1.18) reduces to 3 r^2 / 16
    assert abs(oracle_lib.budget(r, 1.0, 1e-4, 1e-8, 1e-6) - 3 * r * r / 16) <= 1e-15 * r * r


def test_theorem_3_2_1_and_error_propagation(oracle_lib):
    """Thm 3.2.1: with the budget (1.18), ||dR_k|| <= 3 ||R_k|| once adaptive;
    Eq. (1.22) and Sec. 4.1: the filtered and unfiltered iterates stay within
    about tol of each other."""
    a = w.tridiagonal(400)
    n = a.n
    tol = 1e-12
    adaptive_seen = False
    for k in range(0, 12):
        r1 = oracle_lib.nsf(a, tol=tol, filter="exact", max_iter=k)
        r0 = oracle_lib.nsf(a, tol=0.0, filter="none", max_iter=r1.iters)
        assert r0.iters == r1.iters
        X0, X1 = r0.to_dense(n), r1.to_dense(n)
        R0 = np.eye(n) - X0 @ X0
        R1 = np.eye(n) - X1 @ X1
        nr0 = np.linalg.norm(R0) / math.sqrt(n)
        dR = np.linalg.norm(R1 - R0) / math.sqrt(n)
        assert dR <= 3 * nr0 + 1e-14
        assert np.linalg.norm(X1 - X0) / math.sqrt(n) <= 10 * tol
        adaptive_seen |= bool(np.any(r1.trace["resid"][:r1.iters] < 1e-6))
        if r1.status == oracle_lib.OK:
            break
    assert r1.status == oracle_lib.OK and adaptive_seen
    assert np.any(r1.trace["fnorm"][:r1.iters] > 0)  # the filter did drop entries


# --------------------------------------------------------------------------
# mixed precision (step a8)
# --------------------------------------------------------------------------
def test_mixed_precision_stage_and_drift(oracle_lib):
    a = w.tridiagonal(600)
    r64 = oracle_lib.nsf(a, tol=1e-10, filter="exact")
    rmx = oracle_lib.nsf(a, tol=1e-10, filter="exact", mixed=True)
    assert r64.status == rmx.status == oracle_lib.OK
    prec = list(rmx.trace["prec"])
    assert prec[0] == 32 and prec[-1] == 64 and prec == sorted(prec)
    # every FP32-stage check is above the switch residual except the last one
    res32 = [r for r, p in zip(rmx.trace["resid"], prec) if p == 32]
    assert all(r >= 1e-4 for r in res32[:-1]) and res32[-1] < 1e-4
    S64, Smx = r64.to_dense(a.n), rmx.to_dense(a.n)
    ref = _sign_eig(a.to_dense())
    err = np.linalg.norm(Smx - ref) / np.linalg.norm(ref)
    assert 1e-12 < err < 1e-6  # FP32 drift survives the FP64 finish
    assert np.linalg.norm(Smx @ Smx - np.eye(a.n)) / math.sqrt(a.n) < 1e-9  # still an involution
    d = a.to_dense()
    comm = np.linalg.norm(Smx @ d - d @ Smx) / np.linalg.norm(d)
    assert comm > 1e-12  # the commutator exposes the drift


# --------------------------------------------------------------------------
# edge cases and statuses
# --------------------------------------------------------------------------
def test_edge_cases(oracle_lib):
    one = w.csr_from_dense(np.array([[-3.0]]))
    r = oracle_lib.nsf(one, tol=1e-14)
    assert r.status == oracle_lib.OK and r.val[0] == -1.0 and r.iters == 0
    # zero matrix: no scale exists
    z = w.CSR(3, np.array([0, 0, 0, 0], np.int64), np.zeros(0, np.int32), np.zeros(0))
    with pytest.raises(RuntimeError):
        oracle_lib.nsf(z)
    # unsorted columns are rejected
    bad = w.CSR(2, np.array([0, 2, 3], np.int64), np.array([1, 0, 1], np.int32), np.ones(3))
    with pytest.raises(RuntimeError):
        oracle_lib.nsf(bad)
    # unscaled 3*I leaves the region of convergence (||I - A^2|| >= 1)
    big = w.csr_from_dense(3.0 * np.eye(4))
    r = oracle_lib.nsf(big, scale_1norm=False, filter="none")
    assert r.status == oracle_lib.EDIVERGED
    # a singular matrix (empty row) never converges
    sing = w.csr_from_dense(np.diag([1.0, 0.0, -2.0]))
    r = oracle_lib.nsf(sing, tol=1e-12, max_iter=30)
    assert r.status == oracle_lib.ENOTCONV and r.iters == 30


# --------------------------------------------------------------------------
# variants of the readings (NEXT: filtered T, 2-norm budget)
# --------------------------------------------------------------------------
def test_norm2_estimate_converges_to_the_spectral_norm(oracle_lib):
    """The power iteration on X^T X from (1,...,1)/sqrt(n): exact on a diagonal
    matrix, a lower bound that converges to sigma_max on a random matrix with
    a gap, and non-decreasing in the number of steps."""
    d = np.diag([3.0, -1.0, 0.5, 0.2] + [0.1] * 20)
    a = w.csr_from_dense(d)
    assert abs(oracle_lib.norm2_est(a.n, a.rowptr, a.col, a.val, 8) - 3.0) < 1e-12
    rng = np.random.default_rng(1)
    U, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    V, _ = np.linalg.qr(rng.standard_normal((30, 30)))
    s = np.r_[10.0, np.linspace(6.0, 0.1, 29)]
    M = (U * s) @ V.T
    b = w.csr_from_dense(M)
    est = [oracle_lib.norm2_est(b.n, b.rowptr, b.col, b.val, k) for k in (1, 2, 4, 8, 16)]
    assert all(e <= 10.0 * (1 + 1e-14) for e in est)
    assert all(e2 >= e1 - 1e-12 for e1, e2 in zip(est, est[1:]))
    assert abs(est[-1] - 10.0) < 1e-6


def test_filtered_t_variant_steps_and_theorem_3_2_1(oracle_lib):
    """filter_t: each update multiplies by T filtered with the iterate's own
    budget (checked step by step against the oracle's primitives), and the
    run still satisfies Thm 3.2.1 and stays within 10 tol of plain NS."""
    a = w.banded(300, 4, w.BASE_SEED + 61)
    n = a.n
    tol = 1e-12
    run = oracle_lib.nsf(a, tol=tol, filter="exact", filter_t=True)
    assert run.status == oracle_lib.OK
    tr = run.trace
    assert np.any(tr["nnz_that"][:run.iters] < tr["nnz_t"][:run.iters])  # T really was filtered
    for k in (1, 3):
        xk = oracle_lib.nsf(a, tol=tol, filter="exact", filter_t=True, max_iter=k)
        x1 = oracle_lib.nsf(a, tol=tol, filter="exact", filter_t=True, max_iter=k + 1)
        X = (xk.rowptr, xk.col, xk.val)
        T = oracle_lib.spgemm(n, X, X)
        b = math.sqrt(n) * tr["beta"][k]
        Th, _, _ = oracle_lib.filter_csr(n, T, "exact", b)
        assert Th[0][-1] == tr["nnz_that"][k]
        Xb = oracle_lib.ns_update(n, X, Th)
        Xn, _, _ = oracle_lib.filter_csr(n, Xb, "exact", b)
        assert np.array_equal(Xn[1], x1.col) and np.array_equal(Xn[2], x1.val)
    for k in range(run.iters + 1):
        r1 = oracle_lib.nsf(a, tol=tol, filter="exact", filter_t=True, max_iter=k)
        r0 = oracle_lib.nsf(a, tol=0.0, filter="none", max_iter=r1.iters)
        X0, X1 = r0.to_dense(n), r1.to_dense(n)
        R0, R1 = np.eye(n) - X0 @ X0, np.eye(n) - X1 @ X1
        assert np.linalg.norm(R1 - R0) <= 3 * np.linalg.norm(R0) + 1e-13
        assert np.linalg.norm(X1 - X0) / math.sqrt(n) <= 10 * tol
    S = run.to_dense(n)
    assert np.linalg.norm(S - _sign_eig(a.to_dense())) / np.linalg.norm(S) < 1e-10


def test_budget_norm_variant_uses_the_spectral_estimate(oracle_lib):
    """budget_norm='2': in the adaptive phase beta = 3/4 r^2 / (3 x + x^3) with
    x the power-iteration estimate of ||X_k||_2 (within 1e-6 of numpy's 2-norm
    here); the converged sign matches the eigendecomposition."""
    a = w.tridiagonal(500)
    n = a.n
    run = oracle_lib.nsf(a, tol=1e-13, filter="exact", budget_norm="2")
    assert run.status == oracle_lib.OK
    tr = run.trace
    adaptive = [k for k in range(run.iters) if tr["resid"][k] < 1e-6]
    assert adaptive
    for k in adaptive:
        xk = oracle_lib.nsf(a, tol=1e-13, filter="exact", budget_norm="2", max_iter=k)
        x2 = oracle_lib.norm2_est(n, xk.rowptr, xk.col, xk.val, 8)
        assert abs(x2 - np.linalg.norm(xk.to_dense(n), 2)) < 1e-6
        r = tr["resid"][k]
        assert tr["beta"][k] == 0.75 * r * r / (3.0 * x2 + x2 * x2 * x2)
    S = run.to_dense(n)
    assert np.linalg.norm(S - _sign_eig(a.to_dense())) / np.linalg.norm(S) < 1e-10
