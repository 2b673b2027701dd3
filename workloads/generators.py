"""Seeded synthetic sparse matrices for the filtered Newton-Schulz sign solver.

This module only builds input matrices. It holds none of the sign method's
arithmetic, and both the CPU oracle and the CUDA path take their inputs from
here, so that the two sides see the same bytes.

Every matrix is returned as CSR in the layout the library expects:
``rowptr`` int64[n+1], ``col`` int32[nnz] (ascending inside each row, no
duplicates), ``val`` float64[nnz].

Random numbers come from SplitMix64 used as a counter-based generator: draw
``i`` of a stream with seed ``s`` is ``mix(s + (i + 1) * 0x9E3779B97F4A7C15)``
(mod 2**64), and a uniform in [0, 1) is ``(z >> 11) * 2**-53``. SplitMix64 is
Steele, Lea and Flood, "Fast splittable pseudorandom number generators"
(OOPSLA 2014). Seeds are ``221003356 + 1000 * workload_index (+ matrix index)``.

Workloads (sizes are those of the benchmark suite of this library):

* ``tridiagonal``: symmetric tridiagonal, n=2000. Diagonal s_i*(1+u_i) with
  s_i = +-1 (p = 1/2), off-diagonal 0.3*U[-1,1]. Gershgorin keeps every
  eigenvalue outside (-0.4, 0.4).
* ``laplacian2d``: 5-point Dirichlet Laplacian on an m x m grid minus sigma*I,
  sigma mid-gap next to the spectral centre 4 (n = m*m; m = 256 is n = 65,536).
* ``laplacian3d``: 7-point Laplacian on m^3 minus sigma*I, sigma mid-gap at the
  centre 6.
* ``banded_batch``: independent symmetric banded matrices, n log-uniform in
  [200, 8000], half-bandwidth uniform in {1..10}, diagonal +-(1+U[0,1)),
  off-diagonals U[-1,1] scaled so every row's off-diagonal sum is <= 0.8.
* ``ode_block``: the block matrix [[0, B], [I, 0]] of the paper's Sec. 4.2
  (Eq. 1.25-1.26), B = tridiag(1/16, 7/8, 1/16).
* ``spd_random``: random sparse symmetric positive definite matrices, the
  stand-in for the paper's ``sprandsym(n, 0.01, 1)`` inputs of Sec. 4.1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

BASE_SEED = 221003356
_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+count-1`` of the SplitMix64 stream ``seed``."""
    i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed % (1 << 64)) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits each."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


@dataclass
class CSR:
    """One square sparse matrix in CSR."""

    n: int
    rowptr: np.ndarray  # int64[n+1]
    col: np.ndarray  # int32[nnz]
    val: np.ndarray  # float64[nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.rowptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.rowptr))
        d[rows, self.col] = self.val
        return d


def csr_from_coo(n: int, rows, cols, vals, name: str = "") -> CSR:
    """Builds CSR with sorted, de-duplicated columns (duplicates must not occur)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    if rows.size > 1:
        dup = (rows[1:] == rows[:-1]) & (cols[1:] == cols[:-1])
        if dup.any():
            raise ValueError("duplicate entries")
    counts = np.bincount(rows, minlength=n)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return CSR(n, rowptr, cols.astype(np.int32), vals, name)


def csr_from_dense(d: np.ndarray, name: str = "") -> CSR:
    r, c = np.nonzero(d)
    return csr_from_coo(d.shape[0], r, c, d[r, c], name)


# --------------------------------------------------------------------------
# tridiagonal, n = 2000 (the small correctness workload)
# --------------------------------------------------------------------------
def tridiagonal(n: int = 2000, seed: int = BASE_SEED + 0) -> CSR:
    """Symmetric tridiagonal; stream layout: signs[n], magnitudes[n], off[n-1]."""
    u = uniform01(seed, 3 * n - 1)
    sign = np.where(u[:n] < 0.5, -1.0, 1.0)
    diag = sign * (1.0 + u[n:2 * n])
    off = 0.3 * (2.0 * u[2 * n:] - 1.0)
    i = np.arange(n)
    j = np.arange(n - 1)
    rows = np.concatenate([i, j, j + 1])
    cols = np.concatenate([i, j + 1, j])
    vals = np.concatenate([diag, off, off])
    return csr_from_coo(n, rows, cols, vals, f"tridiagonal n={n}")


# --------------------------------------------------------------------------
# shifted Laplacians with closed-form spectra
# --------------------------------------------------------------------------
def _path_eigs(m: int) -> np.ndarray:
    """Eigenvalues 2 - 2cos(i*pi/(m+1)), i = 1..m, of tridiag(-1, 2, -1)."""
    i = np.arange(1, m + 1)
    return 2.0 - 2.0 * np.cos(i * math.pi / (m + 1))


def laplacian_shift(m: int, dim: int) -> float:
    """Mid-gap shift sigma for the dim-D Dirichlet Laplacian on m^dim points.

    The spectrum is symmetric about its centre c = 2*dim. If c is itself an
    eigenvalue (numerically, within 1e-12), sigma is the midpoint between c
    and the nearest distinct eigenvalue above it; otherwise sigma = c, which
    then lies midway between the nearest eigenvalues below and above.
    """
    e = _path_eigs(m)
    c = 2.0 * dim
    if dim == 2:
        lam = (e[:, None] + e[None, :]).ravel()
    elif dim == 3:
        lam = (e[:, None, None] + e[None, :, None] + e[None, None, :]).ravel()
    else:
        lam = e
    d = lam - c
    if np.min(np.abs(d)) < 1e-12:
        above = np.min(d[d > 1e-12])
        return c + above / 2.0
    return c


def laplacian_eigs(m: int, dim: int) -> np.ndarray:
    e = _path_eigs(m)
    if dim == 1:
        return e
    if dim == 2:
        return (e[:, None] + e[None, :]).ravel()
    return (e[:, None, None] + e[None, :, None] + e[None, None, :]).ravel()


def laplacian(m: int, dim: int, sigma: float | None = None) -> CSR:
    """Dirichlet Laplacian L on an m^dim grid, returns L - sigma*I.

    Grid point (x, y, z) has index x + m*y + m*m*z (0-based).
    """
    if sigma is None:
        sigma = laplacian_shift(m, dim)
    n = m ** dim
    idx = np.arange(n)
    coords = [(idx // (m ** a)) % m for a in range(dim)]
    rows = [idx]
    cols = [idx]
    vals = [np.full(n, 2.0 * dim - sigma)]
    for a in range(dim):
        stride = m ** a
        for step in (-1, 1):
            ok = (coords[a] + step >= 0) & (coords[a] + step < m)
            rows.append(idx[ok])
            cols.append(idx[ok] + step * stride)
            vals.append(np.full(int(ok.sum()), -1.0))
    return csr_from_coo(n, np.concatenate(rows), np.concatenate(cols),
                        np.concatenate(vals), f"laplacian{dim}d m={m} sigma={sigma!r}")


def laplacian2d(m: int = 256) -> CSR:
    return laplacian(m, 2)


def laplacian3d(m: int = 64) -> CSR:
    return laplacian(m, 3)


# --------------------------------------------------------------------------
# batch of banded matrices
# --------------------------------------------------------------------------
def banded(n: int, b: int, seed: int) -> CSR:
    """Symmetric banded matrix with half-bandwidth b.

    Stream layout: signs[n], magnitudes[n], then the upper off-diagonals
    diagonal by diagonal (d = 1..b, i = 0..n-d-1). Off-diagonals are U[-1,1]
    mirrored; with s_i = min(1, 0.8 / sum_j |a_ij|) every a_ij is multiplied by
    min(s_i, s_j), which keeps symmetry and every off-diagonal row sum <= 0.8.
    """
    b = min(b, n - 1)
    noff = sum(n - d for d in range(1, b + 1))
    u = uniform01(seed, 2 * n + noff, offset=2)
    sign = np.where(u[:n] < 0.5, -1.0, 1.0)
    diag = sign * (1.0 + u[n:2 * n])
    rows, cols, vals = [np.arange(n)], [np.arange(n)], [diag]
    pos = 2 * n
    ur, uc, uv = [], [], []
    for d in range(1, b + 1):
        i = np.arange(n - d)
        ur.append(i)
        uc.append(i + d)
        uv.append(2.0 * u[pos:pos + n - d] - 1.0)
        pos += n - d
    if b > 0:
        ur = np.concatenate(ur)
        uc = np.concatenate(uc)
        uv = np.concatenate(uv)
        rowsum = np.bincount(ur, weights=np.abs(uv), minlength=n) + \
            np.bincount(uc, weights=np.abs(uv), minlength=n)
        with np.errstate(divide="ignore"):
            s = np.where(rowsum > 0, np.minimum(1.0, 0.8 / np.where(rowsum > 0, rowsum, 1.0)), 1.0)
        uv = uv * np.minimum(s[ur], s[uc])
        rows += [ur, uc]
        cols += [uc, ur]
        vals += [uv, uv]
    return csr_from_coo(n, np.concatenate(rows), np.concatenate(cols),
                        np.concatenate(vals), f"banded n={n} b={b}")


def banded_batch_shapes(count: int = 512, seed0: int = BASE_SEED + 3000,
                        nmin: int = 200, nmax: int = 8000) -> list[tuple[int, int, int]]:
    """(n, b, seed) for each matrix of the batch; draws 0 and 1 of each stream."""
    out = []
    for k in range(count):
        seed = seed0 + k
        u = uniform01(seed, 2)
        n = int(round(math.exp(math.log(nmin) + u[0] * (math.log(nmax) - math.log(nmin)))))
        b = 1 + min(9, int(u[1] * 10))
        out.append((n, b, seed))
    return out


def banded_batch(count: int = 512, seed0: int = BASE_SEED + 3000,
                 nmin: int = 200, nmax: int = 8000) -> list[CSR]:
    return [banded(n, b, s) for n, b, s in banded_batch_shapes(count, seed0, nmin, nmax)]


# --------------------------------------------------------------------------
# the paper's Sec. 4.2 block matrix and Sec. 4.1-style SPD inputs
# --------------------------------------------------------------------------
def ode_tridiag(n: int, lam: float = 1.0 / 16.0) -> CSR:
    """B = tridiag(lam, 1 - 2 lam, lam) of order n (Eq. 1.25)."""
    i = np.arange(n)
    j = np.arange(n - 1)
    rows = np.concatenate([i, j, j + 1])
    cols = np.concatenate([i, j + 1, j])
    vals = np.concatenate([np.full(n, 1.0 - 2.0 * lam), np.full(n - 1, lam), np.full(n - 1, lam)])
    return csr_from_coo(n, rows, cols, vals, f"ode B n={n}")


def ode_block(n: int, lam: float = 1.0 / 16.0) -> CSR:
    """A = [[0, B], [I, 0]] of order 2n (Eq. 1.26)."""
    B = ode_tridiag(n, lam)
    brow = np.repeat(np.arange(n), np.diff(B.rowptr))
    rows = np.concatenate([brow, n + np.arange(n)])
    cols = np.concatenate([n + B.col.astype(np.int64), np.arange(n)])
    vals = np.concatenate([B.val, np.ones(n)])
    return csr_from_coo(2 * n, rows, cols, vals, f"ode block 2n={2 * n}")


def spd_random(n: int, density: float = 0.01, seed: int = BASE_SEED + 7000) -> CSR:
    """Random sparse symmetric positive definite matrix.

    Off-diagonal pattern: each upper pair (i, j) is present with probability
    about density/2 (so the full matrix has about density * n^2 entries),
    values U[-1, 1]; the diagonal is the absolute off-diagonal row sum plus
    U[0.5, 1.5), so the matrix is strictly diagonally dominant with positive
    diagonal, hence SPD.
    """
    m = int(round(density * n * n / 2.0))
    z = splitmix64(seed, 3 * m + n)
    i = (z[:m] % np.uint64(n)).astype(np.int64)
    j = (z[m:2 * m] % np.uint64(n)).astype(np.int64)
    u = (z[2 * m:3 * m] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    keep = i != j
    lo, hi, v = np.minimum(i, j)[keep], np.maximum(i, j)[keep], (2.0 * u[keep] - 1.0)
    key = lo * n + hi
    _, first = np.unique(key, return_index=True)
    lo, hi, v = lo[first], hi[first], v[first]
    rowsum = np.bincount(lo, weights=np.abs(v), minlength=n) + np.bincount(hi, weights=np.abs(v), minlength=n)
    ud = (z[3 * m:] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    diag = rowsum + 0.5 + ud
    rows = np.concatenate([np.arange(n), lo, hi])
    cols = np.concatenate([np.arange(n), hi, lo])
    vals = np.concatenate([diag, v, v])
    return csr_from_coo(n, rows, cols, vals, f"spd n={n} density={density}")


def sprand_like(n: int, density: float = 0.01, seed: int = BASE_SEED + 8000) -> CSR:
    """Random sparse nonsymmetric matrix, the stand-in for sprand(n, n, density)
    of the paper's first filter-error test (Sec. 4.1, Fig. 4.1.1).

    About density * n^2 off-diagonal entries at uniformly drawn positions,
    values U[0, 1) (as sprand draws them), plus a diagonal s_i (1 + u_i) with
    random signs s_i = +-1. The diagonal keeps the matrix nonsingular and its
    eigenvalues off the imaginary axis (the off-diagonal part alone would
    leave empty rows at this density), so Newton's method converges.
    """
    m = int(round(density * n * n))
    z = splitmix64(seed, 3 * m + 2 * n)
    i = (z[:m] % np.uint64(n)).astype(np.int64)
    j = (z[m:2 * m] % np.uint64(n)).astype(np.int64)
    u = (z[2 * m:3 * m] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    keep = i != j
    i, j, u = i[keep], j[keep], u[keep]
    _, first = np.unique(i * n + j, return_index=True)
    i, j, u = i[first], j[first], u[first]
    ud = (z[3 * m:3 * m + n] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    sd = np.where((z[3 * m + n:] >> np.uint64(63)) == np.uint64(1), -1.0, 1.0)
    rows = np.concatenate([np.arange(n), i])
    cols = np.concatenate([np.arange(n), j])
    vals = np.concatenate([sd * (1.0 + ud), u])
    return csr_from_coo(n, rows, cols, vals, f"sprand-like n={n} density={density}")


def block_diagonal(mats: list[CSR]) -> CSR:
    """Concatenates matrices into one block-diagonal CSR (column indices shifted)."""
    offs = np.cumsum([0] + [a.n for a in mats])
    rowptrs = [np.zeros(1, dtype=np.int64)]
    base = 0
    for a in mats:
        rowptrs.append(a.rowptr[1:] + base)
        base += a.nnz
    cols = np.concatenate([a.col.astype(np.int64) + o for a, o in zip(mats, offs[:-1])])
    return CSR(int(offs[-1]), np.concatenate(rowptrs), cols.astype(np.int32),
               np.concatenate([a.val for a in mats]), "block-diagonal")
