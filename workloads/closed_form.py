"""Exact sign functions of the synthetic workloads whose spectra are known in
closed form, used to check results (never a step of the solve).

- Shifted Dirichlet Laplacians on an m^dim grid: L = sum of 1-D path
  Laplacians, eigenvectors the tensor products of the sine basis
  q[x, i] = sqrt(2/(m+1)) sin((x+1) i pi/(m+1)), eigenvalues
  sum_a (2 - 2 cos(i_a pi/(m+1))); sign(L - sigma I) = V sign(Lambda - sigma) V^T.
- Sec. 4.2's ODE block matrix A = [[0, B], [I, 0]]: sign(A) =
  [[0, B^1/2], [B^-1/2, 0]] (Eq. 1.26), B = tridiag(lam, 7/8, lam) with the
  same sine eigenbasis.
"""
from __future__ import annotations

import math

import numpy as np

from .generators import laplacian_shift


def laplacian_sign_entries(m: int, dim: int, p, pp) -> np.ndarray:
    """S[p, pp] of sign(L - sigma I) (sigma = laplacian_shift(m, dim)) for grid
    indices p, pp (x + m y + m^2 z); an O(m^dim) sum per entry."""
    sigma = laplacian_shift(m, dim)
    h = math.pi / (m + 1)
    k = np.arange(1, m + 1)
    lam1 = 2 - 2 * np.cos(k * h)
    q = np.sqrt(2.0 / (m + 1)) * np.sin(np.outer(np.arange(1, m + 1), k) * h)  # q[x, i]

    def coord(idx, a):
        return (idx // m ** a) % m

    f = [q[coord(p, a)] * q[coord(pp, a)] for a in range(dim)]  # (samples, m) each
    if dim == 2:
        sgn = np.sign(lam1[:, None] + lam1[None, :] - sigma)
        return np.einsum("si,ij,sj->s", f[0], sgn, f[1])
    sgn = np.sign(lam1[:, None, None] + lam1[None, :, None] + lam1[None, None, :] - sigma)
    return np.einsum("si,sj,sk,ijk->s", f[0], f[1], f[2], sgn)


def csr_entries(rowptr, col, val, p, pp) -> np.ndarray:
    """Entries (p, pp) of a CSR matrix (0 where absent)."""
    out = np.zeros(len(p))
    for t, (i, j) in enumerate(zip(p, pp)):
        lo, hi = rowptr[i], rowptr[i + 1]
        k = np.searchsorted(col[lo:hi], j)
        if k < hi - lo and col[lo + k] == j:
            out[t] = val[lo + k]
    return out


def ode_block_sign(nb: int, lam: float = 1.0 / 16.0) -> np.ndarray:
    """sign([[0, B], [I, 0]]) = [[0, B^1/2], [B^-1/2, 0]] (Eq. 1.26) for
    B = tridiag(lam, 7/8, lam) of order nb, from B's sine eigenbasis:
    eigenvalues 7/8 + 2 lam cos(j pi/(nb+1)), eigenvectors
    sqrt(2/(nb+1)) sin(i j pi/(nb+1))."""
    j = np.arange(1, nb + 1)
    h = np.pi / (nb + 1)
    V = np.sqrt(2.0 / (nb + 1)) * np.sin(np.outer(j, j) * h)
    mu = 7.0 / 8.0 + 2.0 * lam * np.cos(j * h)
    S = np.zeros((2 * nb, 2 * nb))
    S[:nb, nb:] = (V * np.sqrt(mu)) @ V.T
    S[nb:, :nb] = (V / np.sqrt(mu)) @ V.T
    return S
