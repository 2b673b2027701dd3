"""Seeded synthetic inputs shared by the CPU oracle tests and the CUDA path."""
from .generators import (BASE_SEED, CSR, banded, banded_batch, banded_batch_shapes,
                         block_diagonal, csr_from_coo, csr_from_dense, laplacian,
                         laplacian2d, laplacian3d, laplacian_eigs, laplacian_shift,
                         ode_block, ode_tridiag, spd_random, splitmix64, sprand_like, tridiagonal,
                         uniform01)

__all__ = ["BASE_SEED", "CSR", "banded", "banded_batch", "banded_batch_shapes",
           "block_diagonal", "csr_from_coo", "csr_from_dense", "laplacian",
           "laplacian2d", "laplacian3d", "laplacian_eigs", "laplacian_shift",
           "ode_block", "ode_tridiag", "spd_random", "splitmix64", "sprand_like", "tridiagonal",
           "uniform01"]
