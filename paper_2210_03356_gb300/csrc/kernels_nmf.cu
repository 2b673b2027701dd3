// Newton's method with filtering (NMF, Alg. 3.1.1): the dense inverse of the
// current iterate and the Newton update Xbar = (X + X^-1) / 2.
//
// The inverse follows LU with partial pivoting (right-looking: for each
// column c the first row of largest magnitude at or below c becomes the
// pivot, the rows below are reduced by l = a_rc / a_cc with one rounded
// product and one rounded subtraction per entry), then, for each column e of
// the identity, the forward substitution L y = P e and the back substitution
// U x = y with their sums in ascending index order. The column solves are
// independent and run one per thread. Every operation is an explicitly
// rounded FP64 operation, so the inverse is the same on every run.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace sgn {

namespace {

constexpr int PIVOT_THREADS = 1024;

// The pivot of column c: the first row r >= c of largest |lu[r][c]| (a NaN
// diagonal keeps row c, as a sequential scan from row c would); a largest
// magnitude of 0 marks the matrix singular.
__global__ void __launch_bounds__(PIVOT_THREADS)
    k_lu_pivot(int n, int ld, const double *lu, int c, int *pivot, int *singular) {
  __shared__ double sv[PIVOT_THREADS / 32];
  __shared__ int si[PIVOT_THREADS / 32];
  if (*singular) return;
  double best = -1.0;
  int bi = n;
  for (int r = c + int(threadIdx.x); r < n; r += PIVOT_THREADS) {
    const double v = fabs(lu[int64_t(r) * ld + c]);
    if (v > best) {  // rows ascend within a thread: ties keep the first
      best = v;
      bi = r;
    }
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) {
      best = ov;
      bi = oi;
    }
  }
  if (lane == 0) {
    sv[w] = best;
    si[w] = bi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < PIVOT_THREADS / 32; ++i)
      if (sv[i] > best || (sv[i] == best && si[i] < bi)) {
        best = sv[i];
        bi = si[i];
      }
    const double d = fabs(lu[int64_t(c) * ld + c]);
    if (d != d) {  // NaN pivot candidate at c: kept, as a scan from row c would
      best = d;
      bi = c;
    }
    if (best == 0.0) *singular = 1;
    *pivot = bi < n ? bi : c;
  }
}

__global__ void k_lu_swap(int n, int ld, double *lu, int c, const int *pivot, int *perm,
                          const int *singular) {
  if (*singular) return;
  const int pr = *pivot;
  if (pr == c) return;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const double t = lu[int64_t(c) * ld + j];
    lu[int64_t(c) * ld + j] = lu[int64_t(pr) * ld + j];
    lu[int64_t(pr) * ld + j] = t;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const int t = perm[c];
    perm[c] = perm[pr];
    perm[pr] = t;
  }
}

// rows r > c, columns j > c: lu[r][j] -= (lu[r][c] / lu[c][c]) lu[c][j]
__global__ void k_lu_update(int n, int ld, double *lu, int c, const int *singular) {
  if (*singular) return;
  const int j = c + 1 + blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double piv = lu[int64_t(c) * ld + c], ucj = lu[int64_t(c) * ld + j];
  for (int r = c + 1 + blockIdx.y; r < n; r += gridDim.y) {
    const double l = __ddiv_rn(lu[int64_t(r) * ld + c], piv);
    double *a = lu + int64_t(r) * ld + j;
    *a = __dsub_rn(*a, __dmul_rn(l, ucj));
  }
}

// the multipliers into column c (after the rows were reduced with them)
__global__ void k_lu_store_l(int n, int ld, double *lu, int c, const int *singular) {
  if (*singular) return;
  const double piv = lu[int64_t(c) * ld + c];
  for (int r = c + 1 + blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += gridDim.x * blockDim.x)
    lu[int64_t(r) * ld + c] = __ddiv_rn(lu[int64_t(r) * ld + c], piv);
}

// column e of the inverse: L y = P e_e, then U x = y (in place in inv)
__global__ void k_lu_solve(int n, int ld, const double *lu, const int *perm, double *inv,
                           const int *singular) {
  if (*singular) return;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  for (int i = 0; i < n; ++i) {
    double s = perm[i] == e ? 1.0 : 0.0;
    const double *li = lu + int64_t(i) * ld;
    for (int j = 0; j < i; ++j) s = __dsub_rn(s, __dmul_rn(li[j], inv[int64_t(j) * ld + e]));
    inv[int64_t(i) * ld + e] = s;
  }
  for (int i = n - 1; i >= 0; --i) {
    const double *ui = lu + int64_t(i) * ld;
    double s = inv[int64_t(i) * ld + e];
    for (int j = i + 1; j < n; ++j) s = __dsub_rn(s, __dmul_rn(ui[j], inv[int64_t(j) * ld + e]));
    inv[int64_t(i) * ld + e] = __ddiv_rn(s, ui[i]);
  }
}

// part[i] = sum_j inv_ij^2 (warp per row, fixed order)
__global__ void k_inv_rowsq(int n, int ld, const double *inv, double *part) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < n; i += nw) {
    double a = 0.0;
    for (int j = lane; j < n; j += 32) a = __fma_rn(inv[i * ld + j], inv[i * ld + j], a);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = __dadd_rn(a, __shfl_xor_sync(0xffffffffu, a, o));
    if (lane == 0) part[i] = a;
  }
}

// *out = sqrt(sum_i part[i]) / sqrt(n), the rows added in order
__global__ void k_inv_norm(int n, const double *part, double *out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s = __dadd_rn(s, part[i]);
  *out = __ddiv_rn(__dsqrt_rn(s), __dsqrt_rn(double(n)));
}

__global__ void k_nmf_densify(int n, int ld, const int64_t *rp, const int32_t *col,
                              const double *val, int64_t row0, double *dx) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; i < n; i += nw)
    for (int64_t p = rp[row0 + i] + lane; p < rp[row0 + i + 1]; p += 32)
      dx[i * ld + (col[p] - row0)] = val[p];
}

// Xbar = (X + X^-1) / 2 as n full rows of slots from slot0 (global columns
// from row0), every entry kept (the filter drops the exact zeros)
__global__ void k_nmf_combine(int n, int ld, const double *dx, const double *inv, int64_t row0,
                              int64_t slot0, int64_t *rs, int64_t *re, int32_t *ccol,
                              double *cval) {
  const int64_t total = int64_t(n) * n;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < total;
       t += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = t / n, j = t - i * n;
    ccol[slot0 + t] = int32_t(row0 + j);
    cval[slot0 + t] = __dmul_rn(0.5, __dadd_rn(dx[i * ld + j], inv[i * ld + j]));
    if (j == 0) {
      rs[row0 + i] = slot0 + i * n;
      re[row0 + i] = slot0 + (i + 1) * n;
    }
  }
}

// Eq. (1.13): c4 tol while r >= switch_resid, else r^2 / (x + ||X^-1||)
__global__ void k_nmf_budget(int m, int64_t n, const double *xinv, double c4, double tol,
                             double switch_resid, MatScalars *ms) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double r = ms[m].r, x = ms[m].x;
  const double beta = r >= switch_resid ? __dmul_rn(c4, tol)
                                        : __ddiv_rn(__dmul_rn(r, r), __dadd_rn(x, *xinv));
  ms[m].beta = beta;
  ms[m].b = __dmul_rn(__dsqrt_rn(double(n)), beta);
}

__global__ void k_perm_init(int n, int *perm) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) perm[i] = i;
}

int blocks_for(int64_t items, int per) {
  int64_t g = (items + per - 1) / per;
  return int(g < 1 ? 1 : (g > 152 * 32 ? 152 * 32 : g));
}

}  // namespace

void launch_dense_inverse(int n, int ld, double *lu, int *perm, int *pivot, int *singular,
                          double *inv, cudaStream_t s) {
  if (n <= 0) return;
  SGN_CUDA(cudaMemsetAsync(singular, 0, sizeof(int), s));
  k_perm_init<<<blocks_for(n, 256), 256, 0, s>>>(n, perm);
  SGN_LAUNCH_CHECK();
  for (int c = 0; c < n; ++c) {
    k_lu_pivot<<<1, PIVOT_THREADS, 0, s>>>(n, ld, lu, c, pivot, singular);
    SGN_LAUNCH_CHECK();
    k_lu_swap<<<blocks_for(n, 256), 256, 0, s>>>(n, ld, lu, c, pivot, perm, singular);
    SGN_LAUNCH_CHECK();
    if (c + 1 < n) {
      const int cols = n - c - 1;
      dim3 g(unsigned((cols + 127) / 128), unsigned(std::min(cols, 1024)));
      k_lu_update<<<g, 128, 0, s>>>(n, ld, lu, c, singular);
      SGN_LAUNCH_CHECK();
      k_lu_store_l<<<blocks_for(cols, 256), 256, 0, s>>>(n, ld, lu, c, singular);
      SGN_LAUNCH_CHECK();
    }
  }
  k_lu_solve<<<(n + 63) / 64, 64, 0, s>>>(n, ld, lu, perm, inv, singular);
  SGN_LAUNCH_CHECK();
}

void launch_inv_norm(int n, int ld, const double *inv, double *part, double *out,
                     cudaStream_t s) {
  if (n <= 0) return;
  k_inv_rowsq<<<blocks_for(n, 8), 256, 0, s>>>(n, ld, inv, part);
  SGN_LAUNCH_CHECK();
  k_inv_norm<<<1, 32, 0, s>>>(n, part, out);
  SGN_LAUNCH_CHECK();
}

void launch_nmf_densify(int n, int ld, const int64_t *rp, const int32_t *col, const double *val,
                        int64_t row0, double *dx, cudaStream_t s) {
  if (n <= 0) return;
  k_nmf_densify<<<blocks_for(n, 8), 256, 0, s>>>(n, ld, rp, col, val, row0, dx);
  SGN_LAUNCH_CHECK();
}

void launch_nmf_combine(int n, int ld, const double *dx, const double *inv, int64_t row0,
                        int64_t slot0, int64_t *rs, int64_t *re, int32_t *col, double *val,
                        cudaStream_t s) {
  if (n <= 0) return;
  k_nmf_combine<<<blocks_for(int64_t(n) * n, 256), 256, 0, s>>>(n, ld, dx, inv, row0, slot0, rs,
                                                                 re, col, val);
  SGN_LAUNCH_CHECK();
}

void launch_nmf_budget(int m, int64_t n, const double *xinv, double c4, double tol,
                       double switch_resid, MatScalars *ms, cudaStream_t s) {
  k_nmf_budget<<<1, 32, 0, s>>>(m, n, xinv, c4, tol, switch_resid, ms);
  SGN_LAUNCH_CHECK();
}

}  // namespace sgn
