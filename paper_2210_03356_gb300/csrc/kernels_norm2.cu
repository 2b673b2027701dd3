// The 2-norm reading of ||X|| in the budget of Eq. (1.18) (the budget_norm
// variant): per matrix, a fixed number of power steps on X^T X.
//
//   v_0 = (1, ..., 1) / sqrt(n);  then POW_STEPS times:  y = X v,  z = X^T y,
//   v = z / ||z||;  and finally x2 = ||X v||.
//
// x2 is a lower bound of ||X||_2 that converges to it; for iterates close to
// sign(A) every singular value is close to 1, so the estimate settles in a
// few steps. Every sum has a fixed order or is exact, so the estimate is the
// same on every run: y_i sums row i in the order of the lanes and a fixed
// shuffle tree; z = X^T y adds the products x_ij y_i as integers on a grid
// 2^(g - 62) below a bound 2^g of every |x_ij y_i| of the matrix (128-bit
// sums, order-independent); the norms are per-row squares reduced per matrix
// in a fixed order.
#include <cmath>

#include "common.cuh"
#include "kernels.h"

namespace sgn {

namespace {

// only the matrices in the adaptive phase of the budget use the estimate
__device__ __forceinline__ bool wanted(const MatScalars *ms, int m, double switch_resid) {
  return ms[m].r < switch_resid;
}

__device__ __forceinline__ double val_at(const void *val, int f32, int64_t p) {
  return f32 ? double(static_cast<const float *>(val)[p]) : static_cast<const double *>(val)[p];
}

// floor(log2 v) for v > 0 from the bits of a non-negative double (subnormals
// count as 2^-1023, still an upper bound's exponent after the + 1 below)
__device__ __forceinline__ int exp_of(unsigned long long bits) {
  const int e = int((bits >> 52) & 0x7FFULL);
  return e == 0 ? -1023 : e - 1023;
}

__global__ void k_n2_init(int64_t n, const int32_t *seg, const int64_t *moff, const MatScalars *ms,
                          double sw, double *v) {
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
       r += int64_t(gridDim.x) * blockDim.x) {
    const int m = seg[r];
    if (!wanted(ms, m, sw)) continue;
    v[r] = __ddiv_rn(1.0, __dsqrt_rn(double(moff[m + 1] - moff[m])));
  }
}

__global__ void k_n2_absmax(int64_t n, const int32_t *seg, const int64_t *rs, const int64_t *re,
                            const void *val, int f32, const MatScalars *ms, double sw,
                            unsigned long long *xmax) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; r < n; r += nwarps) {
    if (!wanted(ms, seg[r], sw)) continue;
    double mx = 0.0;
    for (int64_t p = rs[r] + lane; p < re[r]; p += 32) mx = fmax(mx, fabs(val_at(val, f32, p)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0 && mx > 0.0)
      atomicMax(&xmax[seg[r]], (unsigned long long)__double_as_longlong(mx));
  }
}

// y = X v; ymax[m] = max |y_i|; part[i] = y_i^2
__global__ void k_n2_spmv(int64_t n, const int32_t *seg, const int64_t *rs, const int64_t *re,
                          const int32_t *col, const void *val, int f32, const MatScalars *ms,
                          double sw, const double *v, double *y, unsigned long long *ymax,
                          double *part) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; r < n; r += nwarps) {
    if (!wanted(ms, seg[r], sw)) continue;
    double a = 0.0;
    for (int64_t p = rs[r] + lane; p < re[r]; p += 32)
      a = __fma_rn(val_at(val, f32, p), v[col[p]], a);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = __dadd_rn(a, __shfl_xor_sync(0xffffffffu, a, o));
    if (lane == 0) {
      y[r] = a;
      part[r] = __dmul_rn(a, a);
      if (a != 0.0) atomicMax(&ymax[seg[r]], (unsigned long long)__double_as_longlong(fabs(a)));
    }
  }
}

// z += X^T y on each matrix's integer grid (128-bit signed column sums)
__global__ void k_n2_spmv_t(int64_t n, const int32_t *seg, const int64_t *rs, const int64_t *re,
                            const int32_t *col, const void *val, int f32, const MatScalars *ms,
                            double sw, const double *y, const unsigned long long *xmax,
                            const unsigned long long *ymax, unsigned long long *zacc) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; r < n; r += nwarps) {
    if (!wanted(ms, seg[r], sw)) continue;
    const double yr = y[r];
    if (yr == 0.0) continue;
    const int m = seg[r];
    const unsigned long long xb = xmax[m], yb = ymax[m];
    if (!xb || !yb) continue;
    const int g = exp_of(xb) + exp_of(yb) + 2;  // every |x_ij y_i| < 2^g
    const double scale = ldexp(1.0, 62 - g);
    for (int64_t p = rs[r] + lane; p < re[r]; p += 32) {
      const double t = __dmul_rn(val_at(val, f32, p), yr);
      const long long q = __double2ll_rn(__dmul_rn(t, scale));
      if (!q) continue;
      unsigned long long *z = zacc + 2 * int64_t(col[p]);
      const unsigned long long lo = (unsigned long long)q;
      unsigned long long hi = q < 0 ? ~0ULL : 0ULL;
      const unsigned long long old = atomicAdd(&z[0], lo);
      if (old + lo < old) ++hi;
      if (hi) atomicAdd(&z[1], hi);
    }
  }
}

// z_j from its 128-bit sum (then cleared); part[j] = z_j^2
__global__ void k_n2_zfinal(int64_t n, const int32_t *seg, const MatScalars *ms, double sw,
                            const unsigned long long *xmax, const unsigned long long *ymax,
                            unsigned long long *zacc, double *z, double *part) {
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n;
       j += int64_t(gridDim.x) * blockDim.x) {
    const int m = seg[j];
    if (!wanted(ms, m, sw)) continue;
    const unsigned long long lo = zacc[2 * j], hi = zacc[2 * j + 1];
    zacc[2 * j] = 0ULL;
    zacc[2 * j + 1] = 0ULL;
    double zj = 0.0;
    const unsigned long long xb = xmax[m], yb = ymax[m];
    if (xb && yb && (lo | hi)) {
      const int g = exp_of(xb) + exp_of(yb) + 2;
      const double v = __dadd_rn(__dmul_rn(double((long long)hi), 18446744073709551616.0),
                                 double(lo));
      zj = __dmul_rn(v, ldexp(1.0, g - 62));
    }
    z[j] = zj;
    part[j] = __dmul_rn(zj, zj);
  }
}

// v = z / ||z|| per matrix (v unchanged where ||z|| = 0: then X^T X v = 0 and
// every later step gives the same ||X v||)
__global__ void k_n2_scale(int64_t n, const int32_t *seg, const MatScalars *ms, double sw,
                           const double *z, const double *nz2, double *v) {
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n;
       j += int64_t(gridDim.x) * blockDim.x) {
    if (!wanted(ms, seg[j], sw)) continue;
    const double s = __dsqrt_rn(nz2[seg[j]]);
    if (s > 0.0) v[j] = __ddiv_rn(z[j], s);
  }
}

__global__ void k_n2_final(int nb, const double *ny2, double *x2) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < nb) x2[m] = __dsqrt_rn(ny2[m]);
}

// Eq. (1.18) with x = x2 for the matrices in the adaptive phase
__global__ void k_budget_x2(int nb, const int64_t *moff, const double *x2, double switch_resid,
                            MatScalars *ms) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nb) return;
  const double r = ms[m].r;
  if (!(r < switch_resid)) return;
  const double x = x2[m];
  const double beta = __ddiv_rn(__dmul_rn(__dmul_rn(0.75, r), r),
                                __dadd_rn(__dmul_rn(3.0, x), __dmul_rn(__dmul_rn(x, x), x)));
  ms[m].beta = beta;
  ms[m].b = __dmul_rn(__dsqrt_rn(double(moff[m + 1] - moff[m])), beta);
}

int grid_of(int64_t items, int per_block) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t g = (items + per_block - 1) / per_block;
  const int64_t cap = int64_t(sms > 0 ? sms : 1) * 16;
  if (g > cap) g = cap;
  return int(g < 1 ? 1 : g);
}

}  // namespace

void launch_norm2_est(int nb, const int64_t *moff, const int32_t *seg, int64_t n, const Rows &X,
                      const void *val, int val_f32, const MatScalars *ms, double switch_resid,
                      const Norm2Work &wk, double *x2, cudaStream_t s) {
  if (n == 0 || nb == 0) return;
  const int gr = grid_of(n, 256), gw = grid_of(n, 8);
  const double sw = switch_resid;
  SGN_CUDA(cudaMemsetAsync(wk.xmax, 0, sizeof(unsigned long long) * size_t(nb), s));
  SGN_CUDA(cudaMemsetAsync(wk.zacc, 0, sizeof(unsigned long long) * 2 * size_t(n), s));
  k_n2_init<<<gr, 256, 0, s>>>(n, seg, moff, ms, sw, wk.v);
  SGN_LAUNCH_CHECK();
  k_n2_absmax<<<gw, 256, 0, s>>>(n, seg, X.rs, X.re, val, val_f32, ms, sw, wk.xmax);
  SGN_LAUNCH_CHECK();
  for (int step = 0; step <= NORM2_STEPS; ++step) {
    SGN_CUDA(cudaMemsetAsync(wk.ymax, 0, sizeof(unsigned long long) * size_t(nb), s));
    k_n2_spmv<<<gw, 256, 0, s>>>(n, seg, X.rs, X.re, X.col, val, val_f32, ms, sw, wk.v, wk.y,
                                 wk.ymax, wk.part);
    SGN_LAUNCH_CHECK();
    if (step == NORM2_STEPS) break;
    k_n2_spmv_t<<<gw, 256, 0, s>>>(n, seg, X.rs, X.re, X.col, val, val_f32, ms, sw, wk.y,
                                   wk.xmax, wk.ymax, wk.zacc);
    SGN_LAUNCH_CHECK();
    k_n2_zfinal<<<gr, 256, 0, s>>>(n, seg, ms, sw, wk.xmax, wk.ymax, wk.zacc, wk.z, wk.part);
    SGN_LAUNCH_CHECK();
    launch_seg_reduce(nb, moff, wk.part, 1, wk.nrm, s);
    k_n2_scale<<<gr, 256, 0, s>>>(n, seg, ms, sw, wk.z, wk.nrm, wk.v);
    SGN_LAUNCH_CHECK();
  }
  launch_seg_reduce(nb, moff, wk.part, 1, wk.nrm, s);
  k_n2_final<<<(nb + 127) / 128, 128, 0, s>>>(nb, wk.nrm, x2);
  SGN_LAUNCH_CHECK();
}

void launch_budget_x2(int nb, const int64_t *moff, const double *x2, double switch_resid,
                      MatScalars *ms, cudaStream_t s) {
  if (nb == 0) return;
  k_budget_x2<<<(nb + 127) / 128, 128, 0, s>>>(nb, moff, x2, switch_resid, ms);
  SGN_LAUNCH_CHECK();
}

}  // namespace sgn
