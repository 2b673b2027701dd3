// CSR utilities of the sign solver: validation, the reproducible 1-norm and
// scaling of step a1, prefix scans, block-diagonal assembly of batches and
// deterministic per-matrix reductions.
#include <cfloat>

#include "common.cuh"
#include "kernels.h"

namespace sgn {

namespace {

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

template <typename F>
__device__ __forceinline__ void for_each_row_warp(int64_t n, F f) {
  int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = warp; r < n; r += nwarps) f(r);
}

// Rows taken by groups of 8 lanes, four rows per warp at a time: for short
// rows (an input A has a few to a few tens of entries per row). f(r, has, gl)
// is called by every lane of the warp, has = false for a group without a row.
template <typename F>
__device__ __forceinline__ void for_each_row_group8(int64_t n, F f) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r0 = warp * 4; r0 < n; r0 += nwarps * 4) {
    const int64_t r = r0 + (lane >> 3);
    f(r < n ? r : r0, r < n, lane & 7);
  }
}

int grid_for(int64_t items, int per_block, int cap = 152 * 16) {
  int64_t g = (items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return int(g);
}

// ------------------------------------------------------------ validation
__global__ void k_validate(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *col,
                           const double *val, int *flag) {
  int lane = lane_id();
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (rp[0] != 0 || rp[n] != nnz) atomicOr(flag, 1);
  }
  for_each_row_warp(n, [&](int64_t r) {
    int64_t b = rp[r], e = rp[r + 1];
    if (e < b || b < 0 || e > nnz) {
      if (lane == 0) atomicOr(flag, 1);
      return;
    }
    bool bad = false;
    for (int64_t p = b + lane; p < e; p += 32) {
      int32_t c = col[p];
      if (c < 0 || c >= n) bad = true;
      if (p > b && col[p - 1] >= c) bad = true;
      if (!isfinite(val[p])) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(flag, 1);
  });
}

// The same checks for a batch of matrices in one launch: 8 lanes per row of
// all of them (row_off: exclusive prefix of the row counts), the matrix
// found by binary search; thread m also checks matrix m's first and last
// row pointer.
__global__ void k_validate_batch(int count, const ValidateJob *jobs, const int64_t *row_off,
                                 int *flags) {
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (tid < count) {
    const ValidateJob &j = jobs[tid];
    if (j.rp[0] != 0 || j.rp[j.n] != j.nnz) atomicOr(flags + tid, 1);
  }
  for_each_row_group8(row_off[count], [&](int64_t g, bool has, int gl) {
    if (!has) return;
    int lo = 0, hi = count - 1;  // the last matrix whose first row is <= g
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (row_off[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const ValidateJob &j = jobs[lo];
    const int64_t r = g - row_off[lo];
    const int64_t b = j.rp[r], e = j.rp[r + 1];
    if (e < b || b < 0 || e > j.nnz) {
      if (gl == 0) atomicOr(flags + lo, 1);
      return;
    }
    bool bad = false;
    for (int64_t p = b + gl; p < e; p += 8) {
      const int32_t c = j.col[p];
      if (c < 0 || c >= j.n) bad = true;
      if (p > b && j.col[p - 1] >= c) bad = true;
      if (!isfinite(j.val[p])) bad = true;
    }
    if (bad) atomicOr(flags + lo, 1);
  });
}

// ------------------------------------------------------------ gathered copies
// One CTA per chunk (grid-stride): 16-byte words when both ends and the
// length allow it, else 4-byte words (every chunk's length is a multiple of 4).
__global__ void k_copy_chunks(int count, const CopyChunk *chunks) {
  for (int c = blockIdx.x; c < count; c += gridDim.x) {
    const CopyChunk ch = chunks[c];
    const uintptr_t a = reinterpret_cast<uintptr_t>(ch.src), b = reinterpret_cast<uintptr_t>(ch.dst);
    if (((a | b | uintptr_t(ch.bytes)) & 15u) == 0) {
      // four 16-byte words per thread in flight (the far side may be host memory)
      const int4 *s4 = static_cast<const int4 *>(ch.src);
      int4 *d4 = static_cast<int4 *>(ch.dst);
      const int64_t n4 = ch.bytes >> 4;
      const int64_t T = blockDim.x;
      int64_t i = threadIdx.x;
      for (; i + 3 * T < n4; i += 4 * T) {
        const int4 v0 = s4[i], v1 = s4[i + T], v2 = s4[i + 2 * T], v3 = s4[i + 3 * T];
        d4[i] = v0;
        d4[i + T] = v1;
        d4[i + 2 * T] = v2;
        d4[i + 3 * T] = v3;
      }
      for (; i < n4; i += T) d4[i] = s4[i];
    } else {
      const uint32_t *s1 = static_cast<const uint32_t *>(ch.src);
      uint32_t *d1 = static_cast<uint32_t *>(ch.dst);
      const int64_t n1 = ch.bytes >> 2;
      for (int64_t i = threadIdx.x; i < n1; i += blockDim.x) d1[i] = s1[i];
    }
  }
}

// ------------------------------------------------------------ footprint statistics
// Per row: diagonal magnitude, off-diagonal sum and farthest column, folded
// into the matrix-wide Gershgorin gap, row-sum bound and half-bandwidth.
__global__ void k_gersh(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                        GershStats *g) {
  int lane = lane_id();
  for_each_row_warp(n, [&](int64_t r) {
    double diag = 0.0, off = 0.0;
    long long bw = 0;
    for (int64_t p = rp[r] + lane; p < rp[r + 1]; p += 32) {
      int64_t c = col[p];
      double a = fabs(val[p]);
      if (c == r) diag += a; else off += a;
      long long d = c > r ? c - r : r - c;
      bw = d > bw ? d : bw;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      diag += __shfl_xor_sync(0xffffffffu, diag, o);
      off += __shfl_xor_sync(0xffffffffu, off, o);
      long long b2 = __shfl_xor_sync(0xffffffffu, bw, o);
      bw = b2 > bw ? b2 : bw;
    }
    if (lane == 0) {
      double gap = diag - off, rowsum = diag + off;
      if (gap > 0.0)
        atomicMin(&g->min_gap_bits, (unsigned long long)__double_as_longlong(gap));
      else
        atomicOr(&g->nogap, 1);
      atomicMax(&g->max_rowsum_bits, (unsigned long long)__double_as_longlong(rowsum));
      atomicMax(&g->max_bw, bw);
    }
  });
}

// ------------------------------------------------------------ scan
constexpr int SCAN_T = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_T * SCAN_ITEMS;

// Exclusive scan of v over the block (1024 threads); *total gets the sum.
__device__ int64_t block_excl_scan(int64_t v, int64_t *sm, int64_t *total) {
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t t = sm[lane];
    int64_t u = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, u, o);
      if (lane >= o) u += y;
    }
    sm[lane] = u - t;
    if (lane == 31) sm[32] = u;
  }
  __syncthreads();
  int64_t r = sm[warp] + x - v;
  if (total) *total = sm[32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(int64_t n, const int64_t *cnt,
                                                        int64_t *tmp) {
  __shared__ int64_t sm[33];
  int64_t base = int64_t(blockIdx.x) * SCAN_TILE + int64_t(threadIdx.x) * SCAN_ITEMS;
  int64_t v = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i)
    if (base + i < n) v += cnt[base + i];
  int64_t total;
  block_excl_scan(v, sm, &total);
  if (threadIdx.x == 0) tmp[blockIdx.x] = total;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_blocks(int64_t nblocks, int64_t *tmp) {
  __shared__ int64_t sm[33];
  int64_t carry = 0;
  for (int64_t b0 = 0; b0 < nblocks; b0 += SCAN_T) {
    int64_t i = b0 + threadIdx.x;
    int64_t v = i < nblocks ? tmp[i] : 0;
    int64_t total;
    int64_t ex = block_excl_scan(v, sm, &total);
    if (i < nblocks) tmp[i] = carry + ex;
    carry += total;
  }
}

__global__ void __launch_bounds__(SCAN_T) k_scan_final(int64_t n, const int64_t *cnt,
                                                       const int64_t *tmp, int64_t *out) {
  __shared__ int64_t sm[33];
  int64_t base = int64_t(blockIdx.x) * SCAN_TILE + int64_t(threadIdx.x) * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    v[i] = base + i < n ? cnt[base + i] : 0;
    s += v[i];
  }
  int64_t ex = block_excl_scan(s, sm, nullptr) + tmp[blockIdx.x];
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    ex += v[i];
    if (base + i < n) out[base + i + 1] = ex;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
}

// ------------------------------------------------------------ assembly
__device__ __forceinline__ int find_block(const int64_t *off, int nb, int64_t r) {
  int lo = 0, hi = nb;  // off[lo] <= r < off[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (off[mid] <= r)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

__global__ void k_asm_lens(int nblocks, const AsmBlock *blocks, const int64_t *boff, int64_t n,
                           int64_t *lens) {
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
       r += int64_t(gridDim.x) * blockDim.x) {
    int b = find_block(boff, nblocks, r);
    const AsmBlock &B = blocks[b];
    int64_t sr = B.row0 + (r - boff[b]);
    lens[r] = B.rp[sr + 1] - B.rp[sr];
  }
}

__global__ void k_asm_vals(int nblocks, const AsmBlock *blocks, const int64_t *boff, int64_t n,
                           const int64_t *drp, int32_t *dcol, void *dval, int dst_f32) {
  // 8 lanes per row, four rows per warp at a time (rows are short)
  constexpr int L = 8;
  const int lane = lane_id(), gl = lane % L;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = warp * (32 / L) + lane / L; r < n; r += nwarps * (32 / L)) {
    int b = find_block(boff, nblocks, r);
    const AsmBlock B = blocks[b];
    int64_t sr = B.row0 + (r - boff[b]);
    int64_t sb = B.rp[sr], se = B.rp[sr + 1], d = drp[r] - sb;
    if (B.val_f32 && dst_f32) {  // FP32 to FP32: the values as they are
      const float *sv = static_cast<const float *>(B.val);
      float *dv = static_cast<float *>(dval);
      for (int64_t p = sb + gl; p < se; p += L) {
        dcol[d + p] = int32_t(B.col[p] + B.col_shift);
        dv[d + p] = sv[p];
      }
    } else {
      for (int64_t p = sb + gl; p < se; p += L) {
        dcol[d + p] = int32_t(B.col[p] + B.col_shift);
        double v = B.val_f32 ? double(static_cast<const float *>(B.val)[p])
                             : static_cast<const double *>(B.val)[p];
        if (dst_f32)
          static_cast<float *>(dval)[d + p] = __double2float_rn(v);
        else
          static_cast<double *>(dval)[d + p] = v;
      }
    }
  }
}

__global__ void k_fill_seg(int nb, const int64_t *moff, int64_t n, int32_t *seg) {
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
       r += int64_t(gridDim.x) * blockDim.x)
    seg[r] = find_block(moff, nb, r);
}

// ------------------------------------------------------------ 1-norm (step a1)
// ||A||_1 = max_j sum_i |a_ij|, made independent of summation order: with
// M = max |a_ij| < 2^e every |a_ij| is put on the grid 2^(e-62) by one
// round-to-nearest-even conversion of the exact product |a| * 2^(62-e); the
// column sums are exact 128-bit integers (two 64-bit atomics with carry), and
// the largest one, hi * 2^64 + lo, comes back as
// ((double)hi * 2^64 + (double)lo) * 2^(e-62).

__device__ __forceinline__ void add128(unsigned long long *lohi, unsigned long long q) {
  unsigned long long old = atomicAdd(&lohi[0], q);
  if (old + q < old) atomicAdd(&lohi[1], 1ULL);
}

__global__ void k_absmax(int64_t n, const int32_t *seg, const int64_t *rp, const double *val,
                         unsigned long long *mmax) {
  for_each_row_group8(n, [&](int64_t r, bool has, int gl) {
    double m = 0.0;
    if (has)
      for (int64_t p = rp[r] + gl; p < rp[r + 1]; p += 8) m = fmax(m, fabs(val[p]));
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o, 8));
    if (has && gl == 0 && m > 0.0)
      atomicMax(&mmax[seg[r]], (unsigned long long)__double_as_longlong(m));
  });
}

__global__ void k_colsum(int64_t n, const int32_t *seg, const int64_t *rp, const int32_t *col,
                         const double *val, const unsigned long long *mmax,
                         unsigned long long *colsum) {
  for_each_row_group8(n, [&](int64_t r, bool has, int gl) {
    if (!has) return;
    double M = __longlong_as_double((long long)mmax[seg[r]]);
    if (M == 0.0) return;
    int e;
    frexp(M, &e);
    for (int64_t p = rp[r] + gl; p < rp[r + 1]; p += 8) {
      unsigned long long q = __double2ull_rn(ldexp(fabs(val[p]), 62 - e));
      if (q) add128(&colsum[2 * int64_t(col[p])], q);
    }
  });
}

__global__ void k_colmax_hi(int64_t n, const int32_t *seg, const unsigned long long *colsum,
                            unsigned long long *maxhi) {
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n;
       j += int64_t(gridDim.x) * blockDim.x)
    if (colsum[2 * j] | colsum[2 * j + 1]) atomicMax(&maxhi[seg[j]], colsum[2 * j + 1]);
}

__global__ void k_colmax_lo(int64_t n, const int32_t *seg, const unsigned long long *colsum,
                            const unsigned long long *maxhi, unsigned long long *maxlo) {
  for (int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; j < n;
       j += int64_t(gridDim.x) * blockDim.x)
    if (colsum[2 * j + 1] == maxhi[seg[j]]) atomicMax(&maxlo[seg[j]], colsum[2 * j]);
}

__global__ void k_norm_final(int nb, const unsigned long long *mmax,
                             const unsigned long long *maxhi, const unsigned long long *maxlo,
                             double *norm) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nb) return;
  double M = __longlong_as_double((long long)mmax[m]);
  if (M == 0.0) {
    norm[m] = 0.0;
    return;
  }
  int e;
  frexp(M, &e);
  double d = __dadd_rn(__dmul_rn(__ull2double_rn(maxhi[m]), 18446744073709551616.0),
                       __ull2double_rn(maxlo[m]));
  norm[m] = ldexp(d, e - 62);
}

__global__ void k_scale(int64_t n, const int32_t *seg, const int64_t *rp, double *val,
                        const double *norm) {
  for_each_row_group8(n, [&](int64_t r, bool has, int gl) {
    if (!has) return;
    double s = norm[seg[r]];
    for (int64_t p = rp[r] + gl; p < rp[r + 1]; p += 8) val[p] = __ddiv_rn(val[p], s);
  });
}

__global__ void k_gather_offsets(int nb, const int64_t *moff, const int64_t *rp, int64_t *out) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m <= nb) out[m] = rp[moff[m]];
}

// ------------------------------------------------------------ reductions
constexpr int RED_T = 256;
__global__ void __launch_bounds__(RED_T) k_seg_reduce(const int64_t *moff, const double *part,
                                                      int ncomp, double *out) {
  __shared__ double sm[RED_T];
  int m = blockIdx.x;
  int64_t b = moff[m], e = moff[m + 1];
  for (int c = 0; c < ncomp; ++c) {
    double acc = 0.0;
    for (int64_t r = b + threadIdx.x; r < e; r += RED_T) acc += part[r * ncomp + c];
    sm[threadIdx.x] = acc;
    __syncthreads();
    for (int s = RED_T / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[int64_t(m) * ncomp + c] = sm[0];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(RED_T) k_seg_count(const int64_t *moff, const int64_t *rs,
                                                     const int64_t *re, int64_t *out) {
  __shared__ int64_t sm[RED_T];
  int m = blockIdx.x;
  int64_t acc = 0;
  for (int64_t r = moff[m] + threadIdx.x; r < moff[m + 1]; r += RED_T) acc += re[r] - rs[r];
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = RED_T / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[m] = sm[0];
}

// One CTA per extracted matrix: rebased row pointers, shifted columns,
// values widened to FP64.
// blockIdx.y walks the blocks; the gridDim.x CTAs of a block share its rows
// and entries, so that a large matrix is copied by many SMs.
__global__ void k_extract(int nblocks, const ExtractBlock *blocks) {
  for (int b = blockIdx.y; b < nblocks; b += gridDim.y) {
    const ExtractBlock B = blocks[b];
    const int64_t t0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t step = int64_t(gridDim.x) * blockDim.x;
    const int64_t e0 = B.rp[B.row0];
    for (int64_t i = t0; i <= B.nrows; i += step) B.drp[i] = B.rp[B.row0 + i] - e0;
    const int64_t ne = B.rp[B.row0 + B.nrows] - e0;
    for (int64_t p = t0; p < ne; p += step) {
      B.dcol[p] = int32_t(B.col[e0 + p] + B.col_shift);
      B.dval[p] = B.val_f32 ? double(static_cast<const float *>(B.val)[e0 + p])
                            : static_cast<const double *>(B.val)[e0 + p];
    }
  }
}

__global__ void k_row_lengths(int64_t n, const int64_t *rs, const int64_t *re, int64_t *out) {
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
       r += int64_t(gridDim.x) * blockDim.x)
    out[r] = re[r] - rs[r];
}

__global__ void k_compact_rows(int64_t n, const int64_t *rs, const int64_t *re,
                               const int32_t *col, const void *val, int vsize, const int64_t *orp,
                               int32_t *ocol, void *oval) {
  int lane = lane_id();
  for_each_row_warp(n, [&](int64_t r) {
    int64_t b = rs[r], e = re[r], d = orp[r];
    for (int64_t p = b + lane; p < e; p += 32) {
      ocol[d + (p - b)] = col[p];
      if (vsize == 8)
        static_cast<double *>(oval)[d + (p - b)] = static_cast<const double *>(val)[p];
      else
        static_cast<float *>(oval)[d + (p - b)] = static_cast<const float *>(val)[p];
    }
  });
}

}  // namespace

void launch_row_lengths(int64_t n, const int64_t *rs, const int64_t *re, int64_t *out,
                        cudaStream_t s) {
  if (n == 0) return;
  k_row_lengths<<<grid_for(n, 256), 256, 0, s>>>(n, rs, re, out);
  SGN_LAUNCH_CHECK();
}

void launch_compact_rows(int64_t n, const int64_t *rs, const int64_t *re, const int32_t *col,
                         const void *val, int vsize, const int64_t *orp, int32_t *ocol,
                         void *oval, cudaStream_t s) {
  if (n == 0) return;
  k_compact_rows<<<grid_for(n, 8), 256, 0, s>>>(n, rs, re, col, val, vsize, orp, ocol, oval);
  SGN_LAUNCH_CHECK();
}

void launch_seg_count(int nb, const int64_t *moff, const int64_t *rs, const int64_t *re,
                      int64_t *out, cudaStream_t s) {
  if (nb == 0) return;
  k_seg_count<<<nb, RED_T, 0, s>>>(moff, rs, re, out);
  SGN_LAUNCH_CHECK();
}

void launch_extract(int nblocks, const ExtractBlock *blocks, int64_t max_entries, cudaStream_t s) {
  if (nblocks == 0) return;
  // about 8 entries per thread of a 512-thread CTA, at most 152 CTAs per block
  const int64_t per = (max_entries + 4095) / 4096;
  dim3 grid(unsigned(per < 1 ? 1 : (per > 152 ? 152 : per)), unsigned(nblocks < 65535 ? nblocks : 65535));
  k_extract<<<grid, 512, 0, s>>>(nblocks, blocks);
  SGN_LAUNCH_CHECK();
}

void launch_gersh(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                  GershStats *g, cudaStream_t s) {
  k_gersh<<<grid_for(n, 8), 256, 0, s>>>(n, rp, col, val, g);
  SGN_LAUNCH_CHECK();
}

void launch_validate(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *col,
                     const double *val, int *flag, cudaStream_t s) {
  k_validate<<<grid_for(n, 8), 256, 0, s>>>(n, nnz, rp, col, val, flag);
  SGN_LAUNCH_CHECK();
}

void launch_validate_batch(int count, const ValidateJob *jobs, const int64_t *row_off,
                           int64_t total_rows, int *flags, cudaStream_t s) {
  if (count < 1) return;
  const int64_t items = total_rows > count ? total_rows : count;
  k_validate_batch<<<grid_for(items, 32), 256, 0, s>>>(count, jobs, row_off, flags);
  SGN_LAUNCH_CHECK();
}

void launch_copy_chunks(int count, const CopyChunk *chunks, cudaStream_t s) {
  if (count < 1) return;
  k_copy_chunks<<<count < 152 * 8 ? count : 152 * 8, 256, 0, s>>>(count, chunks);
  SGN_LAUNCH_CHECK();
}

int64_t scan_tmp_elems(int64_t n) { return (n + SCAN_TILE - 1) / SCAN_TILE + 1; }

void launch_scan(int64_t n, const int64_t *cnt, int64_t *out, int64_t *tmp, cudaStream_t s) {
  int64_t nblocks = (n + SCAN_TILE - 1) / SCAN_TILE;
  if (nblocks == 0) {
    SGN_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
    return;
  }
  k_scan_reduce<<<unsigned(nblocks), SCAN_T, 0, s>>>(n, cnt, tmp);
  SGN_LAUNCH_CHECK();
  k_scan_blocks<<<1, SCAN_T, 0, s>>>(nblocks, tmp);
  SGN_LAUNCH_CHECK();
  k_scan_final<<<unsigned(nblocks), SCAN_T, 0, s>>>(n, cnt, tmp, out);
  SGN_LAUNCH_CHECK();
}

void launch_assemble_rows(int nblocks, const AsmBlock *blocks, const int64_t *boff, int64_t n_dst,
                          int64_t *lens, int64_t *dst_rp, int64_t *scan_tmp, cudaStream_t s) {
  if (n_dst > 0) {
    k_asm_lens<<<grid_for(n_dst, 256), 256, 0, s>>>(nblocks, blocks, boff, n_dst, lens);
    SGN_LAUNCH_CHECK();
  }
  launch_scan(n_dst, lens, dst_rp, scan_tmp, s);
}

void launch_assemble_vals(int nblocks, const AsmBlock *blocks, const int64_t *boff, int64_t n_dst,
                          const int64_t *dst_rp, int32_t *dst_col, void *dst_val, int dst_f32,
                          cudaStream_t s) {
  if (n_dst == 0) return;
  k_asm_vals<<<grid_for(n_dst, 32), 256, 0, s>>>(nblocks, blocks, boff, n_dst, dst_rp, dst_col,
                                                  dst_val, dst_f32);
  SGN_LAUNCH_CHECK();
}

void launch_fill_seg(int nb, const int64_t *moff, int64_t n, int32_t *seg, cudaStream_t s) {
  if (n == 0) return;
  k_fill_seg<<<grid_for(n, 256), 256, 0, s>>>(nb, moff, n, seg);
  SGN_LAUNCH_CHECK();
}

void launch_onenorm(int nb, const int64_t *moff, const int32_t *seg, int64_t n, const int64_t *rp,
                    const int32_t *col, const double *val, unsigned long long *work, double *norm,
                    cudaStream_t s) {
  (void)moff;
  unsigned long long *colsum = work;            // 2n
  unsigned long long *mmax = work + 2 * n;      // nb
  unsigned long long *maxhi = mmax + nb;        // nb
  unsigned long long *maxlo = maxhi + nb;       // nb
  SGN_CUDA(cudaMemsetAsync(work, 0, sizeof(unsigned long long) * size_t(2 * n + 3 * nb), s));
  k_absmax<<<grid_for(n, 32), 256, 0, s>>>(n, seg, rp, val, mmax);
  SGN_LAUNCH_CHECK();
  k_colsum<<<grid_for(n, 32), 256, 0, s>>>(n, seg, rp, col, val, mmax, colsum);
  SGN_LAUNCH_CHECK();
  k_colmax_hi<<<grid_for(n, 256), 256, 0, s>>>(n, seg, colsum, maxhi);
  SGN_LAUNCH_CHECK();
  k_colmax_lo<<<grid_for(n, 256), 256, 0, s>>>(n, seg, colsum, maxhi, maxlo);
  SGN_LAUNCH_CHECK();
  k_norm_final<<<(nb + 127) / 128, 128, 0, s>>>(nb, mmax, maxhi, maxlo, norm);
  SGN_LAUNCH_CHECK();
}

void launch_scale(int64_t n, const int32_t *seg, const int64_t *rp, double *val,
                  const double *norm, cudaStream_t s) {
  k_scale<<<grid_for(n, 32), 256, 0, s>>>(n, seg, rp, val, norm);
  SGN_LAUNCH_CHECK();
}

void launch_gather_offsets(int nb, const int64_t *moff, const int64_t *rp, int64_t *out,
                           cudaStream_t s) {
  k_gather_offsets<<<(nb + 1 + 127) / 128, 128, 0, s>>>(nb, moff, rp, out);
  SGN_LAUNCH_CHECK();
}

void launch_seg_reduce(int nb, const int64_t *moff, const double *part, int ncomp, double *out,
                       cudaStream_t s) {
  if (nb == 0) return;
  k_seg_reduce<<<nb, RED_T, 0, s>>>(moff, part, ncomp, out);
  SGN_LAUNCH_CHECK();
}

}  // namespace sgn
