// Row-wise sparse products of the Newton-Schulz step (steps a2 and a3):
//   MODE_SQUARE:  T = X X, plus per-row partial sums for ||T - I||_F and ||X||_F
//   MODE_UPDATE:  Xbar = 1.5 X - 0.5 X T   (= 1/2 X (3I - X^2), Alg. 3.2.1 step 3)
//
// Operands are row ranges [rs[i], re[i]) into (col, val) with ascending
// columns, so both compact CSR (rs = rowptr, re = rowptr + 1) and the slotted
// outputs of earlier products can be read.
//
// Row i of C = A B is accumulated in shared memory over its column range
// [lo_i, lo_i + len_i) (union of the ranges of the rows B_k, k in A_i), indexed
// by column - lo_i, so the output comes out in ascending column order without
// hashing or sorting. Rows with len <= WARP_W go to one warp each; wider rows
// to one CTA each, in chunks of CTA_W columns.
//
// No symbolic pass: each output row gets a slot of ub_i = min(len_i, work_i)
// entries (work_i = multiply-adds of the row, plus the row of A itself in
// MODE_UPDATE), which bounds its number of distinct columns; the numeric
// kernel writes the row at the start of its slot and records where it ends.
//
// Accumulation order: the k of A_i are visited in ascending order, one at a
// time; within one k the lanes (threads) stride over the entries of B_k,
// whose columns are distinct, so no two lanes touch the same slot, and a
// barrier separates consecutive k. Every slot therefore receives its
// products in ascending k with one fused multiply-add each, starting from
// +0: the result is the same bit for bit on every run and launch shape.
#include <climits>

#include "common.cuh"
#include "kernels.h"

namespace sgn {

namespace {

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// 1.5 x - 0.5 p with each product and the difference rounded once.
__device__ __forceinline__ double ns_combine(double x, double p) {
  return __dsub_rn(__dmul_rn(1.5, x), __dmul_rn(0.5, p));
}
__device__ __forceinline__ float ns_combine(float x, float p) {
  return __fsub_rn(__fmul_rn(1.5f, x), __fmul_rn(0.5f, p));
}

// Sum of squares of the values of one type, in FP64 precision. For float
// values it avoids FP64 arithmetic (1/64 rate on this part): v^2 = p + e
// exactly (p = v*v rounded, e = fma(v, v, -p)), accumulated as an unevaluated
// float pair with an error-free two-sum, so the sum carries ~48 bits.
template <typename T>
struct SqAcc;
template <>
struct SqAcc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add_sq(double v) { s = __fma_rn(v, v, s); }
  __device__ __forceinline__ double value() const { return s; }
};
template <>
struct SqAcc<float> {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float a) {
    float t = __fadd_rn(hi, a);
    float bb = __fsub_rn(t, hi);
    float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bb)), __fsub_rn(a, bb));
    hi = t;
    lo = __fadd_rn(lo, err);
  }
  __device__ __forceinline__ void add_sq(float v) {
    float p = __fmul_rn(v, v);
    float e = __fmaf_rn(v, v, -p);
    add(p);
    lo = __fadd_rn(lo, e);
  }
  __device__ __forceinline__ double value() const { return double(hi) + double(lo); }
};

__device__ __forceinline__ int64_t lower_bound(const int32_t *a, int64_t lo, int64_t hi,
                                               int64_t v) {
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (a[mid] < v)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

constexpr int BOUNDS_TILE = 256;  // rows per CTA of k_bounds; lists keep this order
static_assert(BOUNDS_TILE % 16 == 0, "band tiles are aligned groups of 16 rows");
// A 16-row group goes to a band tile when its multiply-adds are at least a
// fraction band_min_eff (a schedule option, 0.08 by default) of the tile's
// estimated FMA slots: the band kernel spends about 2.5 instructions per slot,
// the row-wise product tens per multiply-add.

// Row grouping of k_bounds: GROUPS_NONE keeps every row on 32 lanes.
// GROUPS_THROUGHPUT (FP64 products, bound by the FP64 pipe) picks the group
// size that leaves the fewest lanes idle in a k-step. GROUPS_PAIRS (FP32
// products, bound by instruction issue and gather latency) sends every row
// that fits half a warp's accumulator to the pair kernel, where neighbouring
// rows share their passes over B (pair_rows).
enum { GROUPS_NONE = 0, GROUPS_THROUGHPUT = 1, GROUPS_PAIRS = 2 };

// Lane utilization of one k-step with g lanes and a B row of avg entries.
__device__ __forceinline__ float lane_use(float avg, int g) {
  float rounds = ceilf(avg / float(g));
  return avg / (rounds * float(g));
}

// Per row k of B: (first column, last column, entries, 0), so that k_bounds
// reads one 16-byte record per k instead of a chain of dependent loads.
__global__ void k_row_info(int64_t n, const int64_t *rs, const int64_t *re, const int32_t *col,
                           int4 *info) {
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
       r += int64_t(gridDim.x) * blockDim.x) {
    const int64_t a = rs[r], b = re[r];
    info[r] = b > a ? make_int4(col[a], col[b - 1], int(b - a), 0) : make_int4(0, -1, 0, 0);
  }
}

// Rows of A with more entries than this are walked by a whole warp in k_bounds.
constexpr int64_t BOUNDS_LONG = 256;

// The bounds and class of one row of sparse work, from its k hull [kf, kl],
// its column hull [mn, mx] (mx < 0: no output) and its multiply-adds wk;
// writes lo, len, ub, work of row r and, for band tiles, the row's statistics.
__device__ __forceinline__ int bounds_row(int64_t r, int m, int64_t na, int32_t mn, int32_t mx,
                                          int32_t kf, int32_t kl, int64_t wk, int mode,
                                          int groups, float group_margin, int band, int32_t *lo,
                                          int32_t *len, int64_t *ub, double *work, int *sseg,
                                          int *slo, int *sL, int *skf, int *skl, int *sna,
                                          float *swk) {
  int cls = RC_NONE;
  if (mx < 0) {
    ub[r] = 0;
    len[r] = 0;
    lo[r] = 0;
    work[r] = double(wk);
  } else {
    const int32_t L = mx - mn + 1;
    const int64_t bound = wk + (mode == MODE_UPDATE ? na : 0);
    if (L > WARP_W) {
      cls = RC_CTA;
    } else if (!groups) {
      cls = RC_G32;
    } else if (groups == GROUPS_PAIRS) {
      cls = L <= WARP_W / 2 ? RC_G16 : RC_G32;
    } else {
      const float avg = float(wk) / float(na > 0 ? na : 1);
      const float u32 = lane_use(avg, 32), u16 = lane_use(avg, 16), u8 = lane_use(avg, 8);
      cls = RC_G32;
      if (L <= WARP_W / 2 && u16 > u32 + group_margin) cls = RC_G16;
      if (L <= WARP_W / 4 && u8 > (cls == RC_G16 ? u16 : u32) + group_margin) cls = RC_G8;
    }
    lo[r] = mn;
    len[r] = L;
    ub[r] = bound < L ? bound : L;
    work[r] = double(wk);
  }
  if (band) {
    *sseg = m;
    *slo = mx < 0 ? 0 : mn;
    *sL = mx < 0 ? 0 : mx - mn + 1;
    *skf = kf;
    *skl = kl;
    *sna = int(na);
    *swk = float(wk);
  }
  return cls;
}

// counters: [RC_*] list lengths, [RC_QUEUE + RC_*] work-queue heads of the numeric kernels.
__global__ void __launch_bounds__(BOUNDS_TILE)
    k_bounds(int64_t n, const int64_t *ars, const int64_t *are, const int32_t *acol,
             const int4 *binfo, const int32_t *seg,
             const int *active, int mode, int groups, float group_margin, int band,
             float band_min_eff, const int *dslot,
             const int64_t *moff, int32_t *lo, int32_t *len, int64_t *ub, int32_t *lists,
             int *counters, double *work, double *band_work, unsigned char *bandrow) {
  __shared__ unsigned char s_cls[BOUNDS_TILE];
  __shared__ int s_cnt[BOUNDS_TILE / 32][RC_N];
  __shared__ int s_base[RC_N];
  // per-row statistics of the band decision (rows of sparse work only)
  __shared__ int s_seg[BOUNDS_TILE], s_lo[BOUNDS_TILE], s_L[BOUNDS_TILE];
  __shared__ int s_kf[BOUNDS_TILE], s_kl[BOUNDS_TILE], s_na[BOUNDS_TILE];
  __shared__ float s_wk[BOUNDS_TILE];
  __shared__ unsigned char s_band[BOUNDS_TILE / 16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = BOUNDS_TILE / 32;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t ntiles = (n + BOUNDS_TILE - 1) / BOUNDS_TILE;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t t0 = tile * BOUNDS_TILE;
    // One thread per row: its own pass over A_i (four B records in flight),
    // with no reductions across lanes. Rows of more than BOUNDS_LONG entries
    // are left to the whole warp afterwards.
    const int i = threadIdx.x;
    const int64_t r = t0 + i;
    int cls = RC_NONE;
    bool longrow = false;
    s_seg[i] = -1;  // not eligible for a band tile
    int m = 0;
    int64_t a0 = 0, a1 = 0;
    if (r < n) {
      m = seg[r];
      if (!active[m] || (dslot && dslot[m] >= 0)) {
        // inactive, or on the dense path: no sparse work; a dense row of an
        // update gets a whole row of slots for 1.5 X - 0.5 X T
        const bool dense = active[m] && dslot && dslot[m] >= 0;
        ub[r] = dense && mode == MODE_UPDATE ? moff[m + 1] - moff[m] : 0;
        len[r] = 0;
        lo[r] = 0;
        work[r] = 0.0;
      } else {
        a0 = ars[r];
        a1 = are[r];
        if (a1 - a0 > BOUNDS_LONG) {
          longrow = true;
        } else {
          int32_t mn = INT_MAX, mx = -1;
          int64_t wk = 0;
          int64_t p = a0;
          for (; p + 4 <= a1; p += 4) {
            const int32_t k0 = acol[p], k1 = acol[p + 1], k2 = acol[p + 2], k3 = acol[p + 3];
            const int4 b0 = binfo[k0], b1 = binfo[k1], b2 = binfo[k2], b3 = binfo[k3];
            wk += int64_t(b0.z) + b1.z + b2.z + b3.z;
            // an empty B row has first column 0 and last -1: no effect on either
            mn = min(mn, min(min(b0.z ? b0.x : INT_MAX, b1.z ? b1.x : INT_MAX),
                             min(b2.z ? b2.x : INT_MAX, b3.z ? b3.x : INT_MAX)));
            mx = max(mx, max(max(b0.y, b1.y), max(b2.y, b3.y)));
          }
          for (; p < a1; ++p) {
            const int4 bi = binfo[acol[p]];
            wk += bi.z;
            if (bi.z > 0) mn = min(mn, bi.x);
            mx = max(mx, bi.y);
          }
          const int32_t kf = a1 > a0 ? acol[a0] : INT_MAX, kl = a1 > a0 ? acol[a1 - 1] : -1;
          if (mode == MODE_UPDATE && a1 > a0) {  // the columns of X_i itself (ascending)
            mn = min(mn, kf);
            mx = max(mx, kl);
          }
          cls = bounds_row(r, m, a1 - a0, mn, mx, kf, kl, wk, mode, groups, group_margin, band,
                           lo, len, ub, work, s_seg + i, s_lo + i, s_L + i, s_kf + i, s_kl + i,
                           s_na + i, s_wk + i);
        }
      }
    }
    s_cls[i] = (unsigned char)cls;
    // long rows: the warp walks each with its lanes striding over A_i
    unsigned lm = __ballot_sync(0xffffffffu, longrow);
    while (lm) {
      const int src = __ffs(lm) - 1;
      lm &= lm - 1;
      const int li = warp * 32 + src;
      const int64_t lr = t0 + li;
      const int lmat = __shfl_sync(0xffffffffu, m, src);
      const int64_t la0 = __shfl_sync(0xffffffffu, a0, src), la1 = __shfl_sync(0xffffffffu, a1, src);
      int32_t mn = INT_MAX, mx = -1;
      int64_t wk = 0;
      for (int64_t p = la0 + lane; p < la1; p += 32) {
        const int4 bi = binfo[acol[p]];
        wk += bi.z;
        if (bi.z > 0) mn = min(mn, bi.x);
        mx = max(mx, bi.y);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        wk += __shfl_xor_sync(0xffffffffu, wk, o);
      }
      if (lane == src) {
        const int32_t kf = acol[la0], kl = acol[la1 - 1];
        if (mode == MODE_UPDATE) {
          mn = min(mn, kf);
          mx = max(mx, kl);
        }
        s_cls[li] = (unsigned char)bounds_row(lr, lmat, la1 - la0, mn, mx, kf, kl, wk, mode,
                                              groups, group_margin, band, lo, len, ub, work,
                                              s_seg + li, s_lo + li, s_L + li, s_kf + li,
                                              s_kl + li, s_na + li, s_wk + li);
      }
    }
    __syncthreads();
    // band tiles: aligned groups of 16 rows of one matrix, all with sparse
    // work, whose estimated FMA slots the multiply-adds fill well enough
    if (band && threadIdx.x < BOUNDS_TILE / 16) {
      const int b0 = threadIdx.x * 16;
      bool ok = s_seg[b0] >= 0;
      int jlo = INT_MAX, jhi = -1, klo = INT_MAX, khi = -1;
      float wsum = 0.0f, nsum = 0.0f;
      double wexact = 0.0;
      for (int i = b0; i < b0 + 16 && ok; ++i) {
        ok = s_seg[i] == s_seg[b0];
        if (s_L[i] > 0) {
          jlo = min(jlo, s_lo[i]);
          jhi = max(jhi, s_lo[i] + s_L[i] - 1);
        }
        klo = min(klo, s_kf[i]);
        khi = max(khi, s_kl[i]);
        wsum += s_wk[i];
        wexact += double(s_wk[i]);
        nsum += float(s_na[i]);
      }
      if (ok && jhi >= 0 && khi >= 0) {
        const int nwords = (jhi >> 5) - (jlo >> 5) + 1;
        const float bavg = wsum / fmaxf(nsum, 1.0f);  // mean entries of a B row
        const float kc = fminf(float(khi - klo + 1), bavg + 35.0f);
        const float slots = 16.0f * 32.0f * float(nwords) * kc;
        ok = nwords <= BAND_JW && khi - klo < BAND_KT - 3 && wsum >= band_min_eff * slots;
      } else {
        ok = false;
      }
      s_band[threadIdx.x] = ok ? 1 : 0;
      if (ok && band_work) atomicAdd(band_work, wexact);  // multiply-adds of the band tiles
    }
    __syncthreads();
    // ordered compaction of the tile's rows into one list per class
    int my = s_cls[threadIdx.x];
    const bool inband = band && s_band[threadIdx.x >> 4];
    if (inband) my = (threadIdx.x & 15) == 0 ? RC_BAND : RC_NONE;
    if (bandrow && t0 + threadIdx.x < n) bandrow[t0 + threadIdx.x] = inband ? 1 : 0;
    unsigned bal[RC_N];
#pragma unroll
    for (int c = 0; c < RC_N; ++c) {
      bal[c] = __ballot_sync(0xffffffffu, my == c);
      if (lane == 0) s_cnt[warp][c] = __popc(bal[c]);
    }
    __syncthreads();
    if (threadIdx.x < RC_N) {
      int c = threadIdx.x, tot = 0;
      for (int w = 0; w < nw; ++w) tot += s_cnt[w][c];
      s_base[c] = tot ? atomicAdd(&counters[c], tot) : 0;
    }
    __syncthreads();
    if (my < RC_N) {
      int off = s_base[my];
      for (int w = 0; w < warp; ++w) off += s_cnt[w][my];
      off += __popc(bal[my] & lt);
      lists[int64_t(my) * n + off] = int32_t(t0 + threadIdx.x);
    }
    __syncthreads();
  }
}

// Touched slots. With MARK = false every product sets the slot's byte flag
// f[j] = 1. With MARK = true (FP32 accumulators) an untouched slot holds -0.0
// and no flag is written: each product is fma(a, b, acc) + 0, and adding +0
// turns a -0 result into +0 and leaves every other value as it is. A slot
// reads -0 only until its first product, and its values are those of an
// accumulation from +0 (which can never produce -0) bit for bit.
template <typename T, bool MARK>
__device__ __forceinline__ bool untouched(T v) {
  if constexpr (MARK)
    return __float_as_uint(v) == 0x80000000u;
  else
    return false;
}
template <typename T, bool MARK>
__device__ __forceinline__ void mac(T *acc, unsigned char *f, int j, T a, T v) {
  static_assert(!MARK || sizeof(T) == 4, "the -0 marker is used for FP32 accumulators");
  if constexpr (MARK) {
    acc[j] = __fadd_rn(fma_rn(a, v, acc[j]), 0.0f);
  } else {
    acc[j] = fma_rn(a, v, acc[j]);
    f[j] = 1;
  }
}

// One k of the accumulation: lanes stride over B_k = [q0, q1) and add
// a * b_kj into acc[col - c0], up to four independent products per lane in
// flight. The columns of B_k are distinct, so the slots of one call never
// collide.
template <typename T, int STRIDE, bool MARK = false>
__device__ __forceinline__ void accumulate_k(T a, int64_t q0, int64_t q1, const int32_t *bcol,
                                             const T *bval, int64_t c0, T *acc,
                                             unsigned char *f, int tid) {
  if constexpr (sizeof(T) == 8) {
    // FP64 (DFMA-bound): passes of STRIDE entries taken four, then two, then
    // one at a time, the same for every lane of the group, so that only the
    // row's last pass is partly active. A DFMA costs the FP64 pipe the same
    // whatever its active lanes, and lanes running different unrollings
    // would issue the instructions of each. 64-bit positions (~1% faster
    // here than offsets).
    const int np = int((q1 - q0 + STRIDE - 1) / STRIDE);  // group-uniform
    int64_t q = q0 + tid;
    int pass = 0;
    for (; pass + 4 <= np; pass += 4, q += 4 * STRIDE) {
      const bool ok3 = q + 3 * STRIDE < q1;  // only the last pass can be partial
      const int j0 = int(bcol[q] - c0), j1 = int(bcol[q + STRIDE] - c0);
      const int j2 = int(bcol[q + 2 * STRIDE] - c0);
      const int j3 = ok3 ? int(bcol[q + 3 * STRIDE] - c0) : 0;
      const T v0 = bval[q], v1 = bval[q + STRIDE], v2 = bval[q + 2 * STRIDE];
      const T v3 = ok3 ? bval[q + 3 * STRIDE] : T(0);
      mac<T, MARK>(acc, f, j0, a, v0);
      mac<T, MARK>(acc, f, j1, a, v1);
      mac<T, MARK>(acc, f, j2, a, v2);
      if (ok3) mac<T, MARK>(acc, f, j3, a, v3);
    }
    if (pass + 2 <= np) {
      const bool ok1 = q + STRIDE < q1;
      const int j0 = int(bcol[q] - c0), j1 = ok1 ? int(bcol[q + STRIDE] - c0) : 0;
      const T v0 = bval[q], v1 = ok1 ? bval[q + STRIDE] : T(0);
      mac<T, MARK>(acc, f, j0, a, v0);
      if (ok1) mac<T, MARK>(acc, f, j1, a, v1);
      pass += 2;
      q += 2 * STRIDE;
    }
    if (pass < np && q < q1) mac<T, MARK>(acc, f, int(bcol[q] - c0), a, bval[q]);
  } else {
    // FP32 (issue-bound): 32-bit offsets from the start of B_k, one 64-bit
    // address per k (~4% faster)
    const int n = int(q1 - q0);
    const int32_t *bc = bcol + q0;
    const T *bv = bval + q0;
    const int32_t cz = int32_t(c0);
    int i = tid;
    for (; i + 3 * STRIDE < n; i += 4 * STRIDE) {
      int j0 = bc[i] - cz, j1 = bc[i + STRIDE] - cz;
      int j2 = bc[i + 2 * STRIDE] - cz, j3 = bc[i + 3 * STRIDE] - cz;
      T v0 = bv[i], v1 = bv[i + STRIDE], v2 = bv[i + 2 * STRIDE], v3 = bv[i + 3 * STRIDE];
      mac<T, MARK>(acc, f, j0, a, v0);
      mac<T, MARK>(acc, f, j1, a, v1);
      mac<T, MARK>(acc, f, j2, a, v2);
      mac<T, MARK>(acc, f, j3, a, v3);
    }
    if (i + STRIDE < n) {
      int j0 = bc[i] - cz, j1 = bc[i + STRIDE] - cz;
      T v0 = bv[i], v1 = bv[i + STRIDE];
      mac<T, MARK>(acc, f, j0, a, v0);
      mac<T, MARK>(acc, f, j1, a, v1);
      i += 2 * STRIDE;
    }
    if (i < n) mac<T, MARK>(acc, f, bc[i] - cz, a, bv[i]);
  }
}

// accumulate_k for one k shared by two rows (a_ik and a_i'k): every entry of
// B_k is loaded once and added into both rows' accumulators.
template <typename T, bool MARK>
__device__ __forceinline__ void accumulate_k2(T a, T b, int64_t q0, int64_t q1,
                                              const int32_t *bcol, const T *bval, int32_t ca,
                                              T *acca, unsigned char *fa, int32_t cb, T *accb,
                                              unsigned char *fb, int tid) {
  const int n = int(q1 - q0);
  const int32_t *bc = bcol + q0;
  const T *bv = bval + q0;
  int i = tid;
  for (; i + 96 < n; i += 128) {
    int32_t c0 = bc[i], c1 = bc[i + 32], c2 = bc[i + 64], c3 = bc[i + 96];
    T v0 = bv[i], v1 = bv[i + 32], v2 = bv[i + 64], v3 = bv[i + 96];
    mac<T, MARK>(acca, fa, c0 - ca, a, v0);
    mac<T, MARK>(acca, fa, c1 - ca, a, v1);
    mac<T, MARK>(acca, fa, c2 - ca, a, v2);
    mac<T, MARK>(acca, fa, c3 - ca, a, v3);
    mac<T, MARK>(accb, fb, c0 - cb, b, v0);
    mac<T, MARK>(accb, fb, c1 - cb, b, v1);
    mac<T, MARK>(accb, fb, c2 - cb, b, v2);
    mac<T, MARK>(accb, fb, c3 - cb, b, v3);
  }
  // at most three entries per lane are left: two loaded together, then one
  if (i + 32 < n) {
    int32_t c0 = bc[i], c1 = bc[i + 32];
    T v0 = bv[i], v1 = bv[i + 32];
    mac<T, MARK>(acca, fa, c0 - ca, a, v0);
    mac<T, MARK>(acca, fa, c1 - ca, a, v1);
    mac<T, MARK>(accb, fb, c0 - cb, b, v0);
    mac<T, MARK>(accb, fb, c1 - cb, b, v1);
    i += 64;
  }
  if (i < n) {
    int32_t c = bc[i];
    T v = bv[i];
    mac<T, MARK>(acca, fa, c - ca, a, v);
    mac<T, MARK>(accb, fb, c - cb, b, v);
  }
}

// The k-loop of two rows run by one warp (rows of the 16-lane pair class).
// Their k lists, each ascending, are merged: a k found in both rows is one
// step that feeds both accumulators from a single pass over B_k, a k of one
// row only is a step of that row alone. Each row thus still receives its k in
// ascending order, one FMA per slot per k, exactly as with a warp of its own.
// Rows of a banded iterate that are neighbours share almost all of their k,
// so the pair gathers B about half as often as two warps would.
// Row x has k entries [pa, ea) and accumulator (acca, fa) for columns from
// ca; row y likewise (an absent row has pb == eb).
template <typename T, bool MARK>
__device__ __forceinline__ void pair_rows(int64_t pa, int64_t ea, int64_t pb, int64_t eb,
                                          const int32_t *acol, const T *aval,
                                          const int64_t *brs, const int64_t *bre,
                                          const int32_t *bcol, const T *bval, int32_t ca,
                                          T *acca, unsigned char *fa, int32_t cb, T *accb,
                                          unsigned char *fb, int lane) {
  constexpr unsigned FULL = 0xffffffffu;
  // lane l holds the (k, a_k, start, length) of the l-th k of each row's window
  int ka = INT_MAX, kb = INT_MAX, na = 0, nb = 0;
  T va = T(0), vb = T(0);
  int64_t qa = 0, qb = 0;
  {
    int64_t p = pa + lane;
    if (p < ea) {
      ka = acol[p];
      va = aval[p];
      qa = brs[ka];
      na = int(bre[ka] - qa);
    }
    p = pb + lane;
    if (p < eb) {
      kb = acol[p];
      vb = aval[p];
      qb = brs[kb];
      nb = int(bre[kb] - qb);
    }
  }
  int ia = 0, ib = 0;
  for (;;) {
    if (ia == 32) {  // window of row x used up: the next 32 k
      pa += 32;
      ia = 0;
      int64_t p = pa + lane;
      ka = INT_MAX;
      if (p < ea) {
        ka = acol[p];
        va = aval[p];
        qa = brs[ka];
        na = int(bre[ka] - qa);
      }
    }
    if (ib == 32) {
      pb += 32;
      ib = 0;
      int64_t p = pb + lane;
      kb = INT_MAX;
      if (p < eb) {
        kb = acol[p];
        vb = aval[p];
        qb = brs[kb];
        nb = int(bre[kb] - qb);
      }
    }
    const int ha = __shfl_sync(FULL, ka, ia), hb = __shfl_sync(FULL, kb, ib);
    if (ha == INT_MAX && hb == INT_MAX) break;
    if (ha == hb) {
      const T a = __shfl_sync(FULL, va, ia), b = __shfl_sync(FULL, vb, ib);
      const int64_t q0 = __shfl_sync(FULL, qa, ia);
      const int n = __shfl_sync(FULL, na, ia);
      accumulate_k2<T, MARK>(a, b, q0, q0 + n, bcol, bval, ca, acca, fa, cb, accb, fb, lane);
      ++ia;
      ++ib;
    } else if (ha < hb) {
      const T a = __shfl_sync(FULL, va, ia);
      const int64_t q0 = __shfl_sync(FULL, qa, ia);
      const int n = __shfl_sync(FULL, na, ia);
      accumulate_k<T, 32, MARK>(a, q0, q0 + n, bcol, bval, ca, acca, fa, lane);
      ++ia;
    } else {
      const T b = __shfl_sync(FULL, vb, ib);
      const int64_t q0 = __shfl_sync(FULL, qb, ib);
      const int n = __shfl_sync(FULL, nb, ib);
      accumulate_k<T, 32, MARK>(b, q0, q0 + n, bcol, bval, cb, accb, fb, lane);
      ++ib;
    }
    __syncwarp();
  }
}

constexpr int PAIR_OCC = 8;  // CTAs per SM of the pair kernel: 64 registers, no spills
template <typename T>
struct WarpOcc;  // CTAs per SM of the warp kernel (shared memory and registers)
template <> struct WarpOcc<double> { static constexpr int value = 6; };
template <> struct WarpOcc<float> { static constexpr int value = 10; };

// G lanes per row, 32/G rows per warp; each group owns WARP_W*G/32 slots of
// its warp's accumulator and runs the ascending-k accumulation of its own row
// with group-wide barriers, so the result is the same as with a whole warp.
// PAIR (with G = 16): the two rows of a warp share its k-loop (pair_rows);
// the rest of the kernel is that of 16-lane groups.
template <typename T, int MODE, int G, bool PAIR = false>
__global__ void __launch_bounds__(WARPS_PER_CTA * 32, PAIR ? PAIR_OCC : WarpOcc<T>::value)
    k_num_group(const int64_t *ars, const int64_t *are, const int32_t *acol, const T *aval,
                const int64_t *brs, const int64_t *bre, const int32_t *bcol, const T *bval,
                const int32_t *lo, const int32_t *len, const int32_t *list, int *counters,
                int cls, const int64_t *cs, int64_t *ce, int32_t *ccol, T *cval, double *part) {
  static_assert(!PAIR || G == 16, "pairs are two 16-lane groups");
  constexpr bool MARK = sizeof(T) == 4;  // untouched FP32 slots hold -0 (see mac)
  constexpr int NG = 32 / G;
  constexpr int SLOTS = WARP_W / NG;
  // group bases staggered across shared-memory banks: without it the groups of
  // a warp (or of a half-warp, for 8-byte values) start on the same bank and
  // their lanes, which touch neighbouring slots, collide
  constexpr int PAD = G == 32 ? 0 : (sizeof(T) == 4 ? G : (G == 8 ? 8 : 0));
  __shared__ T acc_all[WARPS_PER_CTA][WARP_W + 3 * PAD];
  __shared__ unsigned char flags[WARPS_PER_CTA][WARP_W + 3 * PAD];
  const int lane = lane_id(), w = threadIdx.x >> 5;
  const int g = lane / G, gl = lane % G;
  const unsigned gbits = G == 32 ? 0xffffffffu : ((1u << G) - 1u);
  const unsigned gmask = gbits << (g * G);
  const unsigned lt = (1u << gl) - 1u;
  T *acc = acc_all[w] + g * (SLOTS + PAD);
  unsigned char *f = flags[w] + g * (SLOTS + PAD);
  const int total = counters[cls];
  for (;;) {
    int base = 0;
    if (lane == 0) base = atomicAdd(&counters[RC_QUEUE + cls], NG);
    base = __shfl_sync(0xffffffffu, base, 0);
    if (base >= total) break;
    const int idx = base + g;
    if (PAIR || idx < total) {
      const bool has = idx < total;  // the second row of the last pair may be absent
      const int32_t r = has ? list[idx] : 0;
      const int L = has ? len[r] : 0;
      const int32_t c0 = has ? lo[r] : 0;
      for (int s = gl; s < L; s += G) {
        acc[s] = MARK ? T(-0.0) : T(0);
        if (!MARK || MODE == MODE_UPDATE) f[s] = 0;
      }
      const int64_t a0 = has ? ars[r] : 0, a1 = has ? are[r] : 0;
      if (PAIR) {
        __syncwarp();
        constexpr unsigned FULL = 0xffffffffu;
        pair_rows<T, MARK>(__shfl_sync(FULL, a0, 0), __shfl_sync(FULL, a1, 0),
                     __shfl_sync(FULL, a0, G), __shfl_sync(FULL, a1, G), acol, aval, brs, bre,
                     bcol, bval, __shfl_sync(FULL, c0, 0), acc_all[w], flags[w],
                     __shfl_sync(FULL, c0, G), acc_all[w] + (SLOTS + PAD),
                     flags[w] + (SLOTS + PAD), lane);
      } else {
        __syncwarp(gmask);
        // ascending k; the (a_ik, start, end) of G k at a time are fetched by
        // the group's lanes together and broadcast inside the group
        for (int64_t pb = a0; pb < a1; pb += G) {
          const int nk = int(min(int64_t(G), a1 - pb));
          T av = T(0);
          int64_t qs = 0, qe = 0;
          if (gl < nk) {
            int32_t k = acol[pb + gl];
            av = aval[pb + gl];
            qs = brs[k];
            qe = bre[k];
          }
          for (int t = 0; t < nk; ++t) {
            T a = __shfl_sync(gmask, av, t, G);
            int64_t q0 = __shfl_sync(gmask, qs, t, G);
            int64_t q1 = __shfl_sync(gmask, qe, t, G);
            accumulate_k<T, G, MARK>(a, q0, q1, bcol, bval, c0, acc, f, gl);
            __syncwarp(gmask);
          }
        }
      }
      if (has) {  // group-uniform
        if (MODE == MODE_UPDATE) {
          for (int64_t p = a0 + gl; p < a1; p += G) {
            int j = acol[p] - c0;
            T xt = acc[j];
            if (untouched<T, MARK>(xt)) xt = T(0);
            acc[j] = ns_combine(aval[p], xt);
            f[j] = 3;
          }
          __syncwarp(gmask);
        }
        int64_t out = cs[r];
        SqAcc<T> racc;
        double rdiag = 0.0;
        bool diag = false;
        for (int s0 = 0; s0 < L; s0 += G) {
          int s = s0 + gl;
          int fl = 0;
          if (s < L) {
            if (MARK) {  // touched: a product (acc is not -0) or, in an update, x_ij
              fl = MODE == MODE_UPDATE ? f[s] : 0;
              if (!fl && !untouched<T, MARK>(acc[s])) fl = 1;
            } else {
              fl = f[s];
            }
          }
          unsigned m = (__ballot_sync(gmask, fl != 0) >> (g * G)) & gbits;
          if (fl) {
            int64_t pos = out + __popc(m & lt);
            int32_t cj = c0 + s;
            T v = acc[s];
            if (MODE == MODE_UPDATE && !(fl & 2)) v = ns_combine(T(0), v);
            ccol[pos] = cj;
            cval[pos] = v;
            if (MODE == MODE_SQUARE) {
              if (cj == r) {  // (t_ii - 1)^2 in FP64, once per row
                double d = double(v) - 1.0;
                rdiag = d * d;
                diag = true;
              } else {
                racc.add_sq(v);
              }
            }
          }
          out += __popc(m);
        }
        if (gl == 0) ce[r] = out;
        if (MODE == MODE_SQUARE) {
          SqAcc<T> xacc;
          for (int64_t p = a0 + gl; p < a1; p += G) xacc.add_sq(aval[p]);
          double rs = racc.value() + rdiag, xs = xacc.value();
  #pragma unroll
          for (int o = G / 2; o > 0; o >>= 1) {
            rs += __shfl_xor_sync(gmask, rs, o, G);
            xs += __shfl_xor_sync(gmask, xs, o, G);
          }
          bool any_diag = __any_sync(gmask, diag);
          if (gl == 0) {
            part[2 * int64_t(r)] = any_diag ? rs : rs + 1.0;
            part[2 * int64_t(r) + 1] = xs;
          }
        }
        __syncwarp(gmask);
      }
    }
    __syncwarp();
  }
}

template <typename T>
constexpr size_t num_cta_smem() {
  return size_t(CtaW<T>::value) * (sizeof(T) + 1) + 2 * K_BATCH * sizeof(int64_t);
}

template <typename T, int MODE>
__global__ void __launch_bounds__(CTA_THREADS)
    k_num_cta(const int64_t *ars, const int64_t *are, const int32_t *acol, const T *aval,
              const int64_t *brs, const int64_t *bre, const int32_t *bcol, const T *bval,
              const int32_t *lo, const int32_t *len, const int32_t *clist, int *counters,
              const int64_t *cs, int64_t *ce, int32_t *ccol, T *cval, double *part) {
  constexpr int CW = CtaW<T>::value;
  // the CTA class uses counters[RC_CTA] (length) and counters[RC_QUEUE + RC_CTA] (queue head)
  constexpr int NW = CTA_THREADS / 32;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int64_t *ks = reinterpret_cast<int64_t *>(smem_raw);
  int64_t *ke = ks + K_BATCH;
  T *acc = reinterpret_cast<T *>(ke + K_BATCH);
  unsigned char *f = reinterpret_cast<unsigned char *>(acc + CW);
  __shared__ int s_idx;
  __shared__ int s_cnt[NW];
  __shared__ double s_red[2][NW];
  int lane = lane_id(), w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  for (;;) {
    if (threadIdx.x == 0) s_idx = atomicAdd(&counters[RC_QUEUE + RC_CTA], 1);
    __syncthreads();
    int idx = s_idx;
    __syncthreads();
    if (idx >= counters[RC_CTA]) break;
    int32_t r = clist[idx];
    int64_t L = len[r];
    int64_t base = lo[r];
    int64_t a0 = ars[r], a1 = are[r];
    int64_t nA = a1 - a0;
    bool multi = L > CW;
    int64_t out = cs[r];
    double rs = 0.0;
    bool diag = false;
    for (int64_t c0 = base; c0 < base + L; c0 += CW) {
      int W = int(min(int64_t(CW), base + L - c0));
      for (int s = threadIdx.x; s < W; s += CTA_THREADS) {
        acc[s] = T(0);
        f[s] = 0;
      }
      __syncthreads();
      for (int64_t kb = 0; kb < nA; kb += K_BATCH) {
        int nk = int(min(int64_t(K_BATCH), nA - kb));
        if (threadIdx.x < nk) {
          int32_t k = acol[a0 + kb + threadIdx.x];
          int64_t s = brs[k], e = bre[k];
          if (multi) {
            s = lower_bound(bcol, s, e, c0);
            e = lower_bound(bcol, s, e, c0 + W);
          }
          ks[threadIdx.x] = s;
          ke[threadIdx.x] = e;
        }
        __syncthreads();
        for (int t = 0; t < nk; ++t) {  // ascending k
          accumulate_k<T, CTA_THREADS>(aval[a0 + kb + t], ks[t], ke[t], bcol, bval, c0, acc, f,
                                       threadIdx.x);
          __syncthreads();
        }
      }
      if (MODE == MODE_UPDATE) {
        for (int64_t p = a0 + threadIdx.x; p < a1; p += CTA_THREADS) {
          int64_t j = int64_t(acol[p]) - c0;
          if (j >= 0 && j < W) {
            acc[j] = ns_combine(aval[p], acc[j]);
            f[j] = 3;
          }
        }
        __syncthreads();
      }
      // ordered emission: round g covers words g*NW .. g*NW+NW-1, warp w one word
      for (int s0 = 0; s0 < W; s0 += 32 * NW) {
        int s = s0 + w * 32 + lane;
        int fl = s < W ? f[s] : 0;
        unsigned m = __ballot_sync(0xffffffffu, fl != 0);
        if (lane == 0) s_cnt[w] = __popc(m);
        __syncthreads();
        int64_t wbase = out;
        int64_t round_total = 0;
        for (int i = 0; i < NW; ++i) {
          if (i < w) wbase += s_cnt[i];
          round_total += s_cnt[i];
        }
        if (fl) {
          int64_t pos = wbase + __popc(m & lt);
          int64_t cj = c0 + s;
          T v = acc[s];
          if (MODE == MODE_UPDATE && !(fl & 2)) v = ns_combine(T(0), v);
          ccol[pos] = int32_t(cj);
          cval[pos] = v;
          if (MODE == MODE_SQUARE) {
            double d = double(v);
            if (cj == r) {
              d = d - 1.0;
              diag = true;
            }
            rs += d * d;
          }
        }
        out += round_total;
        __syncthreads();
      }
    }
    if (threadIdx.x == 0) ce[r] = out;
    if (MODE == MODE_SQUARE) {
      double xs = 0.0;
      for (int64_t p = a0 + threadIdx.x; p < a1; p += CTA_THREADS) {
        double x = double(aval[p]);
        xs += x * x;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        rs += __shfl_xor_sync(0xffffffffu, rs, o);
        xs += __shfl_xor_sync(0xffffffffu, xs, o);
      }
      int any_diag = __syncthreads_or(diag ? 1 : 0);
      if (lane == 0) {
        s_red[0][w] = rs;
        s_red[1][w] = xs;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < NW; ++i) {
          a += s_red[0][i];
          b += s_red[1][i];
        }
        part[2 * int64_t(r)] = any_diag ? a : a + 1.0;
        part[2 * int64_t(r) + 1] = b;
      }
      __syncthreads();
    }
  }
}

// Rows with an empty column range: their slot stays empty (ce = cs) and, in
// MODE_SQUARE, they still contribute (0 - 1)^2 = 1 for the missing diagonal
// and sum_k a_ik^2 to the norms.
template <typename T>
__global__ void k_rows_empty(int64_t n, const int64_t *ars, const int64_t *are, const T *aval,
                             const int32_t *len, const int64_t *cs, int64_t *ce, double *part) {
  int lane = lane_id();
  const int g = lane >> 3, gl = lane & 7;  // four groups of 8 lanes
  int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  // a lane per row finds the empty ones, 32 at a time; the warp's four groups
  // of 8 lanes serve them four at a time
  for (int64_t r0 = warp * 32; r0 < n; r0 += nwarps * 32) {
    unsigned empty = __ballot_sync(0xffffffffu, r0 + lane < n && len[r0 + lane] == 0);
    while (empty) {
      int my = -1;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (!empty) break;
        if (k == g) my = __ffs(empty) - 1;
        empty &= empty - 1;
      }
      const bool has = my >= 0;
      const int64_t r = r0 + (has ? my : 0);
      if (has && gl == 0) ce[r] = cs[r];
      if (!part) continue;
      double xs = 0.0;
      if (has)
        for (int64_t p = ars[r] + gl; p < are[r]; p += 8) {
          double x = double(aval[p]);
          xs += x * x;
        }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) xs += __shfl_xor_sync(0xffffffffu, xs, o, 8);
      if (has && gl == 0) {
        part[2 * r] = 1.0;
        part[2 * r + 1] = xs;
      }
    }
  }
}

int sm_count() {
  static const int n = [] {  // once, thread-safe (server lanes launch from several threads)
    int dev = 0, v = 0;
    SGN_CUDA(cudaGetDevice(&dev));
    SGN_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    return v;
  }();
  return n;
}

int grid_cap(int64_t items, int per_block, int per_sm) {
  int64_t g = (items + per_block - 1) / per_block;
  int64_t cap = int64_t(sm_count()) * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return int(g);
}

}  // namespace

void launch_bounds(int64_t n, const Rows &A, const Rows &B, const int32_t *seg, const int *active,
                   int mode, int groups, float group_margin, int band, float band_min_eff,
                   const int *dslot, const int64_t *moff, int32_t *lo, int32_t *len,
                   int64_t *ub, int32_t *lists, int *counters, double *work,
                   double *band_work, unsigned char *bandrow, int4 *binfo, cudaStream_t s) {
  if (n == 0) return;
  k_row_info<<<grid_cap(n, 256, 8), 256, 0, s>>>(n, B.rs, B.re, B.col, binfo);
  SGN_LAUNCH_CHECK();
  int tiles = int((n + BOUNDS_TILE - 1) / BOUNDS_TILE);
  int g = tiles < sm_count() * 8 ? tiles : sm_count() * 8;
  k_bounds<<<g, BOUNDS_TILE, 0, s>>>(n, A.rs, A.re, A.col, binfo, seg, active, mode, groups,
                                     group_margin, band, band_min_eff, dslot, moff, lo, len, ub,
                                     lists, counters, work, band_work, bandrow);
  SGN_LAUNCH_CHECK();
}

template <typename T, int MODE, int G, bool PAIR = false>
static void group_launch(int64_t n, const Rows &A, const T *aval, const Rows &B, const T *bval,
                         const int32_t *lo, const int32_t *len, const int32_t *lists, int *ctr,
                         int cls, const int64_t *cs, int64_t *ce, int32_t *ccol, T *cval,
                         double *part, cudaStream_t s) {
  k_num_group<T, MODE, G, PAIR><<<grid_cap(n, WARPS_PER_CTA * (32 / G),
                                           PAIR ? PAIR_OCC : WarpOcc<T>::value),
                                  WARPS_PER_CTA * 32, 0, s>>>(
      A.rs, A.re, A.col, aval, B.rs, B.re, B.col, bval, lo, len, lists + int64_t(cls) * n, ctr,
      cls, cs, ce, ccol, cval, part);
  SGN_LAUNCH_CHECK();
}

template <typename T, int MODE>
static void num_launch(int64_t n, const Rows &A, const T *aval, const Rows &B, const T *bval,
                       const int32_t *lo, const int32_t *len, const int32_t *lists, int *ctr,
                       const int64_t *cs, int64_t *ce, int32_t *ccol, T *cval, double *part,
                       cudaStream_t s) {
  group_launch<T, MODE, 32>(n, A, aval, B, bval, lo, len, lists, ctr, RC_G32, cs, ce, ccol, cval,
                            part, s);
  // FP32: the 16-lane class holds row pairs (GROUPS_PAIRS)
  group_launch<T, MODE, 16, sizeof(T) == 4>(n, A, aval, B, bval, lo, len, lists, ctr, RC_G16, cs,
                                            ce, ccol, cval, part, s);
  group_launch<T, MODE, 8>(n, A, aval, B, bval, lo, len, lists, ctr, RC_G8, cs, ce, ccol, cval,
                           part, s);
  constexpr size_t sm = num_cta_smem<T>();
  static const bool attr = [] {  // once, thread-safe
    SGN_CUDA(cudaFuncSetAttribute(k_num_cta<T, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(sm)));
    return true;
  }();
  (void)attr;
  k_num_cta<T, MODE><<<grid_cap(n, 1, 2), CTA_THREADS, sm, s>>>(
      A.rs, A.re, A.col, aval, B.rs, B.re, B.col, bval, lo, len, lists + int64_t(RC_CTA) * n, ctr,
      cs, ce, ccol, cval, part);
  SGN_LAUNCH_CHECK();
}

template <typename T>
void launch_numeric(int64_t n, const Rows &A, const T *aval, const Rows &B, const T *bval,
                    int mode, const int32_t *lo, const int32_t *len, const int32_t *lists,
                    const int *counters, const int64_t *cs, int64_t *ce, int32_t *ccol, T *cval,
                    double *part, cudaStream_t s) {
  if (n == 0) return;
  int *ctr = const_cast<int *>(counters);
  k_rows_empty<T><<<grid_cap(n, 8 * 32, 16), 256, 0, s>>>(n, A.rs, A.re, aval, len, cs, ce,
                                                      mode == MODE_SQUARE ? part : nullptr);
  SGN_LAUNCH_CHECK();
  if (mode == MODE_SQUARE)
    num_launch<T, MODE_SQUARE>(n, A, aval, B, bval, lo, len, lists, ctr, cs, ce, ccol, cval, part,
                               s);
  else
    num_launch<T, MODE_UPDATE>(n, A, aval, B, bval, lo, len, lists, ctr, cs, ce, ccol, cval, part,
                               s);
}

template void launch_numeric<double>(int64_t, const Rows &, const double *, const Rows &,
                                     const double *, int, const int32_t *, const int32_t *,
                                     const int32_t *, const int *, const int64_t *, int64_t *,
                                     int32_t *, double *, double *, cudaStream_t);
template void launch_numeric<float>(int64_t, const Rows &, const float *, const Rows &,
                                    const float *, int, const int32_t *, const int32_t *,
                                    const int32_t *, const int *, const int64_t *, int64_t *,
                                    int32_t *, float *, double *, cudaStream_t);

}  // namespace sgn
