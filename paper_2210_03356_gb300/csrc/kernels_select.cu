// Budget, element threshold and filter of the NSF step (steps a4-a6).
//
// Budget (Eq. 1.18 with the fixed phase of Sec. 3.2 / Sec. 4): the RMS budget
// is c4 * tol_stage while r >= switch_resid, else 3/4 r^2 / (3x + x^3), with
// r = ||T - I||_F / sqrt(n) and x = ||X||_F / sqrt(n) of the current iterate;
// the filter's absolute Frobenius bound is b = sqrt(n) * beta.
//
// EXACT threshold: tau is the smallest magnitude v such that the squares of
// all entries with |x| <= v sum to more than b^2 (every |x| < tau is
// dropped, every |x| >= tau kept, so equal magnitudes share their fate); if
// all entries with |x| <= b fit, tau is the smallest magnitude above b
// (+inf if there is none). It is found by a radix select on the IEEE bit
// pattern of |x| (positive doubles order like unsigned integers): a
// histogram of the top 16 bits over a 1024-bucket window below b, then six
// 8-bit digits over the candidates of the crossing bucket. The squares are
// summed as exact 128-bit integers on a fixed grid of the matrix, q(x) =
// floor(x^2 / 2^(2e - 62)) with 2^e <= b < 2^(e+1), against Q = q(b): the
// decision does not depend on the order of the additions, and it is the exact
// one up to the flooring, less than one grid step (2^-62 b^2) per entry.
#include "common.cuh"
#include "kernels.h"

namespace sgn {

namespace {

constexpr int NB0 = 1024;        // level-0 buckets
constexpr int NDIG = 256;        // digit buckets

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__global__ void k_matrix_scalars(int nb, const int64_t *moff, const double *sums, double c4,
                                 double tol_stage, double switch_resid, MatScalars *ms) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nb) return;
  double sn = __dsqrt_rn(double(moff[m + 1] - moff[m]));
  double r = __ddiv_rn(__dsqrt_rn(sums[2 * m]), sn);
  double x = __ddiv_rn(__dsqrt_rn(sums[2 * m + 1]), sn);
  double beta;
  if (r >= switch_resid)
    beta = __dmul_rn(c4, tol_stage);
  else
    beta = __ddiv_rn(__dmul_rn(__dmul_rn(0.75, r), r),
                     __dadd_rn(__dmul_rn(3.0, x), __dmul_rn(__dmul_rn(x, x), x)));
  ms[m].r = r;
  ms[m].x = x;
  ms[m].beta = beta;
  ms[m].b = __dmul_rn(sn, beta);
}

__global__ void k_select_bound(int nb, const int *active, MatScalars *ms) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nb || !active[m]) return;
  int64_t c = ms[m].nnz_bar;
  ms[m].tau = c > 0 ? __ddiv_rn(ms[m].b, __dsqrt_rn(double(c))) : __longlong_as_double(0x7ff0000000000000LL);
}

// ------------------------------------------------------------ EXACT select
struct SelState {
  unsigned long long prefix;              // key bits known so far
  unsigned long long below_lo, below_hi;  // 128-bit sum of q strictly below the prefix range
  unsigned long long below0_lo, below0_hi;  // the same below the crossing level-0 bucket
  int found;                              // 1: a crossing exists; 0: everything <= b fits
  int pad;
};

// Scratch: 128-bit sums (lo, hi) per bucket for the level-0 and digit
// histograms, the smallest key above b per matrix, the select states, the
// candidate count and the candidates (key, row of the values).
struct SelScratch {
  unsigned long long *hist0;    // nb * NB0 * 2
  unsigned long long *hdig;     // nb * NDIG * 2
  unsigned long long *minabove; // nb
  SelState *st;                 // nb
  unsigned long long *ncand;    // 1
  unsigned long long *cand;     // cap
  int *cand_r;                  // cap
  unsigned long long cap;       // candidate room; *ncand may count past it (overflow)
};

static_assert(sizeof(SelState) <= kSelStateBytes, "select state outgrew its scratch slot");
static_assert(NB0 == 1024 && NDIG == 256, "scratch layout in kernels.h assumes these sizes");

inline size_t align_up(size_t x) { return sel_align(x); }

SelScratch carve(void *base, int nb, int64_t cap) {
  char *p = static_cast<char *>(base);
  SelScratch s;
  s.hist0 = reinterpret_cast<unsigned long long *>(p);
  p += align_up(size_t(nb) * NB0 * 2 * 8);
  s.hdig = reinterpret_cast<unsigned long long *>(p);
  p += align_up(size_t(nb) * NDIG * 2 * 8);
  s.minabove = reinterpret_cast<unsigned long long *>(p);
  p += align_up(size_t(nb) * 8);
  s.st = reinterpret_cast<SelState *>(p);
  p += align_up(size_t(nb) * kSelStateBytes);
  s.ncand = reinterpret_cast<unsigned long long *>(p);
  p += align_up(8);
  s.cand = reinterpret_cast<unsigned long long *>(p);
  p += align_up(size_t(cap > 0 ? cap : 1) * 8);
  s.cand_r = reinterpret_cast<int *>(p);
  s.cap = (unsigned long long)(cap > 0 ? cap : 1);
  return s;
}

// Rows of the values to select over: row r holds entries [rs[r], re[r]) and
// belongs to matrix seg[r]; with rs == nullptr the values are one flat array
// of flat_nnz entries cut into rows of FLAT_ROW, all of matrix 0.
constexpr int64_t FLAT_ROW = kFlatRow;
constexpr int SEL_THREADS = 256;

__device__ __forceinline__ int row_mat(const SelRows &R, int64_t r) { return R.seg ? R.seg[r] : 0; }

constexpr unsigned long long INF_KEY = 0x7FF0000000000000ULL;

// The filter's rule on keys: x is kept when x != 0 and |x| >= tau, tau given
// by its bit pattern. For every |x| that is not NaN this is the comparison of
// the two doubles (non-negative doubles order like their bit patterns); NaN
// entries are dropped, as by the floating-point comparison. The count and
// the write of a filter both decide with this one function.
__device__ __forceinline__ bool keep_key(unsigned long long key, unsigned long long tkey) {
  return key != 0ULL && key <= INF_KEY && key >= tkey;
}

__device__ __forceinline__ void row_range(const SelRows &R, int64_t r, int64_t &b, int64_t &e) {
  if (R.rs) {
    b = R.rs[r];
    e = R.re[r];
  } else {
    b = r * FLAT_ROW;
    e = min(b + FLAT_ROW, R.flat_nnz);
  }
}

// Bit pattern of |x| as an FP64 number. For FP32 values of the normal range
// it is built with integer operations (exponent rebiased by 1023 - 127 = 896,
// mantissa widened by 29 bits): the same bits as the exact conversion, with
// no work for the FP64 pipe, which this GPU runs at 1/64 of its FP32 rate.
__device__ __forceinline__ unsigned long long key_f32(float x) {
  const uint32_t b = __float_as_uint(x) & 0x7FFFFFFFu, e = b >> 23;
  if (e != 0u && e != 0xFFu)
    return ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29);
  if (b == 0u) return 0ULL;
  return (unsigned long long)__double_as_longlong(fabs(double(x)));  // subnormal, inf, NaN
}

__device__ __forceinline__ unsigned long long key_f64(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFULL;
}

template <typename T>
__device__ __forceinline__ unsigned long long key_t(T x);
template <>
__device__ __forceinline__ unsigned long long key_t<float>(float x) { return key_f32(x); }
template <>
__device__ __forceinline__ unsigned long long key_t<double>(double x) { return key_f64(x); }

// (hi, lo) += x^2 for FP32 x, exactly: the square's rounding error comes from
// an FMA and the sum's from TwoSum; all in FP32, which this GPU runs at 64x
// its FP64 rate. Inputs are scaled by 2^48 (exact), so that squares of
// entries from 2^-111 to 2^16 stay normal FP32 numbers.
__device__ __forceinline__ void ff_add_sq48(float x, float &hi, float &lo) {
  const float y = __fmul_rn(x, 281474976710656.0f);  // 2^48
  const float p = __fmul_rn(y, y), e = __fmaf_rn(y, y, -p);
  const float s = __fadd_rn(hi, p), bb = __fsub_rn(s, hi);
  lo = __fadd_rn(lo, __fadd_rn(__fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(p, bb)), e));
  hi = s;
}

__device__ __forceinline__ void ff_add(float &hi, float &lo, float h2, float l2) {
  const float s = __fadd_rn(hi, h2), bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(h2, bb));
  lo = __fadd_rn(__fadd_rn(lo, l2), err);
  hi = s;
}

// q = floor(x^2 / 2^(2e - 62)) for 0 < |x| <= b, with |x| given by its FP64
// bit pattern (significand M, biased exponent E; a subnormal counts as E = 1)
// and e the biased exponent of b (likewise): x^2 / 2^(2e - 62) = M^2 2^-s with
// s = 42 + 2 (e - E) >= 42, so q is M^2 shifted right by s, exactly, in
// integers (q < 2^64 since |x| <= b). q >= 1 exactly when E >= e - 31.
// FP32 values have M = m 2^29 with m < 2^24, and q = m^2 2^(58 - s) needs one
// 32 x 32-bit product.
template <typename T>
__device__ __forceinline__ unsigned long long qval(unsigned long long key, int eb) {
  const int ex = int(key >> 52);
  const int s = 42 + 2 * (eb - (ex ? ex : 1));
  if (s >= 106) return 0ULL;
  const unsigned long long M = (key & 0xFFFFFFFFFFFFFULL) | (ex ? (1ULL << 52) : 0ULL);
  if constexpr (sizeof(T) == 4) {
    const unsigned m = unsigned(M >> 29);
    const unsigned long long m2 = (unsigned long long)m * m;  // < 2^48
    return s <= 58 ? m2 << (58 - s) : m2 >> (s - 58);
  } else {
    const unsigned long long lo = M * M, hi = __umul64hi(M, M);
    if (s >= 64) return hi >> (s - 64);
    return (lo >> s) | (hi << (64 - s));
  }
}

// Per matrix: e (the biased exponent of b, 1 for a subnormal b), Q = q(b) and
// the smallest key with q >= 1 (the key of 2^(e - 31 - 1023)). b = 0, +inf or
// NaN: no key is summed (tiny = all ones), every q counts as 0.
__global__ void k_sel_prepare(int nb, MatScalars *ms) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nb) return;
  const unsigned long long bkey = (unsigned long long)__double_as_longlong(ms[m].b);
  const int e = int(bkey >> 52);
  if (bkey == 0ULL || e >= 0x7FF) {  // b <= 0 (sign bit) is caught here as well
    ms[m].sel_e = 0;
    ms[m].sel_q = 0ULL;
    ms[m].tiny = ~0ULL;
    return;
  }
  const int eb = e ? e : 1;
  ms[m].sel_e = eb;
  ms[m].sel_q = qval<double>(bkey, eb);
  ms[m].tiny = eb > 32 ? (unsigned long long)(eb - 31) << 52 : 0ULL;
}

// (lo, hi) += (alo, ahi) atomically in memory; exact, order-independent.
__device__ __forceinline__ void add128(unsigned long long *lohi, unsigned long long alo,
                                       unsigned long long ahi) {
  unsigned long long old = atomicAdd(&lohi[0], alo);
  if (old + alo < old) ++ahi;
  if (ahi) atomicAdd(&lohi[1], ahi);
}

__device__ __forceinline__ int bucket0(unsigned long long key, unsigned long long bkey) {
  long long base = (long long)(bkey >> 48) - (NB0 - 1);
  long long t = (long long)(key >> 48);
  if (base < 0) base = 0;
  return t <= base ? 0 : int(t - base);
}

// A chunk of consecutive rows, their extents and matrices staged in shared
// memory by one thread per row, so that a warp's loop over the chunk's rows
// waits on the values only, not on the chain row -> matrix -> scalars.
// Rows of inactive matrices are staged empty.
constexpr int RPC = 64;  // rows per chunk (row lists); flat values: 32 rows of kFlatRow
__device__ __forceinline__ int64_t chunk_rows(const SelRows &R) { return R.rs ? RPC : 32; }

struct ChunkRows {
  int64_t b[RPC], e[RPC];
  int m[RPC];
};

// Stages rows [r0, r1) (r1 - r0 <= RPC) and returns the thread's row
// slot (-1 if none) with its matrix in m; the caller adds its own per-row
// scalars, then synchronises.
__device__ __forceinline__ int stage_rows(const SelRows &R, const int *active, int64_t r0,
                                          int64_t r1, ChunkRows &cr, int &m) {
  const int t = threadIdx.x;
  if (t >= r1 - r0) return -1;
  const int64_t r = r0 + t;
  m = row_mat(R, r);
  int64_t b, e;
  row_range(R, r, b, e);
  cr.b[t] = b;
  cr.e[t] = active[m] ? e : b;
  cr.m[t] = m;
  return t;
}

constexpr int HIST_LPR = 8;  // lanes per row of the level-0 histogram

// Level-0 histogram. A CTA takes a chunk of consecutive rows, a warp
// 32 / HIST_LPR rows at a time with HIST_LPR lanes each (the per-row work is
// then spread over more entries per lane), each lane a contiguous run of the
// row's entries. Neighbouring entries of a row have similar magnitudes, so a
// lane sums its run per bucket in registers and adds the run's total once
// when the bucket changes: into a shared histogram for the chunk's first
// matrix (almost every row: matrices span many chunks), else into the global
// one.

template <typename T>
__global__ void __launch_bounds__(SEL_THREADS)
    k_sel_hist0(SelRows R, const int *active, const T *val, const MatScalars *ms, SelScratch sc) {
  __shared__ unsigned long long s_h[NB0 * 2];
  __shared__ unsigned long long s_min;
  __shared__ ChunkRows cr;
  __shared__ unsigned long long s_bkey[RPC], s_tiny[RPC];
  __shared__ int s_eb[RPC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = SEL_THREADS / 32;
  const int64_t rpc = chunk_rows(R);
  const int64_t nchunks = (R.nrows + rpc - 1) / rpc;
  for (int64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int64_t r0 = c * rpc, r1 = min(r0 + rpc, R.nrows);
    for (int t = threadIdx.x; t < 2 * NB0; t += SEL_THREADS) s_h[t] = 0ULL;
    if (threadIdx.x == 0) s_min = ~0ULL;
    int mt = 0;
    const int t = stage_rows(R, active, r0, r1, cr, mt);
    if (t >= 0) {
      s_bkey[t] = (unsigned long long)__double_as_longlong(ms[mt].b);
      s_eb[t] = ms[mt].sel_e;
      s_tiny[t] = ms[mt].tiny;
    }
    __syncthreads();
    const int m0 = cr.m[0];
    // HIST_LPR lanes per row, 32 / HIST_LPR rows of the chunk per warp at a time
    const int g = lane / HIST_LPR, gl = lane % HIST_LPR;
    const int nr = int(r1 - r0);
    for (int i0 = warp * (32 / HIST_LPR); i0 < nr; i0 += nw * (32 / HIST_LPR)) {
      const int i = i0 + g;
      const bool has = i < nr;
      const int64_t e0 = has ? cr.b[i] : 0, e1 = has ? cr.e[i] : 0;
      const int m = has ? cr.m[i] : m0;
      const unsigned long long bkey = has ? s_bkey[i] : 0ULL, tiny = has ? s_tiny[i] : ~0ULL;
      const int eb = has ? s_eb[i] : 0;
      unsigned long long *hist = m == m0 ? s_h : sc.hist0 + size_t(m) * NB0 * 2;
      const int64_t per = (e1 - e0 + HIST_LPR - 1) / HIST_LPR;
      const int64_t p0 = e0 + gl * per, p1 = min(p0 + per, e1);
      int cur = -1;
      unsigned long long clo = 0, chi = 0, mymin = ~0ULL;
      // four independent loads in flight, then the entries in order
      for (int64_t pb = p0; pb < p1; pb += 4) {
        unsigned long long keys[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) keys[u] = pb + u < p1 ? key_t<T>(val[pb + u]) : 0ULL;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const unsigned long long key = keys[u];
          if (pb + u >= p1) break;
          if (key > bkey) {
            mymin = key < mymin ? key : mymin;
            continue;
          }
          if (key < tiny) continue;
          unsigned long long q = qval<T>(key, eb);
          if (!q) continue;
          int bk = bucket0(key, bkey);
          if (bk != cur) {
            if (cur >= 0) add128(hist + 2 * cur, clo, chi);
            cur = bk;
            clo = q;
            chi = 0;
          } else {
            clo += q;
            if (clo < q) ++chi;
          }
        }
      }
      if (cur >= 0) add128(hist + 2 * cur, clo, chi);
#pragma unroll
      for (int o = HIST_LPR / 2; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, mymin, o, HIST_LPR);
        mymin = w < mymin ? w : mymin;
      }
      if (gl == 0 && has && mymin != ~0ULL) {
        if (m == m0)
          atomicMin(&s_min, mymin);
        else
          atomicMin(&sc.minabove[m], mymin);
      }
    }
    __syncthreads();
    if (active[m0]) {
      unsigned long long *g = sc.hist0 + size_t(m0) * NB0 * 2;
      for (int t2 = threadIdx.x; t2 < NB0; t2 += SEL_THREADS)
        if (s_h[2 * t2] | s_h[2 * t2 + 1]) add128(g + 2 * t2, s_h[2 * t2], s_h[2 * t2 + 1]);
      if (threadIdx.x == 0 && s_min != ~0ULL) atomicMin(&sc.minabove[m0], s_min);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void u128_add(unsigned long long &lo, unsigned long long &hi,
                                         unsigned long long alo, unsigned long long ahi) {
  unsigned long long o = lo;
  lo += alo;
  hi += ahi + (lo < o ? 1ULL : 0ULL);
}

// (hi, lo) > Q ?
__device__ __forceinline__ bool exceeds(unsigned long long lo, unsigned long long hi,
                                        unsigned long long Q) {
  return hi != 0ULL || lo > Q;
}

// The first of nbk buckets (128-bit sums h[2c], h[2c+1]) at which the running
// sum, started at (lo, hi), exceeds Q = q(b), found by one warp: 32 buckets at a
// time, lane c of a round holding bucket c and an inclusive prefix sum over
// the round by shuffles. The sums are exact integers, so the crossing is the
// one a serial walk finds. Returns the bucket (or -1, with (lo, hi) the total)
// and leaves in (lo, hi) the sum of the buckets below it.
__device__ __forceinline__ int warp_crossing(const unsigned long long *h, int nbk,
                                             unsigned long long Q, unsigned long long &lo,
                                             unsigned long long &hi) {
  const int lane = threadIdx.x & 31;
  for (int c0 = 0; c0 < nbk; c0 += 32) {
    const int c = c0 + lane;
    const unsigned long long blo = c < nbk ? h[2 * c] : 0ULL, bhi = c < nbk ? h[2 * c + 1] : 0ULL;
    unsigned long long plo = blo, phi = bhi;  // inclusive prefix of the round
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long ulo = __shfl_up_sync(0xffffffffu, plo, o);
      const unsigned long long uhi = __shfl_up_sync(0xffffffffu, phi, o);
      if (lane >= o) u128_add(plo, phi, ulo, uhi);
    }
    unsigned long long rlo = lo, rhi = hi;
    u128_add(rlo, rhi, plo, phi);
    const unsigned over = __ballot_sync(0xffffffffu, c < nbk && exceeds(rlo, rhi, Q));
    if (over) {
      const int f = __ffs(over) - 1;
      // the sum below bucket f: start + inclusive prefix of f - h[f]
      unsigned long long elo = rlo - blo, ehi = rhi - bhi - (rlo < blo ? 1ULL : 0ULL);
      lo = __shfl_sync(0xffffffffu, elo, f);
      hi = __shfl_sync(0xffffffffu, ehi, f);
      return c0 + f;
    }
    lo = __shfl_sync(0xffffffffu, rlo, 31);
    hi = __shfl_sync(0xffffffffu, rhi, 31);
  }
  return -1;
}

// One warp per matrix: the level-0 bucket where the exact sums cross Q.
__global__ void k_sel_find0(int nb, const int *active, const MatScalars *ms, SelScratch sc) {
  const int m = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (m == 0 && lane == 0) *sc.ncand = 0ULL;
  if (m >= nb) return;
  SelState st = {};
  if (active[m]) {
    unsigned long long bkey = (unsigned long long)__double_as_longlong(ms[m].b);
    long long base = (long long)(bkey >> 48) - (NB0 - 1);
    if (base < 0) base = 0;
    unsigned long long lo = 0, hi = 0;
    const int c = warp_crossing(sc.hist0 + size_t(m) * NB0 * 2, NB0, ms[m].sel_q, lo, hi);
    if (c >= 0) {
      st.found = 1;
      st.prefix = (unsigned long long)(base + c) << 48;
      st.below_lo = st.below0_lo = lo;
      st.below_hi = st.below0_hi = hi;
    }
  }
  if (lane == 0) sc.st[m] = st;
}

// Per-lane square sums of dropped entries: FP32 values exactly in FP32 pairs
// (scaled by 2^96), FP64 values by FMA.
struct DropSum {
  float hi = 0.0f, lo = 0.0f;
  double d = 0.0;
  __device__ __forceinline__ void add(float x) { ff_add_sq48(x, hi, lo); }
  __device__ __forceinline__ void add(double x) { d = __fma_rn(x, x, d); }
  // the total over each group of W lanes (W divides 32), valid in every lane
  template <typename T, int W>
  __device__ __forceinline__ double group_total() {
    if constexpr (sizeof(T) == 4) {
      if (!__any_sync(0xffffffffu, hi != 0.0f)) return 0.0;
#pragma unroll
      for (int o = W / 2; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o, W);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o, W);
        ff_add(hi, lo, h2, l2);
      }
      return (double(hi) + double(lo)) * 0x1p-96;  // exact scaling, one rounding as ldexp
    } else {
      if (!__any_sync(0xffffffffu, d != 0.0)) return 0.0;  // FP64 adds only for rows that drop
#pragma unroll
      for (int o = W / 2; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o, W);
      return d;
    }
  }
};

constexpr int EX_U = 4;  // entries per lane of a row loaded at once
constexpr int FLT_LPR = 8;  // lanes per row of the candidate pass and the filter write

// Candidates: the entries of the crossing bucket (top 16 bits of the key equal
// to the prefix, 0 < key <= b), appended with one atomic per warp.
// With cnt (the filter of a solve) the same pass also counts, per row, what
// does not depend on where tau falls inside the crossing bucket: entries
// above the bucket or above b are kept (cnt[r]); entries below it are
// dropped, their squares summed into dropped[r] as in k_filter_count. A
// matrix without a crossing already has its tau (the smallest key above b),
// so every entry is decided here. k_sel_cand_keep adds the kept candidates
// once tau is final; the dropped candidates' squares come from the select's
// exact sums (k_sel_drop_fix). Rows of inactive matrices get 0 and 0.
template <typename T>
__global__ void __launch_bounds__(SEL_THREADS)
    k_sel_extract(SelRows R, const int *active, const T *val, const MatScalars *ms,
                  SelScratch sc, int64_t *cnt, double *dropped) {
  __shared__ ChunkRows cr;
  __shared__ unsigned long long s_bkey[RPC], s_top[RPC], s_tkey[RPC];
  __shared__ int s_found[RPC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = SEL_THREADS / 32;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t rpc = chunk_rows(R);
  const int64_t nchunks = (R.nrows + rpc - 1) / rpc;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int64_t r0 = ch * rpc, r1 = min(r0 + rpc, R.nrows);
    __syncthreads();  // the previous chunk's rows are read
    int mt = 0;
    const int t = stage_rows(R, active, r0, r1, cr, mt);
    if (t >= 0) {
      const bool found = active[mt] && sc.st[mt].found != 0;
      const unsigned long long above = sc.minabove[mt];
      s_found[t] = found;
      s_bkey[t] = (unsigned long long)__double_as_longlong(ms[mt].b);
      s_top[t] = found ? sc.st[mt].prefix >> 48 : 0ULL;
      s_tkey[t] = above == ~0ULL ? INF_KEY : above;  // tau without a crossing
    }
    __syncthreads();
    // FLT_LPR lanes per row, 32 / FLT_LPR rows of the chunk per warp at a time
    const int g = lane / FLT_LPR, gl = lane % FLT_LPR;
    const int nr = int(r1 - r0);
    for (int i0 = warp * (32 / FLT_LPR); i0 < nr; i0 += nw * (32 / FLT_LPR)) {
      const int i = i0 + g;
      const bool has = i < nr && (cnt || s_found[i] != 0);
      const int64_t r = r0 + i;
      const bool found = has && s_found[i] != 0;
      // empty for inactive matrices: 0 and 0 written
      const int64_t e0 = has ? cr.b[i] : 0, e1 = has ? cr.e[i] : 0;
      const unsigned long long bkey = has ? s_bkey[i] : 0ULL, top = has ? s_top[i] : 0ULL;
      const unsigned long long tkey = has ? s_tkey[i] : INF_KEY;
      int c = 0;
      DropSum ds;
      for (int64_t p0 = e0;; p0 += FLT_LPR * EX_U) {
        if (!__any_sync(0xffffffffu, p0 < e1)) break;  // every row of the warp done
        T x[EX_U];
#pragma unroll
        for (int u = 0; u < EX_U; ++u) {
          const int64_t p = p0 + FLT_LPR * u + gl;
          x[u] = p < e1 ? val[p] : T(0);  // a zero is neither counted nor dropped
        }
        bool take[EX_U];
#pragma unroll
        for (int u = 0; u < EX_U; ++u) {
          const unsigned long long key = key_t<T>(x[u]);
          take[u] = false;
          if (key == 0ULL) continue;
          bool drop;
          if (found) {
            const unsigned long long t16 = key >> 48;
            take[u] = key <= bkey && t16 == top;
            if (take[u] || !cnt) continue;
            drop = !(key <= INF_KEY && (t16 > top || key > bkey));
          } else {
            drop = !keep_key(key, tkey);
          }
          if (drop)
            ds.add(x[u]);
          else
            ++c;
        }
#pragma unroll
        for (int u = 0; u < EX_U; ++u) {
          const unsigned mask = __ballot_sync(0xffffffffu, take[u]);
          if (!mask) continue;
          unsigned long long base = 0;
          if (lane == 0) base = atomicAdd(sc.ncand, (unsigned long long)__popc(mask));
          base = __shfl_sync(0xffffffffu, base, 0);
          if (take[u]) {
            const unsigned long long slot = base + __popc(mask & lt);
            if (slot < sc.cap) {  // past the room: counted only (the caller retries with more)
              sc.cand[slot] = key_t<T>(x[u]);
              sc.cand_r[slot] = int(r);
            }
          }
        }
      }
      if (!cnt) continue;
#pragma unroll
      for (int o = FLT_LPR / 2; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o, FLT_LPR);
      const double d = ds.group_total<T, FLT_LPR>();
      if (gl == 0 && has) {
        cnt[r] = c;
        dropped[r] = d;
      }
    }
  }
}

// The kept candidates (key >= tau, tau final) into their rows' counts.
__global__ void k_sel_cand_keep(SelRows R, const MatScalars *ms, SelScratch sc, int64_t *cnt) {
  unsigned long long total = *sc.ncand;
  if (total > sc.cap) total = sc.cap;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const int64_t r = sc.cand_r[i];
    const unsigned long long tkey =
        (unsigned long long)__double_as_longlong(ms[row_mat(R, r)].tau);
    if (keep_key(sc.cand[i], tkey))
      atomicAdd(reinterpret_cast<unsigned long long *>(cnt + r), 1ULL);
  }
}

// sums[m] += the squares of the dropped candidates: the exact sum of their q
// (the select's sum below tau minus its sum below the crossing bucket) in
// grid steps 2^(2e - 62). A candidate's magnitude is at least b / sqrt(1.1
// nnz) (a bucket spans a factor 2^(1/16)), so its q is above 2^62 / (1.1 nnz)
// and its flooring to an integer is far below the FP64 rounding of the sum.
__global__ void k_sel_drop_fix(int nb, const int *active, SelScratch sc, const MatScalars *ms,
                               double *sums) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nb || !active[m] || !sc.st[m].found) return;
  const SelState st = sc.st[m];
  const unsigned long long lo = st.below_lo - st.below0_lo;
  const unsigned long long hi = st.below_hi - st.below0_hi - (st.below_lo < st.below0_lo ? 1ULL : 0ULL);
  const double q = __fma_rn(double(hi), 18446744073709551616.0, double(lo));
  sums[m] = __dadd_rn(sums[m], ldexp(q, 2 * (ms[m].sel_e - 1023) - 62));
}

__global__ void k_sel_hist_digit(SelRows R, const MatScalars *ms, SelScratch sc, int shift) {
  unsigned long long total = *sc.ncand;
  if (total > sc.cap) total = sc.cap;
  for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    int m = row_mat(R, sc.cand_r[i]);
    unsigned long long key = sc.cand[i];
    if ((key >> (shift + 8)) != (sc.st[m].prefix >> (shift + 8))) continue;
    int d = int((key >> shift) & 255ULL);
    unsigned long long q = qval<double>(key, ms[m].sel_e);
    if (q) add128(sc.hdig + (size_t(m) * NDIG + d) * 2, q, 0ULL);
  }
}

// One warp per matrix: the digit at `shift` where the sums cross Q.
__global__ void k_sel_find_digit(int nb, const MatScalars *ms, SelScratch sc, int shift) {
  const int m = int((int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5);
  if (m >= nb) return;
  SelState &st = sc.st[m];
  if (!st.found) return;
  unsigned long long lo = st.below_lo, hi = st.below_hi;
  unsigned long long *h = sc.hdig + size_t(m) * NDIG * 2;
  const int d = warp_crossing(h, NDIG, ms[m].sel_q, lo, hi);
  __syncwarp();
  // the buckets are read: cleared here for the next digit, instead of a memset
  for (int c = threadIdx.x & 31; c < 2 * NDIG; c += 32) h[c] = 0ULL;
  if (d >= 0 && (threadIdx.x & 31) == 0) {
    st.prefix |= (unsigned long long)d << shift;
    st.below_lo = lo;
    st.below_hi = hi;
  }
}

__global__ void k_sel_final(int nb, const int *active, SelScratch sc, MatScalars *ms) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nb || !active[m]) return;
  if (sc.st[m].found) {
    ms[m].tau = __longlong_as_double((long long)sc.st[m].prefix);
  } else {
    unsigned long long k = sc.minabove[m];
    ms[m].tau = k == ~0ULL ? __longlong_as_double(0x7ff0000000000000LL)
                           : __longlong_as_double((long long)k);
  }
}

// ------------------------------------------------------------ filter
__global__ void k_filter_count(int64_t n, const int32_t *seg, const int *active,
                               const int64_t *rs, const int64_t *re, const void *val, int f32,
                               const MatScalars *ms, int64_t *cnt, double *dropped) {
  int lane = lane_id();
  int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = warp; r < n; r += nwarps) {
    int m = seg[r];
    const unsigned long long tkey = (unsigned long long)__double_as_longlong(ms[m].tau);
    int c = 0;
    double d2 = 0.0;
    if (active[m] && f32) {
      const float *v = static_cast<const float *>(val);
      float hi = 0.0f, lo = 0.0f;  // dropped squares, scaled by 2^96
      const int64_t pe = re[r];
#pragma unroll 4
      for (int64_t p = rs[r] + lane; p < pe; p += 32) {
        const float x = v[p];
        const unsigned long long key = key_f32(x);
        if (keep_key(key, tkey))
          ++c;
        else if (key != 0ULL)
          ff_add_sq48(x, hi, lo);
      }
      c = __reduce_add_sync(0xffffffffu, c);
      if (__any_sync(0xffffffffu, hi != 0.0f)) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
          const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
          ff_add(hi, lo, h2, l2);
        }
        if (lane == 0) d2 = (double(hi) + double(lo)) * 0x1p-96;  // exact scaling, one rounding as ldexp
      }
    } else if (active[m]) {
      const double *v = static_cast<const double *>(val);
      const int64_t pe = re[r];
#pragma unroll 4
      for (int64_t p = rs[r] + lane; p < pe; p += 32) {
        double x = v[p];
        if (keep_key(key_f64(x), tkey))
          ++c;
        else
          d2 = __fma_rn(x, x, d2);
      }
      c = __reduce_add_sync(0xffffffffu, c);
      if (__any_sync(0xffffffffu, d2 != 0.0)) {  // FP64 adds only for rows that drop
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d2 += __shfl_xor_sync(0xffffffffu, d2, o);
      }
    }
    if (lane == 0) {
      cnt[r] = c;
      dropped[r] = d2;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(SEL_THREADS)
    k_filter_write(int64_t n, const int32_t *seg, const int *active, const int64_t *rs,
                   const int64_t *re, const int32_t *col, const T *val, const MatScalars *ms,
                   const int64_t *orp, int32_t *ocol, T *oval) {
  __shared__ ChunkRows cr;
  __shared__ int64_t s_out[RPC], s_oend[RPC];
  __shared__ unsigned long long s_tkey[RPC];
  const int lane = lane_id(), warp = threadIdx.x >> 5, nw = SEL_THREADS / 32;
  const SelRows R{n, seg, rs, re, 0};
  const int64_t nchunks = (n + RPC - 1) / RPC;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int64_t r0 = ch * RPC, r1 = min(r0 + RPC, n);
    __syncthreads();  // the previous chunk's rows are read
    int mt = 0;
    const int t = stage_rows(R, active, r0, r1, cr, mt);
    if (t >= 0) {
      s_out[t] = orp[r0 + t];
      s_oend[t] = orp[r0 + t + 1];
      s_tkey[t] = (unsigned long long)__double_as_longlong(ms[mt].tau);
    }
    __syncthreads();
    // FLT_LPR lanes per row, 32 / FLT_LPR rows of the chunk per warp at a time
    const int g = lane / FLT_LPR, gl = lane % FLT_LPR;
    const unsigned gbits = (1u << FLT_LPR) - 1u, glt = (1u << gl) - 1u;
    const int nr = int(r1 - r0);
    for (int i0 = warp * (32 / FLT_LPR); i0 < nr; i0 += nw * (32 / FLT_LPR)) {
      const int i = i0 + g;
      const bool has = i < nr;
      // the row's room from the counts; the same rule decides both, and the
      // bound keeps a write inside the row whatever the values are
      const unsigned long long tkey = has ? s_tkey[i] : INF_KEY;
      int64_t out = has ? s_out[i] : 0;
      const int64_t oend = has ? s_oend[i] : 0, b = has ? cr.b[i] : 0, e = has ? cr.e[i] : 0;
      for (int64_t p0 = b;; p0 += FLT_LPR * EX_U) {
        if (!__any_sync(0xffffffffu, p0 < e)) break;  // every row of the warp done
        T x[EX_U];
        int32_t c[EX_U];
#pragma unroll
        for (int u = 0; u < EX_U; ++u) {
          const int64_t p = p0 + FLT_LPR * u + gl;
          x[u] = p < e ? val[p] : T(0);  // a zero is never kept
          c[u] = p < e ? col[p] : 0;
        }
#pragma unroll
        for (int u = 0; u < EX_U; ++u) {
          const bool keep = keep_key(key_t<T>(x[u]), tkey);
          const unsigned gm = (__ballot_sync(0xffffffffu, keep) >> (g * FLT_LPR)) & gbits;
          const int64_t pos = out + __popc(gm & glt);
          if (keep && pos < oend) {
            ocol[pos] = c[u];
            oval[pos] = x[u];
          }
          out += __popc(gm);
        }
      }
    }
  }
}

int grid_for(int64_t items, int per_block, int cap = 152 * 16) {
  int64_t g = (items + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  return int(g);
}

__global__ void k_store_nnz_bar(int nb, const int64_t *nnz, MatScalars *ms) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < nb) ms[m].nnz_bar = nnz[m];
}

}  // namespace

void launch_matrix_scalars(int nb, const int64_t *moff, const double *sums, double c4,
                           double tol_stage, double switch_resid, MatScalars *ms, cudaStream_t s) {
  k_matrix_scalars<<<(nb + 127) / 128, 128, 0, s>>>(nb, moff, sums, c4, tol_stage, switch_resid,
                                                    ms);
  SGN_LAUNCH_CHECK();
}

void launch_store_nnz_bar(int nb, const int64_t *nnz, MatScalars *ms, cudaStream_t s) {
  k_store_nnz_bar<<<(nb + 127) / 128, 128, 0, s>>>(nb, nnz, ms);
  SGN_LAUNCH_CHECK();
}

void launch_select_bound(int nb, const int *active, MatScalars *ms, cudaStream_t s) {
  k_select_bound<<<(nb + 127) / 128, 128, 0, s>>>(nb, active, ms);
  SGN_LAUNCH_CHECK();
}

const unsigned long long *select_cand_count(void *scratch, int nb) {
  return carve(scratch, nb, 1).ncand;
}

void launch_select_exact(int nb, const SelRows &R, int64_t cand_cap, const int *active,
                         const void *val, int val_f32, MatScalars *ms, void *scratch,
                         int64_t *cnt, double *dropped, cudaStream_t s) {
  SelScratch sc = carve(scratch, nb, cand_cap);
  SGN_CUDA(cudaMemsetAsync(sc.hist0, 0, size_t(nb) * NB0 * 2 * 8, s));
  SGN_CUDA(cudaMemsetAsync(sc.minabove, 0xff, size_t(nb) * 8, s));
  k_sel_prepare<<<(nb + 127) / 128, 128, 0, s>>>(nb, ms);
  SGN_LAUNCH_CHECK();
  const int64_t rpc = R.rs ? RPC : 32;
  {
    ProfScope ps(KC_SEL_HIST, s, 0.0, 0.0);
    if (R.nrows > 0) {
      const int g = grid_for((R.nrows + rpc - 1) / rpc, 1, 152 * 8);
      if (val_f32)
        k_sel_hist0<float><<<g, SEL_THREADS, 0, s>>>(R, active, static_cast<const float *>(val),
                                                     ms, sc);
      else
        k_sel_hist0<double><<<g, SEL_THREADS, 0, s>>>(R, active,
                                                      static_cast<const double *>(val), ms, sc);
      SGN_LAUNCH_CHECK();
    }
    k_sel_find0<<<(nb + 3) / 4, 128, 0, s>>>(nb, active, ms, sc);
    SGN_LAUNCH_CHECK();
  }
  {
    ProfScope ps(KC_SEL_EXTRACT, s, 0.0, 0.0);
    if (R.nrows > 0) {
      const int g = grid_for((R.nrows + rpc - 1) / rpc, 1, 152 * 8);
      if (val_f32)
        k_sel_extract<float><<<g, SEL_THREADS, 0, s>>>(R, active, static_cast<const float *>(val),
                                                       ms, sc, cnt, dropped);
      else
        k_sel_extract<double><<<g, SEL_THREADS, 0, s>>>(
            R, active, static_cast<const double *>(val), ms, sc, cnt, dropped);
      SGN_LAUNCH_CHECK();
    }
  }
  ProfScope ps(KC_SEL_DIGITS, s, 0.0, 0.0);
  // zeroed once; after each level the matrices that fill buckets (those with
  // a crossing) clear them again in k_sel_find_digit
  SGN_CUDA(cudaMemsetAsync(sc.hdig, 0, size_t(nb) * NDIG * 2 * 8, s));
  for (int level = 0; level < 6; ++level) {
    int shift = 40 - 8 * level;
    k_sel_hist_digit<<<152 * 4, 256, 0, s>>>(R, ms, sc, shift);
    SGN_LAUNCH_CHECK();
    k_sel_find_digit<<<(nb + 3) / 4, 128, 0, s>>>(nb, ms, sc, shift);
    SGN_LAUNCH_CHECK();
  }
  k_sel_final<<<(nb + 127) / 128, 128, 0, s>>>(nb, active, sc, ms);
  SGN_LAUNCH_CHECK();
  if (cnt) {
    k_sel_cand_keep<<<152 * 2, 256, 0, s>>>(R, ms, sc, cnt);
    SGN_LAUNCH_CHECK();
  }
}

void launch_select_drop_fix(int nb, const int *active, void *scratch, const MatScalars *ms,
                            double *sums, cudaStream_t s) {
  k_sel_drop_fix<<<(nb + 127) / 128, 128, 0, s>>>(nb, active, carve(scratch, nb, 1), ms, sums);
  SGN_LAUNCH_CHECK();
}

void launch_filter_count(int64_t n, const int32_t *seg, const int *active, const int64_t *rs,
                         const int64_t *re, const void *val, int val_f32, const MatScalars *ms,
                         int64_t *cnt, double *dropped, cudaStream_t s) {
  if (n == 0) return;
  k_filter_count<<<grid_for(n, 8), 256, 0, s>>>(n, seg, active, rs, re, val, val_f32, ms, cnt,
                                                 dropped);
  SGN_LAUNCH_CHECK();
}

void launch_filter_write(int64_t n, const int32_t *seg, const int *active, const int64_t *rs,
                         const int64_t *re, const int32_t *col, const void *val, int val_f32,
                         const MatScalars *ms, const int64_t *orp, int32_t *ocol, void *oval,
                         cudaStream_t s) {
  if (n == 0) return;
  if (val_f32)
    k_filter_write<float><<<grid_for(n, RPC, 152 * 8), SEL_THREADS, 0, s>>>(
        n, seg, active, rs, re, col, static_cast<const float *>(val), ms, orp, ocol,
        static_cast<float *>(oval));
  else
    k_filter_write<double><<<grid_for(n, RPC, 152 * 8), SEL_THREADS, 0, s>>>(
        n, seg, active, rs, re, col, static_cast<const double *>(val), ms, orp, ocol,
        static_cast<double *>(oval));
  SGN_LAUNCH_CHECK();
}

}  // namespace sgn
