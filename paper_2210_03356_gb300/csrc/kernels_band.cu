// Band tiles: the FP32 sparse products (steps a2 and a3) of rows whose
// operands are narrow bands, computed as small dense products.
//
// The filtered iterates of banded inputs keep a band around the diagonal that
// is almost full (about 97% of the positions between a row's first and last
// column hold an entry), and their rows are short (tens to a few hundred
// entries). The row-wise gather product then spends most of its instructions
// on per-k bookkeeping. Here 16 consecutive rows form a tile; for each chunk
// of 32 output columns the tile's rows of A and the rows of B that reach the
// chunk are staged densely in shared memory (zeros in the holes), and every
// lane accumulates a 4 x 4 block of outputs in registers with one fused
// multiply-add per k, in ascending k.
//
// Why the values are those of the row-wise product bit for bit: an output
// c_ij receives fma(a_ik, b_kj, c) for every k of the chunk's k range in
// ascending order, starting from +0. For a k with a_ik or b_kj not stored,
// the staged operand is +0, so a_ik b_kj is an exact zero and the fma returns
// c unchanged (c is never -0: a sum that starts at +0 cannot become -0 under
// round-to-nearest). What remains is the stored products in ascending k, one
// fused multiply-add each, as in the oracle's Gustavson product.
//
// The pattern (the entries the product creates, exact zeros included) comes
// from bit masks: row i of C holds column j iff some stored k of A_i has j
// stored in B_k; in an update also iff x_ij is stored (Xbar = 1.5 X - 0.5 X T
// on the union pattern). The outputs go into the row slots of the other
// product kernels, in ascending column order.
#include <climits>

#include "common.cuh"
#include "kernels.h"

namespace sgn {

namespace {

constexpr int BT_WARPS = 2;     // warps per CTA, each on tiles of its own
constexpr int BT_CTAS = 6;      // CTAs per SM (shared memory: ~18.5 KB per warp)
constexpr int BT_KS = 32;       // k per slab
constexpr int BT_AST = BT_KS + 4;  // row stride of the A slab (16-byte rows)

__device__ __forceinline__ float ns_combine_f(float x, float p) {
  return __fsub_rn(__fmul_rn(1.5f, x), __fmul_rn(0.5f, p));
}

// The float-pair sum of squares of the other FP32 product kernels: v^2 =
// p + e exactly, accumulated with an error-free two-sum (~48 bits).
struct SqPair {
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

__device__ __forceinline__ int warp_min(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_max(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------------- band layout
__global__ void k_band_spans(int64_t n, const int64_t *rs, const int64_t *re, const int32_t *col,
                             int32_t *fc, int32_t *nf, int64_t *span) {
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
       r += int64_t(gridDim.x) * blockDim.x) {
    int64_t a = rs[r], b = re[r];
    int32_t f = 0, w = 0;
    if (b > a) {
      int32_t first = col[a], last = col[b - 1];
      f = first & ~3;
      w = ((last + 4) & ~3) - f;
    }
    fc[r] = f;
    nf[r] = w;
    span[r] = w;
  }
}

// The band layout of the rows of a product from their column ranges
// [lo, lo + len): the first and last column of a product row are stored
// entries (each is the first or last column of some B_k), so this is the
// layout k_band_spans gives for the finished rows.
__global__ void k_band_spans_range(int64_t n, const int32_t *lo, const int32_t *len, int32_t *fc,
                                   int32_t *nf, int64_t *span) {
  for (int64_t r = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
       r += int64_t(gridDim.x) * blockDim.x) {
    const int32_t L = len[r];
    int32_t f = 0, w = 0;
    if (L > 0) {
      f = lo[r] & ~3;
      w = ((lo[r] + L - 1 + 4) & ~3) - f;
    }
    fc[r] = f;
    nf[r] = w;
    span[r] = w;
  }
}

constexpr int FILL_LPR = 8;  // lanes per row of the band layout

// FILL_LPR lanes per row (rows with skip[r] set are left alone): the row's
// band and pattern words are cleared, then its values scattered and its
// pattern bits OR-ed in (one atomic per run of a word's columns).

__global__ void k_band_fill(int64_t n, const int64_t *rs, const int64_t *re, const int32_t *col,
                            const float *val, const int64_t *pos, const int32_t *fc,
                            const int32_t *nf, const unsigned char *skip, float *bval,
                            unsigned *bmask) {
  // FILL_LPR lanes per row, 32 / FILL_LPR rows per warp at a time
  constexpr int L = FILL_LPR;
  const int lane = threadIdx.x & 31, g = lane / L, gl = lane % L;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  for (int64_t r0 = warp * (32 / L); r0 < n; r0 += nwarps * (32 / L)) {
    const int64_t r = r0 + g;
    const int32_t w = r < n ? nf[r] : 0;
    const bool has = w > 0 && !(skip && skip[r]);
    const int64_t a = has ? rs[r] : 0, b = has ? re[r] : 0;
    const int64_t p0 = has ? pos[r] : 0;
    const int32_t f = has ? fc[r] : 0;
    if (has) {
      float4 *z = reinterpret_cast<float4 *>(bval + p0);
      for (int t = gl; t < w / 4; t += L) z[t] = make_float4(0.f, 0.f, 0.f, 0.f);
      unsigned *dz = bmask + p0 / 2 - (f >> 5);
      for (int x = (f >> 5) + gl; x <= (f + w - 1) >> 5; x += L) dz[x] = 0u;
    }
    __syncwarp();
    unsigned *dm = bmask + p0 / 2 - (f >> 5);
    float *dv = bval + p0 - f;
    for (int64_t p = a;; p += L) {
      if (!__any_sync(0xffffffffu, p < b)) break;  // every row of the warp done
      const bool ok = p + gl < b;
      int32_t c = ok ? col[p + gl] : INT_MAX;
      if (ok) dv[c] = val[p + gl];
      int wd = ok ? (c >> 5) : INT_MAX;
      unsigned bits = ok ? (1u << (c & 31)) : 0u;
      // suffix OR over the group's lanes holding the same word (columns ascend)
#pragma unroll
      for (int d = 1; d < L; d <<= 1) {
        unsigned ob = __shfl_down_sync(0xffffffffu, bits, d, L);
        int ow = __shfl_down_sync(0xffffffffu, wd, d, L);
        if (gl + d < L && ow == wd) bits |= ob;
      }
      int pw = __shfl_up_sync(0xffffffffu, wd, 1, L);
      if (ok && (gl == 0 || pw != wd)) atomicOr(dm + wd, bits);
    }
  }
}

// ---------------------------------------------------------------- tile product
// 16-byte global -> shared copy that completes asynchronously; src_bytes = 0
// writes 16 zero bytes and reads nothing.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(gmem),
               "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

struct BandSmem {
  float a[2][16][BT_AST];          // A slabs: a[i][kk] = a_{r0+i, k0+kk}
  float b[2][BT_KS][32];           // B slabs: b[kk][j] = b_{k0+kk, j0+j}
  unsigned bm[2][BT_KS];           // pattern word of B row k0+kk over the chunk's columns
  unsigned am[2][16][2];           // pattern words of A row r0+i holding k0 .. k0+31
  int64_t koff[BAND_KT + 4];       // band of B row kb + t: B.val + koff[t] ...
  int32_t kfc[BAND_KT + 4], kend[BAND_KT + 4];  // ... over columns [kfc[t], kend[t])
  int64_t aoff[16];                // band of A row r0 + i at A.val + aoff[i]
  int32_t afc[16], aend[16];
  int64_t coff[16];                // (SQUARE) band of C row r0 + i being written
  int32_t cfc[16], cend[16];
};
static_assert(sizeof(BandSmem) % 16 == 0, "per-warp areas stay 16-byte aligned");
static_assert(BT_CTAS * (BT_WARPS * sizeof(BandSmem) + 1024) <= 228 * 1024, "CTAs per SM fit");

// 4-byte copy of the same kind (a pattern word; zero when src_bytes = 0)
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem, int src_bytes) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(gmem),
               "r"(src_bytes)
               : "memory");
}

template <int MODE>
__global__ void __launch_bounds__(BT_WARPS * 32, BT_CTAS)
    k_band(const int64_t *ars, const int64_t *are, const int32_t *acol, const float *aval,
           Band A, Band B, BandOut Cb, const int32_t *lo, const int32_t *len,
           const int32_t *list, int *counters, int cls, const int64_t *cs, int64_t *ce,
           int32_t *ccol, float *cval, double *part) {
  extern __shared__ __align__(16) unsigned char band_smem[];
  BandSmem &sm = reinterpret_cast<BandSmem *>(band_smem)[threadIdx.x >> 5];
  constexpr unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int rg = lane >> 3, cg = lane & 7;  // rows rg*4.., columns cg*4.. of a chunk
  const int hi = lane & 15, hh = lane >> 4;  // row and half of the pattern phase
  const int total = counters[cls];
  for (;;) {
    int idx = 0;
    if (lane == 0) idx = atomicAdd(&counters[RC_QUEUE + cls], 1);
    idx = __shfl_sync(FULL, idx, 0);
    if (idx >= total) break;
    const int32_t r0 = list[idx];
    // lane i < 16 holds row r0 + i
    int Li = 0, c0i = 0;
    int64_t a0i = 0, a1i = 0, outi = 0;
    if (lane < 16) {
      const int32_t r = r0 + lane;
      Li = len[r];
      c0i = lo[r];
      a0i = ars[r];
      a1i = are[r];
      outi = cs[r];
    }
    const int jlo = warp_min(Li > 0 ? c0i : INT_MAX);
    const int jhi = warp_max(Li > 0 ? c0i + Li - 1 : -1);
    const int kt0 = warp_min(a1i > a0i ? acol[a0i] : INT_MAX);
    const int kt1 = warp_max(a1i > a0i ? acol[a1i - 1] : -1);
    if (jhi < 0 || kt1 < 0) continue;  // no output (every row's slot is empty)
    // k_bounds guarantees kt1 - kt0 < BAND_KT - 3, so nkm <= BAND_KT
    const int jw0 = jlo >> 5, nw = (jhi >> 5) - jw0 + 1;
    const int kb = kt0 & ~3, nkm = kt1 - kb + 1;

    // ---- stage the bands' row descriptors
    for (int t = lane; t < nkm; t += 32) {
      const int32_t f = B.fc[kb + t];
      sm.kfc[t] = f;
      sm.kend[t] = f + B.nf[kb + t];
      sm.koff[t] = B.pos[kb + t] - f;
    }
    if (lane < 16) {
      const int32_t f = A.fc[r0 + lane];
      sm.afc[lane] = f;
      sm.aend[lane] = f + A.nf[r0 + lane];
      sm.aoff[lane] = A.pos[r0 + lane] - f;
    } else if (MODE == MODE_SQUARE && Cb.val) {
      const int32_t i = lane - 16, f = Cb.fc[r0 + i];
      sm.cfc[i] = f;
      sm.cend[i] = f + Cb.nf[r0 + i];
      sm.coff[i] = Cb.pos[r0 + i] - f;
    }
    __syncwarp();

    // ---- (SQUARE) ||x_i||^2: lane (hi, hh) sums every other entry of row hi
    double my_xs = 0.0;
    if (MODE == MODE_SQUARE) {
      const int64_t a0 = __shfl_sync(FULL, a0i, hi), a1 = __shfl_sync(FULL, a1i, hi);
      SqPair xacc;
#pragma unroll 4
      for (int64_t p = a0 + hh; p < a1; p += 2) xacc.add_sq(aval[p]);
      my_xs = xacc.value();
      my_xs += __shfl_xor_sync(FULL, my_xs, 16);  // lanes hi and hi + 16 hold row hi
    }
    SqPair racc[4];
    double rdiag[4] = {0.0, 0.0, 0.0, 0.0};
    bool hasdiag[4] = {false, false, false, false};

    // ---- chunks of 32 output columns; k slabs double-buffered with cp.async
    auto krange = [&](int j0, int &klo, int &khi) {
      // rows of B (within the tile's k hull) with a band position in [j0, j0+32)
      int l = INT_MAX, h = -1;
      for (int t = (kt0 - kb) + lane; t < nkm; t += 32) {
        if (sm.kfc[t] < j0 + 32 && sm.kend[t] > j0) {
          l = min(l, t);
          h = max(h, t);
        }
      }
      klo = warp_min(l);
      khi = warp_max(h);
    };
    // queues the copies of slab [ks, ks + 32) x [j0, j0 + 32) into buffer bf
    auto issue = [&](int bf, int j0, int ks) {  // ks relative to kb, a multiple of 4
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int item = lane + 32 * m, i = item >> 3, u = item & 7;
        const int k = kb + ks + 4 * u;
        const bool in = k >= sm.afc[i] && k < sm.aend[i];
        const float *src = A.val + (in ? sm.aoff[i] + k : 0);
        cp_async16(&sm.a[bf][i][4 * u], src, in ? 16 : 0);
      }
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int item = lane + 32 * m, kk = item >> 3, u = item & 7;
        const int t = ks + kk, j = j0 + 4 * u;
        const bool in = t < nkm && j >= sm.kfc[t] && j < sm.kend[t];
        const float *src = B.val + (in ? sm.koff[t] + j : 0);
        cp_async16(&sm.b[bf][kk][4 * u], src, in ? 16 : 0);
      }
      {  // pattern word of B row ks + lane over the chunk (word j0 / 32)
        const int t = ks + lane, wj = j0 >> 5;
        bool in = t < nkm && sm.kend[t] > sm.kfc[t];
        int64_t at = 0;
        if (in) {
          const int wf = sm.kfc[t] >> 5;
          in = wj >= wf && wj <= (sm.kend[t] - 1) >> 5;
          at = (sm.koff[t] + sm.kfc[t]) / 2 + (wj - wf);
        }
        cp_async4(&sm.bm[bf][lane], B.mask + at, in ? 4 : 0);
      }
      {  // pattern words of A row hi holding k = kb + ks .. kb + ks + 31
        const int wk = ((kb + ks) >> 5) + hh, f = sm.afc[hi], e = sm.aend[hi];
        bool in = e > f;
        int64_t at = 0;
        if (in) {
          const int wf = f >> 5;
          in = wk >= wf && wk <= (e - 1) >> 5;
          at = (sm.aoff[hi] + f) / 2 + (wk - wf);
        }
        cp_async4(&sm.am[bf][hi][hh], A.mask + at, in ? 4 : 0);
      }
      cp_async_commit();
    };
    // the slab sequence: chunk c, k from ks to kend (relative to kb)
    int c = 0, klo = 0, khi = -1;
    auto next_chunk = [&](int cc, int &lo_, int &hi_) {  // first chunk >= cc with a k range
      while (cc < nw) {
        krange((jw0 + cc) * 32, lo_, hi_);
        if (hi_ >= lo_) break;
        ++cc;
      }
      return cc;
    };
    c = next_chunk(0, klo, khi);
    int ks = klo & ~3;
    int bf = 0;
    if (c < nw) issue(0, (jw0 + c) * 32, ks);
    for (int cc = 0; cc < nw; ++cc) {
      float acc[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] = 0.0f;
      unsigned patw = 0u;  // lane (hi, hh): part of row hi's pattern word of the chunk
      if (cc == c) {
        // the slabs of this chunk
        for (;;) {
          const int nk4 = min(BT_KS, ((khi + 1 - ks) + 3) & ~3);
          // queue the next slab (of this chunk or the next) before computing
          int nc = c, nklo = klo, nkhi = khi, nks = ks + BT_KS;
          if (nks > khi) {
            nc = next_chunk(c + 1, nklo, nkhi);
            nks = nklo & ~3;
          }
          if (nc < nw) {
            issue(bf ^ 1, (jw0 + nc) * 32, nks);
            cp_async_wait<1>();
          } else {
            cp_async_wait<0>();
          }
          __syncwarp();
          {  // the chunk's pattern: B words of the stored k of row hi (every other)
            const unsigned sh = unsigned(kb + ks) & 31u;
            const unsigned m = __funnelshift_r(sm.am[bf][hi][0], sm.am[bf][hi][1], sh);
            // the 16 k of this lane's half, unrolled: independent loads, no chain
#pragma unroll
            for (int t = 0; t < 32; t += 2) {
              const int tt = t + hh;
              const unsigned bw = sm.bm[bf][tt];
              patw |= ((m >> tt) & 1u) ? bw : 0u;
            }
          }
          for (int kk = 0; kk < nk4; kk += 4) {
            float4 av[4], bv[4];
#pragma unroll
            for (int r = 0; r < 4; ++r)
              av[r] = *reinterpret_cast<const float4 *>(&sm.a[bf][rg * 4 + r][kk]);
#pragma unroll
            for (int q = 0; q < 4; ++q)
              bv[q] = *reinterpret_cast<const float4 *>(&sm.b[bf][kk + q][cg * 4]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {  // ascending k
#pragma unroll
              for (int r = 0; r < 4; ++r) {
                const float a = q == 0 ? av[r].x : q == 1 ? av[r].y : q == 2 ? av[r].z : av[r].w;
                acc[r][0] = __fmaf_rn(a, bv[q].x, acc[r][0]);
                acc[r][1] = __fmaf_rn(a, bv[q].y, acc[r][1]);
                acc[r][2] = __fmaf_rn(a, bv[q].z, acc[r][2]);
                acc[r][3] = __fmaf_rn(a, bv[q].w, acc[r][3]);
              }
            }
          }
          __syncwarp();  // the buffer is free for the copy after next
          bf ^= 1;
          const bool same = nc == c;
          c = nc;
          klo = nklo;
          khi = nkhi;
          ks = nks;
          if (!same) break;
        }
      }
      // ---- emit chunk cc: row slots in ascending column order
      const int j0 = (jw0 + cc) * 32;
      patw |= __shfl_xor_sync(FULL, patw, 16);
      if (MODE == MODE_UPDATE) {  // the union with X_i's own pattern
        const int f = sm.afc[hi], e = sm.aend[hi], wj = j0 >> 5;
        if (e > f && wj >= (f >> 5) && wj <= (e - 1) >> 5)
          patw |= A.mask[(sm.aoff[hi] + f) / 2 + (wj - (f >> 5))];
      }
      if (MODE == MODE_SQUARE && Cb.val) {
        // the rows' band (values at every position of the band, +0 outside
        // the pattern, where every product was zero) and pattern words
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int ri = rg * 4 + r;
          const int j = j0 + cg * 4;
          if (j >= sm.cfc[ri] && j < sm.cend[ri])
            *reinterpret_cast<float4 *>(Cb.val + sm.coff[ri] + j) =
                make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
        }
        if (lane < 16) {
          const int32_t f = sm.cfc[lane], e = sm.cend[lane], wj = j0 >> 5;
          if (e > f && wj >= (f >> 5) && wj <= (e - 1) >> 5)
            Cb.mask[(sm.coff[lane] + f) / 2 + (wj - (f >> 5))] = patw;
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int ri = rg * 4 + r;
        const unsigned wbits = __shfl_sync(FULL, patw, ri);
        int64_t pos = __shfl_sync(FULL, outi, ri) + __popc(wbits & ((1u << (cg * 4)) - 1u));
        const unsigned bits = (wbits >> (cg * 4)) & 15u;
        float xv[4] = {0.f, 0.f, 0.f, 0.f};
        if (MODE == MODE_UPDATE && bits) {
          const int j = j0 + cg * 4;
          if (j >= sm.afc[ri] && j < sm.aend[ri]) {
            const float4 v = *reinterpret_cast<const float4 *>(A.val + sm.aoff[ri] + j);
            xv[0] = v.x;
            xv[1] = v.y;
            xv[2] = v.z;
            xv[3] = v.w;
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (!((bits >> q) & 1u)) continue;
          const int32_t cj = j0 + cg * 4 + q;
          const float v = MODE == MODE_UPDATE ? ns_combine_f(xv[q], acc[r][q]) : acc[r][q];
          ccol[pos] = cj;
          cval[pos] = v;
          ++pos;
          if (MODE == MODE_SQUARE) {
            if (cj == r0 + ri) {  // (t_ii - 1)^2 in FP64, once per row
              const double d = double(v) - 1.0;
              rdiag[r] = d * d;
              hasdiag[r] = true;
            } else {
              racc[r].add_sq(v);
            }
          }
        }
      }
      outi += __popc(patw);  // lanes < 16: row lane
    }
    if (lane < 16 && Li > 0) ce[r0 + lane] = outi;
    if (MODE == MODE_SQUARE) {
      // per row: the 8 lanes of its row group hold its column groups
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        double rs = racc[r].value() + rdiag[r];
        int any = hasdiag[r] ? 1 : 0;
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
          rs += __shfl_xor_sync(FULL, rs, o);
          any |= __shfl_xor_sync(FULL, any, o);
        }
        const int ri = rg * 4 + r;
        const double xs = __shfl_sync(FULL, my_xs, ri);
        const int Lr = __shfl_sync(FULL, Li, ri);
        if (cg == 0 && Lr > 0) {
          part[2 * int64_t(r0 + ri)] = any ? rs : rs + 1.0;
          part[2 * int64_t(r0 + ri) + 1] = xs;
        }
      }
    }
    __syncwarp();
  }
}

int sm_count_band() {
  static const int n = [] {
    int dev = 0, v = 0;
    SGN_CUDA(cudaGetDevice(&dev));
    SGN_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    return v;
  }();
  return n;
}

}  // namespace

void launch_band_spans(int64_t n, const Rows &R, int32_t *fc, int32_t *nf, int64_t *span,
                       cudaStream_t s) {
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > int64_t(sm_count_band()) * 8) g = int64_t(sm_count_band()) * 8;
  k_band_spans<<<unsigned(g), 256, 0, s>>>(n, R.rs, R.re, R.col, fc, nf, span);
  SGN_LAUNCH_CHECK();
}

void launch_band_spans_range(int64_t n, const int32_t *lo, const int32_t *len, int32_t *fc,
                             int32_t *nf, int64_t *span, cudaStream_t s) {
  if (n == 0) return;
  int64_t g = (n + 255) / 256;
  if (g > int64_t(sm_count_band()) * 8) g = int64_t(sm_count_band()) * 8;
  k_band_spans_range<<<unsigned(g), 256, 0, s>>>(n, lo, len, fc, nf, span);
  SGN_LAUNCH_CHECK();
}

void launch_band_fill(int64_t n, const Rows &R, const float *val, const int64_t *pos,
                      const int32_t *fc, const int32_t *nf, const unsigned char *skip, float *bval,
                      unsigned *bmask, cudaStream_t s) {
  if (n == 0) return;
  int64_t g = (n + 8 * (32 / FILL_LPR) - 1) / (8 * (32 / FILL_LPR));  // 8 warps per CTA
  if (g > int64_t(sm_count_band()) * 16) g = int64_t(sm_count_band()) * 16;
  k_band_fill<<<unsigned(g), 256, 0, s>>>(n, R.rs, R.re, R.col, val, pos, fc, nf, skip, bval,
                                          bmask);
  SGN_LAUNCH_CHECK();
}

void launch_band_product(int64_t n, int mode, const Rows &A, const float *aval, const Band &bandA,
                         const Band &bandB, const BandOut &bandC, const int32_t *lo,
                         const int32_t *len, const int32_t *lists, int *counters,
                         const int64_t *cs, int64_t *ce, int32_t *ccol, float *cval, double *part,
                         cudaStream_t s) {
  if (n == 0) return;
  const int32_t *list = lists + int64_t(RC_BAND) * n;
  constexpr size_t smem = sizeof(BandSmem) * BT_WARPS;
  static const bool attr = [] {  // once, thread-safe
    SGN_CUDA(cudaFuncSetAttribute(k_band<MODE_SQUARE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(smem)));
    SGN_CUDA(cudaFuncSetAttribute(k_band<MODE_UPDATE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(smem)));
    return true;
  }();
  (void)attr;
  const int g = sm_count_band() * BT_CTAS;
  if (mode == MODE_SQUARE)
    k_band<MODE_SQUARE><<<g, BT_WARPS * 32, smem, s>>>(A.rs, A.re, A.col, aval, bandA, bandB,
                                                       bandC, lo, len, list, counters, RC_BAND, cs,
                                                       ce, ccol, cval, part);
  else
    k_band<MODE_UPDATE><<<g, BT_WARPS * 32, smem, s>>>(A.rs, A.re, A.col, aval, bandA, bandB,
                                                       BandOut{}, lo, len, list, counters, RC_BAND,
                                                       cs, ce, ccol, cval, part);
  SGN_LAUNCH_CHECK();
}

}  // namespace sgn
