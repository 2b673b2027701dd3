// FP64-accurate dense products on the BF16 tensor cores, from exact integer
// slices (the error-free splitting of matrix products published by Ozaki,
// Ogita, Oishi and Rump, 2012), for matrices on the dense path in the FP64
// stage. GB300 runs FP64 at about 1/64 of its FP32 rate; this path moves the
// FP64 products of filled-in iterates to the tensor cores.
//
// Splitting. Row i of A (M x K) is scaled by its power of two 2^e_i >
// max_k |a_ik| and rounded to the grid 2^(e_i - 55); the integer q_ik
// (|q| < 2^55) is written as eight balanced base-128 digits,
//   a_ik ~= 2^(e_i + 1) * sum_{s=1..8} d_ik^(s) 2^(-7 s),   |d| <= 64,
// and likewise the rows of Bt (N x K) with 2^(f_j + 1). Every digit is a
// small integer, exact in BF16.
//
// Products. For a digit pair (s, t) the tensor cores form the integer matrix
// D_s E_t^T with FP32 accumulation: each product is at most 64 * 64 = 2^12 in
// magnitude and K is taken in blocks of at most 4096, so every partial sum of
// a block is an integer of magnitude at most 2^24 and its accumulation is
// exact in any order. The epilogue adds, block by block,
//   C_ij += (D_s E_t^T)_ij * 2^(e_i + 1) 2^(f_j + 1) 2^(-7 (s + t))
// in FP64: the scale is a power of two, so each term is exact and is built
// from the FP32 bits with integer operations; one FP64 addition per term.
// The pairs with s + t <= 9 (36 of the 64) are kept, in the order of
// increasing weight; the dropped ones and the rounding of the inputs to the
// 2^-55 grid stay below 2^-41 * 2^(e_i + f_j) * K / 4096 in the worst case
// (digits of equal sign), about the error bound of an FP64 dot product; the
// FP64 sums of the blocks add their own rounding.
//
// Kernel: persistent, one CTA per SM, 320 threads, laid out as the
// split-TF32 kernel but with eight epilogue warps (two per 32 TMEM lanes,
// one per half of the columns). A work unit is one 128 x 256 tile of C; its
// CTA runs the (digit pair, K block) steps one after another, each a K loop
// into one of two 256-column TMEM accumulators, so that the epilogue warps add
// step u into C while the MMAs of step u + 1 run. A thread's loads of C for a
// 32-column chunk are all issued before its stores, to keep them in flight
// together. The producer thread streams 32-wide K slices of the pair's A and
// Bt digits with TMA into an eight-stage ring (64-byte swizzle); the MMA
// thread issues two kind::f16 (BF16) MMAs per stage. Every wait has a clock
// budget, as in the split-TF32 kernel.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/sign.h"
#include "common.cuh"
#include "kernels.h"
#include "tc.cuh"

namespace sgn {

namespace {

using namespace tc;

constexpr int XM = 128;    // tile rows (UMMA M)
constexpr int XN = 256;    // tile columns (UMMA N)
constexpr int XK = 32;     // K slice per stage: 32 BF16 = 64 bytes = one swizzle span
constexpr int XSTAGE = 8;  // ring of stages
constexpr int XSPAN = XK * 2;
constexpr int XA_BYTES = XM * XK * 2;  // 8 KB
constexpr int XB_BYTES = XN * XK * 2;  // 16 KB
constexpr int XSTAGE_BYTES = XA_BYTES + XB_BYTES;
constexpr int XTHREADS = 320;  // producer, MMA, eight epilogue warps
constexpr uint32_t XTMEM_COLS = 2 * XN;
constexpr int XSMEM = XSTAGE * XSTAGE_BYTES + 1024;  // ring and alignment slack
constexpr int DIGIT_BITS = 7;
constexpr int MAX_LEVEL = F64X_DIGITS + 1;  // pairs with s + t <= MAX_LEVEL
constexpr int KBLK = F64X_MAX_K / XK;       // K stages per exact block (integer sums <= 2^24)

// The kept digit pairs, smallest weight first: s + t from MAX_LEVEL down to 2.
struct PairList {
  int n;
  unsigned char s[F64X_DIGITS * F64X_DIGITS], t[F64X_DIGITS * F64X_DIGITS];
};
constexpr PairList make_pairs() {
  PairList p{};
  p.n = 0;
  for (int lv = MAX_LEVEL; lv >= 2; --lv)
    for (int s = 1; s <= F64X_DIGITS; ++s) {
      int t = lv - s;
      if (t >= 1 && t <= F64X_DIGITS) {
        p.s[p.n] = (unsigned char)s;
        p.t[p.n] = (unsigned char)t;
        ++p.n;
      }
    }
  return p;
}
constexpr PairList kPairs = make_pairs();
__constant__ PairList c_pairs = kPairs;

// v 2^sc as an FP64 value, built from the bits of the FP32 integer v (exact):
// the epilogue then spends one FP64 addition per term, GB300's FP64 pipe
// being the scarce unit there. Falls back to ldexp outside the normal range.
__device__ __forceinline__ double exact_scaled(float v, int sc) {
  const uint32_t b = __float_as_uint(v);
  if ((b & 0x7FFFFFFFu) == 0u) return 0.0;
  const int e = int((b >> 23) & 0xFFu) - 127 + sc + 1023;
  if (e <= 0 || e >= 2047) return ldexp(double(v), sc);
  return __longlong_as_double(
      (long long)((uint64_t(b >> 31) << 63) | (uint64_t(e) << 52) | (uint64_t(b & 0x7FFFFFu) << 29)));
}

// Tile t of the launch -> job and tile origin (m0, n0); M blocks run fastest.
__device__ __forceinline__ void xtile_of(int t, const SliceJob *jobs, const int *tile_start,
                                         int njobs, int &j, int &m0, int &n0) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (tile_start[mid] <= t) lo = mid; else hi = mid - 1;
  }
  j = lo;
  const int local = t - tile_start[j];
  const int tm = (jobs[j].M + XM - 1) / XM;
  m0 = (local % tm) * XM;
  n0 = (local / tm) * XN;
}

// maps[2 j]: the digits of A of job j as one (8 M) x K array, maps[2 j + 1]
// those of Bt as (8 N) x K; digit s of row r is row (s - 1) rows + r.
__global__ void __launch_bounds__(XTHREADS, 1)
    k_gemm_slices(const SliceJob *jobs, const CUtensorMap *maps, const int *tile_start,
                  int njobs, int ntiles, int *err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[XSTAGE], empty[XSTAGE], tfull[2], tempty[2], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort, s_consumed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
  volatile int *abort = &s_abort;
  const int npairs = c_pairs.n;
  if (tid == 0) {
    for (int i = 0; i < XSTAGE; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 8);
    }
    mbar_init(&done, 1);
    s_abort = 0;
    s_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(&tmem_slot, XTMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  int issued = 0;

  if (warp == 0) {
    if (lane == 0) {
      for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
        int j, m0, n0;
        xtile_of(t, jobs, tile_start, njobs, j, m0, n0);
        const SliceJob &J = jobs[j];
        const CUtensorMap *mp = maps + 2 * j;
        const int nk = (J.K + XK - 1) / XK, nblk = (nk + KBLK - 1) / KBLK;
        for (int u = 0; u < npairs * nblk && !*abort; ++u) {
          const int p = u / nblk, k0 = (u % nblk) * KBLK, k1 = min(nk, k0 + KBLK);
          const int ya = (c_pairs.s[p] - 1) * J.M + m0, yb = (c_pairs.t[p] - 1) * J.N + n0;
          for (int kb = k0; kb < k1; ++kb, ++issued) {
            const int st = issued % XSTAGE;
            if (!bounded_wait(&empty[st], ((issued / XSTAGE) & 1) ^ 1, abort)) break;
            const uint32_t d = sbase + uint32_t(st * XSTAGE_BYTES);
            mbar_expect_tx(&full[st], XSTAGE_BYTES);
            tma_load_2d(d, mp + 0, kb * XK, ya, &full[st]);
            tma_load_2d(d + XA_BYTES, mp + 1, kb * XK, yb, &full[st]);
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(XM, XN);
      int it = 0, uc = 0;  // stages consumed, units (tile, pair) done
      bool any = false, ok = true;
      for (int t = blockIdx.x; t < ntiles && ok && !*abort; t += gridDim.x) {
        int j, m0, n0;
        xtile_of(t, jobs, tile_start, njobs, j, m0, n0);
        const int nk = (jobs[j].K + XK - 1) / XK, nblk = (nk + KBLK - 1) / KBLK;
        for (int u = 0; u < npairs * nblk && ok; ++u, ++uc) {
          const int k0 = (u % nblk) * KBLK, k1 = min(nk, k0 + KBLK);
          const int a = uc & 1;
          if (!bounded_wait(&tempty[a], ((uc >> 1) & 1) ^ 1, abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t acc = tmem + uint32_t(a * XN);
          for (int kb = k0; kb < k1; ++kb, ++it) {
            const int st = it % XSTAGE;
            if (!bounded_wait(&full[st], (it / XSTAGE) & 1, abort)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t d = sbase + uint32_t(st * XSTAGE_BYTES);
#pragma unroll
            for (int s = 0; s < XK / 16; ++s) {
              const uint32_t ko = uint32_t(s) * 32u;
              mma_bf16(acc, smem_desc_sw<XSPAN>(d + ko), smem_desc_sw<XSPAN>(d + XA_BYTES + ko),
                       idesc, ((kb - k0) | s) != 0 ? 1u : 0u);
            }
            any = true;
            mma_commit(&empty[st]);
          }
          if (!ok) break;
          mma_commit(&tfull[a]);
        }
      }
      s_consumed = it;
      if (any) {
        mma_commit(&done);
        if (!drain_wait(&done, 0, WAIT_BUDGET)) *abort = 1;
      }
    }
  } else {
    const int q = warp & 3;           // this warp's 32 TMEM lanes (rows)
    const int half = (warp - 2) >> 2;  // and its half of the tile's columns
    int uc = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
      int j, m0, n0;
      xtile_of(t, jobs, tile_start, njobs, j, m0, n0);
      const SliceJob J = jobs[j];
      const int gr = m0 + q * 32 + lane;
      const int ea = gr < J.M ? J.ea[gr] : 0;
      const int nk = (J.K + XK - 1) / XK, nblk = (nk + KBLK - 1) / KBLK;
      bool stop = false;
      for (int u = 0; u < npairs * nblk; ++u, ++uc) {
        const int p = u / nblk;
        const int a = uc & 1;
        if (!bounded_wait(&tfull[a], (uc >> 1) & 1, abort)) {
          stop = true;
          break;
        }
        tc_fence_after();
        // exponent of 2^(e_i + 1) 2^(-7 (s + t)); the column's is added per term
        const int er = ea - DIGIT_BITS * (c_pairs.s[p] + c_pairs.t[p]);
#pragma unroll 1
        for (int c = 0; c < XN / 64; ++c) {
          uint32_t v[32];
          const int col = half * (XN / 2) + c * 32;  // this warp's columns of the tile
          __syncwarp();
          tmem_ld_32x32(tmem + (uint32_t(q * 32) << 16) + uint32_t(a * XN + col), v);
          tmem_wait_ld();
          const int gc = n0 + col;
          if (gr >= J.M) continue;
          double *crow = J.C + int64_t(gr) * J.ldc + gc;
          const bool add = u != 0 || J.accum;  // C holds earlier terms
          if (gc + 32 <= J.N) {
            // all sixteen loads of the row's chunk in flight before any store
            double2 c2[16];
            if (add) {
#pragma unroll
              for (int i = 0; i < 16; ++i) c2[i] = reinterpret_cast<const double2 *>(crow)[i];
            }
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int2 eb = reinterpret_cast<const int2 *>(J.eb + gc)[i];
              double2 t2 = make_double2(exact_scaled(__uint_as_float(v[2 * i]), er + eb.x),
                                        exact_scaled(__uint_as_float(v[2 * i + 1]), er + eb.y));
              if (add) {
                t2.x = c2[i].x + t2.x;
                t2.y = c2[i].y + t2.y;
              }
              reinterpret_cast<double2 *>(crow)[i] = t2;
            }
          } else {
            // ragged last chunk (N and ldc even, C 16-byte aligned: column pairs)
#pragma unroll
            for (int k = 0; k < 32; k += 2) {
              if (gc + k >= J.N) break;
              const int2 eb = *reinterpret_cast<const int2 *>(J.eb + gc + k);
              double2 t2 = make_double2(exact_scaled(__uint_as_float(v[k]), er + eb.x),
                                        exact_scaled(__uint_as_float(v[k + 1]), er + eb.y));
              double2 *cp = reinterpret_cast<double2 *>(crow + k);
              if (add) {
                const double2 c2 = *cp;
                t2.x = c2.x + t2.x;
                t2.y = c2.y + t2.y;
              }
              *cp = t2;
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[a]);
      }
      if (stop) break;
    }
  }

  __syncthreads();
  if (warp == 0 && lane == 0) {
    for (int i = s_consumed; i < issued; ++i)
      if (!drain_wait(&full[i % XSTAGE], (i / XSTAGE) & 1, WAIT_BUDGET)) {
        *abort = 1;
        break;
      }
  }
  if (tid == 0 && *abort) atomicOr(err, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, XTMEM_COLS);
}

// Digits of the rows of x (rows x K, leading dimension ldx), or of its
// columns when transpose: digit s of row r at out[(s - 1) rows ld + r ld + k],
// zero for K <= k < ld; w[r] = e_r + 1 with 2^e_r > max_k |x_rk|.
__global__ void k_slices(int rows, int K, const double *x, int ldx, int transpose,
                         uint16_t *out, int ld, int *w) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  const int64_t plane = int64_t(rows) * ld;
  for (int64_t r = warp; r < rows; r += nwarps) {
    auto at = [&](int k) { return transpose ? x[int64_t(k) * ldx + r] : x[r * ldx + k]; };
    double mx = 0.0;
    for (int k = lane; k < K; k += 32) mx = fmax(mx, fabs(at(k)));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    int e = 0;
    frexp(mx, &e);  // mx < 2^e (e = 0 for a zero row)
    if (lane == 0) w[r] = e + 1;
    for (int k = lane; k < ld; k += 32) {
      // |x| < 2^e: q = x 2^(55 - e) rounded to an integer, |q| < 2^55
      long long q = k < K ? __double2ll_rn(ldexp(at(k), 55 - e)) : 0ll;
#pragma unroll
      for (int s = 1; s <= F64X_DIGITS; ++s) {
        const int shift = DIGIT_BITS * (F64X_DIGITS - s);
        long long d = q;
        if (shift > 0) {
          d = (q + (1ll << (shift - 1))) >> shift;  // nearest, |d| <= 64
          q -= d << shift;
        }
        // |d| <= 64 has at most 7 significant bits: its BF16 bits are the top
        // half of its FP32 bits, exactly
        out[(s - 1) * plane + r * ld + k] = uint16_t(__float_as_uint(float(d)) >> 16);
      }
    }
  }
}

// Warp-per-row helpers of the FP64 dense path (same row loop as the FP32 one).
template <typename F>
__device__ __forceinline__ void dense_rows(int64_t n, F f) {
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = warp; r < n; r += nwarps) f(r);
}

__global__ void k_densify64(int64_t n, const int32_t *seg, const int *dslot, const int64_t *moff,
                            const int64_t *rp, const int32_t *col, const double *val,
                            const DenseBuf64 *bufs) {
  const int lane = threadIdx.x & 31;
  dense_rows(n, [&](int64_t r) {
    const int m = seg[r], d = dslot[m];
    if (d < 0) return;
    const DenseBuf64 B = bufs[d];
    const int64_t r0 = moff[m], i = r - r0;
    for (int64_t p = rp[r] + lane; p < rp[r + 1]; p += 32) B.X[i * B.ld + (col[p] - r0)] = val[p];
  });
}

__global__ void k_dense_resid64(int64_t n, const int32_t *seg, const int *dslot,
                                const int64_t *moff, const DenseBuf64 *bufs, double *part,
                                unsigned long long *tcount) {
  const int lane = threadIdx.x & 31;
  dense_rows(n, [&](int64_t r) {
    const int m = seg[r], d = dslot[m];
    if (d < 0) return;
    const DenseBuf64 B = bufs[d];
    const int64_t i = r - moff[m];
    double rs = 0.0, xs = 0.0;
    unsigned cnt = 0;
    for (int j = lane; j < B.n; j += 32) {
      const double t = B.TT[i * B.ld + j], x = B.X[i * B.ld + j];
      const double e = j == i ? t - 1.0 : t;
      rs = fma(e, e, rs);
      xs = fma(x, x, xs);
      cnt += t != 0.0;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      rs += __shfl_xor_sync(0xffffffffu, rs, o);
      xs += __shfl_xor_sync(0xffffffffu, xs, o);
      cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) {
      part[2 * r] = rs;
      part[2 * r + 1] = xs;
      atomicAdd(&tcount[d], (unsigned long long)cnt);
    }
  });
}

__global__ void k_dense_emit64(int64_t n, const int32_t *seg, const int *dslot,
                               const int64_t *moff, const int *active, const DenseBuf64 *bufs,
                               const int64_t *cs, int64_t *ce, int32_t *ccol, double *cval) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  dense_rows(n, [&](int64_t r) {
    const int m = seg[r], d = dslot[m];
    if (d < 0 || !active[m]) return;
    const DenseBuf64 B = bufs[d];
    const int64_t r0 = moff[m], i = r - r0;
    int64_t out = cs[r];
    for (int j0 = 0; j0 < B.n; j0 += 32) {
      const int j = j0 + lane;
      double v = 0.0;
      if (j < B.n)
        v = __dsub_rn(__dmul_rn(1.5, B.X[i * B.ld + j]), __dmul_rn(0.5, B.P[i * B.ld + j]));
      const bool keep = v != 0.0;
      const unsigned mk = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int64_t pos = out + __popc(mk & lt);
        ccol[pos] = int32_t(r0 + j);
        cval[pos] = v;
      }
      out += __popc(mk);
    }
    if (lane == 0) ce[r] = out;
  });
}

int rows_grid(int64_t n) {
  int64_t g = (n + 7) / 8;
  return int(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

size_t scratch_maps_x(int njobs) {
  return size_t(njobs) * 2 + (size_t(njobs + 1) * sizeof(int) + sizeof(CUtensorMap) - 1) /
                                 sizeof(CUtensorMap);
}

}  // namespace

int f64x_pairs() { return kPairs.n; }

void launch_densify64(int64_t n, const int32_t *seg, const int *dslot, const int64_t *moff,
                      const int64_t *rp, const int32_t *col, const double *val,
                      const DenseBuf64 *bufs, cudaStream_t s) {
  if (n == 0) return;
  k_densify64<<<rows_grid(n), 256, 0, s>>>(n, seg, dslot, moff, rp, col, val, bufs);
  SGN_LAUNCH_CHECK();
}

void launch_dense_resid64(int64_t n, const int32_t *seg, const int *dslot, const int64_t *moff,
                          const DenseBuf64 *bufs, double *part, unsigned long long *tcount,
                          cudaStream_t s) {
  if (n == 0) return;
  k_dense_resid64<<<rows_grid(n), 256, 0, s>>>(n, seg, dslot, moff, bufs, part, tcount);
  SGN_LAUNCH_CHECK();
}

void launch_dense_emit64(int64_t n, const int32_t *seg, const int *dslot, const int64_t *moff,
                         const int *active, const DenseBuf64 *bufs, const int64_t *cs,
                         int64_t *ce, int32_t *ccol, double *cval, cudaStream_t s) {
  if (n == 0) return;
  k_dense_emit64<<<rows_grid(n), 256, 0, s>>>(n, seg, dslot, moff, active, bufs, cs, ce, ccol,
                                              cval);
  SGN_LAUNCH_CHECK();
}

size_t f64x_digits_bytes(int rows, int ld) {
  return size_t(F64X_DIGITS) * size_t(rows) * size_t(ld) * sizeof(uint16_t);
}

size_t slice_jobs_scratch_bytes(int njobs) { return scratch_maps_x(njobs) * sizeof(CUtensorMap); }

void launch_slices(int rows, int K, const double *x, int ldx, int transpose, uint16_t *digits,
                   int ld, int *w, cudaStream_t s) {
  if (rows <= 0) return;
  int64_t g = (int64_t(rows) + 7) / 8;
  k_slices<<<unsigned(std::min<int64_t>(g, 152 * 16)), 256, 0, s>>>(rows, K, x, ldx, transpose,
                                                                   digits, ld, w);
  SGN_LAUNCH_CHECK();
}

void launch_slice_jobs(int njobs, const SliceJob *jobs_host, SliceJob *jobs_dev, void *scratch,
                       int *err, cudaStream_t s) {
  if (njobs <= 0) return;
  static const int nsm = [] {  // once, thread-safe
    int dev = 0, n = 0;
    SGN_CUDA(cudaGetDevice(&dev));
    SGN_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    SGN_CUDA(cudaFuncSetAttribute(k_gemm_slices, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  XSMEM));
    return n;
  }();
  thread_local std::vector<CUtensorMap> host;
  host.resize(scratch_maps_x(njobs));
  CUtensorMap *maps = host.data();
  int *tile_start = reinterpret_cast<int *>(host.data() + size_t(njobs) * 2);
  int ntiles = 0;
  for (int j = 0; j < njobs; ++j) {
    const SliceJob &J = jobs_host[j];
    if (J.M <= 0 || J.N <= 0 || J.K <= 0 || J.lda % 8 || J.ldb % 8 ||
        J.ldc % 2 || J.N % 2)
      throw Error(SIGN_EINVAL, "slice job with bad shape");
    const CUtensorMapDataType bf = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    maps[2 * j + 0] = tc::operand_map(J.A, bf, 2, F64X_DIGITS * J.M, J.K, J.lda, XK, XM);
    maps[2 * j + 1] = tc::operand_map(J.B, bf, 2, F64X_DIGITS * J.N, J.K, J.ldb, XK, XN);
    tile_start[j] = ntiles;
    ntiles += ((J.M + XM - 1) / XM) * ((J.N + XN - 1) / XN);
  }
  tile_start[njobs] = ntiles;
  SGN_CUDA(cudaMemcpyAsync(scratch, host.data(), host.size() * sizeof(CUtensorMap),
                           cudaMemcpyHostToDevice, s));
  SGN_CUDA(cudaMemcpyAsync(jobs_dev, jobs_host, sizeof(SliceJob) * size_t(njobs),
                           cudaMemcpyHostToDevice, s));
  const unsigned char *sc = static_cast<const unsigned char *>(scratch);
  k_gemm_slices<<<std::min(ntiles, nsm), XTHREADS, XSMEM, s>>>(
      jobs_dev, reinterpret_cast<const CUtensorMap *>(sc),
      reinterpret_cast<const int *>(sc + size_t(njobs) * 2 * sizeof(CUtensorMap)), njobs, ntiles,
      err);
  SGN_LAUNCH_CHECK();
}

}  // namespace sgn

// ---------------------------------------------------------------------------
namespace sgn {
void set_last_error(const std::string &msg);
}

extern "C" sign_status sign_dense_product_f64(int M, int N, int K, const double *A, int lda,
                                              const double *B, int ldb, double *C, int ldc,
                                              void *cuda_stream) {
  using namespace sgn;
  set_last_error("");
  if (M < 0 || N < 0 || K < 0 || !A || !B || !C || lda < K || ldb < N || ldc < N)
    return set_last_error("bad dimensions or NULL pointer"), SIGN_EINVAL;
  if (N % 2 || ldc % 2 || (reinterpret_cast<uintptr_t>(C) & 15u))
    return set_last_error("need N and ldc even, C 16-byte aligned"), SIGN_EINVAL;
  if (M == 0 || N == 0) return SIGN_OK;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  try {
    if (K == 0) {
      SGN_CUDA(cudaMemset2DAsync(C, sizeof(double) * size_t(ldc), 0, sizeof(double) * size_t(N),
                                 size_t(M), s));
      SGN_CUDA(cudaStreamSynchronize(s));
      return SIGN_OK;
    }
    const int kp = (K + 7) / 8 * 8;
    DevBuf dig, wts, err, job, scratch;
    uint16_t *da = static_cast<uint16_t *>(
        dig.ensure(f64x_digits_bytes(M, kp) + f64x_digits_bytes(N, kp) + 256, s));
    uint16_t *db = da + f64x_digits_bytes(M, kp) / sizeof(uint16_t);
    int *wa = static_cast<int *>(wts.ensure(sizeof(int) * size_t(M + N + 4), s));
    int *wb = wa + ((M + 3) / 4 * 4);  // 16-byte aligned
    launch_slices(M, K, A, lda, 0, da, kp, wa, s);
    launch_slices(N, K, B, ldb, 1, db, kp, wb, s);  // Bt = B^T: the columns of B
    SliceJob J{M, N, kp, da, kp, db, kp, wa, wb, C, ldc};  // digits are zero for K <= k < kp
    job.ensure(sizeof(SliceJob), s);
    scratch.ensure(slice_jobs_scratch_bytes(1), s);
    err.ensure(sizeof(int), s);
    SGN_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    {
      ProfScope ps(KC_DENSE64, s, 2.0 * kPairs.n * double(M) * double(N) * double(kp), 0.0);
      launch_slice_jobs(1, &J, job.as<SliceJob>(), scratch.p, err.as<int>(), s);
    }
    int herr = 0;
    SGN_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SGN_CUDA(cudaStreamSynchronize(s));
    if (herr) return set_last_error("tensor-core wait gave up"), SIGN_ETIMEOUT;
  } catch (const Error &e) {
    set_last_error(e.what());
    return sign_status(e.status);
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    return SIGN_ENOMEM;
  } catch (const std::exception &e) {
    set_last_error(e.what());
    return SIGN_ECUDA;
  }
  return SIGN_OK;
}
