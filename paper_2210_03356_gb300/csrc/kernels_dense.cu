// Dense products on the 5th-generation tensor cores (tcgen05), for matrices
// whose iterate has filled in (step a9, FP32 stage of the mixed mode).
//
// C = A B for dense row-major FP32 A (M x K) and B (K x N), computed with
// split TF32: x = hi + lo with hi = x rounded to TF32 and lo = x - hi (exact),
// and C = A_hi B_hi + A_hi B_lo + A_lo B_hi, three tcgen05.mma of kind::tf32
// per K step, all accumulated in FP32 in tensor memory. The dropped A_lo B_lo
// term is below 2^-22 relative, so the product carries about FP32 accuracy
// (a single TF32 pass would keep only ~10 bits).
//
// Operands are K-major and already split: C = A Bt^T with A (M x K) and Bt
// (N x K) row-major, each given as a hi and a lo array. The kernel is
// persistent (one CTA per SM, tiles of 128 x 256 handed out round-robin over
// all jobs of the launch) and warp-specialised:
//   - warp 0 (one thread) streams K slices of A_hi, A_lo, Bt_hi, Bt_lo with
//     TMA (cp.async.bulk.tensor) into a ring of shared-memory stages laid out
//     in the swizzled K-major canonical form, each stage completing on an
//     mbarrier by transaction count;
//   - warp 1 owns the tensor memory (two 256-column FP32 accumulators) and one
//     of its threads issues the tcgen05.mma (three per K step of 8), releasing
//     a stage with tcgen05.commit once its MMAs have read it and signalling a
//     finished accumulator the same way;
//   - warps 2-5 drain an accumulator with tcgen05.ld (each warp its 32 lanes)
//     while the MMAs of the next tile run in the other one, and write C as
//     FP32 or already split into hi and lo.
// Every wait has a clock budget; a wait that runs out raises a shared abort
// flag, all roles leave their loops, the copies and MMAs already issued are
// waited for (again with a budget) and the tensor memory is freed.
#include <stdint.h>

#include <algorithm>
#include <vector>

#include <cuda.h>

#include "../../include/sign.h"
#include "common.cuh"
#include "tc.cuh"
#include "kernels.h"

namespace sgn {

namespace {

using namespace tc;

constexpr int DM = 128;   // tile rows (UMMA M)
constexpr int DN = 256;   // tile columns (UMMA N)
constexpr int DK = 16;    // K slice per stage: 16 FP32 = 64 bytes = one swizzle span
constexpr int NSTAGE = 4; // ring of stages
constexpr int SWIZZLE_BYTES = DK * 4;
constexpr int A_BYTES = DM * DK * 4;  // one 128 x 16 operand slice (8 KB)
constexpr int B_BYTES = DN * DK * 4;  // one 256 x 16 operand slice (16 KB)
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;
constexpr int DTHREADS = 192;          // producer, MMA, four epilogue warps
constexpr uint32_t TMEM_COLS = 2 * DN; // two FP32 accumulators of 128 lanes x 256 columns
static_assert(SWIZZLE_BYTES == 64 || SWIZZLE_BYTES == 128, "one swizzle span per slice");

// hi = x rounded to nearest TF32 (10 explicit mantissa bits), lo = x - hi
// (exact, so hi + lo == x).
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
  uint32_t b = __float_as_uint(x);
  uint32_t r = (b + 0x1000u) & 0xFFFFE000u;
  hi = __uint_as_float(r);
  if (!isfinite(hi)) hi = x;
  lo = __fsub_rn(x, hi);
}

// Tile t of the launch -> job and tile origin (m0, n0); M blocks run fastest.
__device__ __forceinline__ void tile_of(int t, const DenseJob *jobs, const int *tile_start,
                                        int njobs, int &j, int &m0, int &n0) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {  // last job with tile_start[j] <= t
    int mid = (lo + hi + 1) >> 1;
    if (tile_start[mid] <= t) lo = mid; else hi = mid - 1;
  }
  j = lo;
  const int local = t - tile_start[j];
  const int tm = (jobs[j].M + DM - 1) / DM;
  m0 = (local % tm) * DM;
  n0 = (local / tm) * DN;
}

// maps[4 j + 0..3]: A_hi, A_lo, Bt_hi, Bt_lo of job j (boxes DK x DM and DK x DN).
__global__ void __launch_bounds__(DTHREADS, 1)
    k_gemm_nt(const DenseJob *jobs, const CUtensorMap *maps, const int *tile_start, int njobs,
              int ntiles, int *err) {
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[NSTAGE], empty[NSTAGE], tfull[2], tempty[2], done;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_abort, s_consumed;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // stages 1024-byte aligned (the swizzle pattern follows address bits)
  const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
  volatile int *abort = &s_abort;

  if (tid == 0) {
    for (int i = 0; i < NSTAGE; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 4);
    }
    mbar_init(&done, 1);
    s_abort = 0;
    s_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    tmem_alloc(&tmem_slot, TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  int issued = 0;  // producer: stages filled

  if (warp == 0) {
    if (lane == 0) {
      for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x) {
        int j, m0, n0;
        tile_of(t, jobs, tile_start, njobs, j, m0, n0);
        const CUtensorMap *mp = maps + 4 * j;
        const int nk = (jobs[j].K + DK - 1) / DK;
        for (int kb = 0; kb < nk; ++kb, ++issued) {
          const int st = issued % NSTAGE;
          if (!bounded_wait(&empty[st], ((issued / NSTAGE) & 1) ^ 1, abort)) break;
          const uint32_t d = sbase + uint32_t(st * STAGE_BYTES);
          mbar_expect_tx(&full[st], STAGE_BYTES);
          tma_load_2d(d, mp + 0, kb * DK, m0, &full[st]);
          tma_load_2d(d + A_BYTES, mp + 1, kb * DK, m0, &full[st]);
          tma_load_2d(d + 2 * A_BYTES, mp + 2, kb * DK, n0, &full[st]);
          tma_load_2d(d + 2 * A_BYTES + B_BYTES, mp + 3, kb * DK, n0, &full[st]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_tf32(DM, DN);
      int it = 0, tc = 0;
      bool any = false;
      for (int t = blockIdx.x; t < ntiles && !*abort; t += gridDim.x, ++tc) {
        int j, m0, n0;
        tile_of(t, jobs, tile_start, njobs, j, m0, n0);
        const int nkj = (jobs[j].K + DK - 1) / DK;
        const int a = tc & 1;
        if (!bounded_wait(&tempty[a], ((tc >> 1) & 1) ^ 1, abort)) break;
        tc_fence_after();
        const uint32_t acc = tmem + uint32_t(a * DN);
        bool ok = true;
        for (int kb = 0; kb < nkj; ++kb, ++it) {
          const int st = it % NSTAGE;
          if (!bounded_wait(&full[st], (it / NSTAGE) & 1, abort)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = sbase + uint32_t(st * STAGE_BYTES);
#pragma unroll
          for (int s = 0; s < DK / 8; ++s) {
            const uint32_t ko = uint32_t(s) * 32u;
            const uint64_t ah = smem_desc_sw<SWIZZLE_BYTES>(d + ko), al = smem_desc_sw<SWIZZLE_BYTES>(d + A_BYTES + ko);
            const uint64_t bh = smem_desc_sw<SWIZZLE_BYTES>(d + 2 * A_BYTES + ko);
            const uint64_t bl = smem_desc_sw<SWIZZLE_BYTES>(d + 2 * A_BYTES + B_BYTES + ko);
            mma_tf32(acc, ah, bh, idesc, (kb | s) != 0 ? 1u : 0u);
            mma_tf32(acc, ah, bl, idesc, 1u);
            mma_tf32(acc, al, bh, idesc, 1u);
          }
          any = true;
          mma_commit(&empty[st]);  // the stage is free once these MMAs have read it
        }
        if (!ok) break;
        mma_commit(&tfull[a]);
      }
      s_consumed = it;
      if (any) {  // nothing may still write tensor memory when it is freed
        mma_commit(&done);
        if (!drain_wait(&done, 0, WAIT_BUDGET)) *abort = 1;
      }
    }
  } else {
    const int q = warp & 3;  // this warp's 32 TMEM lanes
    int tc = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tc) {
      int j, m0, n0;
      tile_of(t, jobs, tile_start, njobs, j, m0, n0);
      const DenseJob J = jobs[j];
      const int a = tc & 1;
      if (!bounded_wait(&tfull[a], (tc >> 1) & 1, abort)) break;
      tc_fence_after();
      const int gr = m0 + q * 32 + lane;
      float *dh = J.C + int64_t(gr) * J.ldc;
      float *dl = J.C_lo ? J.C_lo + int64_t(gr) * J.ldc : nullptr;
#pragma unroll 1
      for (int c = 0; c < DN / 32; ++c) {
        uint32_t v[32];
        __syncwarp();
        tmem_ld_32x32(tmem + (uint32_t(q * 32) << 16) + uint32_t(a * DN + c * 32), v);
        tmem_wait_ld();
        const int gc = n0 + c * 32;
        // N is a multiple of 4 and the rows 16-byte aligned: whole float4 groups
#pragma unroll
        for (int k = 0; k < 32; k += 4) {
          if (gr >= J.M || gc + k >= J.N) break;
          float4 h = make_float4(__uint_as_float(v[k]), __uint_as_float(v[k + 1]),
                                 __uint_as_float(v[k + 2]), __uint_as_float(v[k + 3]));
          if (dl) {
            float4 l;
            split_tf32(h.x, h.x, l.x);
            split_tf32(h.y, h.y, l.y);
            split_tf32(h.z, h.z, l.z);
            split_tf32(h.w, h.w, l.w);
            *reinterpret_cast<float4 *>(dl + gc + k) = l;
          }
          *reinterpret_cast<float4 *>(dh + gc + k) = h;
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[a]);
    }
  }

  __syncthreads();
  if (warp == 0 && lane == 0) {
    // TMA copies still landing in shared memory (only after an abort)
    for (int i = s_consumed; i < issued; ++i)
      if (!drain_wait(&full[i % NSTAGE], (i / NSTAGE) & 1, WAIT_BUDGET)) {
        *abort = 1;
        break;
      }
  }
  if (tid == 0 && *abort) atomicOr(err, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, TMEM_COLS);
}

// Split into hi/lo, optionally transposing: out[i][j] = in[i][j] (or in[j][i]),
// rows x cols of out, padded columns up to ldo zeroed.
__global__ void k_split(int rows, int cols, const float *in, int ldi, int transpose, float *hi,
                        float *lo, int ldo) {
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < int64_t(rows) * ldo;
       t += int64_t(gridDim.x) * blockDim.x) {
    int i = int(t / ldo), j = int(t % ldo);
    float x = 0.0f;
    if (j < cols) x = transpose ? in[int64_t(j) * ldi + i] : in[int64_t(i) * ldi + j];
    float h, l;
    split_tf32(x, h, l);
    hi[t] = h;
    lo[t] = l;
  }
}

// Densify: the rows of the dense-path matrices of a stage CSR into their
// zeroed blocks, split: X (row-major) and X^T.
__global__ void k_densify(int64_t n, const int32_t *seg, const int *dslot, const int64_t *moff,
                          const int64_t *rp, const int32_t *col, const float *val,
                          const DenseBuf *bufs) {
  int lane = threadIdx.x & 31;
  int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = warp; r < n; r += nwarps) {
    int m = seg[r];
    int d = dslot[m];
    if (d < 0) continue;
    const DenseBuf Bf = bufs[d];
    int64_t r0 = moff[m], i = r - r0;
    for (int64_t p = rp[r] + lane; p < rp[r + 1]; p += 32) {
      int64_t j = col[p] - r0;
      float h, l;
      split_tf32(val[p], h, l);
      Bf.X_hi[i * Bf.ld + j] = h;
      Bf.X_lo[i * Bf.ld + j] = l;
      Bf.XT_hi[j * Bf.ld + i] = h;
      Bf.XT_lo[j * Bf.ld + i] = l;
    }
  }
}

// Residual partials of the dense matrices from T^T (hi + lo): part[2r] =
// sum_j (t_rj - delta_rj)^2 and part[2r+1] = sum_j x_rj^2, as exact float
// pairs (the Frobenius norm of T^T - I is that of T - I, and the diagonal is
// shared); tcount[d] counts the nonzero entries of T.
__global__ void k_dense_resid(int64_t n, const int32_t *seg, const int *dslot, const int64_t *moff,
                              const DenseBuf *bufs, double *part, unsigned long long *tcount) {
  int lane = threadIdx.x & 31;
  int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = warp; r < n; r += nwarps) {
    int m = seg[r];
    int d = dslot[m];
    if (d < 0) continue;
    const DenseBuf Bf = bufs[d];
    int64_t i = r - moff[m];
    float rh = 0.f, rl = 0.f, xh = 0.f, xl = 0.f;
    double rdiag = 0.0;
    unsigned cnt = 0;
    for (int j = lane; j < Bf.n; j += 32) {
      float t = __fadd_rn(Bf.TT_hi[i * Bf.ld + j], Bf.TT_lo[i * Bf.ld + j]);
      float x = __fadd_rn(Bf.X_hi[i * Bf.ld + j], Bf.X_lo[i * Bf.ld + j]);
      cnt += t != 0.0f;
      if (j == i) {
        double dd = double(t) - 1.0;
        rdiag = dd * dd;
      } else {
        float pp = __fmul_rn(t, t), ee = __fmaf_rn(t, t, -pp);
        float s = __fadd_rn(rh, pp), bb = __fsub_rn(s, rh);
        rl = __fadd_rn(rl, __fadd_rn(__fadd_rn(__fsub_rn(rh, __fsub_rn(s, bb)), __fsub_rn(pp, bb)), ee));
        rh = s;
      }
      float px = __fmul_rn(x, x), ex = __fmaf_rn(x, x, -px);
      float sx = __fadd_rn(xh, px), bx = __fsub_rn(sx, xh);
      xl = __fadd_rn(xl, __fadd_rn(__fadd_rn(__fsub_rn(xh, __fsub_rn(sx, bx)), __fsub_rn(px, bx)), ex));
      xh = sx;
    }
    double rs = double(rh) + double(rl) + rdiag, xs = double(xh) + double(xl);
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
  }
}

// Xbar = 1.5 X - 0.5 P for the dense matrices, nonzero entries written in
// column order into the row slots [cs[r], ...), the end stored in ce[r].
__global__ void k_dense_emit(int64_t n, const int32_t *seg, const int *dslot, const int64_t *moff,
                             const int *active, const DenseBuf *bufs, const int64_t *cs,
                             int64_t *ce, int32_t *ccol, float *cval) {
  int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  int64_t nwarps = (int64_t(gridDim.x) * blockDim.x) >> 5;
  for (int64_t r = warp; r < n; r += nwarps) {
    int m = seg[r];
    int d = dslot[m];
    if (d < 0 || !active[m]) continue;
    const DenseBuf Bf = bufs[d];
    int64_t r0 = moff[m], i = r - r0;
    int64_t out = cs[r];
    for (int j0 = 0; j0 < Bf.n; j0 += 32) {
      int j = j0 + lane;
      float v = 0.0f;
      if (j < Bf.n) {
        float x = __fadd_rn(Bf.X_hi[i * Bf.ld + j], Bf.X_lo[i * Bf.ld + j]);
        v = __fsub_rn(__fmul_rn(1.5f, x), __fmul_rn(0.5f, Bf.P[i * Bf.ld + j]));
      }
      bool keep = v != 0.0f;
      unsigned mk = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        int64_t pos = out + __popc(mk & lt);
        ccol[pos] = int32_t(r0 + j);
        cval[pos] = v;
      }
      out += __popc(mk);
    }
    if (lane == 0) ce[r] = out;
  }
}

int dense_grid(int64_t n) {
  int64_t g = (n + 7) / 8;
  return int(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

}  // namespace

size_t dense_gemm_smem() { return size_t(NSTAGE) * STAGE_BYTES + 1024; }

// Tensor maps (4 per job) followed by the tile offsets, in CUtensorMap units.
static size_t scratch_maps(int njobs) {
  return size_t(njobs) * 4 + (size_t(njobs + 1) * sizeof(int) + sizeof(CUtensorMap) - 1) /
                                 sizeof(CUtensorMap);
}

size_t dense_jobs_scratch_bytes(int njobs) { return scratch_maps(njobs) * sizeof(CUtensorMap); }

void launch_dense_jobs(int njobs, const DenseJob *jobs_host, DenseJob *jobs_dev, void *scratch,
                       int *err, cudaStream_t s) {
  if (njobs <= 0) return;
  static const int nsm = [] {  // once, thread-safe
    int dev = 0, n = 0;
    SGN_CUDA(cudaGetDevice(&dev));
    SGN_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
    SGN_CUDA(cudaFuncSetAttribute(k_gemm_nt, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(dense_gemm_smem())));
    return n;
  }();
  thread_local std::vector<CUtensorMap> host;  // 64-byte aligned elements
  host.resize(scratch_maps(njobs));
  CUtensorMap *maps = host.data();
  int *tile_start = reinterpret_cast<int *>(host.data() + size_t(njobs) * 4);
  int ntiles = 0;
  for (int j = 0; j < njobs; ++j) {
    const DenseJob &J = jobs_host[j];
    if (J.M <= 0 || J.N <= 0 || J.K <= 0 || J.lda % 4 || J.ldb % 4 || J.ldc % 4 || J.N % 4)
      throw Error(SIGN_EINVAL, "dense job with bad shape");
    const CUtensorMapDataType f32 = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    maps[4 * j + 0] = tc::operand_map(J.A_hi, f32, 4, J.M, J.K, J.lda, DK, DM);
    maps[4 * j + 1] = tc::operand_map(J.A_lo, f32, 4, J.M, J.K, J.lda, DK, DM);
    maps[4 * j + 2] = tc::operand_map(J.B_hi, f32, 4, J.N, J.K, J.ldb, DK, DN);
    maps[4 * j + 3] = tc::operand_map(J.B_lo, f32, 4, J.N, J.K, J.ldb, DK, DN);
    tile_start[j] = ntiles;
    ntiles += ((J.M + DM - 1) / DM) * ((J.N + DN - 1) / DN);
  }
  tile_start[njobs] = ntiles;
  // pageable source: the copy has taken the bytes when it returns
  SGN_CUDA(cudaMemcpyAsync(scratch, host.data(), host.size() * sizeof(CUtensorMap),
                           cudaMemcpyHostToDevice, s));
  SGN_CUDA(cudaMemcpyAsync(jobs_dev, jobs_host, sizeof(DenseJob) * size_t(njobs),
                           cudaMemcpyHostToDevice, s));
  const unsigned char *sc = static_cast<const unsigned char *>(scratch);
  k_gemm_nt<<<std::min(ntiles, nsm), DTHREADS, dense_gemm_smem(), s>>>(
      jobs_dev, reinterpret_cast<const CUtensorMap *>(sc),
      reinterpret_cast<const int *>(sc + size_t(njobs) * 4 * sizeof(CUtensorMap)), njobs, ntiles,
      err);
  SGN_LAUNCH_CHECK();
}

void launch_split(int rows, int cols, const float *in, int ldi, int transpose, float *hi,
                  float *lo, int ldo, cudaStream_t s) {
  int64_t total = int64_t(rows) * ldo;
  if (total == 0) return;
  int g = int(std::min<int64_t>((total + 255) / 256, 152 * 32));
  k_split<<<g, 256, 0, s>>>(rows, cols, in, ldi, transpose, hi, lo, ldo);
  SGN_LAUNCH_CHECK();
}

void launch_densify(int64_t n, const int32_t *seg, const int *dslot, const int64_t *moff,
                    const int64_t *rp, const int32_t *col, const float *val, const DenseBuf *bufs,
                    cudaStream_t s) {
  if (n == 0) return;
  k_densify<<<dense_grid(n), 256, 0, s>>>(n, seg, dslot, moff, rp, col, val, bufs);
  SGN_LAUNCH_CHECK();
}

void launch_dense_resid(int64_t n, const int32_t *seg, const int *dslot, const int64_t *moff,
                        const DenseBuf *bufs, double *part, unsigned long long *tcount,
                        cudaStream_t s) {
  if (n == 0) return;
  k_dense_resid<<<dense_grid(n), 256, 0, s>>>(n, seg, dslot, moff, bufs, part, tcount);
  SGN_LAUNCH_CHECK();
}

void launch_dense_emit(int64_t n, const int32_t *seg, const int *dslot, const int64_t *moff,
                       const int *active, const DenseBuf *bufs, const int64_t *cs, int64_t *ce,
                       int32_t *ccol, float *cval, cudaStream_t s) {
  if (n == 0) return;
  k_dense_emit<<<dense_grid(n), 256, 0, s>>>(n, seg, dslot, moff, active, bufs, cs, ce, ccol,
                                             cval);
  SGN_LAUNCH_CHECK();
}

}  // namespace sgn

// ---------------------------------------------------------------------------
namespace sgn {
void set_last_error(const std::string &msg);
}

extern "C" sign_status sign_dense_product(int M, int N, int K, const float *A, int lda,
                                          const float *B, int ldb, float *C, int ldc,
                                          void *cuda_stream) {
  using namespace sgn;
  set_last_error("");
  if (M < 0 || N < 0 || K < 0 || !A || !B || !C || lda < K || ldb < N || ldc < N)
    return set_last_error("bad dimensions or NULL pointer"), SIGN_EINVAL;
  if ((K | N | lda | ldb | ldc) % 4 != 0 ||
      ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) |
        reinterpret_cast<uintptr_t>(C)) & 15u) != 0)
    return set_last_error("K, N and the leading dimensions must be multiples of 4 and the "
                          "arrays 16-byte aligned"),
           SIGN_EINVAL;
  if (M == 0 || N == 0) return SIGN_OK;
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  try {
    if (K == 0) {
      SGN_CUDA(cudaMemset2DAsync(C, sizeof(float) * size_t(ldc), 0, sizeof(float) * size_t(N),
                                 size_t(M), s));
      SGN_CUDA(cudaStreamSynchronize(s));
      return SIGN_OK;
    }
    // split A (M x K) and B^T (N x K) into TF32 hi/lo parts, K padded to 4
    const int kp = (K + 3) / 4 * 4;
    DevBuf ws, err, job, scratch;
    size_t na = size_t(M) * kp, nbt = size_t(N) * kp;
    float *w = static_cast<float *>(ws.ensure(sizeof(float) * 2 * (na + nbt) + 64, s));
    float *a_hi = w, *a_lo = w + na, *b_hi = w + 2 * na, *b_lo = w + 2 * na + nbt;
    launch_split(M, K, A, lda, 0, a_hi, a_lo, kp, s);
    launch_split(N, K, B, ldb, 1, b_hi, b_lo, kp, s);
    DenseJob J{M, N, K, a_hi, a_lo, kp, b_hi, b_lo, kp, C, nullptr, ldc};
    job.ensure(sizeof(DenseJob), s);
    scratch.ensure(dense_jobs_scratch_bytes(1), s);
    err.ensure(sizeof(int), s);
    SGN_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    {
      ProfScope ps(KC_DENSE, s, 3.0 * 2.0 * double(M) * double(N) * double(K), 0.0);
      launch_dense_jobs(1, &J, job.as<DenseJob>(), scratch.p, err.as<int>(), s);
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
