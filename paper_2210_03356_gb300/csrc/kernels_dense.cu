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
// One CTA of 128 threads computes a 128 x 128 tile of C:
//   - the threads stage a 128 x 32 slice of A and of B^T (split into hi and
//     lo) in shared memory, in the no-swizzle K-major core-matrix layout
//     (core matrix = 8 rows x 16 bytes; along K the cores are 128 bytes apart,
//     along M/N the 8-row groups 1024 bytes apart);
//   - thread 0 issues the 12 MMAs of the slice (4 K steps of 8 x 3 splits)
//     and commits them to an mbarrier; everybody waits on it (with a clock
//     budget) before the slice is overwritten;
//   - at the end each warp reads its 32 TMEM lanes (rows) with tcgen05.ld.
#include <stdint.h>

#include "common.cuh"
#include "kernels.h"

namespace sgn {

namespace {

constexpr int DM = 128;  // tile rows (UMMA M)
constexpr int DN = 128;  // tile columns (UMMA N)
constexpr int DK = 32;   // K slice staged per round
constexpr int DTHREADS = 128;
constexpr int TILE_BYTES = DM * DK * 4;  // one 128 x 32 FP32 operand tile (16 KB)
constexpr uint32_t TMEM_COLS = 128;      // FP32 accumulator: 128 lanes x 128 columns
constexpr long long WAIT_BUDGET = 4000000000LL;  // clock cycles (~2 s) per wait

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// D[tmem] (+)= A[smem desc] * B[smem desc]^T, kind::tf32
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n"
      ".reg .pred p;\n"
      "setp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

// 32 TMEM lanes x 32 consecutive 32-bit columns; thread t of the warp gets lane
// (base lane + t).
__device__ __forceinline__ void tmem_ld_32x32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor: no swizzle, K-major, start address,
// leading-dimension byte offset (between core matrices along K) and stride
// byte offset (between 8-row groups), version 1 (tcgen05).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= uint64_t((saddr >> 4) & 0x3FFFu);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;
  return d;
}

// Instruction descriptor of kind::tf32: FP32 accumulator, A and B TF32, both
// K-major, N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(m >> 4) << 24);
}

// Byte offset of element (row, k) of a 128 x 32 tile in the core-matrix layout.
__device__ __forceinline__ uint32_t core_off(int row, int k) {
  return uint32_t(((row >> 3) * (DK / 4) + (k >> 2)) * 128 + (row & 7) * 16 + (k & 3) * 4);
}

// hi = x rounded to nearest TF32 (10 explicit mantissa bits), lo = x - hi.
__device__ __forceinline__ void split_tf32(float x, float &hi, float &lo) {
  uint32_t b = __float_as_uint(x);
  uint32_t r = (b + 0x1000u) & 0xFFFFE000u;
  hi = __uint_as_float(r);
  if (!isfinite(hi)) hi = x;
  lo = __fsub_rn(x, hi);
}

// One 128 x 128 tile (m0, n0) of C = A B; smem = 4 operand tiles.
__device__ __forceinline__ void gemm_tile(int M, int N, int K, const float *__restrict__ A,
                                          int lda, const float *__restrict__ B, int ldb,
                                          float *__restrict__ C, int ldc, int m0, int n0,
                                          unsigned char *smem, int *err) {
  unsigned char *a_hi = smem;
  unsigned char *a_lo = smem + TILE_BYTES;
  unsigned char *b_hi = smem + 2 * TILE_BYTES;
  unsigned char *b_lo = smem + 3 * TILE_BYTES;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 0) {
    tmem_alloc(&tmem_base, TMEM_COLS);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    s_fail = 0;
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_tf32(DM, DN);
  const uint32_t sa_hi = smem_u32(a_hi), sa_lo = smem_u32(a_lo);
  const uint32_t sb_hi = smem_u32(b_hi), sb_lo = smem_u32(b_lo);

  const int nk = (K + DK - 1) / DK;
  uint32_t phase = 0;
  for (int kb = 0; kb < nk; ++kb) {
    const int k0 = kb * DK;
    // A slice: rows m0.., k0..k0+31 ; 128 rows x 8 float4
    for (int i = tid; i < DM * (DK / 4); i += DTHREADS) {
      int row = i / (DK / 4), kc = i % (DK / 4);
      int gr = m0 + row, gk = k0 + kc * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gr < M && gk < K) v = *reinterpret_cast<const float4 *>(A + int64_t(gr) * lda + gk);
      float4 h, l;
      split_tf32(v.x, h.x, l.x);
      split_tf32(v.y, h.y, l.y);
      split_tf32(v.z, h.z, l.z);
      split_tf32(v.w, h.w, l.w);
      uint32_t off = core_off(row, kc * 4);
      *reinterpret_cast<float4 *>(a_hi + off) = h;
      *reinterpret_cast<float4 *>(a_lo + off) = l;
    }
    // B^T slice: tile row n = column n0+n of B, k = k0..k0+31 ; read B rows (k) as float4 along n
    for (int i = tid; i < DK * (DN / 4); i += DTHREADS) {
      int kk = i / (DN / 4), nc = i % (DN / 4);
      int gk = k0 + kk, gn = n0 + nc * 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gk < K && gn < N) v = *reinterpret_cast<const float4 *>(B + int64_t(gk) * ldb + gn);
      float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float h, l;
        split_tf32(vv[e], h, l);
        uint32_t off = core_off(nc * 4 + e, kk);
        *reinterpret_cast<float *>(b_hi + off) = h;
        *reinterpret_cast<float *>(b_lo + off) = l;
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int s = 0; s < DK / 8; ++s) {
        uint32_t koff = uint32_t(s) * 2u * 128u;  // K step of 8 = two core matrices
        uint64_t ah = smem_desc(sa_hi + koff, 128, 1024), al = smem_desc(sa_lo + koff, 128, 1024);
        uint64_t bh = smem_desc(sb_hi + koff, 128, 1024), bl = smem_desc(sb_lo + koff, 128, 1024);
        uint32_t first = (kb == 0 && s == 0) ? 0u : 1u;
        mma_tf32(tmem, ah, bh, idesc, first);
        mma_tf32(tmem, ah, bl, idesc, 1u);
        mma_tf32(tmem, al, bh, idesc, 1u);
      }
      mma_commit(&bar);
    }
    // wait for the MMAs of this slice before the buffers are overwritten
    long long t0 = clock64();
    bool done = false;
    while (!done) {
      done = mbar_try_wait(&bar, phase);
      if (!done && clock64() - t0 > WAIT_BUDGET) {
        s_fail = 1;
        break;
      }
    }
    phase ^= 1u;
    __syncthreads();
    if (s_fail) break;
  }
  tc_fence_after();
  if (!s_fail && nk > 0) {
    // epilogue: warp w holds rows 32w..32w+31 of the tile
#pragma unroll 1
    for (int c = 0; c < DN / 32; ++c) {
      uint32_t v[32];
      tmem_ld_32x32(tmem + (uint32_t(warp * 32) << 16) + uint32_t(c * 32), v);
      tmem_wait_ld();
      int gr = m0 + warp * 32 + lane;
      int gc = n0 + c * 32;
      if (gr < M) {
        float *dst = C + int64_t(gr) * ldc + gc;
        if (gc + 32 <= N) {
#pragma unroll
          for (int j = 0; j < 32; j += 4)
            *reinterpret_cast<float4 *>(dst + j) =
                make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                            __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
        } else {
          for (int j = 0; j < 32 && gc + j < N; ++j) dst[j] = __uint_as_float(v[j]);
        }
      }
    }
  } else if (nk == 0) {
    for (int i = tid; i < DM * DN; i += DTHREADS) {
      int r = m0 + i / DN, c = n0 + i % DN;
      if (r < M && c < N) C[int64_t(r) * ldc + c] = 0.0f;
    }
  }
  if (s_fail && tid == 0) atomicOr(err, 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, TMEM_COLS);
}

__global__ void __launch_bounds__(DTHREADS)
    k_gemm_tf32x3(int M, int N, int K, const float *__restrict__ A, int lda,
                  const float *__restrict__ B, int ldb, float *__restrict__ C, int ldc,
                  int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  gemm_tile(M, N, K, A, lda, B, ldb, C, ldc, blockIdx.y * DM, blockIdx.x * DN, smem, err);
}

// Several independent products in one launch: blockIdx.z is the job.
__global__ void __launch_bounds__(DTHREADS) k_gemm_tf32x3_jobs(const DenseJob *jobs, int *err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const DenseJob J = jobs[blockIdx.z];
  const int m0 = blockIdx.y * DM, n0 = blockIdx.x * DN;
  if (m0 >= J.M || n0 >= J.N) return;  // before any tensor-memory allocation
  gemm_tile(J.M, J.N, J.K, J.A, J.lda, J.B, J.ldb, J.C, J.ldc, m0, n0, smem, err);
}

// Densify: rows of the dense matrices of a stage CSR into their zeroed
// row-major blocks (global columns minus the matrix's first row).
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
    int64_t r0 = moff[m];
    float *row = Bf.X + (r - r0) * Bf.ld;
    for (int64_t p = rp[r] + lane; p < rp[r + 1]; p += 32) row[col[p] - r0] = val[p];
  }
}

// Residual partials of the dense matrices from T = X X: part[2r] =
// sum_j (t_rj - delta_rj)^2 and part[2r+1] = sum_j x_rj^2, as exact float
// pairs; tcount[d] counts the nonzero entries of T.
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
    const float *trow = Bf.T + i * Bf.ld;
    const float *xrow = Bf.X + i * Bf.ld;
    float rh = 0.f, rl = 0.f, xh = 0.f, xl = 0.f;
    double rdiag = 0.0;
    unsigned cnt = 0;
    for (int j = lane; j < Bf.n; j += 32) {
      float t = trow[j], x = xrow[j];
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
    int64_t r0 = moff[m];
    int64_t i = r - r0;
    const float *xrow = Bf.X + i * Bf.ld;
    const float *prow = Bf.P + i * Bf.ld;
    int64_t out = cs[r];
    for (int j0 = 0; j0 < Bf.n; j0 += 32) {
      int j = j0 + lane;
      float v = 0.0f;
      if (j < Bf.n)
        v = __fsub_rn(__fmul_rn(1.5f, xrow[j]), __fmul_rn(0.5f, prow[j]));
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

}  // namespace

size_t dense_gemm_smem() { return size_t(4) * TILE_BYTES; }

int dense_grid(int64_t n) {
  int64_t g = (n + 7) / 8;
  return int(g < 1 ? 1 : (g > 152 * 16 ? 152 * 16 : g));
}

void launch_dense_jobs(int njobs, const DenseJob *jobs, int max_m, int max_n, int *err,
                       cudaStream_t s) {
  if (njobs <= 0) return;
  static bool attr = false;
  if (!attr) {
    SGN_CUDA(cudaFuncSetAttribute(k_gemm_tf32x3_jobs, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(dense_gemm_smem())));
    attr = true;
  }
  dim3 grid((max_n + DN - 1) / DN, (max_m + DM - 1) / DM, njobs);
  k_gemm_tf32x3_jobs<<<grid, DTHREADS, dense_gemm_smem(), s>>>(jobs, err);
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

void launch_dense_gemm_tf32x3(int M, int N, int K, const float *A, int lda, const float *B,
                              int ldb, float *C, int ldc, int *err, cudaStream_t s) {
  if (M <= 0 || N <= 0) return;
  static bool attr = false;
  if (!attr) {
    SGN_CUDA(cudaFuncSetAttribute(k_gemm_tf32x3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  int(dense_gemm_smem())));
    attr = true;
  }
  dim3 grid((N + DN - 1) / DN, (M + DM - 1) / DM);
  k_gemm_tf32x3<<<grid, DTHREADS, dense_gemm_smem(), s>>>(M, N, K, A, lda, B, ldb, C, ldc, err);
  SGN_LAUNCH_CHECK();
}

}  // namespace sgn

// ---------------------------------------------------------------------------
#include <string>

#include "../../include/sign.h"

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
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  try {
    DevBuf err;
    err.ensure(sizeof(int), s);
    SGN_CUDA(cudaMemsetAsync(err.p, 0, sizeof(int), s));
    launch_dense_gemm_tf32x3(M, N, K, A, lda, B, ldb, C, ldc, err.as<int>(), s);
    int herr = 0;
    SGN_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    SGN_CUDA(cudaStreamSynchronize(s));
    if (herr) return set_last_error("tensor-core wait gave up"), SIGN_ETIMEOUT;
  } catch (const Error &e) {
    set_last_error(e.what());
    return sign_status(e.status);
  }
  return SIGN_OK;
}

