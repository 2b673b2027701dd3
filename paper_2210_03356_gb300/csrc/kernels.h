// Host-side launchers of the sign solver's CUDA kernels. Every pointer is a
// device pointer; every launcher enqueues on `s` and returns immediately.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sgn {

// ---------------------------------------------------------------- csr utils
// flag |= 1 if the CSR is malformed (rowptr not monotone or not ending at
// nnz, column out of range or not strictly ascending, value not finite).
void launch_validate(int64_t n, int64_t nnz, const int64_t *rp, const int32_t *col,
                     const double *val, int *flag, cudaStream_t s);
// launch_validate for `count` matrices in one launch: jobs[m] describes matrix
// m (device pointers), row_off (count + 1, on the device) the exclusive prefix
// of their row counts, total_rows = row_off[count]; flags[m] |= 1 if matrix m
// is malformed.
struct ValidateJob {
  int64_t n, nnz;
  const int64_t *rp;
  const int32_t *col;
  const double *val;
};
void launch_validate_batch(int count, const ValidateJob *jobs, const int64_t *row_off,
                           int64_t total_rows, int *flags, cudaStream_t s);

// Copies `count` chunks (src, dst: device-accessible pointers, e.g. device
// memory or mapped pinned host memory; bytes a multiple of 4, the chunks not
// overlapping) in one launch.
struct CopyChunk {
  const void *src;
  void *dst;
  int64_t bytes;
};
void launch_copy_chunks(int count, const CopyChunk *chunks, cudaStream_t s);

// Matrix-wide statistics for the server's footprint model. Initialise
// min_gap_bits to the bits of +inf and the rest to 0; then min_gap_bits holds
// the bits of min over rows with a positive gap of |a_ii| - sum_{j!=i}|a_ij|,
// nogap = 1 if any row has no positive gap, max_rowsum_bits the bits of
// max_i sum_j |a_ij| and max_bw max |i - j| over the entries.
struct GershStats {
  unsigned long long min_gap_bits, max_rowsum_bits;
  long long max_bw;
  int nogap;
};
void launch_gersh(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                  GershStats *g, cudaStream_t s);

// out[0] = 0, out[i+1] = sum_{r<=i} cnt[r] for i < n. tmp holds
// scan_tmp_elems(n) int64 values.
int64_t scan_tmp_elems(int64_t n);
void launch_scan(int64_t n, const int64_t *cnt, int64_t *out, int64_t *tmp, cudaStream_t s);

// One block of a block-diagonal assembly: rows [row0, row0+nrows) of a source
// CSR whose column indices are shifted by col_shift on the way.
struct AsmBlock {
  const int64_t *rp;
  const int32_t *col;
  const void *val;
  int64_t row0, nrows, col_shift;
  int val_f32;  // source values are float
};
// Writes dst rowptr (n_dst+1) from the blocks, laid out one after another.
// blocks/boff are device arrays: boff[b] is the first destination row of
// block b (boff[nblocks] = n_dst). lens is an int64[n_dst] scratch.
void launch_assemble_rows(int nblocks, const AsmBlock *blocks, const int64_t *boff, int64_t n_dst,
                          int64_t *lens, int64_t *dst_rp, int64_t *scan_tmp, cudaStream_t s);
void launch_assemble_vals(int nblocks, const AsmBlock *blocks, const int64_t *boff, int64_t n_dst,
                          const int64_t *dst_rp, int32_t *dst_col, void *dst_val, int dst_f32,
                          cudaStream_t s);

// seg[r] = matrix of row r, from moff (nb+1 row offsets).
void launch_fill_seg(int nb, const int64_t *moff, int64_t n, int32_t *seg, cudaStream_t s);

// Reproducible ||A||_1 per matrix (see kernels_csr.cu) and X_1 = A / ||A||_1.
// work: 2*n + 4*nb uint64 scratch. norm: double[nb].
void launch_onenorm(int nb, const int64_t *moff, const int32_t *seg, int64_t n, const int64_t *rp,
                    const int32_t *col, const double *val, unsigned long long *work, double *norm,
                    cudaStream_t s);
void launch_scale(int64_t n, const int32_t *seg, const int64_t *rp, double *val,
                  const double *norm, cudaStream_t s);

// out[m] = sum over the rows r of matrix m of (re[r] - rs[r]) (entries per
// matrix of a slotted CSR).
void launch_seg_count(int nb, const int64_t *moff, const int64_t *rs, const int64_t *re,
                      int64_t *out, cudaStream_t s);

// out[r] = re[r] - rs[r]; and the copy of slotted rows into a compact CSR
// whose row pointers orp are the scan of those lengths (vsize: 4 or 8 bytes).
void launch_row_lengths(int64_t n, const int64_t *rs, const int64_t *re, int64_t *out,
                        cudaStream_t s);
void launch_compact_rows(int64_t n, const int64_t *rs, const int64_t *re, const int32_t *col,
                         const void *val, int vsize, const int64_t *orp, int32_t *ocol,
                         void *oval, cudaStream_t s);

// Copies whole matrices out of a compact stage CSR in one launch: block b
// takes rows [row0, row0 + nrows) of (rp, col, val), rebases the row pointers
// to start at 0, shifts the columns by col_shift and widens FP32 values.
struct ExtractBlock {
  const int64_t *rp;
  const int32_t *col;
  const void *val;
  int val_f32;
  int64_t row0, nrows, col_shift;
  int64_t *drp;
  int32_t *dcol;
  double *dval;
};
// max_entries: the most entries of one block (sizes the grid).
void launch_extract(int nblocks, const ExtractBlock *blocks, int64_t max_entries, cudaStream_t s);

// out[m] = rp[moff[m]] for m = 0..nb (entry offsets of the matrices).
void launch_gather_offsets(int nb, const int64_t *moff, const int64_t *rp, int64_t *out,
                           cudaStream_t s);

// out[m*ncomp + c] = sum over rows r of matrix m of part[r*ncomp + c], in a
// fixed order (deterministic).
void launch_seg_reduce(int nb, const int64_t *moff, const double *part, int ncomp, double *out,
                       cudaStream_t s);

// ---------------------------------------------------------------- spgemm
enum ProductMode { MODE_SQUARE = 0, MODE_UPDATE = 1 };

// An operand's rows: row i holds entries [rs[i], re[i]) of col (and the
// values), columns ascending. Compact CSR: rs = rowptr, re = rowptr + 1.
struct Rows {
  const int64_t *rs;
  const int64_t *re;
  const int32_t *col;
};

// Row classes of the numeric kernels: groups of 32, 16 or 8 lanes per row,
// one CTA per row, or band tiles of 16 rows (FP32 only; the list holds each
// tile's first row).
enum RowClass { RC_G32 = 0, RC_CTA = 1, RC_G16 = 2, RC_G8 = 3, RC_BAND = 4, RC_NONE = 5, RC_N = 5 };
constexpr int RC_QUEUE = RC_N;        // counters[RC_QUEUE + c]: work-queue head of class c
constexpr int RC_COUNTERS = 2 * RC_N;  // ints in the counters array

// Per row i of C = A B (rows of inactive matrices are empty): the column
// range [lo, lo+len) of the row (including A's own row in MODE_UPDATE), the
// slot size ub[i] = min(len, work + (UPDATE ? nnz(A_i) : 0)) >= nnz(C_i), and
// work[i] = sum_{k in A_i} nnz(B_k), the multiply-adds of the row. Non-empty
// rows are listed, in row order within tiles, by the numeric kernel that takes
// them: lists holds RC_N lists of n entries (32-, 16- or 8-lane groups, one
// CTA per row, band tiles); counters[c] is the length of list c and
// counters[RC_QUEUE + c] the work-queue head of its kernel (all zeroed by the
// caller). groups: 0 keeps every warp-sized row on 32 lanes; 1 (FP64
// products, bound by the FP64 pipe) picks 32, 16 or 8 lanes by lane
// utilisation, a narrower group only when it raises the use by more than
// group_margin; 2 (FP32 products) lists every row of extent <= 512 in the
// 16-lane class, whose FP32 kernel runs the rows two per warp with shared
// passes over B. band (FP32 products only): aligned groups of 16 rows of one
// matrix whose multiply-adds fill at least band_min_eff of the band tile's
// FMA slots (by the work estimate in k_bounds; at the default 0.08 the tile
// costs fewer instructions than the row-wise product) go to the band list
// instead, and their
// multiply-adds are added to *band_work (nullable; zeroed by the caller);
// bandrow (nullable) gets 1 for the rows of band tiles, 0 for the others.
// binfo: scratch of n records (B's rows' first/last column and length; B has
// n rows, as every operand of a stage).
// dslot (nullable, per matrix): matrices with dslot[m] >= 0 take the dense
// path; their rows get no sparse work, and in MODE_UPDATE a whole row of
// slots (moff gives the matrix sizes).
void launch_bounds(int64_t n, const Rows &A, const Rows &B, const int32_t *seg, const int *active,
                   int mode, int groups, float group_margin, int band, float band_min_eff,
                   const int *dslot, const int64_t *moff, int32_t *lo, int32_t *len,
                   int64_t *ub, int32_t *lists, int *counters, double *work,
                   double *band_work, unsigned char *bandrow, int4 *binfo, cudaStream_t s);

// Band layout of the rows of an FP32 operand: row k's values dense over the
// columns [fc[k], fc[k] + nf[k]) (fc and nf multiples of 4, holes +0) at
// val[pos[k]], pos[k] a multiple of 4 (16-byte aligned rows); its pattern as
// bit words of absolute column blocks, word w (columns 32w .. 32w + 31) at
// mask[pos[k] / 2 + w - (fc[k] >> 5)] (nf/2 words per row always suffice).
struct Band {
  const int64_t *pos;
  const int32_t *fc, *nf;
  const float *val;
  const unsigned *mask;
};
// A band being written (the square T = X X of the band tiles, for the update).
struct BandOut {
  const int64_t *pos = nullptr;
  const int32_t *fc = nullptr, *nf = nullptr;
  float *val = nullptr;
  unsigned *mask = nullptr;
};
constexpr int BAND_JW = 64;   // widest output hull of a band tile, in 32-column words
constexpr int BAND_KT = 312;  // widest k hull (A rows' columns) of a band tile
// fc, nf and span[k] = nf[k] of each row (span is scanned into pos).
void launch_band_spans(int64_t n, const Rows &R, int32_t *fc, int32_t *nf, int64_t *span,
                       cudaStream_t s);
// The same layout from a product's row column ranges [lo, lo + len) (the
// first and last column of a product row are stored entries).
void launch_band_spans_range(int64_t n, const int32_t *lo, const int32_t *len, int32_t *fc,
                             int32_t *nf, int64_t *span, cudaStream_t s);
// Writes the rows' bands (cleared first) from their CSR; rows with skip[r]
// set (skip nullable) are left as they are.
void launch_band_fill(int64_t n, const Rows &R, const float *val, const int64_t *pos,
                      const int32_t *fc, const int32_t *nf, const unsigned char *skip, float *bval,
                      unsigned *bmask, cudaStream_t s);
// The band tiles of an FP32 product (the RC_BAND list of k_bounds): C = A A
// (SQUARE, with the partial sums of launch_numeric) or 1.5 A - 0.5 A B
// (UPDATE), A's rows as CSR (its stored k) and both operands as bands. In
// SQUARE, bandC (val nullable) receives the band of the tiles' rows of C, laid
// out by launch_band_spans_range.
void launch_band_product(int64_t n, int mode, const Rows &A, const float *aval, const Band &bandA,
                         const Band &bandB, const BandOut &bandC, const int32_t *lo,
                         const int32_t *len, const int32_t *lists, int *counters,
                         const int64_t *cs, int64_t *ce, int32_t *ccol, float *cval, double *part,
                         cudaStream_t s);
// Numeric product. Row i is written at cs[i] (exclusive scan of ub) and its
// end stored in ce[i]. MODE_SQUARE: C = A A, and part[2i] = sum_j (C_ij -
// delta_ij)^2, part[2i+1] = sum_k a_ik^2. MODE_UPDATE: C = 1.5 A - 0.5 A B.
template <typename T>
void launch_numeric(int64_t n, const Rows &A, const T *aval, const Rows &B, const T *bval,
                    int mode, const int32_t *lo, const int32_t *len, const int32_t *lists,
                    const int *counters, const int64_t *cs, int64_t *ce, int32_t *ccol, T *cval,
                    double *part, cudaStream_t s);

// ---------------------------------------------------------------- filter
// Per-matrix scalars after the check of the current iterates.
struct MatScalars {
  double r;      // ||T - I||_F / sqrt(n)
  double x;      // ||X||_F / sqrt(n)
  double beta;   // RMS budget (Eq. 1.18 or c4 * tol_stage)
  double b;      // absolute Frobenius budget sqrt(n) * beta
  double tau;    // element threshold of the filter
  double fnorm;  // ||F||_F dropped
  int64_t nnz_x, nnz_t, nnz_bar, nnz_hat;
  // threshold select: squares on the grid 2^(2e - 62) with 2^e <= b < 2^(e+1)
  unsigned long long sel_q;  // q(b) = floor(b^2 / 2^(2e - 62))
  unsigned long long tiny;   // keys below this have q == 0 (all ones: no key is summed)
  int sel_e;                 // e + 1023, the biased exponent of b (1 for a subnormal b)
  int sel_pad;
};
// From sums[2m] = sum (T-I)^2, sums[2m+1] = sum X^2: r, x, beta, b.
void launch_matrix_scalars(int nb, const int64_t *moff, const double *sums, double c4,
                           double tol_stage, double switch_resid, MatScalars *ms, cudaStream_t s);
// ---------------------------------------------------------------- 2-norm
// ||X||_2 estimates for the budget_norm variant (see kernels_norm2.cu):
// v_0 = (1,...,1)/sqrt(n), NORM2_STEPS steps v <- X^T X v / ||X^T X v||, then
// x2[m] = ||X v||. Work arrays: v, y, z, part of n doubles, zacc of 2n
// uint64, xmax, ymax of nb uint64, nrm of nb doubles.
constexpr int NORM2_STEPS = 8;
struct Norm2Work {
  double *v, *y, *z, *part, *nrm;
  unsigned long long *zacc, *xmax, *ymax;
};
// Only the matrices with ms[m].r < switch_resid (the adaptive phase) are
// estimated; x2 of the others is left undefined.
void launch_norm2_est(int nb, const int64_t *moff, const int32_t *seg, int64_t n, const Rows &X,
                      const void *val, int val_f32, const MatScalars *ms, double switch_resid,
                      const Norm2Work &wk, double *x2, cudaStream_t s);

// budget_norm: beta and b of Eq. (1.18) recomputed with x = x2[m] for the
// matrices in the adaptive phase (r < switch_resid).
void launch_budget_x2(int nb, const int64_t *moff, const double *x2, double switch_resid,
                      MatScalars *ms, cudaStream_t s);

// The values a threshold is selected over: row r holds entries [rs[r], re[r])
// of matrix seg[r]; rs == nullptr means one flat array of flat_nnz values of
// matrix 0, cut into rows of kFlatRow values.
constexpr int64_t kFlatRow = 16384;
struct SelRows {
  int64_t nrows;
  const int32_t *seg;
  const int64_t *rs;
  const int64_t *re;
  int64_t flat_nnz;
};

// Threshold selection (EXACT) for every active matrix; writes ms[m].tau.
// The scratch holds, 256-byte aligned each: the level-0 histograms (1024
// 128-bit sums per matrix), the digit histograms (256 per matrix), one
// minimum per matrix, one select state of at most kSelStateBytes per matrix,
// the candidate count, and room for cap candidates (8-byte key + row).
constexpr size_t kSelStateBytes = 64;
constexpr size_t sel_align(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t select_scratch_bytes(int nb, int64_t cap) {
  return sel_align(size_t(nb) * 1024 * 2 * 8) + sel_align(size_t(nb) * 256 * 2 * 8) +
         sel_align(size_t(nb) * 8) + sel_align(size_t(nb) * kSelStateBytes) + sel_align(8) +
         sel_align(size_t(cap > 0 ? cap : 1) * 8) + sel_align(size_t(cap > 0 ? cap : 1) * 4);
}
// cand_cap is the scratch's candidate room. Candidates past it are counted
// but not kept, and the thresholds (and counts) are then not valid: the
// caller compares the count (*select_cand_count) with cand_cap and selects
// again with room for every value when it is exceeded.
// cnt, dropped (nullable, R.nrows each; R must have rows rs/re): the
// filter's per-row kept counts and dropped sums of squares under the
// selected tau, as launch_filter_count gives them, except that the squares of
// the dropped entries of the crossing bucket are left out: add them per
// matrix with launch_select_drop_fix once dropped is summed per matrix.
void launch_select_exact(int nb, const SelRows &R, int64_t cand_cap, const int *active,
                         const void *val, int val_f32, MatScalars *ms, void *scratch,
                         int64_t *cnt, double *dropped, cudaStream_t s);
// sums[m] += the squares of matrix m's dropped entries of its crossing bucket
// (after launch_select_exact with counts, on the same scratch).
void launch_select_drop_fix(int nb, const int *active, void *scratch, const MatScalars *ms,
                            double *sums, cudaStream_t s);
const unsigned long long *select_cand_count(void *scratch, int nb);
// ms[m].nnz_bar = nnz[m].
void launch_store_nnz_bar(int nb, const int64_t *nnz, MatScalars *ms, cudaStream_t s);
// BOUND: tau = b / sqrt(nnz_bar) per matrix.
void launch_select_bound(int nb, const int *active, MatScalars *ms, cudaStream_t s);

// Keeps |x| >= tau_m and x != 0 (filter != NONE), counts kept entries per
// row and the dropped sum of squares per row.
void launch_filter_count(int64_t n, const int32_t *seg, const int *active, const int64_t *rs,
                         const int64_t *re, const void *val, int val_f32, const MatScalars *ms,
                         int64_t *cnt, double *dropped, cudaStream_t s);
void launch_filter_write(int64_t n, const int32_t *seg, const int *active, const int64_t *rs,
                         const int64_t *re, const int32_t *col, const void *val, int val_f32,
                         const MatScalars *ms, const int64_t *orp, int32_t *ocol, void *oval,
                         cudaStream_t s);

// ---------------------------------------------------------------- NMF (Alg. 3.1.1)
// The inverse of the n x n FP64 matrix in lu (leading dimension ld; factored
// in place) by LU with partial pivoting and one forward and back substitution
// per column of the identity, into inv (same ld). perm: n ints; pivot: one
// int; *singular = 1 (and inv undefined) if a pivot column is zero.
void launch_dense_inverse(int n, int ld, double *lu, int *perm, int *pivot, int *singular,
                          double *inv, cudaStream_t s);
// *out = ||inv||_F / sqrt(n) (part: n doubles of scratch).
void launch_inv_norm(int n, int ld, const double *inv, double *part, double *out,
                     cudaStream_t s);
// The n rows of a matrix (rows row0 .. of a compact CSR, columns from row0)
// into the zeroed dense block dx.
void launch_nmf_densify(int n, int ld, const int64_t *rp, const int32_t *col, const double *val,
                        int64_t row0, double *dx, cudaStream_t s);
// Xbar = (X + X^-1) / 2 into n full rows of slots from slot0: rows row0 ..
// of (rs, re, col, val), global columns from row0.
void launch_nmf_combine(int n, int ld, const double *dx, const double *inv, int64_t row0,
                        int64_t slot0, int64_t *rs, int64_t *re, int32_t *col, double *val,
                        cudaStream_t s);
// ms[m].beta and .b by Eq. (1.13): c4 tol while r >= switch_resid, else
// r^2 / (x + ||X^-1||) with *xinv = ||X^-1||_F / sqrt(n).
void launch_nmf_budget(int m, int64_t n, const double *xinv, double c4, double tol,
                       double switch_resid, MatScalars *ms, cudaStream_t s);

// ---------------------------------------------------------------- dense (a9)
// C = A Bt^T on the tensor cores (split TF32: three kind::tf32 MMAs per K step,
// FP32 accumulation in tensor memory). A (M x K) and Bt (N x K) are row-major
// FP32, each given split into hi (rounded to TF32) and lo = x - hi, with
// leading dimensions multiples of 4 and 16-byte aligned rows. C is written
// as FP32, or split into hi (C) and lo (C_lo) when C_lo is not null.
struct DenseJob {
  int M, N, K;
  const float *A_hi, *A_lo;
  int lda;
  const float *B_hi, *B_lo;
  int ldb;
  float *C, *C_lo;
  int ldc;
};
size_t dense_gemm_smem();
// Device scratch launch_dense_jobs needs for njobs jobs (tensor maps, tile offsets).
size_t dense_jobs_scratch_bytes(int njobs);
// jobs_host: the jobs on the host; jobs_dev: room for njobs DenseJob on the
// device; scratch: dense_jobs_scratch_bytes(njobs) device bytes, 64-byte
// aligned. *err |= 1 if a bounded wait gave up.
void launch_dense_jobs(int njobs, const DenseJob *jobs_host, DenseJob *jobs_dev, void *scratch,
                       int *err, cudaStream_t s);
// hi/lo split of a rows x cols matrix (or of the transpose of in), ldo >= cols.
void launch_split(int rows, int cols, const float *in, int ldi, int transpose, float *hi,
                  float *lo, int ldo, cudaStream_t s);

// ---------------------------------------------------------------- dense FP64 (a9)
// C = A Bt^T to about FP64 accuracy on the BF16 tensor cores from exact
// integer digits (see kernels_f64x.cu). The rows of A and of Bt are given as
// F64X_DIGITS digit planes, each rows x ld BF16 (plane s - 1 of an array of
// `rows` rows starts at row (s - 1) rows), with per-row scale exponents ea,
// eb (a_ik ~= 2^ea_i sum_s d_ik^(s) 2^(-7 s)). C is FP64, written (not
// accumulated); K is taken in exact blocks of F64X_MAX_K; lda and ldb
// multiples of 8, N and ldc even, C 16-byte and eb 8-byte aligned.
constexpr int F64X_DIGITS = 8;
constexpr int F64X_MAX_K = 4096;
struct SliceJob {
  int M, N, K;
  const uint16_t *A;
  int lda;
  const uint16_t *B;
  int ldb;
  const int *ea, *eb;
  double *C;
  int ldc;
  int accum;  // 1: C += A Bt^T (a later K block); 0: C = A Bt^T
};
size_t f64x_digits_bytes(int rows, int ld);
size_t slice_jobs_scratch_bytes(int njobs);
// Digit planes and scales of the rows of x (rows x K, leading dimension ldx),
// or of its columns when transpose; digits zero for K <= k < ld.
void launch_slices(int rows, int K, const double *x, int ldx, int transpose, uint16_t *digits,
                   int ld, int *w, cudaStream_t s);
void launch_slice_jobs(int njobs, const SliceJob *jobs_host, SliceJob *jobs_dev, void *scratch,
                       int *err, cudaStream_t s);

int f64x_pairs();  // digit pairs one product multiplies

// The dense blocks of one matrix on the dense path of the FP64 stage, n x n
// with leading dimension ld (a multiple of 8): X, T^T = (X X)^T and P = X T
// in FP64, and the digit planes (rows of kd BF16 digits) and row exponents of
// the two operands of one K block of F64X_MAX_K columns at a time: the
// products run block by block, each block's digits cut from X, X^T (read
// transposed from X) or T^T just before its product, so that no whole-matrix
// digit planes are held.
struct DenseBuf64 {
  double *X, *TT, *P;
  uint16_t *dA, *dB;
  int *eA, *eB;
  int n, ld, kd;
};
// K-block digit row length of a dense FP64 block of leading dimension ld.
constexpr int f64x_kd(int ld) { return ((ld < F64X_MAX_K ? ld : F64X_MAX_K) + 31) / 32 * 32; }
// The FP64 stage's CSR rows of the dense-path matrices into their zeroed X
// blocks.
void launch_densify64(int64_t n, const int32_t *seg, const int *dslot, const int64_t *moff,
                      const int64_t *rp, const int32_t *col, const double *val,
                      const DenseBuf64 *bufs, cudaStream_t s);
// part[2r] = sum_j (t_rj - delta_rj)^2 over row r of T^T, part[2r+1] =
// sum_j x_rj^2 (FP64, fixed order); tcount[d] += nonzeros of T.
void launch_dense_resid64(int64_t n, const int32_t *seg, const int *dslot, const int64_t *moff,
                          const DenseBuf64 *bufs, double *part, unsigned long long *tcount,
                          cudaStream_t s);
// Xbar = 1.5 X - 0.5 P (each product and the difference rounded once), its
// nonzeros in column order into the row slots [cs[r], ce[r]).
void launch_dense_emit64(int64_t n, const int32_t *seg, const int *dslot, const int64_t *moff,
                         const int *active, const DenseBuf64 *bufs, const int64_t *cs,
                         int64_t *ce, int32_t *ccol, double *cval, cudaStream_t s);

// The dense blocks of one matrix on the dense path, n x n with leading
// dimension ld (a multiple of 4): X and X^T split, T^T = (X X)^T split, and
// P = X T.
struct DenseBuf {
  float *X_hi, *X_lo, *XT_hi, *XT_lo, *TT_hi, *TT_lo, *P;
  int n, ld;
};
// dslot[m] = index into bufs for matrices on the dense path, -1 otherwise.
void launch_densify(int64_t n, const int32_t *seg, const int *dslot, const int64_t *moff,
                    const int64_t *rp, const int32_t *col, const float *val, const DenseBuf *bufs,
                    cudaStream_t s);
void launch_dense_resid(int64_t n, const int32_t *seg, const int *dslot, const int64_t *moff,
                        const DenseBuf *bufs, double *part, unsigned long long *tcount,
                        cudaStream_t s);
void launch_dense_emit(int64_t n, const int32_t *seg, const int *dslot, const int64_t *moff,
                       const int *active, const DenseBuf *bufs, const int64_t *cs, int64_t *ce,
                       int32_t *ccol, float *cval, cudaStream_t s);

}  // namespace sgn
