/*
 * sign.h — C ABI of the GB300 filtered Newton-Schulz sign solver.
 *
 * Computes S = sign(A) for a square sparse matrix A with the filtered
 * Newton-Schulz iteration (NSF) of Wu et al., "Two iterative algorithms for
 * the matrix sign function based on the adaptive filtering technology",
 * arXiv 2210.03356, Alg. 3.2.1:
 *
 *   X_1 = A (optionally A / ||A||_1);  e_1 = ||I - X_1^2||
 *   while e_k > tol:
 *       Xbar_{k+1} = 1/2 X_k (3I - X_k^2)            (two sparse products)
 *       X_{k+1}    = Xbar_{k+1} - F_{k+1}            (drop entries below tau_k)
 *       e_{k+1}    = ||I - X_{k+1}^2||
 *
 * The bound on ||F_k|| is c4*tol while e_k >= switch_resid and
 * 3/4 e_k^2 / (3x + x^3), x = ||X_k||, afterwards (Eq. 1.18; Sec. 3.2 and
 * Sec. 4 for the two phases). Norms are Frobenius divided by sqrt(n).
 *
 * Every step runs in CUDA kernels on the current device; there is no CPU
 * fallback. Matrices are CSR with
 *   rowptr int64[n+1] (rowptr[0] = 0, non-decreasing),
 *   col    int32[nnz] (0 <= col < n, strictly ascending inside a row),
 *   val    double[nnz] (finite).
 *
 * Conventions
 *   - Every function returns a sign_status; no C++ exception crosses the ABI.
 *     On failure sign_last_error() describes the last error of the calling
 *     thread (valid until that thread's next call).
 *   - sign_create copies its inputs; the caller keeps ownership of its arrays.
 *   - The CUDA stream passed to sign_create is borrowed, not owned. All work of
 *     a handle is ordered on it; sign_solve and sign_get_csr return after the
 *     stream has finished the work they queued.
 *   - A handle is not thread-safe; distinct handles are independent.
 *   - Device memory is allocated stream-ordered (cudaMallocAsync) on the
 *     handle's stream and released by sign_destroy or the end of a solve.
 */
#ifndef GB300_SIGN_H
#define GB300_SIGN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sign_ctx *sign_t; /* opaque, owned by the library */

typedef enum {
  SIGN_OK = 0,        /* converged: ||X^2 - I||_F/sqrt(n) <= tol            */
  SIGN_EINVAL = 1,    /* invalid argument or malformed CSR                   */
  SIGN_ENOMEM = 2,    /* device allocation failed                            */
  SIGN_ENOTCONV = 3,  /* max_iter updates done without reaching tol          */
  SIGN_EDIVERGED = 4, /* residual non-finite or above div_limit (Sec. 2:
                         convergence needs ||I - X_1^2|| < 1)                 */
  SIGN_ECUDA = 5,     /* a CUDA runtime call failed                          */
  SIGN_ETIMEOUT = 6,  /* a bounded wait of a tensor-core kernel gave up     */
  SIGN_ESTATE = 7,    /* call out of order (e.g. sign_get_csr before solve)  */
  SIGN_EAGAIN = 8     /* server: the request has not finished yet, or a
                         submission was refused for its predicted wait        */
} sign_status;

typedef enum {
  SIGN_FILTER_NONE = 0,  /* plain Newton-Schulz: nothing dropped             */
  SIGN_FILTER_EXACT = 1, /* drop the largest set of smallest magnitudes whose
                            Frobenius norm fits the budget; equal magnitudes
                            are dropped or kept together                     */
  SIGN_FILTER_BOUND = 2  /* drop |x| < b / sqrt(nnz(Xbar)) (never exceeds b) */
} sign_filter;

typedef enum {
  SIGN_METHOD_NSF = 0, /* filtered Newton-Schulz, Alg. 3.2.1                  */
  SIGN_METHOD_NMF = 1  /* Newton's method with filtering, Alg. 3.1.1: X_{k+1} =
                          (Xhat_k + Xhat_k^-1)/2 with a dense inverse (LU with
                          partial pivoting), budget c4*tol, then Eq. (1.13)
                          r^2/(x + ||X^-1||); X_1 = A (no scaling), FP64 only,
                          n <= 32768; filter NONE is Newton's method, Eq. (1.1) */
} sign_method;

typedef enum {
  SIGN_PREC_FP64 = 0,  /* FP64 values and fused multiply-adds throughout     */
  SIGN_PREC_MIXED = 1  /* FP32 values and accumulation until the residual is
                          below fp32_until, then FP64; norms, budgets and
                          thresholds are FP64 in both stages                 */
} sign_prec;

typedef struct {
  double tol;          /* stop when ||X^2 - I||_F/sqrt(n) <= tol; 1e-8       */
  int filter;          /* sign_filter; SIGN_FILTER_EXACT                     */
  double c4;           /* fixed budget factor (Sec. 3.2); 1e-4               */
  double switch_resid; /* fixed -> Eq. (1.18) budget below this; 1e-6        */
  int max_iter;        /* maximum Newton-Schulz updates; 100                 */
  int prec;            /* sign_prec; SIGN_PREC_FP64                          */
  double fp32_until;   /* FP32 stage ends below this residual; 1e-4          */
  double dense_frac;   /* a matrix whose iterate holds at least
                          dense_frac n^2 entries (n <= 65536, a filter on,
                          its dense blocks fitting in the free memory)
                          runs its products on the dense tensor-core path
                          in that round; > 1 turns the path off; 0.25      */
  int scale_1norm;     /* 1: X_1 = A/||A||_1 (default); 0: X_1 = A (paper)   */
  double div_limit;    /* residual above this = diverged; 1e6                */
  int dense64_min_n;   /* the FP64 stage's dense path (36 exact digit-pair
                          products per tile) only for n >= this; 1024      */
  int fp32_band;       /* 1: FP32 products of groups of 16 narrow-band rows
                          run as band tiles (dense register-blocked FMAs in
                          ascending k; the same values bit for bit); 0: the
                          row-wise kernels only; 1                        */
  int filter_t;        /* variant: 1 = T = X^2 is filtered too, with the same
                          budget and filter, before the update uses it (the
                          dense path is then off); 0                       */
  int budget_norm;     /* variant: 1 = x in Eq. (1.18) is ||X||_2, estimated
                          by 8 power steps on X^T X from (1,...,1)/sqrt(n);
                          0 = RMS Frobenius ||X||_F/sqrt(n); 0             */
  int method;          /* sign_method; SIGN_METHOD_NSF                       */
  /* Schedule: which kernel runs which rows. It changes the speed; every
   * schedule gives the same products bit for bit (each still adds its terms
   * in ascending k), and so the same iterates and results, except where a
   * residual within a rounding of a threshold (tol, fp32_until,
   * switch_resid) is summed in another order. sign_tune_batch picks one by
   * timing. */
  double band_min_eff; /* an FP32 group of 16 rows runs as a band tile when its
                          multiply-adds fill at least this fraction of the
                          tile's FMA slots (>= 0); 0.08                     */
  double group_margin; /* an FP64 row moves to 16 or 8 lanes when that raises
                          the lanes' use in a k-step by more than this; < 0
                          keeps every row on 32 lanes; 0.05                */
  int pair_rows;       /* 1: FP32 rows that fit half a warp's accumulator run
                          two per warp, sharing their passes over B; 0: one
                          row per warp; 1                                  */
} sign_opts;

/* Per-iteration record, filled by sign_solve when non-NULL. The arrays are
 * caller-owned with `cap` slots each (any may be NULL). Record k describes
 * the check of iterate X_k (k = 0 is X_1 of the paper) and, when an update
 * followed it, the filter that formed the next iterate. In the mixed mode
 * the iterate at the switch has two records (FP32 check, then FP64 check). */
typedef struct {
  int iters;          /* out: Newton-Schulz updates performed                */
  int status;         /* out: sign_status of this matrix                     */
  double resid;       /* out: final ||X^2 - I||_F / sqrt(n)                  */
  int64_t nnz_final;  /* out: nnz of the result                              */
  int cap;            /* in: slots in each array below                       */
  int count;          /* out: records written                                */
  int64_t *nnz_x;     /* nnz of X_k                                          */
  int64_t *nnz_t;     /* nnz of T = X_k X_k                                  */
  double *resid_k;    /* ||T - I||_F / sqrt(n)                               */
  double *xnorm_k;    /* ||X_k||_F / sqrt(n)                                 */
  double *beta_k;     /* RMS budget for the next filter (0 if none)          */
  double *tau_k;      /* element threshold of the next filter                */
  double *fnorm_k;    /* ||F||_F dropped by the next filter                  */
  int64_t *nnz_bar;   /* nnz of Xbar before the next filter                  */
  int *prec_k;        /* 32 or 64                                            */
  double *mults_t;    /* multiply-adds of T = X_k X_k                        */
  double *mults_bar;  /* multiply-adds of X_k T of the next update           */
  int64_t *nnz_that;  /* nnz of the T the next update multiplies by (after
                         its filter with filter_t, else nnz_t)              */
} sign_info;

/* Fills *o with the defaults listed in sign_opts. */
void sign_default_opts(sign_opts *o);

/* Creates a handle holding a copy of A (n x n, CSR as above).
 * on_device = 1: the three arrays are device pointers; 0: host pointers.
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream).
 * The CSR is validated on the device; malformed input gives SIGN_EINVAL. */
sign_status sign_create(int64_t n, int64_t nnz, const int64_t *rowptr, const int32_t *col,
                        const double *val, int on_device, void *cuda_stream, sign_t *out);

/* sign_create for `count` matrices at once (arrays of their arguments):
 * the copies and checks of all of them are queued back to back on
 * cuda_stream, which is waited for once. When every array is device memory
 * (on_device = 1) or pinned, mapped host memory (cudaMallocHost,
 * cudaHostAlloc, cudaHostRegister), one gather kernel reads them all; other
 * host memory is copied with one cudaMemcpyAsync per array. The checks run
 * as one kernel over all matrices. On any error no handle is created,
 * every out[i] is NULL, and sign_last_error names the first bad matrix. */
sign_status sign_create_batch(int count, const int64_t *n, const int64_t *nnz,
                              const int64_t *const *rowptr, const int32_t *const *col,
                              const double *const *val, int on_device, void *cuda_stream,
                              sign_t *out);

/* Runs the solve (Alg. 3.2.1). Returns the matrix's status (SIGN_OK,
 * SIGN_ENOTCONV or SIGN_EDIVERGED leave a result to read) or an error. */
sign_status sign_solve(sign_t h, const sign_opts *o, sign_info *info);

/* Solves `count` independent matrices together: their rows are processed in
 * the same kernel launches, each matrix with its own residual, budget,
 * threshold, stage and stopping test, so every result is the one a lone
 * sign_solve gives. All work goes to hs[0]'s stream. infos may be NULL or an
 * array of `count`. Returns SIGN_OK if the batch ran (per-matrix outcomes are
 * in infos[i].status) or an error that applies to the whole call. */
sign_status sign_solve_batch(sign_t *hs, int count, const sign_opts *o, sign_info *infos);

/* Schedule tuning for a batch. */
typedef struct {
  int timed;          /* out: batch solves timed (0 when the choice was cached) */
  int cached;         /* out: 1 if the schedule came from the cache             */
  double ms_base;     /* out: best time of a batch solve with base's schedule
                         (0 when cached)                                       */
  double ms_best;     /* out: best time with the chosen schedule (0 when cached) */
} sign_tune_report;

/* Times schedules on this batch and writes the fastest into *best (a copy of
 * *base with band_min_eff, group_margin and pair_rows chosen). The sweep goes
 * one field at a time from base's values: band_min_eff over {0.02, 0.04,
 * 0.08, 0.16, 0.32}, group_margin over {-1, 0, 0.05, 0.15}, pair_rows over
 * {0, 1}; each candidate is timed as `reps` (>= 1) full sign_solve_batch
 * calls, keeping the best time. The choice is cached per workload key (the
 * precision mode, filter, method, count rounded to a power of two, and the
 * powers of two of the mean n and of the mean nnz per row), and a later call
 * with an equal key returns it without timing unless force = 1. The handles
 * are left with the result of the last solve (the same for every schedule).
 * rep may be NULL. Errors of a solve are returned as they are. */
sign_status sign_tune_batch(sign_t *hs, int count, const sign_opts *base, int reps, int force,
                            sign_opts *best, sign_tune_report *rep);

/* Copies the result out. Call first with row_ptr = col = val = NULL to get
 * *nnz_out; then with buffers of n+1, nnz and nnz elements (device pointers if
 * on_device = 1). Columns are ascending inside each row. */
sign_status sign_get_csr(sign_t h, int64_t *nnz_out, int64_t *row_ptr, int32_t *col, double *val,
                         int on_device);

/* sign_get_csr for `count` handles at once (arrays of its arguments): the
 * copies are queued on each handle's stream, which is then waited for once
 * (so a batch solved together costs one wait instead of count). When the
 * handles share one stream and every output array is device memory
 * (on_device = 1) or pinned, mapped host memory, one gather kernel writes
 * them all; otherwise one cudaMemcpyAsync per array. Every handle
 * must hold a result; row_ptr, col and val must all be given, each array with
 * its handle's n+1 and nnz elements. On an error no copy is queued unless the
 * status is SIGN_ECUDA; sign_last_error names the first bad handle. */
sign_status sign_get_csr_batch(int count, const sign_t *hs, int64_t *const *row_ptr,
                               int32_t *const *col, double *const *val, int on_device);

/* Releases the handle and its device memory (NULL is ignored). */
void sign_destroy(sign_t h);

/* sign_destroy for `count` handles (NULL entries are skipped): each distinct
 * stream is waited for once, then every handle is freed. */
void sign_destroy_batch(const sign_t *hs, int count);

/* nnz_out[i] = the stored entries of handle i's result (as sign_get_csr with
 * no arrays). SIGN_ESTATE names the first handle without a result. */
sign_status sign_result_nnz_batch(int count, const sign_t *hs, int64_t *nnz_out);

/* Message of the calling thread's last failed call ("" if none). */
const char *sign_last_error(void);

/* EXACT element threshold (step a5) for one array of values, the rule the
 * solver applies per matrix: tau is the smallest magnitude v such that the
 * squares of all values with |x| <= v sum to more than b^2, so that dropping
 * every |x| < tau keeps the dropped Frobenius norm <= b (Sec. 3.1: the
 * threshold derived from a bound on ||F_k||; equal magnitudes share their
 * fate). If all values with |x| <= b fit, tau is the smallest magnitude above
 * b, and +inf if there is none.
 *   val: nnz doubles, device pointer if on_device = 1, else host.
 *   b:   the absolute Frobenius budget, finite and >= 0.
 *   tau_out: host pointer receiving tau.
 * Allocates its scratch stream-ordered (cudaMallocAsync) on cuda_stream and
 * returns after the stream has finished. SIGN_EINVAL for bad arguments. */
sign_status sign_threshold_exact(const double *val, int64_t nnz, double b, int on_device,
                                 void *cuda_stream, double *tau_out);

/* The same threshold as sign_threshold_exact without any device allocation,
 * for callers that cannot allocate: a process whose own pool already holds
 * the GPU's memory (so a library cudaMalloc would fail or eat into it), or a
 * loop that cannot afford the device-wide synchronization cudaMalloc/cudaFree
 * may cause. The paper has no counterpart; it is a deployment convenience.
 *   val: nnz doubles on the device (no host input: staging would allocate).
 *   nnz: at most SIGN_NOALLOC_MAX_NNZ, else SIGN_EINVAL with a message.
 * Scratch lives in one file-scope device array (about 12 MiB per GPU that
 * loads the library, held until exit). The first call on each device, made
 * with that device current, looks up the array's address
 * (cudaGetSymbolAddress). No call can be captured into a CUDA graph: each
 * copies its small inputs and the threshold through host memory and waits
 * for cuda_stream. All calls share the array: calls that overlap on the GPU
 * race, so the caller must serialize them. Returns after cuda_stream has
 * finished. */
#define SIGN_NOALLOC_MAX_NNZ ((int64_t)1 << 20)
sign_status sign_threshold_exact_noalloc(const double *val, int64_t nnz, double b,
                                         void *cuda_stream, double *tau_out);

/* Dense product C = A B on the tensor cores: the dense path (a9) for
 * matrices whose iterate has filled in. A (M x K), B (K x N) and C (M x N)
 * are row-major FP32 device arrays with leading dimensions lda, ldb, ldc
 * (elements). The product is split TF32: every operand is split as
 * hi + lo (hi rounded to TF32) and C = A_hi B_hi + A_hi B_lo + A_lo B_hi is
 * accumulated in FP32 by tcgen05 MMAs, which keeps about FP32 accuracy
 * (the sparse FP32 stage's products are FP32 FMAs). K, N and the leading
 * dimensions must be multiples of 4 and the arrays 16-byte aligned, else
 * SIGN_EINVAL. SIGN_ETIMEOUT if a bounded wait on the tensor cores gave up.
 * Returns after cuda_stream has finished. */
sign_status sign_dense_product(int M, int N, int K, const float *A, int lda, const float *B,
                               int ldb, float *C, int ldc, void *cuda_stream);

/* Dense product C = A B to about FP64 accuracy on the BF16 tensor cores: the
 * dense path (a9) of the FP64 stage. A (M x K), B (K x N) and C (M x N) are
 * row-major FP64 device arrays with leading dimensions lda, ldb, ldc
 * (elements). Each row of A and each column of B is scaled by a power of
 * two and cut into eight 7-bit integer digits (56 bits below its largest
 * entry); the 36 digit pairs of highest weight are multiplied exactly (BF16
 * digits, FP32 sums that stay integers below 2^24) and summed in FP64. The
 * error of an entry stays below about 2^-41 (K/4096) 2^(e_i + f_j), with
 * 2^e_i, 2^f_j bounding row i of A and column j of B (an FP64 dot product's
 * bound); K is taken in blocks of 4096, each summed exactly, the blocks
 * added in FP64. Needs N and ldc even and C 16-byte aligned, else
 * SIGN_EINVAL; SIGN_ETIMEOUT if a bounded wait on the tensor cores gave up.
 * Returns after cuda_stream has finished. */
sign_status sign_dense_product_f64(int M, int N, int K, const double *A, int lda, const double *B,
                                   int ldb, double *C, int ldc, void *cuda_stream);

/* ---- serving (not part of the paper's method) ---------------------------
 *
 * A server owns worker threads (one per lane) and CUDA streams of its own, on
 * the device current at creation. Requests are submitted from any thread;
 * each lane's worker runs its solver's rounds continuously and admits the
 * lane's waiting requests at each round boundary, first come first served,
 * while the sum of the admitted requests' predicted footprints stays within
 * mem_budget and fewer than max_active are on the GPU (both shared by the
 * lanes). An admitted request joins the next round of its lane's entry
 * stage beside the requests already in flight; each
 * request's arithmetic is that of a lone sign_solve with the server's
 * options, so its result is the same alone or in any mix. A request whose
 * predicted footprint alone exceeds mem_budget is refused at submission.
 *
 * Predicted footprint (bytes) of a request, from its n, nnz, Gershgorin
 * gap delta = min_i (|a_ii| - sum_{j!=i} |a_ij|), row-sum bound
 * rho = max_i sum_j |a_ij| and half-bandwidth bw = max |i - j|:
 *   w = n                                          if delta <= 0,
 *   w = min(n, max(32, ceil(1.5 (rho/delta) (2 bw + 1))))  otherwise,
 *   bytes = 96 n w + 80 n^2 [if 4 w >= n] + 24 nnz.
 * w predicts the filtered iterate's entries per row: the sign of a matrix
 * whose spectrum avoids (-delta, delta) decays away from the band at a rate
 * set by rho/delta; without a Gershgorin gap no decay is assumed (dense).
 * 96 bytes per predicted entry covers the iterate, its square, the update
 * slots and the filtered copy in FP64 (12 bytes per entry each, with the
 * products' upper-bound slots counted twice); 80 bytes per n^2 entry the
 * dense path's FP64 blocks and digit planes, taken when the fill is
 * predicted to reach a quarter of the row; 24 bytes per input entry the
 * input and its scaled copy. */
typedef struct sign_server_s *sign_server_t;

typedef struct {
  sign_opts solve;   /* options of every request                        */
  double mem_budget; /* bytes of predicted footprints in flight (120e9)  */
  int max_active;    /* requests on the GPU at once (1024)               */
  int max_queue;     /* requests waiting for admission (65536)           */
  int lanes;         /* 1, or 2 to give requests predicted to fill in (no
                        Gershgorin gap, or w >= n/4 in the model above) a
                        worker, solver and stream of their own, the other
                        lane's stream having the higher priority (2)      */
  double max_wait_s; /* latency target: a submission whose predicted wait
                        for admission exceeds this many seconds is refused
                        with SIGN_EAGAIN. The prediction is the requests
                        queued ahead on its lane divided by that lane's
                        completion rate over its last 64 completions (no
                        prediction before 8); 0 = no target (0)          */
} sign_server_opts;

typedef struct {
  double t_submit, t_admit, t_done; /* seconds on the server's steady clock */
  double footprint;                 /* predicted bytes, reserved while on the GPU */
  int lane;                         /* lane the request ran on */
} sign_request_times;

typedef struct {
  /* requests, cumulative: submitted counts valid inputs (sign_create's
   * checks passed), refused those of them turned away at submission */
  int64_t submitted, refused, admitted, completed;
  int64_t queued, active;                          /* requests, now          */
  int64_t max_active_seen;  /* most requests on the GPU at once so far       */
  int64_t rounds;           /* solver rounds run                             */
  double reserved;          /* bytes of predicted footprint now in flight    */
} sign_server_stats;

/* The footprint model above (host arithmetic only). */
double sign_footprint_bytes(int64_t n, int64_t nnz, double delta, double rho, int64_t bw);

/* Defaults: sign_default_opts with SIGN_PREC_MIXED, mem_budget 120e9,
 * max_active 1024, max_queue 65536, lanes 2. */
void sign_server_default_opts(sign_server_opts *o);

/* Starts a server. SIGN_EINVAL for bad options. */
sign_status sign_server_create(const sign_server_opts *o, sign_server_t *out);

/* Copies a CSR matrix (the arguments of sign_create) and queues it. Returns
 * after the copy: the caller may reuse its arrays at once. *ticket names the
 * request. SIGN_EINVAL for malformed input, SIGN_ENOMEM when the predicted
 * footprint exceeds mem_budget or max_queue requests are waiting, SIGN_EAGAIN
 * when its predicted wait exceeds max_wait_s (the request is then refused
 * and has no ticket). */
sign_status sign_server_submit(sign_server_t srv, int64_t n, int64_t nnz, const int64_t *rowptr,
                               const int32_t *col, const double *val, int on_device,
                               uint64_t *ticket);

/* SIGN_EAGAIN while the request is queued or running (after waiting up to
 * wait_ms milliseconds for it); SIGN_OK once it has finished, with its
 * outcome in info->status (iters, resid, nnz_final filled; no per-iteration
 * arrays) and its times in *times (either may be NULL). SIGN_EINVAL for an
 * unknown or already taken ticket. */
sign_status sign_server_poll(sign_server_t srv, uint64_t ticket, int wait_ms, sign_info *info,
                             sign_request_times *times);

/* Hands a finished request's result over as a handle (read it with
 * sign_get_csr, free it with sign_destroy); later work on the handle goes to
 * cuda_stream. The ticket is then forgotten. SIGN_EAGAIN if not finished. */
sign_status sign_server_take(sign_server_t srv, uint64_t ticket, void *cuda_stream, sign_t *out);

sign_status sign_server_get_stats(sign_server_t srv, sign_server_stats *out);

/* Stops admitting, lets the requests on the GPU finish, and frees the server
 * with every request not yet taken. The other sign_server_* calls may come
 * from any threads at once; this one must not overlap any of them. */
void sign_server_destroy(sign_server_t srv);

/* ---- observability (not part of the paper's method) -------------------- */

/* Total CUDA kernel launches made by this library in this process. */
int64_t sign_kernel_launches(void);

/* Device memory. The library allocates from its own stream-ordered pool,
 * which keeps freed memory for reuse, and each host thread that solves also
 * keeps the blocks it freed for its next solve (server lanes do not). This
 * returns the calling thread's kept blocks to the pool and the pool's unused
 * memory to the device. It synchronizes the device. Errors: SIGN_ECUDA. */
sign_status sign_trim_memory(void);

/* Per-kernel-class timing. When enabled, every group of launches of one
 * class is bracketed by CUDA events recorded on the stream it runs on.
 * flops counts two per multiply-add of a sparse product (the products the
 * method must do); bytes counts the algorithmic traffic of the class: each
 * operand's values, column indices and row pointers read once and each
 * output written once. Classes named host_* are wall times of the solver's
 * host phases, except host_sync_gap: the device time from the end of the
 * work queued before each of the solver's host synchronizations to the start
 * of the next timed launch, i.e. how long the GPU idles around the waits. */
typedef struct {
  char name[32];
  int64_t launches; /* timed groups of launches                      */
  double ms;        /* summed device time                              */
  double flops;     /* algorithmic floating-point operations           */
  double bytes;     /* algorithmic DRAM bytes                           */
} sign_prof_entry;

/* Peak probe of the FMA pipes (FP64 if fp64, else FP32), for the rooflines
 * of the sparse products: queues one launch of `blocks` x `threads` threads
 * (threads a multiple of 32, at most 1024), each running 8 independent
 * register-resident fused multiply-add chains for `iters` steps, on
 * cuda_stream, and returns at once; the caller times it (CUDA events on that
 * stream). *flops_out receives the launch's flops, 2 per multiply-add.
 * SIGN_EINVAL for bad sizes, SIGN_ECUDA if the launch failed. */
sign_status sign_fma_probe(int fp64, int blocks, int threads, int iters, void *cuda_stream,
                           double *flops_out);

/* Turns timing on (1) or off (0); returns the previous setting. */
int sign_prof_enable(int on);
/* Waits for the recorded events, writes up to cap entries (one per kernel
 * class) and returns the number written (out = NULL: the class count). */
int sign_prof_read(sign_prof_entry *out, int cap);
/* Clears the accumulated timings. */
void sign_prof_reset(void);

#ifdef __cplusplus
}
#endif
#endif
