/*
 * Plain CPU oracle for the filtered Newton-Schulz (NSF) sign iteration.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing on the library's compute path includes,
 * links or calls this code: only the tests, the package smoke check and the
 * benchmark's CPU-baseline leg do. It shares no code with the CUDA path.
 *
 * Every matrix is CSR: rowptr int64[n+1], col int32[nnz] ascending within a
 * row without duplicates, val double[nnz] (or float[nnz] in the FP32 stage).
 * All functions are single-threaded and allocate their outputs with malloc;
 * release them with oracle_free.
 */
#ifndef SIGN_ORACLE_H
#define SIGN_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_FILTER_NONE = 0, OR_FILTER_EXACT = 1, OR_FILTER_BOUND = 2 };
enum { OR_OK = 0, OR_EINVAL = 1, OR_ENOMEM = 2, OR_ENOTCONV = 3, OR_EDIVERGED = 4 };

typedef struct {
  double tol;          /* stop when ||X^2 - I||_F / sqrt(n) <= tol          */
  int filter;          /* OR_FILTER_*                                        */
  double c4;           /* fixed-budget factor, 1e-4 (Sec. 3.2)               */
  double switch_resid; /* fixed -> adaptive budget below this residual, 1e-6 */
  int max_iter;        /* maximum number of Newton-Schulz updates            */
  int mixed;           /* 1: FP32 stage until resid < fp32_until, then FP64  */
  double fp32_until;   /* 1e-4                                               */
  int scale_1norm;     /* 1: X0 = A / ||A||_1, 0: X0 = A                     */
  double div_limit;    /* residual above this (or non-finite) = diverged     */
  int filter_t;        /* variant: 1 = T = X^2 filtered too, with the same
                          budget, before the update uses it                  */
  int budget_norm;     /* variant: 1 = x in Eq. (1.18) is the 2-norm of X,
                          estimated by ORACLE_POW_STEPS power steps on X^T X;
                          0 = RMS Frobenius (the default reading)            */
} oracle_opts;

/* Power steps of the 2-norm estimate (budget_norm = 1). */
#define ORACLE_POW_STEPS 8

/* Per-iteration record. Arrays are caller-owned with `cap` slots; entry k
 * describes the check of iterate X_k (k = 0 is X0) and, when an update
 * follows it, the filter applied to form X_{k+1}. */
typedef struct {
  int cap, count;
  int64_t *nnz_x;   /* nnz of X_k                                */
  int64_t *nnz_t;   /* nnz of T = X_k X_k                         */
  double *resid;    /* ||T - I||_F / sqrt(n)                      */
  double *xnorm;    /* ||X_k||_F / sqrt(n)                        */
  double *beta;     /* RMS budget used for X_{k+1} (0 if none)    */
  double *tau;      /* element threshold used for X_{k+1}         */
  double *fnorm;    /* ||F_{k+1}||_F, the dropped part            */
  int64_t *nnz_bar; /* nnz of Xbar_{k+1} before filtering         */
  int *prec;        /* 32 or 64: precision of iterate k           */
  int64_t *nnz_that; /* nnz of T after its filter (filter_t; else nnz_t); nullable */
} oracle_trace;

typedef struct {
  int64_t n, nnz;
  int64_t *rowptr;
  int32_t *col;
  double *val;
} or_csr;

void oracle_free(void *p);

/* ||A||_1 with reproducible column sums (see oracle.c). */
double oracle_onenorm(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val);

/* C = A B, Gustavson row by row, ascending k, fma accumulation, structural
 * pattern kept (exact zeros included). Returns OR_OK or OR_ENOMEM. */
int oracle_spgemm(int64_t n, const int64_t *arp, const int32_t *acol, const double *aval,
                  const int64_t *brp, const int32_t *bcol, const double *bval,
                  int64_t **crp, int32_t **ccol, double **cval);
int oracle_spgemm_f32(int64_t n, const int64_t *arp, const int32_t *acol, const float *aval,
                      const int64_t *brp, const int32_t *bcol, const float *bval,
                      int64_t **crp, int32_t **ccol, float **cval);

/* ||T - I||_F / sqrt(n) and ||X||_F / sqrt(n). */
double oracle_resid_rms(int64_t n, const int64_t *rp, const int32_t *col, const double *val);
double oracle_resid_rms_f32(int64_t n, const int64_t *rp, const int32_t *col, const float *val);
double oracle_fro_rms(int64_t n, const int64_t *rp, const double *val);

/* Xbar = 1.5 X - 0.5 (X T) on the union pattern (Alg. 3.2.1 step 3). */
int oracle_ns_update(int64_t n, const int64_t *xrp, const int32_t *xcol, const double *xval,
                     const int64_t *trp, const int32_t *tcol, const double *tval,
                     int64_t **orp, int32_t **ocol, double **oval);

/* Filters (Alg. 3.2.1 step 4) given the absolute Frobenius budget b.
 * Outputs the kept matrix, tau and ||F||_F. */
int oracle_filter(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                  int mode, double b, int64_t **orp, int32_t **ocol, double **oval,
                  double *tau, double *fnorm);

/* 2-norm estimate of X: v_0 = (1, ..., 1)/sqrt(n), then `steps` times
 * v <- X^T X v / ||X^T X v||, and ||X v|| of the last v (long double sums).
 * A lower bound of ||X||_2 that converges to it as steps grow. */
double oracle_norm2_est(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                        int steps);

/* Budget (RMS) for the next filter: c4*tol_stage in the fixed phase, else
 * Eq. (1.18) as 3/4 r^2 / (3x + x^3). */
double oracle_budget(double r, double x, double c4, double tol_stage, double switch_resid);

/* Whole NSF / NS solve (filter NONE is plain NS). */
int oracle_nsf(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
               const oracle_opts *o, oracle_trace *tr, int *iters, double *resid,
               int64_t **srp, int32_t **scol, double **sval);

/* Newton's method with filtering (Alg. 3.1.1) on CSR input, dense inverse;
 * o->filter, tol, c4, switch_resid, max_iter and div_limit apply (no scaling,
 * no mixed precision). Outputs as oracle_nsf. */
int oracle_nmf(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
               const oracle_opts *o, oracle_trace *tr, int *iters, double *resid,
               int64_t **srp, int32_t **scol, double **sval);

/* Newton's method X <- (X + X^-1)/2 on a dense row-major matrix, X0 = A. */
int oracle_nm_dense(int64_t n, const double *a, double tol, int max_iter,
                    double *s, int *iters, double *resid);

#ifdef __cplusplus
}
#endif
#endif
