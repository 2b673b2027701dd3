/*
 * Plain CPU oracle for the filtered Newton-Schulz (NSF) sign iteration of
 * Wu et al., "Two iterative algorithms for the matrix sign function based on
 * the adaptive filtering technology" (arXiv 2210.03356).
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the library. It shares no code with
 * the CUDA path.
 *
 * Build with contraction off (-ffp-contract=off) so that every multiply and
 * add rounds on its own, identically on x86-64 and AArch64; products are
 * accumulated with fma() explicitly.
 *
 * What it follows:
 *   - Alg. 3.2.1 (NSF): X1 = A, e1 = ||I - X1^2||; while e_k > tol:
 *     Xbar = 1/2 X (3I - X^2); Xhat = Xbar - F; e = ||I - Xhat^2||.
 *     X (3I - X^2)/2 is evaluated as 1.5 X - 0.5 (X T) with T = X X, the T of
 *     the residual check, so one check and one update cost two products.
 *   - Eq. (1.18) and Sec. 3.2 / Sec. 4: the filter budget is c4*tol while the
 *     residual is >= 1e-6, then 3/4 r^2 / (3x + x^3).
 *   - Sec. 3.1: "filtering" drops the entries below a threshold; the paper
 *     derives the threshold from a bound on ||F|| with an algorithm of its
 *     Ref. [22] that it does not print. EXACT mode takes the largest set of
 *     smallest-magnitude entries whose Frobenius norm fits the bound, with
 *     equal magnitudes dropped or kept together; BOUND mode drops
 *     |x| < b / sqrt(nnz), which can never exceed the bound.
 *   - Eq. (1.1): Newton's method X <- (X + X^-1)/2, dense, for comparison.
 *   - Alg. 3.1.1 (NMF): Newton's method with the same filter, on CSR with a
 *     dense inverse, budget c4*tol and then Thm 3.1.2's bound (Eq. 1.13),
 *     r^2 / (x + x_inv).
 * Norms are Frobenius divided by sqrt(n) ("RMS"); the paper leaves the norm
 * unspecified.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

void oracle_free(void *p) { free(p); }

/* ---------------------------------------------------------------------- */
/* compensated (Neumaier) summation                                        */
/* ---------------------------------------------------------------------- */
typedef struct {
  double s, c;
} ksum;

static void kadd(ksum *k, double x) {
  double t = k->s + x;
  if (fabs(k->s) >= fabs(x))
    k->c += (k->s - t) + x;
  else
    k->c += (x - t) + k->s;
  k->s = t;
}

static double kval(const ksum *k) { return k->s + k->c; }

/* ---------------------------------------------------------------------- */
/* input validation                                                         */
/* ---------------------------------------------------------------------- */
static int valid_csr(int64_t n, const int64_t *rp, const int32_t *col, const double *val) {
  if (n < 1 || rp[0] != 0) return 0;
  for (int64_t i = 0; i < n; ++i) {
    if (rp[i + 1] < rp[i]) return 0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
      if (col[p] < 0 || col[p] >= n) return 0;
      if (p > rp[i] && col[p] <= col[p - 1]) return 0;
      if (!isfinite(val[p])) return 0;
    }
  }
  return 1;
}

/* ---------------------------------------------------------------------- */
/* ||A||_1 = max_j sum_i |a_ij|                                             */
/* ---------------------------------------------------------------------- */
/*
 * Column sums are made independent of summation order: with M = max |a_ij|
 * and M < 2^e, every |a_ij| is put on the fixed-point grid 2^(e-62)
 * (q = round-to-nearest-even of |a| * 2^(62-e), an exact scaling followed by
 * one rounding) and the q of a column are added exactly in 128-bit integers.
 * The largest column sum s is brought back as ((double)hi * 2^64 +
 * (double)lo) * 2^(e-62). The grid step is below 2^-62 of the largest entry,
 * so the result equals the ordinary floating-point 1-norm to within about
 * nnz_col * 2^-62 relative, and it is the same whatever order the entries
 * are visited in.
 */
double oracle_onenorm(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val) {
  double m = 0.0;
  int64_t nnz = rowptr[n];
  for (int64_t p = 0; p < nnz; ++p)
    if (fabs(val[p]) > m) m = fabs(val[p]);
  if (m == 0.0) return 0.0;
  int e;
  frexp(m, &e); /* m = f 2^e, f in [0.5, 1) */
  unsigned __int128 *cs = (unsigned __int128 *)calloc((size_t)n, sizeof(unsigned __int128));
  if (!cs) return NAN;
  for (int64_t p = 0; p < nnz; ++p) {
    double x = nearbyint(ldexp(fabs(val[p]), 62 - e));
    cs[col[p]] += (unsigned __int128)(uint64_t)x;
  }
  unsigned __int128 best = 0;
  for (int64_t j = 0; j < n; ++j)
    if (cs[j] > best) best = cs[j];
  free(cs);
  uint64_t hi = (uint64_t)(best >> 64), lo = (uint64_t)best;
  double d = (double)hi * 18446744073709551616.0 + (double)lo;
  return ldexp(d, e - 62);
}

/* ---------------------------------------------------------------------- */
/* sparse products (Gustavson)                                              */
/* ---------------------------------------------------------------------- */
static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

/* C = A B. Row i of C: for each k of row i of A in ascending order, for each
 * (j, b_kj) of row k of B in ascending order, acc_j = fma(a_ik, b_kj, acc_j)
 * starting from +0. Every column touched is emitted, ascending, even when its
 * sum is exactly zero (the symbolic pattern of the product). */
#define SPGEMM_BODY(T, FMA)                                                                \
  int64_t *mark = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);                          \
  int32_t *list = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);                          \
  T *acc = (T *)malloc(sizeof(T) * (size_t)n);                                             \
  int64_t *rp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));                      \
  int64_t cap = 16 + arp[n] * 2, len = 0;                                                  \
  int32_t *cc = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);                          \
  T *cv = (T *)malloc(sizeof(T) * (size_t)cap);                                            \
  if (!mark || !list || !acc || !rp || !cc || !cv) goto fail;                              \
  for (int64_t j = 0; j < n; ++j) mark[j] = -1;                                            \
  rp[0] = 0;                                                                               \
  for (int64_t i = 0; i < n; ++i) {                                                        \
    int64_t cnt = 0;                                                                       \
    for (int64_t p = arp[i]; p < arp[i + 1]; ++p) {                                        \
      int32_t k = acol[p];                                                                 \
      T a = aval[p];                                                                       \
      for (int64_t q = brp[k]; q < brp[k + 1]; ++q) {                                      \
        int32_t j = bcol[q];                                                               \
        if (mark[j] != i) {                                                                \
          mark[j] = i;                                                                     \
          acc[j] = (T)0;                                                                   \
          list[cnt++] = j;                                                                 \
        }                                                                                  \
        acc[j] = FMA(a, bval[q], acc[j]);                                                  \
      }                                                                                    \
    }                                                                                      \
    qsort(list, (size_t)cnt, sizeof(int32_t), cmp_i32);                                    \
    if (len + cnt > cap) {                                                                 \
      while (len + cnt > cap) cap *= 2;                                                    \
      int32_t *c2 = (int32_t *)realloc(cc, sizeof(int32_t) * (size_t)cap);                 \
      if (!c2) goto fail;                                                                  \
      cc = c2;                                                                             \
      T *v2 = (T *)realloc(cv, sizeof(T) * (size_t)cap);                                   \
      if (!v2) goto fail;                                                                  \
      cv = v2;                                                                             \
    }                                                                                      \
    for (int64_t t = 0; t < cnt; ++t) {                                                    \
      cc[len] = list[t];                                                                   \
      cv[len] = acc[list[t]];                                                              \
      ++len;                                                                               \
    }                                                                                      \
    rp[i + 1] = len;                                                                       \
  }                                                                                        \
  free(mark);                                                                              \
  free(list);                                                                              \
  free(acc);                                                                               \
  *crp = rp;                                                                               \
  *ccol = cc;                                                                              \
  *cval = cv;                                                                              \
  return OR_OK;                                                                            \
  fail:                                                                                    \
  free(mark);                                                                              \
  free(list);                                                                              \
  free(acc);                                                                               \
  free(rp);                                                                                \
  free(cc);                                                                                \
  free(cv);                                                                                \
  return OR_ENOMEM;

int oracle_spgemm(int64_t n, const int64_t *arp, const int32_t *acol, const double *aval,
                  const int64_t *brp, const int32_t *bcol, const double *bval,
                  int64_t **crp, int32_t **ccol, double **cval) {
  SPGEMM_BODY(double, fma)
}

int oracle_spgemm_f32(int64_t n, const int64_t *arp, const int32_t *acol, const float *aval,
                      const int64_t *brp, const int32_t *bcol, const float *bval,
                      int64_t **crp, int32_t **ccol, float **cval) {
  SPGEMM_BODY(float, fmaf)
}

/* ---------------------------------------------------------------------- */
/* norms                                                                    */
/* ---------------------------------------------------------------------- */
/* e = ||I - T||_F / sqrt(n), summed row by row with compensation; a row with
 * no stored diagonal contributes (0 - 1)^2 = 1 for it. */
#define RESID_BODY                                                       \
  ksum s = {0.0, 0.0};                                                   \
  for (int64_t i = 0; i < n; ++i) {                                      \
    int seen = 0;                                                        \
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {                        \
      double d = (double)val[p];                                         \
      if (col[p] == i) {                                                 \
        d = d - 1.0;                                                     \
        seen = 1;                                                        \
      }                                                                  \
      kadd(&s, d * d);                                                   \
    }                                                                    \
    if (!seen) kadd(&s, 1.0);                                            \
  }                                                                      \
  return sqrt(kval(&s)) / sqrt((double)n);

double oracle_resid_rms(int64_t n, const int64_t *rp, const int32_t *col, const double *val) {
  RESID_BODY
}
double oracle_resid_rms_f32(int64_t n, const int64_t *rp, const int32_t *col, const float *val) {
  RESID_BODY
}

double oracle_fro_rms(int64_t n, const int64_t *rp, const double *val) {
  ksum s = {0.0, 0.0};
  for (int64_t p = 0; p < rp[n]; ++p) kadd(&s, val[p] * val[p]);
  return sqrt(kval(&s)) / sqrt((double)n);
}

static double fro_rms_f32(int64_t n, const int64_t *rp, const float *val) {
  ksum s = {0.0, 0.0};
  for (int64_t p = 0; p < rp[n]; ++p) kadd(&s, (double)val[p] * (double)val[p]);
  return sqrt(kval(&s)) / sqrt((double)n);
}

/* ---------------------------------------------------------------------- */
/* Newton-Schulz update, Alg. 3.2.1 step 3                                  */
/* ---------------------------------------------------------------------- */
/* Xbar = 1/2 X (3I - X^2) = 1.5 X - 0.5 P with P = X T, on the union of the
 * patterns of X and P; an entry missing from one side counts as 0. */
#define UPDATE_BODY(T, SPG, C15, C05)                                                      \
  int64_t *prp = NULL;                                                                     \
  int32_t *pcol = NULL;                                                                    \
  T *pval = NULL;                                                                          \
  int rc = SPG(n, xrp, xcol, xval, trp, tcol, tval, &prp, &pcol, &pval);                   \
  if (rc) return rc;                                                                       \
  int64_t cap = xrp[n] + prp[n];                                                           \
  int64_t *rp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));                      \
  int32_t *oc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(cap > 0 ? cap : 1));          \
  T *ov = (T *)malloc(sizeof(T) * (size_t)(cap > 0 ? cap : 1));                            \
  if (!rp || !oc || !ov) {                                                                 \
    free(prp); free(pcol); free(pval); free(rp); free(oc); free(ov);                       \
    return OR_ENOMEM;                                                                      \
  }                                                                                        \
  int64_t len = 0;                                                                         \
  rp[0] = 0;                                                                               \
  for (int64_t i = 0; i < n; ++i) {                                                        \
    int64_t a = xrp[i], ae = xrp[i + 1], b = prp[i], be = prp[i + 1];                      \
    while (a < ae || b < be) {                                                             \
      int32_t ca = a < ae ? xcol[a] : INT32_MAX, cb = b < be ? pcol[b] : INT32_MAX;        \
      int32_t c = ca < cb ? ca : cb;                                                       \
      T xv = (T)0, pv = (T)0;                                                              \
      if (ca == c) xv = xval[a++];                                                         \
      if (cb == c) pv = pval[b++];                                                         \
      oc[len] = c;                                                                         \
      ov[len] = C15 * xv - C05 * pv;                                                       \
      ++len;                                                                               \
    }                                                                                      \
    rp[i + 1] = len;                                                                       \
  }                                                                                        \
  free(prp);                                                                               \
  free(pcol);                                                                              \
  free(pval);                                                                              \
  *orp = rp;                                                                               \
  *ocol = oc;                                                                              \
  *oval = ov;                                                                              \
  return OR_OK;

int oracle_ns_update(int64_t n, const int64_t *xrp, const int32_t *xcol, const double *xval,
                     const int64_t *trp, const int32_t *tcol, const double *tval,
                     int64_t **orp, int32_t **ocol, double **oval) {
  UPDATE_BODY(double, oracle_spgemm, 1.5, 0.5)
}

static int ns_update_f32(int64_t n, const int64_t *xrp, const int32_t *xcol, const float *xval,
                         const int64_t *trp, const int32_t *tcol, const float *tval,
                         int64_t **orp, int32_t **ocol, float **oval) {
  UPDATE_BODY(float, oracle_spgemm_f32, 1.5f, 0.5f)
}

/* ---------------------------------------------------------------------- */
/* filters, Alg. 3.2.1 step 4                                               */
/* ---------------------------------------------------------------------- */
static const double *g_sort_mag; /* single-threaded oracle: sort key source */
static int cmp_mag(const void *a, const void *b) {
  double x = g_sort_mag[*(const int64_t *)a], y = g_sort_mag[*(const int64_t *)b];
  return (x > y) - (x < y);
}

/* Decides which entries of Xbar are dropped; mag[p] = |x_p| in double.
 * EXACT: visit magnitudes in ascending order, one group of equal magnitudes
 * at a time; drop the group while the running sum of squares of everything
 * dropped stays <= b^2; tau is the magnitude of the first group kept (every
 * |x| < tau is dropped, every |x| >= tau kept), +inf if all fit.
 * BOUND: tau = b / sqrt(nnz); drop |x| < tau and exact zeros.
 * NONE: keep everything, tau = 0. */
static int filter_mask(int64_t nnz, const double *mag, int mode, double b, unsigned char *keep,
                       double *tau_out, double *fnorm_out) {
  ksum dropped = {0.0, 0.0};
  double tau = 0.0;
  if (mode == OR_FILTER_NONE) {
    for (int64_t p = 0; p < nnz; ++p) keep[p] = 1;
  } else if (mode == OR_FILTER_BOUND) {
    tau = nnz > 0 ? b / sqrt((double)nnz) : INFINITY;
    for (int64_t p = 0; p < nnz; ++p) {
      keep[p] = !(mag[p] < tau || mag[p] == 0.0);
      if (!keep[p]) kadd(&dropped, mag[p] * mag[p]);
    }
  } else if (mode == OR_FILTER_EXACT) {
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!idx) return OR_ENOMEM;
    for (int64_t p = 0; p < nnz; ++p) idx[p] = p;
    g_sort_mag = mag;
    qsort(idx, (size_t)nnz, sizeof(int64_t), cmp_mag);
    double b2 = b * b;
    tau = INFINITY;
    int64_t t = 0;
    while (t < nnz) {
      double v = mag[idx[t]];
      int64_t g = t;
      ksum trial = dropped;
      while (g < nnz && mag[idx[g]] == v) {
        kadd(&trial, v * v);
        ++g;
      }
      if (kval(&trial) <= b2) {
        dropped = trial;
        t = g;
      } else {
        tau = v;
        break;
      }
    }
    free(idx);
    for (int64_t p = 0; p < nnz; ++p) keep[p] = mag[p] >= tau;
  } else {
    return OR_EINVAL;
  }
  *tau_out = tau;
  *fnorm_out = sqrt(kval(&dropped));
  return OR_OK;
}

#define COMPACT_BODY(T)                                                                    \
  int64_t *rp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));                      \
  int64_t kept = 0;                                                                        \
  for (int64_t p = 0; p < irp[n]; ++p) kept += keep[p];                                    \
  int32_t *oc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(kept > 0 ? kept : 1));        \
  T *ov = (T *)malloc(sizeof(T) * (size_t)(kept > 0 ? kept : 1));                          \
  if (!rp || !oc || !ov) {                                                                 \
    free(rp); free(oc); free(ov);                                                          \
    return OR_ENOMEM;                                                                      \
  }                                                                                        \
  int64_t len = 0;                                                                         \
  rp[0] = 0;                                                                               \
  for (int64_t i = 0; i < n; ++i) {                                                        \
    for (int64_t p = irp[i]; p < irp[i + 1]; ++p)                                          \
      if (keep[p]) {                                                                       \
        oc[len] = icol[p];                                                                 \
        ov[len] = ival[p];                                                                 \
        ++len;                                                                             \
      }                                                                                    \
    rp[i + 1] = len;                                                                       \
  }                                                                                        \
  *orp = rp;                                                                               \
  *ocol = oc;                                                                              \
  *oval = ov;                                                                              \
  return OR_OK;

static int compact_f64(int64_t n, const int64_t *irp, const int32_t *icol, const double *ival,
                       const unsigned char *keep, int64_t **orp, int32_t **ocol, double **oval) {
  COMPACT_BODY(double)
}
static int compact_f32(int64_t n, const int64_t *irp, const int32_t *icol, const float *ival,
                       const unsigned char *keep, int64_t **orp, int32_t **ocol, float **oval) {
  COMPACT_BODY(float)
}

int oracle_filter(int64_t n, const int64_t *rp, const int32_t *col, const double *val, int mode,
                  double b, int64_t **orp, int32_t **ocol, double **oval, double *tau,
                  double *fnorm) {
  int64_t nnz = rp[n];
  double *mag = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  unsigned char *keep = (unsigned char *)malloc((size_t)(nnz > 0 ? nnz : 1));
  if (!mag || !keep) {
    free(mag);
    free(keep);
    return OR_ENOMEM;
  }
  for (int64_t p = 0; p < nnz; ++p) mag[p] = fabs(val[p]);
  int rc = filter_mask(nnz, mag, mode, b, keep, tau, fnorm);
  if (rc == OR_OK) rc = compact_f64(n, rp, col, val, keep, orp, ocol, oval);
  free(mag);
  free(keep);
  return rc;
}

static int filter_f32(int64_t n, const int64_t *rp, const int32_t *col, const float *val, int mode,
                      double b, int64_t **orp, int32_t **ocol, float **oval, double *tau,
                      double *fnorm) {
  int64_t nnz = rp[n];
  double *mag = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  unsigned char *keep = (unsigned char *)malloc((size_t)(nnz > 0 ? nnz : 1));
  if (!mag || !keep) {
    free(mag);
    free(keep);
    return OR_ENOMEM;
  }
  for (int64_t p = 0; p < nnz; ++p) mag[p] = fabs((double)val[p]);
  int rc = filter_mask(nnz, mag, mode, b, keep, tau, fnorm);
  if (rc == OR_OK) rc = compact_f32(n, rp, col, val, keep, orp, ocol, oval);
  free(mag);
  free(keep);
  return rc;
}

/* ---------------------------------------------------------------------- */
/* 2-norm estimate (the budget_norm variant of the reading of ||.||)        */
/* ---------------------------------------------------------------------- */
double oracle_norm2_est(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                        int steps) {
  double *v = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  double *y = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  long double *z = (long double *)malloc(sizeof(long double) * (size_t)(n > 0 ? n : 1));
  double out = NAN;
  if (!v || !y || !z || n <= 0) goto done;
  for (int64_t i = 0; i < n; ++i) v[i] = 1.0 / sqrt((double)n);
  for (int s = 0; s <= steps; ++s) {
    for (int64_t i = 0; i < n; ++i) { /* y = X v */
      long double a = 0.0L;
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) a += (long double)val[p] * v[col[p]];
      y[i] = (double)a;
    }
    if (s == steps) { /* ||X v|| of the last v */
      long double a = 0.0L;
      for (int64_t i = 0; i < n; ++i) a += (long double)y[i] * y[i];
      out = sqrt((double)a);
      break;
    }
    for (int64_t j = 0; j < n; ++j) z[j] = 0.0L; /* z = X^T y */
    for (int64_t i = 0; i < n; ++i)
      for (int64_t p = rp[i]; p < rp[i + 1]; ++p) z[col[p]] += (long double)val[p] * y[i];
    long double a = 0.0L;
    for (int64_t j = 0; j < n; ++j) a += z[j] * z[j];
    double nz = sqrt((double)a);
    if (!(nz > 0.0)) { /* X v = 0 or X^T y = 0: the estimate so far is the norm */
      long double b = 0.0L;
      for (int64_t i = 0; i < n; ++i) b += (long double)y[i] * y[i];
      out = sqrt((double)b);
      break;
    }
    for (int64_t j = 0; j < n; ++j) v[j] = (double)(z[j] / nz);
  }
done:
  free(v);
  free(y);
  free(z);
  return out;
}

/* ---------------------------------------------------------------------- */
/* budget, Eq. (1.18) and the fixed phase of Sec. 3.2 / Sec. 4              */
/* ---------------------------------------------------------------------- */
/* r = ||R_k|| of the iterate being updated, x = ||X_k||; both RMS. The
 * returned RMS budget becomes the absolute Frobenius bound sqrt(n)*beta. */
double oracle_budget(double r, double x, double c4, double tol_stage, double switch_resid) {
  if (r >= switch_resid) return c4 * tol_stage;
  return 0.75 * r * r / (3.0 * x + x * x * x);
}

/* ---------------------------------------------------------------------- */
/* whole solve                                                               */
/* ---------------------------------------------------------------------- */
static void trace_put(oracle_trace *tr, int64_t nnz_x, int64_t nnz_t, double r, double x, int prec) {
  if (!tr || tr->count >= tr->cap) return;
  int k = tr->count++;
  tr->nnz_x[k] = nnz_x;
  tr->nnz_t[k] = nnz_t;
  if (tr->nnz_that) tr->nnz_that[k] = nnz_t;
  tr->resid[k] = r;
  tr->xnorm[k] = x;
  tr->beta[k] = 0.0;
  tr->tau[k] = 0.0;
  tr->fnorm[k] = 0.0;
  tr->nnz_bar[k] = 0;
  tr->prec[k] = prec;
}

static void trace_that(oracle_trace *tr, int64_t nnz_that) {
  if (!tr || tr->count == 0 || tr->count > tr->cap || !tr->nnz_that) return;
  tr->nnz_that[tr->count - 1] = nnz_that;
}

static void trace_filter(oracle_trace *tr, double beta, double tau, double fnorm, int64_t nnz_bar) {
  if (!tr || tr->count == 0 || tr->count > tr->cap) return;
  int k = tr->count - 1;
  tr->beta[k] = beta;
  tr->tau[k] = tau;
  tr->fnorm[k] = fnorm;
  tr->nnz_bar[k] = nnz_bar;
}

int oracle_nsf(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
               const oracle_opts *o, oracle_trace *tr, int *iters, double *resid,
               int64_t **srp, int32_t **scol, double **sval) {
  if (!o || !valid_csr(n, rowptr, col, val)) return OR_EINVAL;
  if (tr) tr->count = 0;
  int64_t nnz = rowptr[n];
  /* X1 = A (Alg. 3.2.1 step 1), optionally scaled by 1/||A||_1. */
  int64_t *xrp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int32_t *xcol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  double *xval = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  float *xf = NULL;
  if (!xrp || !xcol || !xval) goto nomem;
  memcpy(xrp, rowptr, sizeof(int64_t) * (size_t)(n + 1));
  memcpy(xcol, col, sizeof(int32_t) * (size_t)nnz);
  if (o->scale_1norm) {
    double nrm = oracle_onenorm(n, rowptr, col, val);
    if (!(nrm > 0.0) || !isfinite(nrm)) {
      free(xrp);
      free(xcol);
      free(xval);
      return OR_EINVAL;
    }
    for (int64_t p = 0; p < nnz; ++p) xval[p] = val[p] / nrm;
  } else {
    memcpy(xval, val, sizeof(double) * (size_t)nnz);
  }
  int prec = o->mixed ? 32 : 64;
  if (prec == 32) {
    xf = (float *)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
    if (!xf) goto nomem;
    for (int64_t p = 0; p < nnz; ++p) xf[p] = (float)xval[p];
    free(xval);
    xval = NULL;
  }
  int k = 0, status = OR_OK;
  double r = NAN;
  for (;;) {
    if (prec == 32) {
      int64_t *trp;
      int32_t *tcol;
      float *tval;
      if (oracle_spgemm_f32(n, xrp, xcol, xf, xrp, xcol, xf, &trp, &tcol, &tval)) goto nomem;
      r = oracle_resid_rms_f32(n, trp, tcol, tval);
      double x = fro_rms_f32(n, xrp, xf);
      trace_put(tr, xrp[n], trp[n], r, x, 32);
      if (!isfinite(r) || r > o->div_limit) {
        free(trp); free(tcol); free(tval);
        status = OR_EDIVERGED;
        break;
      }
      if (r < o->fp32_until) {
        /* switch: widen X exactly and redo the check in FP64 */
        free(trp); free(tcol); free(tval);
        xval = (double *)malloc(sizeof(double) * (size_t)(xrp[n] > 0 ? xrp[n] : 1));
        if (!xval) goto nomem;
        for (int64_t p = 0; p < xrp[n]; ++p) xval[p] = (double)xf[p];
        free(xf);
        xf = NULL;
        prec = 64;
        continue;
      }
      if (k >= o->max_iter) {
        free(trp); free(tcol); free(tval);
        status = OR_ENOTCONV;
        break;
      }
      double xb = x;
      if (o->budget_norm && r < o->switch_resid) { /* the 2-norm of the widened iterate */
        double *xw = (double *)malloc(sizeof(double) * (size_t)(xrp[n] > 0 ? xrp[n] : 1));
        if (!xw) {
          free(trp); free(tcol); free(tval);
          goto nomem;
        }
        for (int64_t p = 0; p < xrp[n]; ++p) xw[p] = (double)xf[p];
        xb = oracle_norm2_est(n, xrp, xcol, xw, ORACLE_POW_STEPS);
        free(xw);
      }
      double beta = oracle_budget(r, xb, o->c4, o->fp32_until, o->switch_resid);
      if (o->filter_t && o->filter != OR_FILTER_NONE) {
        /* variant: T filtered with the same budget before the update */
        int64_t *frp;
        int32_t *fcol;
        float *fval;
        double ttau = 0.0, tfn = 0.0;
        int rt = filter_f32(n, trp, tcol, tval, o->filter, sqrt((double)n) * beta, &frp, &fcol,
                            &fval, &ttau, &tfn);
        free(trp); free(tcol); free(tval);
        if (rt) goto nomem;
        trp = frp;
        tcol = fcol;
        tval = fval;
        trace_that(tr, trp[n]);
      }
      int64_t *brp;
      int32_t *bcol;
      float *bval;
      int rc = ns_update_f32(n, xrp, xcol, xf, trp, tcol, tval, &brp, &bcol, &bval);
      free(trp); free(tcol); free(tval);
      if (rc) goto nomem;
      int64_t *hrp;
      int32_t *hcol;
      float *hval;
      double tau = 0.0, fn = 0.0;
      rc = filter_f32(n, brp, bcol, bval, o->filter, sqrt((double)n) * beta, &hrp, &hcol, &hval,
                      &tau, &fn);
      trace_filter(tr, beta, tau, fn, brp[n]);
      free(brp); free(bcol); free(bval);
      if (rc) goto nomem;
      free(xrp); free(xcol); free(xf);
      xrp = hrp;
      xcol = hcol;
      xf = hval;
      ++k;
    } else {
      int64_t *trp;
      int32_t *tcol;
      double *tval;
      /* e_k = ||I - X_k^2|| (Alg. 3.2.1 steps 1 and 4) */
      if (oracle_spgemm(n, xrp, xcol, xval, xrp, xcol, xval, &trp, &tcol, &tval)) goto nomem;
      r = oracle_resid_rms(n, trp, tcol, tval);
      double x = oracle_fro_rms(n, xrp, xval);
      trace_put(tr, xrp[n], trp[n], r, x, 64);
      if (r <= o->tol) { /* while e_k > tol (step 2) */
        free(trp); free(tcol); free(tval);
        status = OR_OK;
        break;
      }
      if (!isfinite(r) || r > o->div_limit) {
        free(trp); free(tcol); free(tval);
        status = OR_EDIVERGED;
        break;
      }
      if (k >= o->max_iter) {
        free(trp); free(tcol); free(tval);
        status = OR_ENOTCONV;
        break;
      }
      double xb = x;
      if (o->budget_norm && r < o->switch_resid)
        xb = oracle_norm2_est(n, xrp, xcol, xval, ORACLE_POW_STEPS);
      double beta = oracle_budget(r, xb, o->c4, o->tol, o->switch_resid);
      if (o->filter_t && o->filter != OR_FILTER_NONE) {
        /* variant: T filtered with the same budget before the update */
        int64_t *frp;
        int32_t *fcol;
        double *fval;
        double ttau = 0.0, tfn = 0.0;
        int rt = oracle_filter(n, trp, tcol, tval, o->filter, sqrt((double)n) * beta, &frp, &fcol,
                               &fval, &ttau, &tfn);
        free(trp); free(tcol); free(tval);
        if (rt) goto nomem;
        trp = frp;
        tcol = fcol;
        tval = fval;
        trace_that(tr, trp[n]);
      }
      int64_t *brp;
      int32_t *bcol;
      double *bval;
      int rc = oracle_ns_update(n, xrp, xcol, xval, trp, tcol, tval, &brp, &bcol, &bval);
      free(trp); free(tcol); free(tval);
      if (rc) goto nomem;
      int64_t *hrp;
      int32_t *hcol;
      double *hval;
      double tau = 0.0, fn = 0.0;
      rc = oracle_filter(n, brp, bcol, bval, o->filter, sqrt((double)n) * beta, &hrp, &hcol, &hval,
                         &tau, &fn);
      trace_filter(tr, beta, tau, fn, brp[n]);
      free(brp); free(bcol); free(bval);
      if (rc) goto nomem;
      free(xrp); free(xcol); free(xval);
      xrp = hrp;
      xcol = hcol;
      xval = hval;
      ++k;
    }
  }
  if (prec == 32) { /* stopped inside the FP32 stage: report the widened iterate */
    xval = (double *)malloc(sizeof(double) * (size_t)(xrp[n] > 0 ? xrp[n] : 1));
    if (!xval) goto nomem;
    for (int64_t p = 0; p < xrp[n]; ++p) xval[p] = (double)xf[p];
    free(xf);
    xf = NULL;
  }
  if (iters) *iters = k;
  if (resid) *resid = r;
  *srp = xrp;
  *scol = xcol;
  *sval = xval;
  return status;
nomem:
  free(xrp);
  free(xcol);
  free(xval);
  free(xf);
  return OR_ENOMEM;
}

/* ---------------------------------------------------------------------- */
/* Newton's method, Eq. (1.1), dense                                         */
/* ---------------------------------------------------------------------- */
/* Inverse by LU with partial pivoting (Doolittle), then one triangular
 * solve pair per unit vector. Returns 0 on success, 1 if singular. */
static int dense_inverse(int64_t n, const double *a, double *inv, double *lu, int64_t *piv) {
  memcpy(lu, a, sizeof(double) * (size_t)(n * n));
  for (int64_t i = 0; i < n; ++i) piv[i] = i;
  for (int64_t c = 0; c < n; ++c) {
    int64_t pr = c;
    double best = fabs(lu[c * n + c]);
    for (int64_t r = c + 1; r < n; ++r)
      if (fabs(lu[r * n + c]) > best) {
        best = fabs(lu[r * n + c]);
        pr = r;
      }
    if (best == 0.0) return 1;
    if (pr != c) {
      for (int64_t j = 0; j < n; ++j) {
        double t = lu[c * n + j];
        lu[c * n + j] = lu[pr * n + j];
        lu[pr * n + j] = t;
      }
      int64_t t = piv[c];
      piv[c] = piv[pr];
      piv[pr] = t;
    }
    for (int64_t r = c + 1; r < n; ++r) {
      double l = lu[r * n + c] / lu[c * n + c];
      lu[r * n + c] = l;
      for (int64_t j = c + 1; j < n; ++j) lu[r * n + j] -= l * lu[c * n + j];
    }
  }
  double *y = (double *)malloc(sizeof(double) * (size_t)n);
  if (!y) return 1;
  for (int64_t e = 0; e < n; ++e) {
    /* solve L y = P e_e, then U x = y; x is column e of the inverse */
    for (int64_t i = 0; i < n; ++i) {
      double s = piv[i] == e ? 1.0 : 0.0;
      for (int64_t j = 0; j < i; ++j) s -= lu[i * n + j] * y[j];
      y[i] = s;
    }
    for (int64_t i = n - 1; i >= 0; --i) {
      double s = y[i];
      for (int64_t j = i + 1; j < n; ++j) s -= lu[i * n + j] * inv[j * n + e];
      inv[i * n + e] = s / lu[i * n + i];
    }
  }
  free(y);
  return 0;
}

static double dense_resid(int64_t n, const double *x, double *tmp) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double s = 0.0;
      for (int64_t k = 0; k < n; ++k) s = fma(x[i * n + k], x[k * n + j], s);
      tmp[i * n + j] = s;
    }
  ksum acc = {0.0, 0.0};
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) {
      double d = tmp[i * n + j] - (i == j ? 1.0 : 0.0);
      kadd(&acc, d * d);
    }
  return sqrt(kval(&acc)) / sqrt((double)n);
}

int oracle_nm_dense(int64_t n, const double *a, double tol, int max_iter, double *s, int *iters,
                    double *resid) {
  size_t nn = (size_t)(n * n);
  double *inv = (double *)malloc(sizeof(double) * nn);
  double *lu = (double *)malloc(sizeof(double) * nn);
  int64_t *piv = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  if (!inv || !lu || !piv) {
    free(inv); free(lu); free(piv);
    return OR_ENOMEM;
  }
  memcpy(s, a, sizeof(double) * nn);
  int k = 0, status = OR_ENOTCONV;
  double r = NAN;
  for (;;) {
    r = dense_resid(n, s, lu);
    if (r <= tol) {
      status = OR_OK;
      break;
    }
    if (!isfinite(r)) {
      status = OR_EDIVERGED;
      break;
    }
    if (k >= max_iter) break;
    if (dense_inverse(n, s, inv, lu, piv)) {
      status = OR_EDIVERGED;
      break;
    }
    for (size_t p = 0; p < nn; ++p) s[p] = 0.5 * (s[p] + inv[p]);
    ++k;
  }
  free(inv); free(lu); free(piv);
  if (iters) *iters = k;
  if (resid) *resid = r;
  return status;
}

/* ---------------------------------------------------------------------- */
/* Newton's method with filtering, Alg. 3.1.1                                */
/* ---------------------------------------------------------------------- */
/* X1 = A. While e_k = ||I - X_k^2|| > tol: Xbar_{k+1} = (X_k + X_k^-1)/2
 * with a dense LU inverse, then the filter with an RMS budget of c4*tol in
 * the fixed phase (e_k >= switch_resid) and, in the adaptive phase, the bound
 * of Thm 3.1.2 (Eq. 1.13), ||F|| <= e_k^2 / (||X_k|| + ||X_k^-1||), all RMS
 * norms and taken from the current filtered iterate (the readings used for
 * Eq. 1.18). Xbar holds all n^2 entries of the dense sum; the EXACT and BOUND
 * filters drop its zeros, NONE keeps them, which makes NONE plain Newton. */
int oracle_nmf(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
               const oracle_opts *o, oracle_trace *tr, int *iters, double *resid,
               int64_t **srp, int32_t **scol, double **sval) {
  if (!o || !valid_csr(n, rowptr, col, val)) return OR_EINVAL;
  if (tr) tr->count = 0;
  size_t nn = (size_t)(n * n);
  int64_t nnz = rowptr[n];
  double *dx = (double *)malloc(sizeof(double) * nn);
  double *inv = (double *)malloc(sizeof(double) * nn);
  double *lu = (double *)malloc(sizeof(double) * nn);
  int64_t *piv = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int64_t *brp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int32_t *bcol = (int32_t *)malloc(sizeof(int32_t) * nn);
  double *bval = (double *)malloc(sizeof(double) * nn);
  int64_t *xrp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int32_t *xcol = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  double *xval = (double *)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  if (!dx || !inv || !lu || !piv || !brp || !bcol || !bval || !xrp || !xcol || !xval) {
    free(dx); free(inv); free(lu); free(piv); free(brp); free(bcol); free(bval);
    free(xrp); free(xcol); free(xval);
    return OR_ENOMEM;
  }
  memcpy(xrp, rowptr, sizeof(int64_t) * (size_t)(n + 1));
  if (nnz > 0) {
    memcpy(xcol, col, sizeof(int32_t) * (size_t)nnz);
    memcpy(xval, val, sizeof(double) * (size_t)nnz);
  }
  int k = 0, status = OR_ENOTCONV;
  double r = NAN;
  for (;;) {
    /* e_k = ||I - X_k^2|| (step 5, for k = 1 step 1) */
    int64_t *trp = NULL;
    int32_t *tcol = NULL;
    double *tval = NULL;
    if (oracle_spgemm(n, xrp, xcol, xval, xrp, xcol, xval, &trp, &tcol, &tval) != OR_OK) {
      status = OR_ENOMEM;
      break;
    }
    r = oracle_resid_rms(n, trp, tcol, tval);
    int64_t nnz_t = trp[n];
    free(trp); free(tcol); free(tval);
    double x = oracle_fro_rms(n, xrp, xval);
    trace_put(tr, xrp[n], nnz_t, r, x, 64);
    if (r <= o->tol) {
      status = OR_OK;
      break;
    }
    if (!isfinite(r) || r > o->div_limit) {
      status = OR_EDIVERGED;
      break;
    }
    if (k >= o->max_iter) break;
    /* X_k^-1, dense */
    memset(dx, 0, sizeof(double) * nn);
    for (int64_t i = 0; i < n; ++i)
      for (int64_t p = xrp[i]; p < xrp[i + 1]; ++p) dx[i * n + xcol[p]] = xval[p];
    if (dense_inverse(n, dx, inv, lu, piv)) {
      status = OR_EDIVERGED;  /* singular iterate */
      break;
    }
    ksum isq = {0.0, 0.0};
    for (size_t p = 0; p < nn; ++p) kadd(&isq, inv[p] * inv[p]);
    double xinv = sqrt(kval(&isq)) / sqrt((double)n);
    /* Xbar_{k+1} = (X_k + X_k^-1) / 2 (step 3), every entry kept */
    for (int64_t i = 0; i <= n; ++i) brp[i] = i * n;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) {
        bcol[i * n + j] = (int32_t)j;
        bval[i * n + j] = 0.5 * (dx[i * n + j] + inv[i * n + j]);
      }
    /* budget: fixed phase, else Eq. (1.13) */
    double beta = r >= o->switch_resid ? o->c4 * o->tol : r * r / (x + xinv);
    int64_t *frp = NULL;
    int32_t *fcol = NULL;
    double *fval = NULL;
    double tau = 0.0, fnorm = 0.0;
    int rc = oracle_filter(n, brp, bcol, bval, o->filter, sqrt((double)n) * beta, &frp, &fcol,
                           &fval, &tau, &fnorm);
    if (rc != OR_OK) {
      status = rc;
      break;
    }
    trace_filter(tr, beta, tau, fnorm, (int64_t)nn);
    free(xrp); free(xcol); free(xval);
    xrp = frp;
    xcol = fcol;
    xval = fval;
    ++k;
  }
  free(dx); free(inv); free(lu); free(piv); free(brp); free(bcol); free(bval);
  if (iters) *iters = k;
  if (resid) *resid = r;
  if (srp && scol && sval && (status == OR_OK || status == OR_ENOTCONV || status == OR_EDIVERGED)) {
    *srp = xrp;
    *scol = xcol;
    *sval = xval;
  } else {
    free(xrp); free(xcol); free(xval);
  }
  return status;
}
