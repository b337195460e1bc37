/*
 * oracle.c -- plain, slow, FP64 CPU oracle for the SPD solve path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product (the CUDA library and its
 * Python binding) may call, link or load this file; only the tests, the smoke
 * check and the bench's CPU-baseline leg use it.  It shares no code, header,
 * table or helper with the CUDA path.
 *
 * What it computes (paper: "Software design", the `potrs` workflow: an SPD
 * solve A x = b through a Cholesky factorisation potrf + potrs, optionally
 * returning log det A):
 *
 *   oracle_potrf   A = L L^T, lower, in place; the plain definition of the
 *                  Cholesky factor written as the textbook right-looking scalar
 *                  loop (column j: pivot, scale, rank-1 update of the trailing
 *                  lower triangle).  info = j+1 at the first pivot that is not
 *                  > 0 (this also catches NaN), LAPACK convention.
 *   oracle_potrs   forward substitution L y = b, then back substitution
 *                  L^T x = y, column by column.
 *   oracle_posv    oracle_potrf then oracle_potrs.
 *   oracle_resid_dot2   r = b - A x with A symmetric, lower triangle stored,
 *                  every row sum done by Dot2 (Ogita, Rump and Oishi 2005,
 *                  "Accurate sum and dot product"): TwoProduct by fma,
 *                  TwoSum by Knuth's six-flop sum.  The result is as
 *                  accurate as if computed in twice the working precision and
 *                  then rounded, so it certifies backward errors near 1e-16.
 *   oracle_norm_inf  ||A||_inf of the symmetric matrix held in its lower triangle.
 *   oracle_bwd_err normwise backward error per column (Rigal and Gaches):
 *                  eta_j = ||r_j||_inf / (||A||_inf ||x_j||_inf + ||b_j||_inf).
 *   oracle_bwd_err_rows  the same numbers, bit for bit, with the loops arranged
 *                  so that a matrix of tens of GB is read once (certification
 *                  of full-size results).
 *   oracle_rowmajor_to_colmajor  the layout conversion of the paper's
 *                  "Local memory-layout conversion" stage, by its definition.
 *   oracle_logdet  log det A = 2 sum_i log L_ii (paper: "Software design",
 *                  potrs can also return log det A).
 *   oracle_grad    adjoint of X = A^{-1} B for symmetric A:
 *                  Bbar = A^{-1} Xbar,  Abar = -(Bbar X^T + X Bbar^T)/2.
 *   oracle_ge_solve  Gaussian elimination with partial pivoting on the full
 *                  (symmetrised) matrix, tiny n only: an independent route to
 *                  the same x, used to check oracle_posv.
 *
 * Storage: column-major, element (i,j) at A[i + j*lda]; only the lower
 * triangle (i >= j) of a symmetric matrix is read or written.
 *
 * Build with -ffp-contract=off so that no multiply-add is fused behind the
 * code's back (the Dot2 error-free transformations need that, and it makes
 * results identical on x86-64 and aarch64).  OpenMP, when enabled, only splits
 * independent columns / right-hand sides across threads; it never changes the
 * order of the operations that produce any one element.
 */
#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define AT(M, i, j, ld) (M)[(size_t)(j) * (size_t)(ld) + (size_t)(i)]

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void oracle_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
#else
  (void)t;
#endif
}

/* Cholesky factorisation, lower, in place.  Returns 0 or j+1 (1-based) of the
 * first column whose pivot d = a_jj - sum_{k<j} l_jk^2 is not > 0. */
int oracle_potrf(int n, double* A, int lda) {
  for (int j = 0; j < n; ++j) {
    double d = AT(A, j, j, lda);
    if (!(d > 0.0)) return j + 1;
    double ljj = sqrt(d);
    AT(A, j, j, lda) = ljj;
    for (int i = j + 1; i < n; ++i) AT(A, i, j, lda) = AT(A, i, j, lda) / ljj;
    /* a_ik -= l_ij * l_kj for j < k <= i: each column k is independent. */
#pragma omp parallel for schedule(dynamic, 8) if (n - j > 512)
    for (int k = j + 1; k < n; ++k) {
      double lkj = AT(A, k, j, lda);
      for (int i = k; i < n; ++i) AT(A, i, k, lda) -= AT(A, i, j, lda) * lkj;
    }
  }
  return 0;
}

/* Solve (L L^T) X = B in place on B (n x nrhs, column-major, ldb). */
void oracle_potrs(int n, int nrhs, const double* L, int lda, double* B, int ldb) {
#pragma omp parallel for schedule(dynamic, 1) if (nrhs > 1)
  for (int c = 0; c < nrhs; ++c) {
    double* b = B + (size_t)c * (size_t)ldb;
    /* forward: L y = b */
    for (int j = 0; j < n; ++j) {
      double yj = b[j] / AT(L, j, j, lda);
      b[j] = yj;
      for (int i = j + 1; i < n; ++i) b[i] -= AT(L, i, j, lda) * yj;
    }
    /* back: L^T x = y; row j of L^T is column j of L */
    for (int j = n - 1; j >= 0; --j) {
      double s = b[j];
      for (int i = j + 1; i < n; ++i) s -= AT(L, i, j, lda) * b[i];
      b[j] = s / AT(L, j, j, lda);
    }
  }
}

int oracle_posv(int n, int nrhs, double* A, int lda, double* B, int ldb) {
  int info = oracle_potrf(n, A, lda);
  if (info == 0) oracle_potrs(n, nrhs, A, lda, B, ldb);
  return info;
}

/* element (i,j) of the symmetric matrix whose lower triangle is stored */
static double sym_at(const double* A, int lda, int i, int j) {
  return i >= j ? AT(A, i, j, lda) : AT(A, j, i, lda);
}

/* Error-free transformations (Knuth's TwoSum; TwoProduct through fma). */
static void two_sum(double a, double b, double* s, double* e) {
  double x = a + b;
  double z = x - a;
  *e = (a - (x - z)) + (b - z);
  *s = x;
}
static void two_prod(double a, double b, double* p, double* e) {
  double x = a * b;
  *e = fma(a, b, -x);
  *p = x;
}

/* R = B - A X with A symmetric (lower stored); each entry by Dot2. */
void oracle_resid_dot2(int n, int nrhs, const double* A, int lda, const double* X,
                       int ldx, const double* B, int ldb, double* R, int ldr) {
#pragma omp parallel for schedule(dynamic, 16) collapse(2) if (n > 256)
  for (int c = 0; c < nrhs; ++c) {
    for (int i = 0; i < n; ++i) {
      double s = AT(B, i, c, ldb), comp = 0.0;
      for (int j = 0; j < n; ++j) {
        double p, ep, es;
        two_prod(-sym_at(A, lda, i, j), AT(X, j, c, ldx), &p, &ep);
        two_sum(s, p, &s, &es);
        comp += es + ep;
      }
      AT(R, i, c, ldr) = s + comp;
    }
  }
}

/* ||A||_inf = max_i sum_j |a_ij| of the symmetric matrix (lower stored). */
double oracle_norm_inf(int n, const double* A, int lda) {
  double best = 0.0;
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) s += fabs(sym_at(A, lda, i, j));
    if (s > best || isnan(s)) best = s;
  }
  return best;
}

/* max that lets a NaN through (fmax would drop it) */
static double nan_max(double a, double b) { return (isnan(a) || isnan(b)) ? NAN : (a > b ? a : b); }

/* Normwise backward error per column, written to eta[c]; returns max_c. */
double oracle_bwd_err(int n, int nrhs, const double* A, int lda, const double* X,
                      int ldx, const double* B, int ldb, double* eta) {
  double anorm = oracle_norm_inf(n, A, lda);
  double* r = (double*)malloc(sizeof(double) * (size_t)n * (size_t)(nrhs > 0 ? nrhs : 1));
  oracle_resid_dot2(n, nrhs, A, lda, X, ldx, B, ldb, r, n);
  double worst = 0.0;
  for (int c = 0; c < nrhs; ++c) {
    double rn = 0.0, xn = 0.0, bn = 0.0;
    for (int i = 0; i < n; ++i) {
      rn = nan_max(rn, fabs(r[(size_t)c * n + i]));
      xn = nan_max(xn, fabs(AT(X, i, c, ldx)));
      bn = nan_max(bn, fabs(AT(B, i, c, ldb)));
    }
    double den = anorm * xn + bn;
    double e = (isnan(rn) || isnan(den)) ? NAN : den > 0.0 ? rn / den : (rn > 0.0 ? INFINITY : 0.0);
    if (eta) eta[c] = e;
    if (e > worst || isnan(e)) worst = e;
  }
  free(r);
  return worst;
}

/* The same per-column backward errors as oracle_bwd_err, bit for bit, for
 * matrices too large for its row-by-row sweep.  Every residual entry is still
 * the Dot2 sum over j = 0, 1, ..., n-1 of exactly the operations of
 * oracle_resid_dot2, and every row sum of ||A||_inf runs over j in the same
 * order as in oracle_norm_inf; only the loop nest is arranged differently:
 * rows go in blocks of 32 that advance through j together, each carrying its
 * own running sums for all right-hand sides, so that A is read once, down its
 * columns (lower triangle) and along 32 neighbouring columns (the mirrored
 * half), instead of once per right-hand side along its rows. */
#define ORACLE_ROWS 32
double oracle_bwd_err_rows(int n, int nrhs, const double* A, int lda, const double* X,
                           int ldx, const double* B, int ldb, double* eta) {
  const size_t nr = (size_t)(nrhs > 0 ? nrhs : 1);
  double* r = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1) * nr);
  double* rowsum = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#pragma omp parallel for schedule(dynamic, 1)
  for (int i0 = 0; i0 < n; i0 += ORACLE_ROWS) {
    const int ib = n - i0 < ORACLE_ROWS ? n - i0 : ORACLE_ROWS;
    double* s = (double*)malloc(sizeof(double) * ORACLE_ROWS * nr);
    double* comp = (double*)malloc(sizeof(double) * ORACLE_ROWS * nr);
    double asum[ORACLE_ROWS];
    for (int ii = 0; ii < ib; ++ii) {
      asum[ii] = 0.0;
      for (int c = 0; c < nrhs; ++c) {
        s[(size_t)ii * nr + c] = AT(B, i0 + ii, c, ldb);
        comp[(size_t)ii * nr + c] = 0.0;
      }
    }
    for (int j = 0; j < n; ++j) {
      for (int ii = 0; ii < ib; ++ii) {
        const double a = sym_at(A, lda, i0 + ii, j);
        asum[ii] += fabs(a);
        for (int c = 0; c < nrhs; ++c) {
          double p, ep, es;
          double* sc = &s[(size_t)ii * nr + c];
          two_prod(-a, AT(X, j, c, ldx), &p, &ep);
          two_sum(*sc, p, sc, &es);
          comp[(size_t)ii * nr + c] += es + ep;
        }
      }
    }
    for (int ii = 0; ii < ib; ++ii) {
      rowsum[i0 + ii] = asum[ii];
      for (int c = 0; c < nrhs; ++c)
        r[(size_t)c * n + i0 + ii] = s[(size_t)ii * nr + c] + comp[(size_t)ii * nr + c];
    }
    free(s);
    free(comp);
  }
  double anorm = 0.0;
  for (int i = 0; i < n; ++i)
    if (rowsum[i] > anorm || isnan(rowsum[i])) anorm = rowsum[i];
  double worst = 0.0;
  for (int c = 0; c < nrhs; ++c) {
    double rn = 0.0, xn = 0.0, bn = 0.0;
    for (int i = 0; i < n; ++i) {
      rn = nan_max(rn, fabs(r[(size_t)c * n + i]));
      xn = nan_max(xn, fabs(AT(X, i, c, ldx)));
      bn = nan_max(bn, fabs(AT(B, i, c, ldb)));
    }
    double den = anorm * xn + bn;
    double e = (isnan(rn) || isnan(den)) ? NAN : den > 0.0 ? rn / den : (rn > 0.0 ? INFINITY : 0.0);
    if (eta) eta[c] = e;
    if (e > worst || isnan(e)) worst = e;
  }
  free(r);
  free(rowsum);
  return worst;
}

/* Row-major to column-major order (paper: "Local memory-layout conversion"),
 * out of place, by its definition: the m x n matrix held row-major in `in`
 * (element (i, j) at i n + j) is written column-major to `out` (element (i, j)
 * at i + j m). */
void oracle_rowmajor_to_colmajor(long long m, long long n, const double* in, double* out) {
  for (long long i = 0; i < m; ++i)
    for (long long j = 0; j < n; ++j) out[i + j * m] = in[i * n + j];
}

double oracle_logdet(int n, const double* L, int lda) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += log(AT(L, i, i, lda));
  return 2.0 * s;
}

/* Adjoint of X = A^{-1} B.  Inputs: lower(A), B, upstream Xbar.  Outputs:
 * X, Bbar = A^{-1} Xbar and the full symmetric Abar = -(Bbar X^T + X Bbar^T)/2
 * (n x n, column-major, ldab).  Returns potrf's info. */
int oracle_grad(int n, int nrhs, const double* A, int lda, const double* B, int ldb,
                const double* Xbar, int ldxb, double* X, double* Bbar, double* Abar,
                int ldab) {
  double* L = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  for (int j = 0; j < n; ++j)
    for (int i = j; i < n; ++i) L[(size_t)j * n + i] = AT(A, i, j, lda);
  int info = oracle_potrf(n, L, n);
  if (info) {
    free(L);
    return info;
  }
  for (int c = 0; c < nrhs; ++c)
    for (int i = 0; i < n; ++i) {
      X[(size_t)c * n + i] = AT(B, i, c, ldb);
      Bbar[(size_t)c * n + i] = AT(Xbar, i, c, ldxb);
    }
  oracle_potrs(n, nrhs, L, n, X, n);
  oracle_potrs(n, nrhs, L, n, Bbar, n);
#pragma omp parallel for schedule(static) if (n > 256)
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      for (int c = 0; c < nrhs; ++c)
        s += Bbar[(size_t)c * n + i] * X[(size_t)c * n + j] +
             X[(size_t)c * n + i] * Bbar[(size_t)c * n + j];
      AT(Abar, i, j, ldab) = -0.5 * s;
    }
  free(L);
  return 0;
}

/* Gaussian elimination with partial pivoting on the symmetric matrix held in
 * lower(A); B (n x nrhs) is overwritten with the solution.  Returns 0, or k+1
 * when column k has no non-zero pivot.  Tiny n only (it copies A). */
int oracle_ge_solve(int n, int nrhs, const double* A, int lda, double* B, int ldb) {
  double* M = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) M[(size_t)j * n + i] = sym_at(A, lda, i, j);
  int info = 0;
  for (int k = 0; k < n && !info; ++k) {
    int p = k;
    for (int i = k + 1; i < n; ++i)
      if (fabs(M[(size_t)k * n + i]) > fabs(M[(size_t)k * n + p])) p = i;
    if (M[(size_t)k * n + p] == 0.0) {
      info = k + 1;
      break;
    }
    if (p != k) {
      for (int j = 0; j < n; ++j) {
        double t = M[(size_t)j * n + k];
        M[(size_t)j * n + k] = M[(size_t)j * n + p];
        M[(size_t)j * n + p] = t;
      }
      for (int c = 0; c < nrhs; ++c) {
        double t = AT(B, k, c, ldb);
        AT(B, k, c, ldb) = AT(B, p, c, ldb);
        AT(B, p, c, ldb) = t;
      }
    }
    for (int i = k + 1; i < n; ++i) {
      double f = M[(size_t)k * n + i] / M[(size_t)k * n + k];
      for (int j = k; j < n; ++j) M[(size_t)j * n + i] -= f * M[(size_t)j * n + k];
      for (int c = 0; c < nrhs; ++c) AT(B, i, c, ldb) -= f * AT(B, k, c, ldb);
    }
  }
  if (!info) {
    for (int c = 0; c < nrhs; ++c)
      for (int i = n - 1; i >= 0; --i) {
        double s = AT(B, i, c, ldb);
        for (int j = i + 1; j < n; ++j) s -= M[(size_t)j * n + i] * AT(B, j, c, ldb);
        AT(B, i, c, ldb) = s / M[(size_t)i * n + i];
      }
  }
  free(M);
  return info;
}
