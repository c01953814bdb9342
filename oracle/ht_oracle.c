/*
 * CPU oracle for the Hessenberg-triangular (HT) reduction of Bujanovic,
 * Karlsson and Kressner, "A Householder-based algorithm for
 * Hessenberg-triangular reduction" (arXiv 1710.08538).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA library is checked against.  Nothing in the product path may link,
 * load or call it; it shares no code with the CUDA sources.
 *
 * Everything is FP64, column-major, 0-based (the paper is 1-based).
 *
 * Contents
 *   oracle_house          Householder reflector, Sec. 2.1 (Golub-Van Loan
 *                         Alg. 5.1.1 as cited there), LAPACK-DLARFG sign rule.
 *   oracle_basic_househt  Algorithm 2 (BasicHouseHT, Appendix A): one left
 *                         reflector and one opposite right reflector per
 *                         column, dense LU solve of B(j+1:n,j+1:n) x = e1.
 *                         Theta(n^4); small n only.
 *   oracle_givens_ht      Textbook unblocked Givens HT reduction (the
 *                         Moler-Stewart algorithm the paper compares with,
 *                         Sec. 1 and Sec. 4).  Theta(n^3); the timed CPU
 *                         baseline and the large-n reference.
 *   oracle_philox_normal  Counter-based N(0,1) sample (Philox4x32-10 of
 *                         Salmon et al. 2011 + Box-Muller) used for the
 *                         singular-B perturbation of Remark 2.2 / Sec. 3.2.1.
 *
 * Error behaviour: functions return 0 on success, a negative value -i when
 * argument i is invalid, and 1 on allocation failure.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX(M, ld, i, j) ((M)[(size_t)(j) * (size_t)(ld) + (size_t)(i)])

static const double ORACLE_U = 1.1102230246251565e-16; /* unit roundoff 2^-53 */

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller.         */
/* ------------------------------------------------------------------------ */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  const uint32_t n0 = hi1 ^ c[1] ^ k[0];
  const uint32_t n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k[2] = {key_in[0], key_in[1]};
  for (int r = 0; r < 10; ++r) {
    philox_round(c, k);
    k[0] += 0x9E3779B9u;
    k[1] += 0xBB67AE85u;
  }
  memcpy(out, c, sizeof(c));
}

/* N(0,1) sample for (seed, column, index): counter = (column, index, 0, 0),
 * key = (seed lo, seed hi).  u1 in (0,1], u2 in [0,1) from 32-bit words. */
double oracle_philox_normal(uint64_t seed, uint32_t column, uint32_t index) {
  const uint32_t ctr[4] = {column, index, 0u, 0u};
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t r[4];
  oracle_philox4x32_10(ctr, key, r);
  const double u1 = ((double)r[0] + 1.0) * 2.3283064365386963e-10; /* 2^-32 */
  const double u2 = (double)r[1] * 2.3283064365386963e-10;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

/* ------------------------------------------------------------------------ */
/* Householder reflector (Sec. 2.1).                                         */
/* Given x[0..m-1] (stride incx) compute v (v[0] = 1 implicitly, tail        */
/* returned in place of x[1..m-1]) and beta such that                        */
/* (I - beta v v^T) x = alpha e1.  Sign rule (DLARFG): alpha =              */
/* -sign(x0) ||x|| with sign(0) = +; if the tail is exactly zero the         */
/* reflector is the identity (beta = 0, alpha = x0).                         */
/* ------------------------------------------------------------------------ */
void oracle_house(int m, double* x, int incx, double* beta, double* alpha) {
  if (m <= 0) { *beta = 0.0; *alpha = 0.0; return; }
  const double x0 = x[0];
  double tail2 = 0.0;
  for (int i = 1; i < m; ++i) tail2 += x[(size_t)i * incx] * x[(size_t)i * incx];
  if (tail2 == 0.0) { *beta = 0.0; *alpha = x0; return; }
  const double nrm = sqrt(x0 * x0 + tail2);
  const double a = (x0 >= 0.0) ? -nrm : nrm;
  const double denom = x0 - a; /* = x0 + sign(x0)||x||, no cancellation */
  for (int i = 1; i < m; ++i) x[(size_t)i * incx] /= denom;
  /* beta = 2 / v^T v with v = [1; tail/denom] */
  double vtv = 1.0;
  for (int i = 1; i < m; ++i) vtv += x[(size_t)i * incx] * x[(size_t)i * incx];
  *beta = 2.0 / vtv;
  *alpha = a;
  x[0] = a;
}

/* Apply (I - beta v v^T) from the left to rows r0..r0+m-1 of columns
 * c0..c1-1 of M (v[0] = 1, v tail in vt[1..m-1]). */
static void apply_left(int m, const double* v, double beta, double* M, int ld, int r0, int c0, int c1) {
  if (beta == 0.0) return;
  for (int c = c0; c < c1; ++c) {
    double w = 0.0;
    for (int i = 0; i < m; ++i) w += v[i] * IDX(M, ld, r0 + i, c);
    w *= beta;
    for (int i = 0; i < m; ++i) IDX(M, ld, r0 + i, c) -= w * v[i];
  }
}

/* Apply (I - beta v v^T) from the right to columns c0..c0+m-1 of rows
 * r0..r1-1 of M. */
static void apply_right(int m, const double* v, double beta, double* M, int ld, int c0, int r0, int r1) {
  if (beta == 0.0) return;
  for (int r = r0; r < r1; ++r) {
    double w = 0.0;
    for (int i = 0; i < m; ++i) w += IDX(M, ld, r, c0 + i) * v[i];
    w *= beta;
    for (int i = 0; i < m; ++i) IDX(M, ld, r, c0 + i) -= w * v[i];
  }
}

static double frob(int n, const double* M, int ld) {
  double s = 0.0;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) s += IDX(M, ld, i, j) * IDX(M, ld, i, j);
  return sqrt(s);
}

static void set_identity(int n, double* M, int ld) {
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) IDX(M, ld, i, j) = (i == j) ? 1.0 : 0.0;
}

/* Dense solve C x = e1 (C is m x m, copied into work) by Gaussian
 * elimination with partial pivoting.  A pivot that is exactly zero is
 * replaced by 2 u rho ||B||_F (the perturbation rule of Remark 2.2 applied
 * to the LU pivot; rho ~ N(0,1) from the counter-based generator keyed by
 * (seed, column, pivot index)).  Returns the number of replaced pivots. */
static int lu_solve_e1(int m, double* C, double* x, double bnorm, uint64_t seed, int column) {
  int replaced = 0;
  for (int i = 0; i < m; ++i) x[i] = (i == 0) ? 1.0 : 0.0;
  for (int c = 0; c < m; ++c) {
    int p = c;
    double best = fabs(C[(size_t)c * m + c]);
    for (int i = c + 1; i < m; ++i) {
      const double a = fabs(C[(size_t)c * m + i]);
      if (a > best) { best = a; p = i; }
    }
    if (p != c) {
      for (int jj = 0; jj < m; ++jj) {
        const double t = C[(size_t)jj * m + c];
        C[(size_t)jj * m + c] = C[(size_t)jj * m + p];
        C[(size_t)jj * m + p] = t;
      }
      const double t = x[c]; x[c] = x[p]; x[p] = t;
    }
    if (C[(size_t)c * m + c] == 0.0) {
      C[(size_t)c * m + c] = 2.0 * ORACLE_U * oracle_philox_normal(seed, (uint32_t)column, (uint32_t)c) * bnorm;
      if (C[(size_t)c * m + c] == 0.0) C[(size_t)c * m + c] = 2.0 * ORACLE_U * bnorm;
      ++replaced;
    }
    const double piv = C[(size_t)c * m + c];
    for (int i = c + 1; i < m; ++i) {
      const double l = C[(size_t)c * m + i] / piv;
      if (l == 0.0) continue;
      for (int jj = c + 1; jj < m; ++jj) C[(size_t)jj * m + i] -= l * C[(size_t)jj * m + c];
      x[i] -= l * x[c];
    }
  }
  for (int c = m - 1; c >= 0; --c) {
    double t = x[c];
    for (int jj = c + 1; jj < m; ++jj) t -= C[(size_t)jj * m + c] * x[jj];
    x[c] = t / C[(size_t)c * m + c];
  }
  return replaced;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2, BasicHouseHT (Appendix A).                                   */
/* A (n x n, lda) and B (n x n upper triangular, ldb) are overwritten by H   */
/* and T; Q and Z (n x n, ldq/ldz) receive the transforms (set to I first).  */
/* ------------------------------------------------------------------------ */
int oracle_basic_househt(int n, double* A, int lda, double* B, int ldb, double* Q, int ldq, double* Z, int ldz,
                         uint64_t seed, int* n_perturbed) {
  if (n < 0) return -1;
  if (lda < (n > 1 ? n : 1)) return -3;
  if (ldb < (n > 1 ? n : 1)) return -5;
  if (ldq < (n > 1 ? n : 1)) return -7;
  if (ldz < (n > 1 ? n : 1)) return -9;
  set_identity(n, Q, ldq);
  set_identity(n, Z, ldz);
  if (n_perturbed) *n_perturbed = 0;
  /* B is upper triangular on entry: its strictly lower part is ignored. */
  for (int j = 0; j < n; ++j)
    for (int i = j + 1; i < n; ++i) IDX(B, ldb, i, j) = 0.0;
  if (n <= 2) return 0;
  const double bnorm = frob(n, B, ldb);
  double* v = (double*)malloc(sizeof(double) * (size_t)n);
  double* x = (double*)malloc(sizeof(double) * (size_t)n);
  double* C = (double*)malloc(sizeof(double) * (size_t)n * (size_t)n);
  if (!v || !x || !C) { free(v); free(x); free(C); return 1; }
  for (int j = 0; j <= n - 3; ++j) {
    /* F_j = I_{j+1} (+) House(A(j+1:n, j))  (0-based rows j+1..n-1) */
    const int m = n - j - 1;
    double beta, alpha;
    for (int i = 0; i < m; ++i) v[i] = IDX(A, lda, j + 1 + i, j);
    oracle_house(m, v, 1, &beta, &alpha);
    v[0] = 1.0;
    apply_left(m, v, beta, A, lda, j + 1, 0, n);
    apply_left(m, v, beta, B, ldb, j + 1, 0, n);
    apply_right(m, v, beta, Q, ldq, j + 1, 0, n); /* Q <- Q F_j */
    IDX(A, lda, j + 1, j) = alpha;
    for (int i = j + 2; i < n; ++i) IDX(A, lda, i, j) = 0.0;
    /* solve B(j+1:n, j+1:n) x = e1 (dense) */
    for (int c = 0; c < m; ++c)
      for (int i = 0; i < m; ++i) C[(size_t)c * m + i] = IDX(B, ldb, j + 1 + i, j + 1 + c);
    const int rep = lu_solve_e1(m, C, x, bnorm, seed, j);
    if (n_perturbed) *n_perturbed += rep;
    /* G_j = I_{j+1} (+) House(x) applied from the right to A, B, Z */
    double gamma, xa;
    oracle_house(m, x, 1, &gamma, &xa);
    x[0] = 1.0;
    apply_right(m, x, gamma, A, lda, j + 1, 0, n);
    apply_right(m, x, gamma, B, ldb, j + 1, 0, n);
    apply_right(m, x, gamma, Z, ldz, j + 1, 0, n);
    for (int i = j + 2; i < n; ++i) IDX(B, ldb, i, j + 1) = 0.0;
  }
  free(v); free(x); free(C);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Unblocked Givens HT reduction (Moler-Stewart).                            */
/* For each column j, for i = n-1 down to j+2: a rotation of rows (i-1, i)   */
/* zeros A(i, j) and is applied to A, B and Q; the fill B(i, i-1) it makes   */
/* is zeroed by a rotation of columns (i-1, i) applied to A, B and Z.        */
/* ------------------------------------------------------------------------ */
static void givens(double a, double b, double* c, double* s, double* r) {
  if (b == 0.0) { *c = 1.0; *s = 0.0; *r = a; return; }
  const double h = hypot(a, b);
  *c = a / h; *s = b / h; *r = h;
}

int oracle_givens_ht(int n, double* A, int lda, double* B, int ldb, double* Q, int ldq, double* Z, int ldz) {
  if (n < 0) return -1;
  if (lda < (n > 1 ? n : 1)) return -3;
  if (ldb < (n > 1 ? n : 1)) return -5;
  if (ldq < (n > 1 ? n : 1)) return -7;
  if (ldz < (n > 1 ? n : 1)) return -9;
  set_identity(n, Q, ldq);
  set_identity(n, Z, ldz);
  for (int j = 0; j < n; ++j)
    for (int i = j + 1; i < n; ++i) IDX(B, ldb, i, j) = 0.0;
  for (int j = 0; j + 2 < n; ++j) {
    for (int i = n - 1; i >= j + 2; --i) {
      double c, s, r;
      /* rows (i-1, i): [c s; -s c] [a; b] = [r; 0] */
      givens(IDX(A, lda, i - 1, j), IDX(A, lda, i, j), &c, &s, &r);
      if (s != 0.0) {
        IDX(A, lda, i - 1, j) = r;
        IDX(A, lda, i, j) = 0.0;
        for (int cc = j + 1; cc < n; ++cc) {
          const double t1 = IDX(A, lda, i - 1, cc), t2 = IDX(A, lda, i, cc);
          IDX(A, lda, i - 1, cc) = c * t1 + s * t2;
          IDX(A, lda, i, cc) = -s * t1 + c * t2;
        }
        for (int cc = i - 1; cc < n; ++cc) {
          const double t1 = IDX(B, ldb, i - 1, cc), t2 = IDX(B, ldb, i, cc);
          IDX(B, ldb, i - 1, cc) = c * t1 + s * t2;
          IDX(B, ldb, i, cc) = -s * t1 + c * t2;
        }
        for (int rr = 0; rr < n; ++rr) { /* Q <- Q G^T */
          const double t1 = IDX(Q, ldq, rr, i - 1), t2 = IDX(Q, ldq, rr, i);
          IDX(Q, ldq, rr, i - 1) = c * t1 + s * t2;
          IDX(Q, ldq, rr, i) = -s * t1 + c * t2;
        }
      } else {
        IDX(A, lda, i, j) = 0.0;
      }
      /* columns (i-1, i): zero B(i, i-1) using B(i, i) */
      givens(IDX(B, ldb, i, i), IDX(B, ldb, i, i - 1), &c, &s, &r);
      if (s != 0.0) {
        /* [b(i,i-1) b(i,i)] [c -s; s c]... choose rotation with
           new(i,i-1) = c*b(i,i-1) - s*b(i,i) = 0 and new(i,i) = s*b(i,i-1) + c*b(i,i) = r */
        for (int rr = 0; rr <= i; ++rr) {
          const double t1 = IDX(B, ldb, rr, i - 1), t2 = IDX(B, ldb, rr, i);
          IDX(B, ldb, rr, i - 1) = c * t1 - s * t2;
          IDX(B, ldb, rr, i) = s * t1 + c * t2;
        }
        IDX(B, ldb, i, i - 1) = 0.0;
        IDX(B, ldb, i, i) = r;
        for (int rr = 0; rr < n; ++rr) {
          const double t1 = IDX(A, lda, rr, i - 1), t2 = IDX(A, lda, rr, i);
          IDX(A, lda, rr, i - 1) = c * t1 - s * t2;
          IDX(A, lda, rr, i) = s * t1 + c * t2;
        }
        for (int rr = 0; rr < n; ++rr) {
          const double t1 = IDX(Z, ldz, rr, i - 1), t2 = IDX(Z, ldz, rr, i);
          IDX(Z, ldz, rr, i - 1) = c * t1 - s * t2;
          IDX(Z, ldz, rr, i) = s * t1 + c * t2;
        }
      } else {
        IDX(B, ldb, i, i - 1) = 0.0;
      }
    }
  }
  return 0;
}
