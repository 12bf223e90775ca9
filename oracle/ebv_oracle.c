/*
 * ebv_oracle.c -- plain, slow, obviously correct FP64 CPU oracle for the EbV
 * solver (arXiv 1907.05767).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may call,
 * link or load this file: only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code with the CUDA path.
 *
 * Everything is IEEE binary64, compiled with -O2 -ffp-contract=off (no fused
 * multiply-add is formed by the compiler, no -ffast-math), so results are
 * deterministic.  The optional OpenMP loop splits the independent rows of one
 * elimination step across threads; it does not change any result bit.
 *
 * Storage: row-major, element (i, j) of a dense matrix at a[i*lda + j].
 * Band storage ("row band"): a_ij at ab[i*ldab + (j - i + kl)] for
 * i - kl <= j <= i + ku, with ldab >= kl + ku + 1.
 *
 * Readings of the paper used here:
 *  - Eq. 1: AX = B  <=>  L(UX) = B; solve LY = B by forward substitution, then
 *    UX = Y by backward substitution (the paper prints "UX = B" for the second
 *    system, read as UX = Y).
 *  - Eq. 6a and 6c (Doolittle form): at step r the L vector (the column below
 *    the pivot) is divided by the pivot A_rr and the trailing matrix receives
 *    the rank-1 update A <- A - L * U / A_rr.  L is unit lower triangular and U
 *    keeps the pivots on its diagonal (Eq. 3 draws a unit diagonal on U as well,
 *    which cannot hold for a general A; the Doolittle reading is taken).  The
 *    minus sign printed in Eq. 6a/6b belongs to the elementary transformation,
 *    not to the stored factor.
 *  - The pairing of long and short vectors (Eq. 7) only reassigns the same
 *    operations to threads; the factors it produces are the unique Doolittle
 *    factors, so the oracle computes them in the plain order.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define IDX(i, j, ld) ((int64_t)(i) * (int64_t)(ld) + (int64_t)(j))

int oracle_set_threads(int t) {
#ifdef _OPENMP
  if (t > 0) omp_set_num_threads(t);
  return omp_get_max_threads();
#else
  (void)t;
  return 1;
#endif
}

/*
 * Doolittle LU without pivoting, in place (Eq. 6a, 6c; step r of Eq. 5c).
 * On return the strict lower triangle holds L (unit diagonal implied) and the
 * upper triangle, diagonal included, holds U.
 * Only the first kstop elimination steps are taken when 0 <= kstop < n (a
 * partial factorisation); kstop < 0 means all n steps.
 * Returns 0, or k+1 for the first step k whose pivot is zero or not finite (the
 * elimination continues, as LAPACK's getrf does).
 */
int64_t oracle_lu(int64_t n, double *a, int64_t lda, int64_t kstop) {
  int64_t info = 0;
  int64_t kend = (kstop < 0 || kstop > n) ? n : kstop;
  for (int64_t k = 0; k < kend; ++k) {
    const double p = a[IDX(k, k, lda)];
    if (info == 0 && (p == 0.0 || !isfinite(p))) info = k + 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (n - k > 128)
#endif
    for (int64_t i = k + 1; i < n; ++i) {
      const double lik = a[IDX(i, k, lda)] / p; /* Eq. 6a: L vector over the pivot */
      a[IDX(i, k, lda)] = lik;
      for (int64_t j = k + 1; j < n; ++j) /* Eq. 6c: rank-1 update */
        a[IDX(i, j, lda)] -= lik * a[IDX(k, j, lda)];
    }
  }
  return info;
}

/* Forward substitution LY = B with L unit lower (Eq. 1).  B (n x nrhs, ldb) is
 * overwritten by Y:  y_i = b_i - sum_{j<i} l_ij y_j. */
void oracle_forward(int64_t n, const double *lu, int64_t lda, double *b,
                    int64_t nrhs, int64_t ldb) {
  for (int64_t c = 0; c < nrhs; ++c)
    for (int64_t i = 0; i < n; ++i) {
      double s = b[IDX(i, c, ldb)];
      for (int64_t j = 0; j < i; ++j) s -= lu[IDX(i, j, lda)] * b[IDX(j, c, ldb)];
      b[IDX(i, c, ldb)] = s;
    }
}

/* Backward substitution UX = Y with U upper, non-unit diagonal (Eq. 1).  Y is
 * overwritten by X:  x_i = (y_i - sum_{j>i} u_ij x_j) / u_ii. */
void oracle_backward(int64_t n, const double *lu, int64_t lda, double *b,
                     int64_t nrhs, int64_t ldb) {
  for (int64_t c = 0; c < nrhs; ++c)
    for (int64_t i = n - 1; i >= 0; --i) {
      double s = b[IDX(i, c, ldb)];
      for (int64_t j = i + 1; j < n; ++j) s -= lu[IDX(i, j, lda)] * b[IDX(j, c, ldb)];
      b[IDX(i, c, ldb)] = s / lu[IDX(i, i, lda)];
    }
}

/*
 * Banded Doolittle LU without pivoting, in place on row-band storage.  Without
 * row exchanges the multipliers of step k reach rows k+1..k+kl only and the
 * rank-1 update touches columns k+1..k+ku only, so every fill-in stays inside
 * the band (the sparse case of the paper's first experiment, read as a band).
 * Same arithmetic, in the same order, as oracle_lu restricted to the band.
 */
int64_t oracle_band_lu(int64_t n, int64_t kl, int64_t ku, double *ab, int64_t ldab) {
  int64_t info = 0;
#define AB(i, j) ab[IDX(i, (j) - (i) + kl, ldab)]
  for (int64_t k = 0; k < n; ++k) {
    const double p = AB(k, k);
    if (info == 0 && (p == 0.0 || !isfinite(p))) info = k + 1;
    const int64_t iend = (k + kl < n - 1) ? k + kl : n - 1;
    const int64_t jend = (k + ku < n - 1) ? k + ku : n - 1;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (iend - k > 128)
#endif
    for (int64_t i = k + 1; i <= iend; ++i) {
      const double lik = AB(i, k) / p;
      AB(i, k) = lik;
      for (int64_t j = k + 1; j <= jend; ++j) AB(i, j) -= lik * AB(k, j);
    }
  }
#undef AB
  return info;
}

/* Banded forward then backward substitution (Eq. 1), B overwritten by X. */
void oracle_band_solve(int64_t n, int64_t kl, int64_t ku, const double *ab,
                       int64_t ldab, double *b, int64_t nrhs, int64_t ldb) {
#define AB(i, j) ab[IDX(i, (j) - (i) + kl, ldab)]
  for (int64_t c = 0; c < nrhs; ++c) {
    for (int64_t i = 0; i < n; ++i) {
      double s = b[IDX(i, c, ldb)];
      const int64_t j0 = (i - kl > 0) ? i - kl : 0;
      for (int64_t j = j0; j < i; ++j) s -= AB(i, j) * b[IDX(j, c, ldb)];
      b[IDX(i, c, ldb)] = s;
    }
    for (int64_t i = n - 1; i >= 0; --i) {
      double s = b[IDX(i, c, ldb)];
      const int64_t j1 = (i + ku < n - 1) ? i + ku : n - 1;
      for (int64_t j = i + 1; j <= j1; ++j) s -= AB(i, j) * b[IDX(j, c, ldb)];
      b[IDX(i, c, ldb)] = s / AB(i, i);
    }
  }
#undef AB
}

/*
 * Adjoint of X = A^{-1} B for a loss with dL/dX = G (project addition; the
 * paper has no gradients).  With A = LU, A^T = U^T L^T, so
 *   grad_B = A^{-T} G : solve U^T z = G (lower, non-unit), then L^T w = z
 *                       (upper, unit);  grad_B = w,
 *   grad_A = -grad_B X^T.
 * grad_a may be NULL.  G, X, grad_B are n x nrhs with leading dimension ldx.
 */
void oracle_adjoint(int64_t n, int64_t nrhs, const double *lu, int64_t lda,
                    const double *x, const double *g, int64_t ldx,
                    double *grad_b, double *grad_a, int64_t ldga) {
  for (int64_t c = 0; c < nrhs; ++c) {
    for (int64_t i = 0; i < n; ++i) { /* U^T z = g */
      double s = g[IDX(i, c, ldx)];
      for (int64_t j = 0; j < i; ++j) s -= lu[IDX(j, i, lda)] * grad_b[IDX(j, c, ldx)];
      grad_b[IDX(i, c, ldx)] = s / lu[IDX(i, i, lda)];
    }
    for (int64_t i = n - 1; i >= 0; --i) { /* L^T w = z */
      double s = grad_b[IDX(i, c, ldx)];
      for (int64_t j = i + 1; j < n; ++j) s -= lu[IDX(j, i, lda)] * grad_b[IDX(j, c, ldx)];
      grad_b[IDX(i, c, ldx)] = s;
    }
  }
  if (grad_a) {
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t c = 0; c < nrhs; ++c) s += grad_b[IDX(i, c, ldx)] * x[IDX(j, c, ldx)];
        grad_a[IDX(i, j, ldga)] = -s;
      }
  }
}

/* Error-free transformations (Knuth's TwoSum; TwoProduct through the exact C99
 * fma) used by the compensated dot product Dot2 of Ogita, Rump and Oishi,
 * "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005). */
static void two_sum(double a, double b, double *s, double *e) {
  const double x = a + b;
  const double z = x - a;
  *s = x;
  *e = (a - (x - z)) + (b - z);
}

/* Residual R = B - A X, each entry by Dot2 (about twice the working precision).
 * Dense A: a[i*lda + j].  rows == NULL computes all n rows; otherwise only the
 * nrows listed rows, written to r in that order (r is nrows x nrhs, ldr). */
void oracle_residual(int64_t n, const double *a, int64_t lda, const double *x,
                     int64_t ldx, const double *b, int64_t ldb, int64_t nrhs,
                     const int64_t *rows, int64_t nrows, double *r, int64_t ldr) {
  const int64_t m = rows ? nrows : n;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (m > 64)
#endif
  for (int64_t t = 0; t < m; ++t) {
    const int64_t i = rows ? rows[t] : t;
    for (int64_t c = 0; c < nrhs; ++c) {
      double s = b[IDX(i, c, ldb)], comp = 0.0;
      for (int64_t j = 0; j < n; ++j) {
        const double p = -a[IDX(i, j, lda)] * x[IDX(j, c, ldx)];
        const double pe = fma(-a[IDX(i, j, lda)], x[IDX(j, c, ldx)], -p);
        double se;
        two_sum(s, p, &s, &se);
        comp += pe + se;
      }
      r[IDX(t, c, ldr)] = s + comp;
    }
  }
}

/* Same residual for a row-band A. */
void oracle_band_residual(int64_t n, int64_t kl, int64_t ku, const double *ab,
                          int64_t ldab, const double *x, int64_t ldx,
                          const double *b, int64_t ldb, int64_t nrhs, double *r,
                          int64_t ldr) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (n > 4096)
#endif
  for (int64_t i = 0; i < n; ++i) {
    const int64_t j0 = (i - kl > 0) ? i - kl : 0;
    const int64_t j1 = (i + ku < n - 1) ? i + ku : n - 1;
    for (int64_t c = 0; c < nrhs; ++c) {
      double s = b[IDX(i, c, ldb)], comp = 0.0;
      for (int64_t j = j0; j <= j1; ++j) {
        const double aij = ab[IDX(i, j - i + kl, ldab)];
        const double p = -aij * x[IDX(j, c, ldx)];
        const double pe = fma(-aij, x[IDX(j, c, ldx)], -p);
        double se;
        two_sum(s, p, &s, &se);
        comp += pe + se;
      }
      r[IDX(i, c, ldr)] = s + comp;
    }
  }
}

/*
 * Product-form inverse (Eq. 4a-c) from the packed Doolittle factors A = LU.
 * Eq. 4c writes A^{-1} as a product of elementary transformations, one per
 * elimination step; with the Doolittle reading of the factors they are
 *   L^{-1} = M_{n-1} ... M_2 M_1,     M_k = I - l_k e_k^T
 *            (l_k: column k of L below the diagonal -- the Gauss transform of
 *            step k, Eq. 6a),
 *   U^{-1} = E_1 E_2 ... E_{n-1} D^{-1},  E_k = I - e_k v_k^T, D = diag(u_kk)
 *            (v_k: row k of U right of the diagonal divided by the pivot u_kk;
 *            D^{-1} is the diagonal scaling that the printed Eq. 4a-c omit),
 *   A^{-1} = U^{-1} L^{-1}.
 * X starts as the identity and takes the factors from the right: M_1 first,
 * ..., M_{n-1}; then D^{-1}; then E_{n-1}, ..., E_1.  X (n x n, leading
 * dimension ldx) is overwritten.  The factors must have non-zero pivots.
 */
void oracle_inverse(int64_t n, const double *lu, int64_t lda, double *x, int64_t ldx) {
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) x[IDX(i, j, ldx)] = (i == j) ? 1.0 : 0.0;
  for (int64_t k = 0; k < n; ++k) { /* M_k: rows i > k take -l_ik * row k */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (n - k > 128)
#endif
    for (int64_t i = k + 1; i < n; ++i) {
      const double lik = lu[IDX(i, k, lda)];
      for (int64_t j = 0; j < n; ++j) x[IDX(i, j, ldx)] -= lik * x[IDX(k, j, ldx)];
    }
  }
  for (int64_t k = 0; k < n; ++k) /* D^{-1} */
    for (int64_t j = 0; j < n; ++j) x[IDX(k, j, ldx)] /= lu[IDX(k, k, lda)];
  for (int64_t k = n - 1; k >= 0; --k) { /* E_k: row k takes -v_kq * row q, q > k */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (n > 128)
#endif
    for (int64_t j = 0; j < n; ++j) {
      double s = x[IDX(k, j, ldx)];
      for (int64_t q = k + 1; q < n; ++q) s -= (lu[IDX(k, q, lda)] / lu[IDX(k, k, lda)]) * x[IDX(q, j, ldx)];
      x[IDX(k, j, ldx)] = s;
    }
  }
}
