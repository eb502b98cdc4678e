/* Oracle for dynamical perturbation theory (DPT): plain, slow, obviously correct
 * CPU code in FP64 / complex128.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, __graft_entry__.smoke() and
 * bench.py's CPU-baseline / reference legs may build, load or call this code.
 * The CUDA library never links, loads or calls it, and the two share no code:
 * the oracle is the independent definition the GPU results are checked against.
 *
 * Source: M. Kenmoe, M. Smerlak, A. Zadorin, "Dynamical perturbation theory for
 * eigenvalue problems", arXiv:2002.12872.
 *
 *   ora_solve_full_{r,c}     the bundled map F of Eq. (dyn), iterated from I
 *                            (Sec. II.B), on any subset of columns
 *   ora_step_{r,c}           one application of F plus the eigenvalue read-out
 *   ora_residual_{r,c}       explicit residual M A - A diag(E)
 *   ora_solve_dominant_csr   the single-vector map F_{n*} of Eq. (single_line_dyn)
 *                            for the dominant eigenvector (Sec. II.H), on a CSR
 *                            perturbation with FP32 values promoted to FP64
 *   ora_rs_series_r          Rayleigh-Schroedinger partial sum, Eq. (ARS-alpha)
 *   ora_jacobi_sym           cyclic Jacobi diagonalisation of a real symmetric
 *                            matrix (textbook method, for brute-force checks)
 *
 * All matrices are column-major.  Status codes: see dpt_oracle.h.
 */
#include "dpt_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads for the parallel loops over independent columns (n <= 0 leaves the
 * setting unchanged); returns the number in effect (1 without OpenMP). */
int ora_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
  return omp_get_max_threads();
#else
  (void)n;
  return 1;
#endif
}

/* ---- real FP64 instance ------------------------------------------------- */
#define T double
#define ABS(x) fabs(x)
#define SQ(x) ((x) * (x))
#define FN(name) name##_r
#include "dpt_oracle_body.inc"
#undef T
#undef ABS
#undef SQ
#undef FN

/* ---- complex128 instance ------------------------------------------------ */
#define T double _Complex
#define ABS(x) cabs(x)
#define SQ(x) (creal(x) * creal(x) + cimag(x) * cimag(x))
#define FN(name) name##_c
#include "dpt_oracle_body.inc"
#undef T
#undef ABS
#undef SQ
#undef FN

/* ---- public entry points ---------------------------------------------- */
/* Complex lambda crosses the C boundary as two doubles (re, im). */

int ora_step_r(int64_t n, const double* theta, const double* delta, double lambda,
               const double* A, double* A_next, double* E) {
  return step_all_r(n, theta, delta, lambda, A, A_next, E);
}
double ora_residual_r(int64_t n, const double* theta, const double* delta,
                      double lambda, const double* A, const double* E, double* rho) {
  return residual_all_r(n, theta, delta, lambda, A, E, rho);
}
int ora_solve_full_r(int64_t n, const double* theta, const double* delta,
                     double lambda, int64_t ncols, const int64_t* cols, double tol,
                     int64_t max_iter, int epstein_nesbet, double ramp_alpha,
                     const double* start, double* A_out, double* E_out, ora_info* info) {
  return solve_full_r(n, theta, delta, lambda, ncols, cols, tol, max_iter,
                      epstein_nesbet, ramp_alpha, start, A_out, E_out, info);
}
int ora_step_c(int64_t n, const double _Complex* theta, const double _Complex* delta,
               double lambda_re, double lambda_im, const double _Complex* A,
               double _Complex* A_next, double _Complex* E) {
  return step_all_c(n, theta, delta, CMPLX(lambda_re, lambda_im), A, A_next, E);
}
double ora_residual_c(int64_t n, const double _Complex* theta,
                      const double _Complex* delta, double lambda_re, double lambda_im,
                      const double _Complex* A, const double _Complex* E, double* rho) {
  return residual_all_c(n, theta, delta, CMPLX(lambda_re, lambda_im), A, E, rho);
}
int ora_solve_full_c(int64_t n, const double _Complex* theta,
                     const double _Complex* delta, double lambda_re, double lambda_im,
                     int64_t ncols, const int64_t* cols, double tol, int64_t max_iter,
                     int epstein_nesbet, double ramp_alpha, const double _Complex* start,
                     double _Complex* A_out, double _Complex* E_out, ora_info* info) {
  return solve_full_c(n, theta, delta, CMPLX(lambda_re, lambda_im), ncols, cols, tol,
                      max_iter, epstein_nesbet, ramp_alpha, start, A_out, E_out, info);
}

/* ---- dominant eigenvector, CSR perturbation ------------------------------ */

/* The single-vector map of Eq. (single_line_dyn) for n = n*, the index of the
 * largest unperturbed eigenvalue (Sec. II.H: the dominant eigenvector is the one
 * attached to the largest epsilon_n when M is perturbative):
 *
 *     y     = Delta z
 *     E     = theta_{n*} + lambda * y_{n*}
 *     z'_m  = lambda * (y_m - y_{n*} z_m) / (theta_{n*} - theta_m)   (m != n*)
 *     z'_n* = 1
 *
 * Delta is given in CSR form (row_ptr[n+1], col_idx[nnz], vals[nnz] as FP32);
 * every value is promoted exactly to FP64.  Convergence is judged by the explicit
 * residual ||M z - E z||_2 / (s ||z||_2), with M z = theta o z + lambda Delta z
 * evaluated by a second pass over the matrix and
 * s = max_m |theta_m| + |lambda| * max_m sum_k |Delta_mk|.
 * nstar < 0 selects argmax_m theta_m (first index on ties).  ramp_alpha and start
 * (n values, or NULL for e_{n*}) as for ora_solve_full_r.
 * Returns the statuses of ora_solve_full_r; the degeneracy test concerns the
 * gaps theta_{n*} - theta_m only, the only ones this map divides by. */
int ora_solve_dominant_csr(int64_t n, const double* theta, const int32_t* row_ptr,
                           const int32_t* col_idx, const float* vals,
                           int64_t nstar, double lambda, double tol,
                           int64_t max_iter, double ramp_alpha, const double* start,
                           double* z_out, double* E_out, ora_info* info) {
  if (info) { info->iters = 0; info->residual = NAN; info->status = ORA_ERR_ARG; }
  if (n <= 0 || !theta || !row_ptr || !col_idx || !vals || !z_out || !E_out ||
      max_iter < 0 || nstar >= n || !(ramp_alpha >= 0.0 && ramp_alpha < 1.0))
    return ORA_ERR_ARG;
  if (row_ptr[0] != 0) return ORA_ERR_ARG;
  for (int64_t m = 0; m < n; ++m) {
    if (row_ptr[m + 1] < row_ptr[m]) return ORA_ERR_ARG;
    for (int32_t q = row_ptr[m]; q < row_ptr[m + 1]; ++q)
      if (col_idx[q] < 0 || col_idx[q] >= n) return ORA_ERR_ARG;
  }
  if (nstar < 0) {
    nstar = 0;
    for (int64_t m = 1; m < n; ++m)
      if (theta[m] > theta[nstar]) nstar = m;
  }
  for (int64_t m = 0; m < n; ++m)
    if (m != nstar && theta[m] == theta[nstar]) {
      if (info) info->status = ORA_ERR_DEGENERATE;
      return ORA_ERR_DEGENERATE;
    }

  double tmax = 0.0, rmax = 0.0;
  for (int64_t m = 0; m < n; ++m) {
    if (fabs(theta[m]) > tmax) tmax = fabs(theta[m]);
    double row = 0.0;
    for (int32_t q = row_ptr[m]; q < row_ptr[m + 1]; ++q) row += fabs((double)vals[q]);
    if (row > rmax) rmax = row;
  }
  const double s = tmax + fabs(lambda) * rmax;

  double* z = (double*)malloc(sizeof(double) * (size_t)n);
  double* zn = (double*)malloc(sizeof(double) * (size_t)n);
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  if (!z || !zn || !y) { free(z); free(zn); free(y); return ORA_ERR_ARG; }
  /* z_0 = e_{n*}, or the given start scaled to the chart z_{n*} = 1 */
  if (start) {
    const double piv = start[nstar];
    int ok = piv != 0.0 && isfinite(piv);
    for (int64_t m = 0; m < n; ++m) ok = ok && isfinite(start[m]);
    if (!ok) {
      free(z); free(zn); free(y);
      return ORA_ERR_ARG;
    }
    for (int64_t m = 0; m < n; ++m) z[m] = (m == nstar) ? 1.0 : start[m] / piv;
  } else {
    for (int64_t m = 0; m < n; ++m) z[m] = (m == nstar) ? 1.0 : 0.0;
  }

  int status = ORA_ERR_MAXITER;
  double best = INFINITY, rho = INFINITY, E = 0.0;
  double pw = 1.0;   /* alpha^k */
  int64_t grown = 0, k = 0;
  for (k = 0;; ++k) {
    /* y = Delta z */
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < n; ++m) {
      double acc = 0.0;
      for (int32_t q = row_ptr[m]; q < row_ptr[m + 1]; ++q)
        acc += (double)vals[q] * z[col_idx[q]];
      y[m] = acc;
    }
    const double ys = y[nstar];
    E = theta[nstar] + lambda * ys;
    /* explicit residual of z: (M z)_m - E z_m with (M z)_m = theta_m z_m + lambda (Delta z)_m */
    double rr = 0.0, zz = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : rr, zz)
    for (int64_t m = 0; m < n; ++m) {
      double acc = 0.0;
      for (int32_t q = row_ptr[m]; q < row_ptr[m + 1]; ++q)
        acc += (double)vals[q] * z[col_idx[q]];
      const double r = theta[m] * z[m] + lambda * acc - E * z[m];
      rr += r * r;
      zz += z[m] * z[m];
    }
    rho = sqrt(rr) / (s * sqrt(zz));
    if (!isfinite(rho)) { status = ORA_ERR_DIVERGED; break; }
    if (rho <= tol) { status = ORA_OK; break; }
    if (rho < best) { best = rho; grown = 0; }
    else if (rho > 10.0 * best) {
      if (++grown >= 20) { status = ORA_ERR_DIVERGED; break; }
    } else grown = 0;
    if (k == max_iter) break;
    /* z' = F_{n*}(z), at lambda (1 - alpha^k) for the non-autonomous iteration */
    const double lam_map = ramp_alpha > 0.0 ? lambda * (1.0 - pw) : lambda;
    pw *= ramp_alpha;
#pragma omp parallel for schedule(static)
    for (int64_t m = 0; m < n; ++m)
      zn[m] = (m == nstar) ? 1.0
                           : lam_map * (y[m] - ys * z[m]) / (theta[nstar] - theta[m]);
    double* t = z; z = zn; zn = t;
  }
  memcpy(z_out, z, sizeof(double) * (size_t)n);
  *E_out = E;
  if (info) { info->iters = k; info->residual = rho; info->status = status; }
  free(z); free(zn); free(y);
  return status;
}

/* ---- Rayleigh-Schroedinger series ---------------------------------------- */

/* Partial sums of the RS series, Eq. (ARS-alpha), in column form.  With
 * C^(l) = (a^(l))^T (column i = correction of eigenvector i), the recursion
 *     a^(l) = theta o ( a^(l-1) Delta' - sum_{s=0}^{l-1} (a^(s) Delta') |> a^(l-1-s) ),
 * with X |> B = (I o X) B, becomes
 *     C^(l) = G o ( Delta C^(l-1) - sum_{s=0}^{l-1} C^(l-1-s) diag(Delta C^(s)) ),
 * where G_ji = 1/(theta_i - theta_j) is the transpose of the paper's theta matrix
 * and diag(X) keeps only the diagonal.  C^(0) = I.  The eigenvalue corrections
 * are eps^(l)_i = (Delta C^(l-1))_ii (Supplement B).
 * Outputs:  A_out = sum_{l=0}^{k} lambda^l C^(l),
 *           E_out = theta + sum_{l=1}^{k} lambda^l eps^(l). */
int ora_rs_series_r(int64_t n, const double* theta, const double* delta,
                    double lambda, int64_t k, double* A_out, double* E_out) {
  if (n <= 0 || k < 0 || !theta || !delta || !A_out || !E_out) return ORA_ERR_ARG;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = i + 1; j < n; ++j)
      if (theta[i] == theta[j]) return ORA_ERR_DEGENERATE;
  const size_t nn = (size_t)(n * n);
  double* C = (double*)calloc(nn * (size_t)(k + 1), sizeof(double));   /* C^(0..k) */
  double* DC = (double*)calloc(nn * (size_t)(k + 1), sizeof(double));  /* Delta C^(l) */
  if (!C || !DC) { free(C); free(DC); return ORA_ERR_ARG; }
  for (int64_t i = 0; i < n; ++i) C[i + i * n] = 1.0;
  int64_t* cols = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
  for (int64_t i = 0; i < n; ++i) cols[i] = i;
  product_cols_r(n, n, delta, C, DC);
  for (int64_t l = 1; l <= k; ++l) {
    double* Cl = C + nn * (size_t)l;
    const double* DCp = DC + nn * (size_t)(l - 1);
    for (int64_t i = 0; i < n; ++i) {
      for (int64_t j = 0; j < n; ++j) {
        if (j == i) { Cl[j + i * n] = 0.0; continue; }
        double acc = DCp[j + i * n];
        for (int64_t s = 0; s <= l - 1; ++s) {
          const double* Cb = C + nn * (size_t)(l - 1 - s);
          const double* DCs = DC + nn * (size_t)s;
          acc -= Cb[j + i * n] * DCs[i + i * n];
        }
        Cl[j + i * n] = acc / (theta[i] - theta[j]);
      }
    }
    product_cols_r(n, n, delta, Cl, DC + nn * (size_t)l);
  }
  for (size_t e = 0; e < nn; ++e) A_out[e] = 0.0;
  for (int64_t i = 0; i < n; ++i) E_out[i] = theta[i];
  double lp = 1.0;
  for (int64_t l = 0; l <= k; ++l) {
    const double* Cl = C + nn * (size_t)l;
    for (size_t e = 0; e < nn; ++e) A_out[e] += lp * Cl[e];
    if (l >= 1) {
      const double* DCp = DC + nn * (size_t)(l - 1);
      for (int64_t i = 0; i < n; ++i) E_out[i] += lp * DCp[i + i * n];
    }
    lp *= lambda;
  }
  free(C); free(DC); free(cols);
  return ORA_OK;
}

/* ---- cyclic Jacobi (real symmetric) --------------------------------------- */

/* Eigen-decomposition S = V diag(w) V^T of a real symmetric n x n matrix by
 * cyclic Jacobi rotations (the classical method; see e.g. Golub & Van Loan,
 * "Matrix Computations", Sec. 8.5).  For each off-diagonal pair (p, q) the
 * rotation angle is chosen so that the rotated (p, q) entry vanishes:
 *     tau = (S_qq - S_pp) / (2 S_pq),  t = sign(tau) / (|tau| + sqrt(1 + tau^2)),
 *     c = 1 / sqrt(1 + t^2),  s = t c;
 * S <- J^T S J and V <- V J with J the plane rotation [[c, s], [-s, c]] in (p, q).
 * Sweeps repeat until the off-diagonal Frobenius norm is below
 * 1e-15 * ||S||_F or 100 sweeps have run.  Eigenvalues are not sorted. */
int ora_jacobi_sym(int64_t n, const double* S_in, double* w, double* V) {
  if (n <= 0 || !S_in || !w || !V) return ORA_ERR_ARG;
  double* S = (double*)malloc(sizeof(double) * (size_t)(n * n));
  if (!S) return ORA_ERR_ARG;
  memcpy(S, S_in, sizeof(double) * (size_t)(n * n));
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) V[i + j * n] = (i == j) ? 1.0 : 0.0;
  double fro = 0.0;
  for (int64_t e = 0; e < n * n; ++e) fro += S[e] * S[e];
  fro = sqrt(fro);
  int status = ORA_ERR_MAXITER;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int64_t q = 0; q < n; ++q)
      for (int64_t p = 0; p < n; ++p)
        if (p != q) off += S[p + q * n] * S[p + q * n];
    if (sqrt(off) <= 1e-15 * fro) { status = ORA_OK; break; }
    for (int64_t p = 0; p < n - 1; ++p) {
      for (int64_t q = p + 1; q < n; ++q) {
        const double spq = S[p + q * n];
        if (spq == 0.0) continue;
        const double tau = (S[q + q * n] - S[p + p * n]) / (2.0 * spq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
        const double c = 1.0 / sqrt(1.0 + t * t);
        const double s = t * c;
        /* columns p, q of S <- S J */
        for (int64_t r = 0; r < n; ++r) {
          const double srp = S[r + p * n], srq = S[r + q * n];
          S[r + p * n] = c * srp - s * srq;
          S[r + q * n] = s * srp + c * srq;
        }
        /* rows p, q of S <- J^T S */
        for (int64_t r = 0; r < n; ++r) {
          const double spr = S[p + r * n], sqr_ = S[q + r * n];
          S[p + r * n] = c * spr - s * sqr_;
          S[q + r * n] = s * spr + c * sqr_;
        }
        S[p + q * n] = 0.0;
        S[q + p * n] = 0.0;
        /* V <- V J */
        for (int64_t r = 0; r < n; ++r) {
          const double vrp = V[r + p * n], vrq = V[r + q * n];
          V[r + p * n] = c * vrp - s * vrq;
          V[r + q * n] = s * vrp + c * vrq;
        }
      }
    }
  }
  for (int64_t i = 0; i < n; ++i) w[i] = S[i + i * n];
  free(S);
  return status;
}
