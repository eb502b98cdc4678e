/* Oracle for dynamical perturbation theory (arXiv:2002.12872).
 * TEST INFRASTRUCTURE ONLY: see dpt_oracle.c.  Column-major storage throughout. */
#ifndef DPT_ORACLE_H
#define DPT_ORACLE_H

#include <stdint.h>

#define ORA_OK 0
#define ORA_ERR_ARG (-1)
#define ORA_ERR_DEGENERATE (-2)
#define ORA_ERR_MAXITER (-3)
#define ORA_ERR_DIVERGED (-4)

typedef struct {
  int64_t iters;    /* map applications performed before the returned iterate */
  double residual;  /* max normalised explicit residual of the returned iterate */
  int64_t status;   /* one of ORA_* */
} ora_info;

#ifdef __cplusplus
extern "C" {
#endif

int ora_step_r(int64_t n, const double* theta, const double* delta, double lambda,
               const double* A, double* A_next, double* E);
double ora_residual_r(int64_t n, const double* theta, const double* delta,
                      double lambda, const double* A, const double* E, double* rho);
int ora_solve_full_r(int64_t n, const double* theta, const double* delta,
                     double lambda, int64_t ncols, const int64_t* cols, double tol,
                     int64_t max_iter, int epstein_nesbet, double ramp_alpha,
                     const double* start, double* A_out, double* E_out, ora_info* info);

int ora_step_c(int64_t n, const double _Complex* theta, const double _Complex* delta,
               double lambda_re, double lambda_im, const double _Complex* A,
               double _Complex* A_next, double _Complex* E);
double ora_residual_c(int64_t n, const double _Complex* theta,
                      const double _Complex* delta, double lambda_re, double lambda_im,
                      const double _Complex* A, const double _Complex* E, double* rho);
int ora_solve_full_c(int64_t n, const double _Complex* theta,
                     const double _Complex* delta, double lambda_re, double lambda_im,
                     int64_t ncols, const int64_t* cols, double tol, int64_t max_iter,
                     int epstein_nesbet, double ramp_alpha, const double _Complex* start,
                     double _Complex* A_out, double _Complex* E_out, ora_info* info);

int ora_solve_dominant_csr(int64_t n, const double* theta, const int32_t* row_ptr,
                           const int32_t* col_idx, const float* vals, int64_t nstar,
                           double lambda, double tol, int64_t max_iter,
                           double ramp_alpha, const double* start, double* z_out,
                           double* E_out, ora_info* info);

int ora_rs_series_r(int64_t n, const double* theta, const double* delta,
                    double lambda, int64_t k, double* A_out, double* E_out);

int ora_jacobi_sym(int64_t n, const double* S, double* w, double* V);

/* Threads for the column-parallel loops (n <= 0: unchanged); returns the count in
 * effect.  Timing control only: no result depends on it beyond the summation
 * order of the residual norms. */
int ora_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
