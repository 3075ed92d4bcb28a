/*
 * Unpreconditioned conjugate gradients on the full unreduced system, FP64,
 * OpenMP over the host cores (ORACLE; test infrastructure only: tests/,
 * smoke() and the CPU legs of bench.py use it; the CUDA library never does).
 *
 * The same iteration as oracle.solvers.cg (the paper's outer Krylov method,
 * Sec. 5, without a preconditioner), written as plain loops so that it runs
 * on every host core: q = A p, alpha = <r,r>/<p,q>, x += alpha p,
 * r -= alpha q, beta = <r,r>_new/<r,r>, p = r + beta p, from x = 0.  It stops
 * when ||r|| <= tol ||b|| (recurrence residual) or after maxit iterations.
 * The CG coefficients are returned so that the caller can form the Lanczos
 * tridiagonal (Ritz values bound the spectrum from inside).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <omp.h>

static void spmv(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s += v[e] * x[ci[e]];
    y[i] = s;
  }
}

static double dot(int64_t n, const double* a, const double* b) {
  double s = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : s)
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Returns the iterations run; -1 if a work array could not be allocated.
 * alphas/betas (may be NULL) receive up to maxit coefficients; *seconds the
 * wall time of the iteration loop; *threads the OpenMP threads used. */
int oracle_cg(int64_t n, const int64_t* rp, const int32_t* ci, const double* v, const double* b, double* x,
              int32_t maxit, double tol, int32_t nthreads, double* alphas, double* betas, double* seconds,
              int32_t* threads) {
  if (nthreads > 0) omp_set_num_threads(nthreads);
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* p = (double*)malloc(sizeof(double) * (size_t)n);
  double* q = (double*)malloc(sizeof(double) * (size_t)n);
  if (!r || !p || !q) {
    free(r);
    free(p);
    free(q);
    return -1;
  }
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    x[i] = 0.0;
    r[i] = b[i];
    p[i] = b[i];
  }
  int32_t nt = 1;
#pragma omp parallel
  {
#pragma omp single
    nt = (int32_t)omp_get_num_threads();
  }
  if (threads) *threads = nt;
  const double bn = sqrt(dot(n, b, b));
  double rr = dot(n, r, r);
  int32_t it = 0;
  const double t0 = omp_get_wtime();
  while (it < maxit && sqrt(rr) > tol * bn) {
    spmv(n, rp, ci, v, p, q);
    const double alpha = rr / dot(n, p, q);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * q[i];
    }
    const double rr_new = dot(n, r, r);
    const double beta = rr_new / rr;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    rr = rr_new;
    if (alphas) alphas[it] = alpha;
    if (betas) betas[it] = beta;
    ++it;
  }
  if (seconds) *seconds = omp_get_wtime() - t0;
  free(r);
  free(p);
  free(q);
  return it;
}
