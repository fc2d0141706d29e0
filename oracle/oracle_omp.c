/*
 * Timed CPU baseline of the oracle -- TEST AND MEASUREMENT INFRASTRUCTURE
 * ONLY (see oracle.h): only bench.py's cpu_baseline / reference leg and
 * tests/ load it.
 *
 * The same plain FP64 loops as oracle.c -- Jacobi seed (Section 3),
 * Lanczos for the interval, the coefficients of Section 2.2 / Eq. thetamod
 * / Eq. rhocheb, Algorithm 2 for p_k(A_hat) r and PCG (Section 1) -- with
 * one change: every loop over rows is an OpenMP `parallel for` (inner
 * products as a `reduction(+)`), so the solve uses all host cores.  No
 * blocking, fusion or reordering is added.  The single-thread oracle.c
 * routines used for parity are not changed; this file is built into a
 * library of its own (liboracle_omp.so) together with oracle.c, whose
 * Sturm bisection and coefficient routines it calls for the scalar setup.
 */
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

int oracle_omp_threads(void) { return omp_get_max_threads(); }

static double pdot(int n, const double* x, const double* y) {
  double s = 0.0;
#pragma omp parallel for reduction(+ : s) schedule(static)
  for (int i = 0; i < n; ++i) s += x[i] * y[i];
  return s;
}

static void pspmv(int n, const int* rowptr, const int* col, const double* val, const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) s += val[p] * x[col[p]];
    y[i] = s;
  }
}

typedef struct {
  int n;
  const int *rowptr, *col;
  const double* val;
} mat_t;

/* Algorithm 2 (ChebAlg), as in oracle.c: x_old = r/theta; x = (2 rho_1 /
 * delta)(2 r - A r / theta); for j = 2..k the three-term step. */
static void pcheb(const mat_t* A, int k, double tb, double d, double sb, const double* rho, const double* r,
                  double* out, double* x_old, double* x, double* t, double* zv) {
  int n = A->n;
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) x_old[i] = r[i] / tb;
  if (k == 0) {
    memcpy(out, x_old, sizeof(double) * (size_t)n);
    return;
  }
  pspmv(n, A->rowptr, A->col, A->val, r, t);
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) x[i] = (2.0 * rho[1] / d) * (2.0 * r[i] - t[i] / tb);
  for (int j = 2; j <= k; ++j) {
    pspmv(n, A->rowptr, A->col, A->val, x, t);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) zv[i] = (2.0 / d) * (r[i] - t[i]);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
      double rhat = rho[j] * (2.0 * sb * x[i] - rho[j - 1] * x_old[i] + zv[i]);
      x_old[i] = x[i];
      x[i] = rhat;
    }
  }
  memcpy(out, x, sizeof(double) * (size_t)n);
}

/* Full solve with the interval from `lanczos_steps` Lanczos steps on
 * A_hat = W A W from v0 (no reorthogonalisation, as oracle_lanczos), xi =
 * clip(10 alpha/beta, 1e-6, 1e-2) when xi < 0, and PCG from x = 0 to
 * ||r||/||b|| <= rtol (recursive residual of the scaled system).
 * seconds[0] = setup (scaling, Lanczos, coefficients), seconds[1] = the
 * PCG iterations alone, both wall-clock.  Returns the oracle status. */
int oracle_omp_solve(int n, const int* rowptr, const int* col, const double* val, const double* b, double* x,
                     const double* v0, int k, int lanczos_steps, double xi_in, double rtol, int maxit,
                     oracle_stats* st, double* seconds) {
  if (n <= 0 || k < 0 || lanczos_steps < 1) return -1;
  double t0 = omp_get_wtime();
  int nnz = rowptr[n];
  double* vh = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  double* buf = (double*)calloc((size_t)n * 10, sizeof(double));
  double *bh = buf, *xh = buf + n, *r = buf + 2 * (size_t)n, *z = buf + 3 * (size_t)n, *p = buf + 4 * (size_t)n,
         *q = buf + 5 * (size_t)n, *s1 = buf + 6 * (size_t)n, *s2 = buf + 7 * (size_t)n, *s3 = buf + 8 * (size_t)n,
         *s4 = buf + 9 * (size_t)n;
  double* a = (double*)calloc((size_t)lanczos_steps, sizeof(double));
  double* bl = (double*)calloc((size_t)lanczos_steps, sizeof(double));
  double* rho = (double*)malloc(sizeof(double) * (size_t)(k + 1));
  int rc = 0, it = 0;
  long long mvp = 0, dots = 0;
  double rel = 0.0, alpha = 0.0, beta = 0.0, xi = 0.0;
  int bad = 0;
  /* Section 3: W = diag(A)^{-1/2}, A_hat = W A W */
#pragma omp parallel for schedule(static) reduction(+ : bad)
  for (int i = 0; i < n; ++i) {
    double dd = 0.0;
    for (int pp = rowptr[i]; pp < rowptr[i + 1]; ++pp)
      if (col[pp] == i) dd += val[pp];
    if (!(dd > 0.0)) bad += 1;
    w[i] = dd > 0.0 ? 1.0 / sqrt(dd) : 1.0;
  }
  if (bad) {
    rc = -2;
    goto out;
  }
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i)
    for (int pp = rowptr[i]; pp < rowptr[i + 1]; ++pp) vh[pp] = w[i] * val[pp] * w[col[pp]];
  mat_t A = {n, rowptr, col, vh};
  /* Lanczos on A_hat (lanczos_op of oracle.c, loops in parallel) */
  {
    double *v = s1, *vp = s2, *wv = s3;
    double nv = sqrt(pdot(n, v0, v0));
    int steps = 0;
    if (nv > 0.0) {
#pragma omp parallel for schedule(static)
      for (int i = 0; i < n; ++i) {
        v[i] = v0[i] / nv;
        vp[i] = 0.0;
      }
      double bprev = 0.0;
      for (int j = 0; j < lanczos_steps; ++j) {
        pspmv(n, rowptr, col, vh, v, wv);
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i) wv[i] -= bprev * vp[i];
        a[j] = pdot(n, wv, v);
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i) wv[i] -= a[j] * v[i];
        steps = j + 1;
        if (j == lanczos_steps - 1) break;
        double bj = sqrt(pdot(n, wv, wv));
        if (!(bj > 1e-300)) break;
        bl[j] = bj;
#pragma omp parallel for schedule(static)
        for (int i = 0; i < n; ++i) {
          vp[i] = v[i];
          v[i] = wv[i] / bj;
        }
        bprev = bj;
      }
    }
    if (steps == 0 || oracle_tridiag_extremes(steps, a, bl, &alpha, &beta) != 0) {
      rc = -1;
      goto out;
    }
  }
  xi = xi_in >= 0.0 ? xi_in : fmin(fmax(10.0 * alpha / beta, 1e-6), 1e-2);
  double tb, d, sb;
  if (oracle_cheb_coeffs(alpha, beta, xi, k, &tb, &d, &sb, rho) != 0) {
    rc = -1;
    goto out;
  }
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) {
    bh[i] = w[i] * b[i];
    xh[i] = 0.0;
  }
  double t1 = omp_get_wtime();
  /* PCG (pcg_op of oracle.c, plain variant, x0 = 0) */
  double bnorm = sqrt(pdot(n, bh, bh));
  memcpy(r, bh, sizeof(double) * (size_t)n);
  rel = bnorm > 0.0 ? 1.0 : 0.0;
  if (bnorm == 0.0 || rel <= rtol) goto solved;
  pcheb(&A, k, tb, d, sb, rho, r, z, s1, s2, s3, s4);
  mvp += k;
  memcpy(p, z, sizeof(double) * (size_t)n);
  double rz = pdot(n, r, z);
  ++dots;
  if (!(rz > 0.0)) {
    rc = isfinite(rz) ? -2 : -3;
    goto solved;
  }
  rc = 1;
  while (it < maxit) {
    pspmv(n, rowptr, col, vh, p, q);
    ++mvp;
    double pq = pdot(n, p, q);
    ++dots;
    if (!(pq > 0.0)) {
      rc = isfinite(pq) ? -2 : -3;
      break;
    }
    double al = rz / pq;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) xh[i] += al * p[i];
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) r[i] -= al * q[i];
    ++it;
    double rr = pdot(n, r, r);
    ++dots;
    if (!isfinite(rr)) {
      rc = -3;
      break;
    }
    rel = sqrt(rr) / bnorm;
    if (rel <= rtol) {
      rc = 0;
      break;
    }
    pcheb(&A, k, tb, d, sb, rho, r, z, s1, s2, s3, s4);
    mvp += k;
    double rz_new = pdot(n, r, z);
    ++dots;
    if (!(rz_new > 0.0)) {
      rc = isfinite(rz_new) ? -2 : -3;
      break;
    }
    double be = rz_new / rz;
    rz = rz_new;
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) p[i] = z[i] + be * p[i];
  }
solved:;
  double t2 = omp_get_wtime();
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i) x[i] = w[i] * xh[i];
  if (seconds) {
    seconds[0] = t1 - t0;
    seconds[1] = t2 - t1;
  }
out:
  if (st) {
    st->iterations = it;
    st->mvp = mvp;
    st->dots = dots;
    st->rel_res = rel;
    st->true_rel_res = 0.0;
    st->alpha_hat = alpha;
    st->beta_hat = beta;
    st->xi = xi;
    st->status = rc;
  }
  free(vh);
  free(w);
  free(buf);
  free(a);
  free(bl);
  free(rho);
  return rc;
}
