/*
 * Plain FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Written for clarity, not speed: no blocking, no fusion, no reordering
 * beyond what each cited definition or algorithm states.  Single thread.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */

static double dot(int n, const double* x, const double* y) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += x[i] * y[i];
  return s;
}

static int all_finite(int n, const double* x) {
  for (int i = 0; i < n; ++i)
    if (!isfinite(x[i])) return 0;
  return 1;
}

/* ------------------------------------------------------------------ */
/* Chebyshev coefficients: Section 2.2 and Eq. thetamod, Eq. rhocheb   */
/* ------------------------------------------------------------------ */

/* theta = (beta+alpha)/2, delta = (beta-alpha)/2 (Section 2.2);
 * theta_bar = theta (1 + xi) (Eq. thetamod); delta is kept and
 * sigma_bar = theta_bar / delta, i.e. the polynomial is the Chebyshev
 * polynomial of the shifted interval [theta_bar - delta, theta_bar + delta].
 * This is the reading of the xi-modification that reproduces Table 1.
 * rho_0 = 1/sigma_bar, rho_j = 1/(2 sigma_bar - rho_{j-1}) (Eq. rhocheb). */
int oracle_cheb_coeffs(double alpha, double beta, double xi, int k, double* theta_bar,
                       double* delta, double* sigma_bar, double* rho) {
  if (!(alpha > 0.0) || !(beta > alpha) || k < 0 || xi < 0.0) return -1;
  double theta = 0.5 * (beta + alpha);
  double d = 0.5 * (beta - alpha);
  double tb = theta * (1.0 + xi);
  double sb = tb / d;
  *theta_bar = tb;
  *delta = d;
  *sigma_bar = sb;
  if (rho) {
    rho[0] = 1.0 / sb;
    for (int j = 1; j <= k; ++j) rho[j] = 1.0 / (2.0 * sb - rho[j - 1]);
  }
  return 0;
}

/* Scalar p_k(x) by the three-term recursion Eq. polycheb:
 * p_{-1} = 0, p_0 = 1/theta, p_j = rho_j (2 sigma (1 - x/theta) p_{j-1}
 * - rho_{j-1} p_{j-2} + 2/delta), with theta, sigma replaced by their
 * xi-modified values. */
double oracle_cheb_poly(double x, double alpha, double beta, double xi, int k) {
  double tb, d, sb;
  double* rho = (double*)malloc(sizeof(double) * (size_t)(k + 1));
  if (oracle_cheb_coeffs(alpha, beta, xi, k, &tb, &d, &sb, rho) != 0) {
    free(rho);
    return NAN;
  }
  double pm2 = 0.0;       /* p_{j-2} */
  double pm1 = 1.0 / tb;  /* p_{j-1}; starts as p_0 */
  for (int j = 1; j <= k; ++j) {
    double pj = rho[j] * (2.0 * sb * (1.0 - x / tb) * pm1 - rho[j - 1] * pm2 + 2.0 / d);
    pm2 = pm1;
    pm1 = pj;
  }
  free(rho);
  return pm1;
}

/* ------------------------------------------------------------------ */
/* Linear operators                                                    */
/* ------------------------------------------------------------------ */

void oracle_spmv(int n, const int* rowptr, const int* col, const double* val, const double* x,
                 double* y) {
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) s += val[p] * x[col[p]];
    y[i] = s;
  }
}

typedef struct {
  void (*apply)(const void* ctx, const double* x, double* y);
  const void* ctx;
  int n;
} op_t;

typedef struct {
  int n;
  const int *rowptr, *col;
  const double* val;
} csr_t;

static void csr_apply(const void* c, const double* x, double* y) {
  const csr_t* a = (const csr_t*)c;
  oracle_spmv(a->n, a->rowptr, a->col, a->val, x, y);
}

/* ------------------------------------------------------------------ */
/* Algorithm 2 (ChebAlg): r_hat = P_m r                                */
/* ------------------------------------------------------------------ */

static int cheb_apply_op(const op_t* A, int m, double theta_bar, double delta, double sigma_bar,
                         const double* rho, const double* r, double* out, long long* mvp) {
  int n = A->n;
  double* x_old = (double*)malloc(sizeof(double) * (size_t)n);
  double* x = (double*)malloc(sizeof(double) * (size_t)n);
  double* t = (double*)malloc(sizeof(double) * (size_t)n);
  double* zv = (double*)malloc(sizeof(double) * (size_t)n);
  /* step 2: x_old = r / theta (exit here when m = 0) */
  for (int i = 0; i < n; ++i) x_old[i] = r[i] / theta_bar;
  if (m == 0) {
    memcpy(out, x_old, sizeof(double) * (size_t)n);
  } else {
    /* step 3: x = (2 rho_1 / delta) (2 r - A r / theta) (exit when m = 1) */
    A->apply(A->ctx, r, t);
    if (mvp) ++*mvp;
    for (int i = 0; i < n; ++i) x[i] = (2.0 * rho[1] / delta) * (2.0 * r[i] - t[i] / theta_bar);
    /* steps 4-8: for k = 2..m */
    for (int k = 2; k <= m; ++k) {
      A->apply(A->ctx, x, t);
      if (mvp) ++*mvp;
      for (int i = 0; i < n; ++i) zv[i] = (2.0 / delta) * (r[i] - t[i]);
      for (int i = 0; i < n; ++i) {
        double rhat = rho[k] * (2.0 * sigma_bar * x[i] - rho[k - 1] * x_old[i] + zv[i]);
        x_old[i] = x[i];
        x[i] = rhat;
      }
    }
    memcpy(out, x, sizeof(double) * (size_t)n);
  }
  free(x_old);
  free(x);
  free(t);
  free(zv);
  return all_finite(n, out) ? 0 : -3;
}

int oracle_cheb_apply(int n, const int* rowptr, const int* col, const double* val, double alpha,
                      double beta, double xi, int k, const double* r, double* z) {
  double tb, d, sb;
  double* rho = (double*)malloc(sizeof(double) * (size_t)(k + 1));
  int rc = oracle_cheb_coeffs(alpha, beta, xi, k, &tb, &d, &sb, rho);
  if (rc == 0) {
    csr_t a = {n, rowptr, col, val};
    op_t op = {csr_apply, &a, n};
    rc = cheb_apply_op(&op, k, tb, d, sb, rho, r, z, NULL);
  }
  free(rho);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Algorithm 1 (NewtAlg): Newton-based preconditioner of level nlev    */
/* ------------------------------------------------------------------ */
/* zeta_0 scales the interval to be centred on 1: zeta_0 = 1/theta_bar
 * (= 2/(alpha+beta) when xi = 0).  The lower end of the xi-shifted interval
 * is alpha' = theta_bar - delta, so zeta_1 = 2/(1 + 2 alpha' zeta_0 -
 * (alpha' zeta_0)^2) and zeta_i = 2/(1 + 2 zeta_{i-1} - zeta_{i-1}^2)
 * (Eq. zetaNewt).  P_hat_0 r = zeta_0 r and P_hat_{j+1} r =
 * zeta_{j+1} (2 P_hat_j r - P_hat_j A P_hat_j r) (Eq. newrec0), applied
 * recursively: degree 2^nlev - 1, with 2^nlev - 1 products by A. */
static void newton_rec(const op_t* A, const double* zeta, int j, const double* r, double* out) {
  int n = A->n;
  if (j == 0) {
    for (int i = 0; i < n; ++i) out[i] = zeta[0] * r[i];
    return;
  }
  double* y = (double*)malloc(sizeof(double) * (size_t)n);
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  double* v = (double*)malloc(sizeof(double) * (size_t)n);
  newton_rec(A, zeta, j - 1, r, y);  /* y = P_hat_{j-1} r         */
  A->apply(A->ctx, y, w);            /* w = A P_hat_{j-1} r       */
  newton_rec(A, zeta, j - 1, w, v);  /* v = P_hat_{j-1} A P_hat_{j-1} r */
  for (int i = 0; i < n; ++i) out[i] = zeta[j] * (2.0 * y[i] - v[i]);
  free(y);
  free(w);
  free(v);
}

int oracle_newton_apply(int n, const int* rowptr, const int* col, const double* val,
                        double alpha, double beta, double xi, int nlev, const double* r,
                        double* z) {
  if (nlev < 0 || !(alpha > 0.0) || !(beta > alpha) || xi < 0.0) return -1;
  double theta = 0.5 * (beta + alpha), delta = 0.5 * (beta - alpha);
  double theta_bar = theta * (1.0 + xi);
  double a_shift = theta_bar - delta;
  double* zeta = (double*)malloc(sizeof(double) * (size_t)(nlev + 1));
  zeta[0] = 1.0 / theta_bar;
  if (nlev >= 1) {
    double az = a_shift * zeta[0];
    zeta[1] = 2.0 / (1.0 + 2.0 * az - az * az);
  }
  for (int i = 2; i <= nlev; ++i) zeta[i] = 2.0 / (1.0 + 2.0 * zeta[i - 1] - zeta[i - 1] * zeta[i - 1]);
  csr_t a = {n, rowptr, col, val};
  op_t op = {csr_apply, &a, n};
  newton_rec(&op, zeta, nlev, r, z);
  free(zeta);
  return all_finite(n, z) ? 0 : -3;
}

/* ------------------------------------------------------------------ */
/* Section 3: seed preconditioner W = diag(A)^{-1/2}, A_hat = W^T A W  */
/* ------------------------------------------------------------------ */

int oracle_jacobi_scale(int n, const int* rowptr, const int* col, const double* val,
                        double* val_hat, double* w) {
  for (int i = 0; i < n; ++i) {
    double d = 0.0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p)
      if (col[p] == i) d += val[p];
    if (!(d > 0.0)) return -2;
    w[i] = 1.0 / sqrt(d);
  }
  for (int i = 0; i < n; ++i)
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) val_hat[p] = w[i] * val[p] * w[col[p]];
  return 0;
}

/* ------------------------------------------------------------------ */
/* Lanczos tridiagonalisation and Sturm bisection                      */
/* ------------------------------------------------------------------ */

static int lanczos_op(const op_t* A, const double* v0, int m, double* a, double* b) {
  int n = A->n;
  double* v = (double*)calloc((size_t)n, sizeof(double));
  double* vp = (double*)calloc((size_t)n, sizeof(double));
  double* w = (double*)calloc((size_t)n, sizeof(double));
  double nv = sqrt(dot(n, v0, v0));
  int steps = 0;
  if (nv > 0.0) {
    for (int i = 0; i < n; ++i) v[i] = v0[i] / nv;
    double bprev = 0.0;
    for (int j = 0; j < m; ++j) {
      A->apply(A->ctx, v, w);
      for (int i = 0; i < n; ++i) w[i] -= bprev * vp[i];
      a[j] = dot(n, w, v);
      for (int i = 0; i < n; ++i) w[i] -= a[j] * v[i];
      steps = j + 1;
      if (j == m - 1) break;
      double bj = sqrt(dot(n, w, w));
      if (!(bj > 1e-300)) break; /* invariant subspace found */
      b[j] = bj;
      for (int i = 0; i < n; ++i) {
        vp[i] = v[i];
        v[i] = w[i] / bj;
      }
      bprev = bj;
    }
  }
  free(v);
  free(vp);
  free(w);
  return steps;
}

int oracle_lanczos(int n, const int* rowptr, const int* col, const double* val,
                   const double* v0, int m, double* a, double* b) {
  csr_t c = {n, rowptr, col, val};
  op_t op = {csr_apply, &c, n};
  return lanczos_op(&op, v0, m, a, b);
}

/* number of eigenvalues of T (diag a, off-diag b) smaller than x */
static int sturm_count(int m, const double* a, const double* b, double x) {
  int cnt = 0;
  double d = 1.0;
  for (int i = 0; i < m; ++i) {
    double off = (i > 0) ? b[i - 1] * b[i - 1] / d : 0.0;
    d = a[i] - x - off;
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++cnt;
  }
  return cnt;
}

int oracle_tridiag_extremes(int m, const double* a, const double* b, double* lmin,
                            double* lmax) {
  if (m <= 0) return -1;
  double lo = a[0], hi = a[0];
  for (int i = 0; i < m; ++i) {
    double r = 0.0;
    if (i > 0) r += fabs(b[i - 1]);
    if (i < m - 1) r += fabs(b[i]);
    if (a[i] - r < lo) lo = a[i] - r;
    if (a[i] + r > hi) hi = a[i] + r;
  }
  double span = hi - lo + 1e-300;
  /* smallest eigenvalue: the point where the count goes from 0 to 1 */
  double l = lo - 1e-12 * span, h = hi + 1e-12 * span;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (l + h);
    if (sturm_count(m, a, b, mid) >= 1) h = mid; else l = mid;
  }
  *lmin = 0.5 * (l + h);
  /* largest eigenvalue: the point where the count goes from m-1 to m */
  l = lo - 1e-12 * span;
  h = hi + 1e-12 * span;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (l + h);
    if (sturm_count(m, a, b, mid) >= m) h = mid; else l = mid;
  }
  *lmax = 0.5 * (l + h);
  return 0;
}

/* ------------------------------------------------------------------ */
/* Section 3.1: leftmost eigenpairs for the low-rank acceleration      */
/* ------------------------------------------------------------------ */
/* Lanczos that keeps its basis: q_0 = v0/||v0||; step j forms
 * w = A q_j - b_{j-1} q_{j-1}, a_j = (w, q_j), w -= a_j q_j, then
 * orthogonalises w against every kept q_0..q_j by classical Gram-Schmidt,
 * done twice, and sets b_j = ||w||, q_{j+1} = w / b_j.  Q is n x m with
 * q_j at Q + j n.  b[m-1] is the coupling beta_m to the next (not kept)
 * vector: the Ritz pair (theta, Q y) of T_m has residual beta_m |y_m|. */
static int lanczos_basis_op(const op_t* A, const double* v0, int m, double* a, double* b,
                            double* Q) {
  int n = A->n;
  double* w = (double*)calloc((size_t)n, sizeof(double));
  double* h = (double*)calloc((size_t)m, sizeof(double));
  double nv = sqrt(dot(n, v0, v0));
  int steps = 0;
  if (nv > 0.0) {
    for (int i = 0; i < n; ++i) Q[i] = v0[i] / nv;
    for (int j = 0; j < m; ++j) {
      const double* qj = Q + (size_t)j * n;
      A->apply(A->ctx, qj, w);
      if (j > 0) {
        const double* qp = Q + (size_t)(j - 1) * n;
        for (int i = 0; i < n; ++i) w[i] -= b[j - 1] * qp[i];
      }
      a[j] = dot(n, w, qj);
      for (int i = 0; i < n; ++i) w[i] -= a[j] * qj[i];
      for (int pass = 0; pass < 2; ++pass) {
        for (int l = 0; l <= j; ++l) h[l] = dot(n, Q + (size_t)l * n, w);
        for (int l = 0; l <= j; ++l) {
          const double* ql = Q + (size_t)l * n;
          for (int i = 0; i < n; ++i) w[i] -= h[l] * ql[i];
        }
      }
      b[j] = sqrt(dot(n, w, w));
      steps = j + 1;
      if (j == m - 1) break;
      if (!(b[j] > 1e-300)) break; /* invariant subspace found */
      double* qn = Q + (size_t)(j + 1) * n;
      for (int i = 0; i < n; ++i) qn[i] = w[i] / b[j];
    }
  }
  free(w);
  free(h);
  return steps;
}

int oracle_lanczos_basis(int n, const int* rowptr, const int* col, const double* val,
                         const double* v0, int m, double* a, double* b, double* Q) {
  csr_t c = {n, rowptr, col, val};
  op_t op = {csr_apply, &c, n};
  return lanczos_basis_op(&op, v0, m, a, b, Q);
}

/* Solve the dense m x m system M y = f by Gaussian elimination with
 * partial pivoting (M and f are overwritten); a zero pivot is replaced by
 * tiny, which is what inverse iteration wants at an exact eigenvalue. */
static void dense_solve(int m, double* M, double* f, double* y, double tiny) {
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (fabs(M[(size_t)r * m + c]) > fabs(M[(size_t)piv * m + c])) piv = r;
    if (piv != c) {
      for (int k = 0; k < m; ++k) {
        double t = M[(size_t)c * m + k];
        M[(size_t)c * m + k] = M[(size_t)piv * m + k];
        M[(size_t)piv * m + k] = t;
      }
      double t = f[c];
      f[c] = f[piv];
      f[piv] = t;
    }
    if (fabs(M[(size_t)c * m + c]) < tiny) M[(size_t)c * m + c] = tiny;
    for (int r = c + 1; r < m; ++r) {
      double l = M[(size_t)r * m + c] / M[(size_t)c * m + c];
      if (l == 0.0) continue;
      for (int k = c; k < m; ++k) M[(size_t)r * m + k] -= l * M[(size_t)c * m + k];
      f[r] -= l * f[c];
    }
  }
  for (int r = m - 1; r >= 0; --r) {
    double s = f[r];
    for (int k = r + 1; k < m; ++k) s -= M[(size_t)r * m + k] * y[k];
    y[r] = s / M[(size_t)r * m + r];
  }
}

/* The i-th smallest eigenvalue (i = 0, 1, ...) of the tridiagonal T (diag a,
 * off-diagonal b) by Sturm-sequence bisection, and its unit eigenvector by
 * three steps of inverse iteration on the dense T - lambda I.  The sign is
 * fixed by making the largest-magnitude entry positive. */
int oracle_tridiag_eig(int m, const double* a, const double* b, int i, double* lambda,
                       double* y) {
  if (m <= 0 || i < 0 || i >= m) return -1;
  double lo = a[0], hi = a[0];
  for (int r = 0; r < m; ++r) {
    double rad = 0.0;
    if (r > 0) rad += fabs(b[r - 1]);
    if (r < m - 1) rad += fabs(b[r]);
    if (a[r] - rad < lo) lo = a[r] - rad;
    if (a[r] + rad > hi) hi = a[r] + rad;
  }
  double span = hi - lo + 1e-300;
  double l = lo - 1e-12 * span, h = hi + 1e-12 * span;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (l + h);
    if (sturm_count(m, a, b, mid) >= i + 1) h = mid; else l = mid;
  }
  double lam = 0.5 * (l + h);
  *lambda = lam;
  double* M = (double*)malloc(sizeof(double) * (size_t)m * m);
  double* f = (double*)malloc(sizeof(double) * (size_t)m);
  for (int r = 0; r < m; ++r) y[r] = 1.0 / sqrt((double)m) * (1.0 + 0.01 * r);
  for (int step = 0; step < 3; ++step) {
    for (size_t t = 0; t < (size_t)m * m; ++t) M[t] = 0.0;
    for (int r = 0; r < m; ++r) {
      M[(size_t)r * m + r] = a[r] - lam;
      if (r + 1 < m) M[(size_t)r * m + r + 1] = M[(size_t)(r + 1) * m + r] = b[r];
      f[r] = y[r];
    }
    dense_solve(m, M, f, y, 1e-300 + 1e-15 * span);
    double nrm = sqrt(dot(m, y, y));
    for (int r = 0; r < m; ++r) y[r] /= nrm;
  }
  int big = 0;
  for (int r = 1; r < m; ++r)
    if (fabs(y[r]) > fabs(y[big])) big = r;
  if (y[big] < 0.0)
    for (int r = 0; r < m; ++r) y[r] = -y[r];
  free(M);
  free(f);
  return 0;
}

/* Ritz vectors of the p smallest Ritz values: V_i = Q y_i (n x p). */
static int ritz_vectors(int n, int m, const double* a, const double* b, const double* Q, int p,
                        double* V, double* theta) {
  if (p > m) return -1;
  double* y = (double*)malloc(sizeof(double) * (size_t)m);
  for (int i = 0; i < p; ++i) {
    double th;
    oracle_tridiag_eig(m, a, b, i, &th, y);
    if (theta) theta[i] = th;
    double* vi = V + (size_t)i * n;
    for (int r = 0; r < n; ++r) vi[r] = 0.0;
    for (int j = 0; j < m; ++j)
      for (int r = 0; r < n; ++r) vi[r] += y[j] * Q[(size_t)j * n + r];
  }
  free(y);
  return 0;
}

/* The spectral correction of Section 3.1: P = P_0 + V (V^T A V)^{-1} V^T.
 * G = V^T A V is formed once (p products by A, not counted as PCG work)
 * and factorised by Cholesky, G = L L^T; each application then costs p
 * inner products (V^T r) and one combination of the columns of V. */
typedef struct {
  int p;
  const double* V; /* n x p, column i at V + i n */
  double* L;       /* p x p lower Cholesky factor of G */
} lowrank_t;

static int lowrank_setup(const op_t* A, int p, const double* V, lowrank_t* lr) {
  int n = A->n;
  lr->p = p;
  lr->V = V;
  lr->L = (double*)calloc((size_t)(p > 0 ? p * p : 1), sizeof(double));
  if (p == 0) return 0;
  double* G = (double*)malloc(sizeof(double) * (size_t)p * p);
  double* t = (double*)malloc(sizeof(double) * (size_t)n);
  for (int j = 0; j < p; ++j) {
    A->apply(A->ctx, V + (size_t)j * n, t);
    for (int i = 0; i < p; ++i) G[(size_t)i * p + j] = dot(n, V + (size_t)i * n, t);
  }
  int rc = 0;
  for (int j = 0; j < p && rc == 0; ++j) {
    double d = G[(size_t)j * p + j];
    for (int k = 0; k < j; ++k) d -= lr->L[(size_t)j * p + k] * lr->L[(size_t)j * p + k];
    if (!(d > 0.0)) { rc = -2; break; }
    lr->L[(size_t)j * p + j] = sqrt(d);
    for (int i = j + 1; i < p; ++i) {
      double s = G[(size_t)i * p + j];
      for (int k = 0; k < j; ++k) s -= lr->L[(size_t)i * p + k] * lr->L[(size_t)j * p + k];
      lr->L[(size_t)i * p + j] = s / lr->L[(size_t)j * p + j];
    }
  }
  free(G);
  free(t);
  return rc;
}

/* z += V G^{-1} V^T r */
static void lowrank_add(int n, const lowrank_t* lr, const double* r, double* z) {
  int p = lr->p;
  double* c = (double*)malloc(sizeof(double) * (size_t)p);
  for (int i = 0; i < p; ++i) c[i] = dot(n, lr->V + (size_t)i * n, r);
  for (int i = 0; i < p; ++i) { /* L u = w */
    double s = c[i];
    for (int k = 0; k < i; ++k) s -= lr->L[(size_t)i * p + k] * c[k];
    c[i] = s / lr->L[(size_t)i * p + i];
  }
  for (int i = p - 1; i >= 0; --i) { /* L^T c = u */
    double s = c[i];
    for (int k = i + 1; k < p; ++k) s -= lr->L[(size_t)k * p + i] * c[k];
    c[i] = s / lr->L[(size_t)i * p + i];
  }
  for (int i = 0; i < p; ++i) {
    const double* vi = lr->V + (size_t)i * n;
    for (int r2 = 0; r2 < n; ++r2) z[r2] += c[i] * vi[r2];
  }
  free(c);
}

/* ------------------------------------------------------------------ */
/* PCG with P = p_k(A) (Section 1, Algorithm 2 as the preconditioner)  */
/* ------------------------------------------------------------------ */
/* Standard PCG from x0: r = b - A x, z = P r, p = z; each iteration
 * q = A p, alpha = (r,z)/(p,q), x += alpha p, r -= alpha q, stop when
 * ||r||/||b|| <= rtol, z = P r, beta = (r,z)_new/(r,z)_old, p = z + beta p.
 * Work per iteration: one product by A plus m inside P, and 3 inner
 * products; the preconditioner is not applied after the last iteration,
 * so products = iter (m + 1) and inner products = 3 iter from x0 = 0
 * (the counts of Table 4).
 * flexible = 1 replaces beta by (z_new, r_new - r_old)/(z_old, r_old)
 * (flexible CG; identical in exact arithmetic for a fixed SPD P). */
typedef struct {
  int m;
  double theta_bar, delta, sigma_bar;
  const double* rho;
  lowrank_t lr; /* lr.p = 0: no spectral correction */
} cheb_t;

/* z = P r with P = p_m(A) (+ V G^{-1} V^T, Section 3.1); the p inner
 * products of the correction are counted in dots. */
static int prec_apply(const op_t* A, const cheb_t* P, const double* r, double* z,
                      long long* mvp, long long* dots) {
  int rc = cheb_apply_op(A, P->m, P->theta_bar, P->delta, P->sigma_bar, P->rho, r, z, mvp);
  if (rc || P->lr.p == 0) return rc;
  lowrank_add(A->n, &P->lr, r, z);
  *dots += P->lr.p;
  return all_finite(A->n, z) ? 0 : -3;
}

/* Truncated flexible CG, FCG(m) (Notay 2000), for m >= 2: from x0,
 * r = b - A x, z = M r, p_0 = z; each iteration q_i = A p_i,
 * alpha = (r, p_i)/(p_i, q_i), x += alpha p_i, r -= alpha q_i, stop when
 * ||r||/||b|| <= rtol, z = M r, and the next direction is z made
 * A-orthogonal to the last m directions:
 *   p_{i+1} = z - sum_{j = max(0, i-m+1)}^{i} (z, q_j)/(p_j, q_j) p_j.
 * M may be any operator (a variable or nonsymmetric preconditioner too).
 * Inner products per iteration: (p, q), (r, r), m of (z, q_j) (fewer in the
 * first m - 1 iterations) and (r, p); counted in dots.  dirs (may be NULL)
 * receives the directions p_0, p_1, ... (n each, at most maxit + 1). */
static int fcgm_core(const op_t* A, const op_t* M, const double* b, double* x, int m, int maxit,
                     double rtol, oracle_stats* st, double* dirs, long long* mvp_out,
                     long long* dots_out) {
  int n = A->n;
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* z = (double*)malloc(sizeof(double) * (size_t)n);
  double* P = (double*)calloc((size_t)n * m, sizeof(double));
  double* Q = (double*)calloc((size_t)n * m, sizeof(double));
  double* pq = (double*)calloc((size_t)m, sizeof(double));
  double* pn = (double*)malloc(sizeof(double) * (size_t)n);
  long long mvp = 0, dots = 0;
  int rc = 0, it = 0;
  double bnorm = sqrt(dot(n, b, b));
  int x_zero = 1;
  for (int i = 0; i < n; ++i)
    if (x[i] != 0.0) { x_zero = 0; break; }
  if (x_zero) {
    memcpy(r, b, sizeof(double) * (size_t)n);
  } else {
    A->apply(A->ctx, x, r);
    ++mvp;
    for (int i = 0; i < n; ++i) r[i] = b[i] - r[i];
  }
  double rel = (bnorm > 0.0) ? sqrt(dot(n, r, r)) / bnorm : 0.0;
  if (bnorm == 0.0 || rel <= rtol) goto done;
  M->apply(M->ctx, r, z);
  memcpy(P, z, sizeof(double) * (size_t)n); /* p_0 in slot 0 */
  if (dirs) memcpy(dirs, z, sizeof(double) * (size_t)n);
  double rp = dot(n, r, P);
  ++dots;
  rc = 1;
  while (it < maxit) {
    int s = it % m;
    double* p = P + (size_t)s * n;
    double* q = Q + (size_t)s * n;
    A->apply(A->ctx, p, q);
    ++mvp;
    pq[s] = dot(n, p, q);
    ++dots;
    if (!(pq[s] > 0.0)) { rc = isfinite(pq[s]) ? -2 : -3; break; }
    double alpha = rp / pq[s];
    for (int i = 0; i < n; ++i) x[i] += alpha * p[i];
    for (int i = 0; i < n; ++i) r[i] -= alpha * q[i];
    ++it;
    double rr = dot(n, r, r);
    ++dots;
    if (!isfinite(rr)) { rc = -3; break; }
    rel = sqrt(rr) / bnorm;
    if (rel <= rtol) { rc = 0; break; }
    M->apply(M->ctx, r, z);
    memcpy(pn, z, sizeof(double) * (size_t)n);
    int nv = it < m ? it : m; /* directions p_{it-nv} .. p_{it-1} */
    for (int t = 0; t < nv; ++t) {
      int sj = (s - t + m) % m;
      double beta = -dot(n, z, Q + (size_t)sj * n) / pq[sj];
      ++dots;
      for (int i = 0; i < n; ++i) pn[i] += beta * P[(size_t)sj * n + i];
    }
    int s_new = it % m;
    memcpy(P + (size_t)s_new * n, pn, sizeof(double) * (size_t)n);
    if (dirs) memcpy(dirs + (size_t)it * n, pn, sizeof(double) * (size_t)n);
    rp = dot(n, r, pn);
    ++dots;
    if (!isfinite(rp)) { rc = -3; break; }
    rc = 1;
  }
done:
  if (st) {
    st->iterations = it;
    st->rel_res = rel;
    st->status = rc;
  }
  if (mvp_out) *mvp_out = mvp;
  if (dots_out) *dots_out = dots;
  free(r);
  free(z);
  free(P);
  free(Q);
  free(pq);
  free(pn);
  return rc;
}

/* The solve's preconditioner as an operator (for FCG(m)); counts work. */
typedef struct {
  const op_t* A;
  const cheb_t* P;
  long long mvp, dots;
} precond_op_t;

static void precond_op_apply(const void* c, const double* x, double* y) {
  precond_op_t* pc = (precond_op_t*)c;
  prec_apply(pc->A, pc->P, x, y, &pc->mvp, &pc->dots);
}

typedef struct {
  int n;
  const double* D; /* row-major n x n */
} dense_t;

static void dense_apply(const void* c, const double* x, double* y) {
  const dense_t* d = (const dense_t*)c;
  for (int i = 0; i < d->n; ++i) {
    double s = 0.0;
    for (int j = 0; j < d->n; ++j) s += d->D[(size_t)i * d->n + j] * x[j];
    y[i] = s;
  }
}

int oracle_fcg_dense(int n, const double* A, const double* M, const double* b, double* x, int m,
                     int maxit, double rtol, double* dirs, oracle_stats* st) {
  if (n <= 0 || m < 2 || maxit < 0) return -1;
  dense_t da = {n, A}, dm = {n, M};
  op_t opA = {dense_apply, &da, n}, opM = {dense_apply, &dm, n};
  long long mvp = 0, dots = 0;
  int rc = fcgm_core(&opA, &opM, b, x, m, maxit, rtol, st, dirs, &mvp, &dots);
  if (st) {
    st->mvp = mvp;
    st->dots = dots;
  }
  return rc;
}

static int pcg_op(const op_t* A, const cheb_t* P, const double* b, double* x, int flexible,
                  int maxit, double rtol, oracle_stats* st) {
  if (flexible >= 2) {
    precond_op_t pc = {A, P, 0, 0};
    op_t M = {precond_op_apply, &pc, A->n};
    long long mvp = 0, dots = 0;
    int rc2 = fcgm_core(A, &M, b, x, flexible, maxit, rtol, st, NULL, &mvp, &dots);
    if (st) {
      st->mvp = mvp + pc.mvp;
      st->dots = dots + pc.dots;
    }
    return rc2;
  }
  int n = A->n;
  double* r = (double*)malloc(sizeof(double) * (size_t)n);
  double* z = (double*)malloc(sizeof(double) * (size_t)n);
  double* p = (double*)malloc(sizeof(double) * (size_t)n);
  double* q = (double*)malloc(sizeof(double) * (size_t)n);
  double* r_old = flexible ? (double*)malloc(sizeof(double) * (size_t)n) : NULL;
  long long mvp = 0, dots = 0;
  int rc = 0, it = 0;
  double bnorm = sqrt(dot(n, b, b));
  int x_zero = 1;
  for (int i = 0; i < n; ++i)
    if (x[i] != 0.0) { x_zero = 0; break; }
  if (x_zero) {
    memcpy(r, b, sizeof(double) * (size_t)n);
  } else {
    A->apply(A->ctx, x, q);
    ++mvp;
    for (int i = 0; i < n; ++i) r[i] = b[i] - q[i];
  }
  double rel = (bnorm > 0.0) ? sqrt(dot(n, r, r)) / bnorm : 0.0;
  if (bnorm == 0.0 || rel <= rtol) goto done;
  rc = prec_apply(A, P, r, z, &mvp, &dots);
  if (rc) goto done;
  memcpy(p, z, sizeof(double) * (size_t)n);
  double rz = dot(n, r, z);
  ++dots;
  if (!(rz > 0.0)) { rc = isfinite(rz) ? -2 : -3; goto done; }
  rc = 1;
  while (it < maxit) {
    A->apply(A->ctx, p, q);
    ++mvp;
    double pq = dot(n, p, q);
    ++dots;
    if (!(pq > 0.0)) { rc = isfinite(pq) ? -2 : -3; break; }
    double alpha = rz / pq;
    if (flexible) memcpy(r_old, r, sizeof(double) * (size_t)n);
    for (int i = 0; i < n; ++i) x[i] += alpha * p[i];
    for (int i = 0; i < n; ++i) r[i] -= alpha * q[i];
    ++it;
    double rr = dot(n, r, r);
    ++dots;
    if (!isfinite(rr)) { rc = -3; break; }
    rel = sqrt(rr) / bnorm;
    if (rel <= rtol) { rc = 0; break; }
    rc = prec_apply(A, P, r, z, &mvp, &dots);
    if (rc) break;
    rc = 1;
    double rz_new = dot(n, r, z);
    ++dots;
    double beta;
    if (flexible) {
      double zr_old = dot(n, z, r_old);
      beta = (rz_new - zr_old) / rz;
    } else {
      beta = rz_new / rz;
    }
    if (!(rz_new > 0.0)) { rc = isfinite(rz_new) ? -2 : -3; break; }
    rz = rz_new;
    for (int i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
  }
done:
  if (st) {
    st->iterations = it;
    st->mvp = mvp;
    st->dots = dots;
    st->rel_res = rel;
    st->status = rc;
  }
  free(r);
  free(z);
  free(p);
  free(q);
  free(r_old);
  return rc;
}

static double auto_xi(double a, double b) {
  double xi = 10.0 * a / b;
  if (xi < 1e-6) xi = 1e-6;
  if (xi > 1e-2) xi = 1e-2;
  return xi;
}

/* The interval [alpha, beta]: given, or the extreme Ritz values of
 * lanczos_steps plain Lanczos steps from v0. */
static int pick_interval(const op_t* A, const double* v0, const oracle_options* opt,
                         double* alpha, double* beta) {
  if (opt->interval == 1) {
    *alpha = opt->alpha;
    *beta = opt->beta;
    return 0;
  }
  int m = opt->lanczos_steps > 0 ? opt->lanczos_steps : 10;
  double* a = (double*)calloc((size_t)m, sizeof(double));
  double* b = (double*)calloc((size_t)m, sizeof(double));
  int steps = lanczos_op(A, v0, m, a, b);
  int rc = steps > 0 ? oracle_tridiag_extremes(steps, a, b, alpha, beta) : -1;
  free(a);
  free(b);
  return rc;
}

/* The preconditioned operator B = p_k(A) A used to find the leftmost
 * eigenvectors: a polynomial in A, so it has the eigenvectors of A, and
 * with the xi-shifted polynomial the smallest eigenvalues of A go to the
 * smallest of B (Theorem 2.3) while kappa(B) is far below kappa(A). */
typedef struct {
  const op_t* A;
  const cheb_t* P;
  double* t;
} precop_t;

static void precop_apply(const void* c, const double* x, double* y) {
  const precop_t* pc = (const precop_t*)c;
  pc->A->apply(pc->A->ctx, x, pc->t);
  cheb_apply_op(pc->A, pc->P->m, pc->P->theta_bar, pc->P->delta, pc->P->sigma_bar, pc->P->rho, pc->t, y,
                NULL);
}

/* Section 3.1 vectors: the Ritz vectors of the p smallest Ritz values of m
 * Lanczos steps (full reorthogonalisation, from v0) on B = p_k(A) A, and
 * their Rayleigh quotients theta_i = v_i^T A v_i (unit vectors). */
static int lowrank_vectors_op(const op_t* A, const cheb_t* P, const double* v0, int p, int m,
                              double* V, double* theta) {
  int n = A->n;
  precop_t pc = {A, P, (double*)malloc(sizeof(double) * (size_t)n)};
  op_t B = {precop_apply, &pc, n};
  double* a = (double*)calloc((size_t)m, sizeof(double));
  double* b = (double*)calloc((size_t)m, sizeof(double));
  double* Q = (double*)calloc((size_t)n * m, sizeof(double));
  int steps = lanczos_basis_op(&B, v0, m, a, b, Q);
  int rc = steps >= p ? ritz_vectors(n, steps, a, b, Q, p, V, NULL) : -1;
  if (rc == 0 && theta) {
    for (int i = 0; i < p; ++i) {
      A->apply(A->ctx, V + (size_t)i * n, pc.t);
      theta[i] = dot(n, V + (size_t)i * n, pc.t);
    }
  }
  free(pc.t);
  free(a);
  free(b);
  free(Q);
  return rc;
}

int oracle_lowrank_vectors(int n, const int* rowptr, const int* col, const double* val,
                           const double* v0, double alpha, double beta, double xi, int k, int p,
                           int m, double* V, double* theta) {
  if (p <= 0 || m < p) return -1;
  double* rho = (double*)malloc(sizeof(double) * (size_t)(k + 1));
  cheb_t P;
  P.m = k;
  P.rho = rho;
  P.lr.p = 0;
  int rc = oracle_cheb_coeffs(alpha, beta, xi, k, &P.theta_bar, &P.delta, &P.sigma_bar, rho);
  if (rc == 0) {
    csr_t c = {n, rowptr, col, val};
    op_t op = {csr_apply, &c, n};
    rc = lowrank_vectors_op(&op, &P, v0, p, m, V, theta);
  }
  free(rho);
  return rc;
}

/* Everything the solve needs before its first iteration: the interval, xi,
 * the coefficients and, for opt->lowrank = p > 0, the Section 3.1
 * correction with V = opt->lr_V or the vectors of lowrank_vectors_op
 * (lowrank_steps steps).  The interval is not changed by the correction:
 * as in Section 3.1 the polynomial keeps its lower end and the correction
 * lifts the images of the leftmost eigenvalues.  *Vown receives memory to
 * free. */
static int setup_prec(const op_t* A, const double* v0, const oracle_options* opt, cheb_t* P,
                      double* rho, double* alpha, double* beta, double* xi, double** Vown) {
  *Vown = NULL;
  P->m = opt->k;
  P->rho = rho;
  P->lr.p = 0;
  P->lr.V = NULL;
  P->lr.L = NULL;
  int rc = pick_interval(A, v0, opt, alpha, beta);
  if (rc) return rc;
  *xi = opt->xi >= 0.0 ? opt->xi : auto_xi(*alpha, *beta);
  rc = oracle_cheb_coeffs(*alpha, *beta, *xi, opt->k, &P->theta_bar, &P->delta, &P->sigma_bar, rho);
  if (rc || opt->lowrank <= 0) return rc;
  int p = opt->lowrank;
  const double* V = opt->lr_V;
  if (V == NULL) {
    int n = A->n;
    int m = opt->lowrank_steps > 0 ? opt->lowrank_steps : 30;
    double* theta = (double*)malloc(sizeof(double) * (size_t)p);
    *Vown = (double*)malloc(sizeof(double) * (size_t)n * p);
    rc = lowrank_vectors_op(A, P, v0, p, m, *Vown, theta);
    V = *Vown;
    free(theta);
    if (rc) return rc;
  }
  return lowrank_setup(A, p, V, &P->lr);
}

int oracle_pcg_csr(int n, const int* rowptr, const int* col, const double* val,
                   const double* b, double* x, const double* v0, const oracle_options* opt,
                   oracle_stats* st) {
  if (n <= 0 || opt->k < 0) return -1;
  int nnz = rowptr[n];
  double* vh = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  double* w = (double*)malloc(sizeof(double) * (size_t)n);
  double* bh = (double*)malloc(sizeof(double) * (size_t)n);
  double* xh = (double*)malloc(sizeof(double) * (size_t)n);
  double* rho = (double*)malloc(sizeof(double) * (size_t)(opt->k + 1));
  int rc = 0;
  if (opt->seed_scaling == 1) {
    rc = oracle_jacobi_scale(n, rowptr, col, val, vh, w);
  } else {
    memcpy(vh, val, sizeof(double) * (size_t)nnz);
    for (int i = 0; i < n; ++i) w[i] = 1.0;
  }
  if (rc == 0) {
    csr_t ah = {n, rowptr, col, vh};
    op_t A = {csr_apply, &ah, n};
    /* A_hat x_hat = b_hat with b_hat = W b, x = W x_hat */
    for (int i = 0; i < n; ++i) bh[i] = w[i] * b[i];
    for (int i = 0; i < n; ++i) xh[i] = x[i] / w[i];
    double alpha = 0.0, beta = 0.0, xi = 0.0;
    double* Vown = NULL;
    cheb_t P;
    rc = setup_prec(&A, v0, opt, &P, rho, &alpha, &beta, &xi, &Vown);
    if (rc == 0) {
      rc = pcg_op(&A, &P, bh, xh, opt->flexible, opt->maxit, opt->rtol, st);
      if (st) {
        st->alpha_hat = alpha;
        st->beta_hat = beta;
        st->xi = xi;
      }
      for (int i = 0; i < n; ++i) x[i] = w[i] * xh[i];
      if (st) {
        double* t = (double*)malloc(sizeof(double) * (size_t)n);
        oracle_spmv(n, rowptr, col, val, x, t);
        double num = 0.0;
        for (int i = 0; i < n; ++i) num += (b[i] - t[i]) * (b[i] - t[i]);
        double bn = sqrt(dot(n, b, b));
        st->true_rel_res = bn > 0.0 ? sqrt(num) / bn : 0.0;
        free(t);
      }
    }
    free(P.lr.L);
    free(Vown);
  }
  if (st) st->status = rc;
  free(vh);
  free(w);
  free(bh);
  free(xh);
  free(rho);
  return rc;
}

/* ------------------------------------------------------------------ */
/* Section 4.2: the DFN Schur complement                               */
/* ------------------------------------------------------------------ */
/* A is block diagonal (one SPD block per fracture).  As in the paper, its
 * exact Cholesky factor L_A (block diagonal, fill confined to the band of
 * each block) is computed once; A^{-1} v = L_A^{-T} L_A^{-1} v. */

struct oracle_schur {
  oracle_dfn d;
  int* bw;          /* per-fracture half bandwidth          */
  long long* boff;  /* offset of each block's band storage  */
  double* L;        /* band storage: L[boff + i*(bw+1) + (i-j)] */
};

oracle_schur* oracle_schur_create(const oracle_dfn* d) {
  oracle_schur* s = (oracle_schur*)calloc(1, sizeof(oracle_schur));
  s->d = *d;
  int nf = d->n_f;
  s->bw = (int*)calloc((size_t)nf, sizeof(int));
  s->boff = (long long*)calloc((size_t)nf + 1, sizeof(long long));
  for (int f = 0; f < nf; ++f) {
    long long o = d->offset[f], e = d->offset[f + 1];
    int bw = 0;
    for (long long i = o; i < e; ++i)
      for (int p = d->A_rowptr[i]; p < d->A_rowptr[i + 1]; ++p) {
        long long j = d->A_col[p];
        int dist = (int)(i > j ? i - j : j - i);
        if (dist > bw) bw = dist;
      }
    s->bw[f] = bw;
    s->boff[f + 1] = s->boff[f] + (e - o) * (long long)(bw + 1);
  }
  s->L = (double*)calloc((size_t)s->boff[nf], sizeof(double));
  for (int f = 0; f < nf; ++f) {
    long long o = d->offset[f];
    int nloc = (int)(d->offset[f + 1] - o), bw = s->bw[f];
    double* L = s->L + s->boff[f];
#define LB(i, j) L[(long long)(i) * (bw + 1) + ((i) - (j))]
    /* copy the lower band of the block */
    for (int i = 0; i < nloc; ++i)
      for (int p = d->A_rowptr[o + i]; p < d->A_rowptr[o + i + 1]; ++p) {
        int j = (int)(d->A_col[p] - o);
        if (j <= i) LB(i, j) = d->A_val[p];
      }
    /* banded Cholesky, column by column */
    for (int j = 0; j < nloc; ++j) {
      int k0 = j - bw > 0 ? j - bw : 0;
      double sj = LB(j, j);
      for (int k = k0; k < j; ++k) sj -= LB(j, k) * LB(j, k);
      if (!(sj > 0.0)) {
        oracle_schur_free(s);
        return NULL;
      }
      double ljj = sqrt(sj);
      LB(j, j) = ljj;
      int iend = j + bw < nloc - 1 ? j + bw : nloc - 1;
      for (int i = j + 1; i <= iend; ++i) {
        int kk = i - bw > 0 ? i - bw : 0;
        double sij = LB(i, j);
        for (int k = kk; k < j; ++k) sij -= LB(i, k) * LB(j, k);
        LB(i, j) = sij / ljj;
      }
    }
#undef LB
  }
  return s;
}

void oracle_schur_free(oracle_schur* s) {
  if (!s) return;
  free(s->bw);
  free(s->boff);
  free(s->L);
  free(s);
}

/* y = A_f^{-1} v on one block: forward (L u = v) then backward (L^T y = u). */
static void block_solve(const oracle_schur* s, int f, const double* v, double* y) {
  long long o = s->d.offset[f];
  int nloc = (int)(s->d.offset[f + 1] - o), bw = s->bw[f];
  const double* L = s->L + s->boff[f];
#define LB(i, j) L[(long long)(i) * (bw + 1) + ((i) - (j))]
  for (int i = 0; i < nloc; ++i) {
    double t = v[o + i];
    int k0 = i - bw > 0 ? i - bw : 0;
    for (int k = k0; k < i; ++k) t -= LB(i, k) * y[o + k];
    y[o + i] = t / LB(i, i);
  }
  for (int i = nloc - 1; i >= 0; --i) {
    double t = y[o + i];
    int k1 = i + bw < nloc - 1 ? i + bw : nloc - 1;
    for (int k = i + 1; k <= k1; ++k) t -= LB(k, i) * y[o + k];
    y[o + i] = t / LB(i, i);
  }
#undef LB
}

int oracle_ainv(const oracle_schur* s, const double* v, double* y) {
  for (int f = 0; f < s->d.n_f; ++f) block_solve(s, f, v, y);
  return 0;
}

static void rect_spmv(int nrows, const int* rp, const int* ci, const double* va, const double* x,
                      double* y) {
  for (int i = 0; i < nrows; ++i) {
    double acc = 0.0;
    for (int p = rp[i]; p < rp[i + 1]; ++p) acc += va[p] * x[ci[p]];
    y[i] = acc;
  }
}

/* Algorithm 3, y = S_u r, with the regularisation parameter alpha kept in
 * the products by B^T and C^T as in the expansion
 * S_u = G^u - alpha B^T A^{-1} C - alpha C^T A^{-1} B + C^T A^{-1} G^h A^{-1} C
 * (alpha = 1 gives the algorithm as printed). */
int oracle_schur_apply(const oracle_schur* s, const double* r, double* y) {
  const oracle_dfn* d = &s->d;
  int nh = d->n_h, nu = d->n_u;
  double* v = (double*)calloc((size_t)nh, sizeof(double));
  double* z = (double*)calloc((size_t)nh, sizeof(double));
  double* t = (double*)calloc((size_t)nh, sizeof(double));
  double* w = (double*)calloc((size_t)nh, sizeof(double));
  double* zu = (double*)calloc((size_t)nu, sizeof(double));
  double* tmp = (double*)calloc((size_t)nu, sizeof(double));
  rect_spmv(nh, d->C_rowptr, d->C_col, d->C_val, r, v);           /* v = C r            */
  rect_spmv(nh, d->B_rowptr, d->B_col, d->B_val, r, z);           /* z = B r            */
  oracle_ainv(s, v, t);                                            /* t = A^{-1} v       */
  oracle_ainv(s, z, w);                                            /* w = A^{-1} z       */
  rect_spmv(nu, d->Gu_rowptr, d->Gu_col, d->Gu_val, r, zu);       /* z = G^u r          */
  rect_spmv(nu, d->BT_rowptr, d->BT_col, d->BT_val, t, tmp);      /*   - alpha B^T t    */
  for (int i = 0; i < nu; ++i) zu[i] -= d->alpha_reg * tmp[i];
  rect_spmv(nu, d->CT_rowptr, d->CT_col, d->CT_val, w, tmp);      /*   - alpha C^T w    */
  for (int i = 0; i < nu; ++i) zu[i] -= d->alpha_reg * tmp[i];
  rect_spmv(nh, d->Gh_rowptr, d->Gh_col, d->Gh_val, t, v);        /* v = G^h t          */
  oracle_ainv(s, v, w);                                            /* w = A^{-1} v       */
  rect_spmv(nu, d->CT_rowptr, d->CT_col, d->CT_val, w, tmp);      /* y = z + C^T w      */
  for (int i = 0; i < nu; ++i) y[i] = zu[i] + tmp[i];
  free(v);
  free(z);
  free(t);
  free(w);
  free(zu);
  free(tmp);
  return all_finite(nu, y) ? 0 : -3;
}

/* Algorithm 4: Z = A^{-1} C, T = G^h Z - 2 alpha B, (D_S)_i = G^u_ii + z_i^T t_i.
 * Column i of C touches one fracture, and A^{-1} is block diagonal, so z_i
 * is obtained by solving that fracture's block only; z_i^T t_i then only
 * involves the rows of that block. */
int oracle_schur_diag(const oracle_schur* s, double* ds) {
  const oracle_dfn* d = &s->d;
  int nh = d->n_h, nu = d->n_u;
  /* column access to C and B through their transposes CT, BT */
  double* c = (double*)calloc((size_t)nh, sizeof(double));
  double* zc = (double*)calloc((size_t)nh, sizeof(double));
  double* ghz = (double*)calloc((size_t)nh, sizeof(double));
  double* bcol = (double*)calloc((size_t)nh, sizeof(double));
  for (int i = 0; i < nu; ++i) {
    int f = -1;
    for (int p = d->CT_rowptr[i]; p < d->CT_rowptr[i + 1]; ++p) {
      long long row = d->CT_col[p];
      c[row] = d->CT_val[p];
      int ff = 0;
      while (d->offset[ff + 1] <= row) ++ff;
      if (f >= 0 && ff != f) return -1; /* C must be fracture-local */
      f = ff;
    }
    double gii = 0.0;
    for (int p = d->Gu_rowptr[i]; p < d->Gu_rowptr[i + 1]; ++p)
      if (d->Gu_col[p] == i) gii += d->Gu_val[p];
    double acc = 0.0;
    if (f >= 0) {
      long long o = d->offset[f], e = d->offset[f + 1];
      block_solve(s, f, c, zc);
      for (long long row = o; row < e; ++row) {
        double g = 0.0;
        for (int p = d->Gh_rowptr[row]; p < d->Gh_rowptr[row + 1]; ++p) g += d->Gh_val[p] * zc[d->Gh_col[p]];
        ghz[row] = g;
      }
      for (int p = d->BT_rowptr[i]; p < d->BT_rowptr[i + 1]; ++p) bcol[d->BT_col[p]] += d->BT_val[p];
      for (long long row = o; row < e; ++row) acc += zc[row] * (ghz[row] - 2.0 * d->alpha_reg * bcol[row]);
      for (int p = d->BT_rowptr[i]; p < d->BT_rowptr[i + 1]; ++p) bcol[d->BT_col[p]] = 0.0;
      for (long long row = o; row < e; ++row) zc[row] = 0.0;
    }
    for (int p = d->CT_rowptr[i]; p < d->CT_rowptr[i + 1]; ++p) c[d->CT_col[p]] = 0.0;
    ds[i] = gii + acc;
  }
  free(c);
  free(zc);
  free(ghz);
  free(bcol);
  return all_finite(nu, ds) ? 0 : -3;
}

/* r = W^T M^{-1} f_1 with f_1 = [q; 0] (Eq. schur):
 * M^{-1} f_1 = [A^{-1} q; -A^{-1} G^h A^{-1} q], W^T = [alpha B^T, C^T]. */
int oracle_schur_rhs(const oracle_schur* s, const double* q, double* r) {
  const oracle_dfn* d = &s->d;
  int nh = d->n_h, nu = d->n_u;
  double* a1 = (double*)calloc((size_t)nh, sizeof(double));
  double* g = (double*)calloc((size_t)nh, sizeof(double));
  double* a2 = (double*)calloc((size_t)nh, sizeof(double));
  double* tmp = (double*)calloc((size_t)nu, sizeof(double));
  oracle_ainv(s, q, a1);
  rect_spmv(nh, d->Gh_rowptr, d->Gh_col, d->Gh_val, a1, g);
  oracle_ainv(s, g, a2);
  rect_spmv(nu, d->BT_rowptr, d->BT_col, d->BT_val, a1, r);
  rect_spmv(nu, d->CT_rowptr, d->CT_col, d->CT_val, a2, tmp);
  for (int i = 0; i < nu; ++i) r[i] = d->alpha_reg * r[i] - tmp[i];
  free(a1);
  free(g);
  free(a2);
  free(tmp);
  return all_finite(nu, r) ? 0 : -3;
}

/* h = A^{-1}(q + C u), p = A^{-1}(alpha B u - G^h h) (Section 4.2, with
 * alpha kept as in the first block row of the permuted system). */
int oracle_schur_recover(const oracle_schur* s, const double* q, const double* u, double* h,
                         double* p) {
  const oracle_dfn* d = &s->d;
  int nh = d->n_h;
  double* t = (double*)calloc((size_t)nh, sizeof(double));
  double* g = (double*)calloc((size_t)nh, sizeof(double));
  rect_spmv(nh, d->C_rowptr, d->C_col, d->C_val, u, t);
  for (int i = 0; i < nh; ++i) t[i] += q[i];
  oracle_ainv(s, t, h);
  rect_spmv(nh, d->B_rowptr, d->B_col, d->B_val, u, t);
  rect_spmv(nh, d->Gh_rowptr, d->Gh_col, d->Gh_val, h, g);
  for (int i = 0; i < nh; ++i) t[i] = d->alpha_reg * t[i] - g[i];
  oracle_ainv(s, t, p);
  free(t);
  free(g);
  return 0;
}

/* S_hat = D_S^{-1/2} S_u D_S^{-1/2} (end of Section 4.3) */
typedef struct {
  const oracle_schur* s;
  const double* w; /* D_S^{-1/2} */
  double* tmp;
  double* tmp2;
} schur_scaled_t;

static void schur_scaled_apply(const void* c, const double* x, double* y) {
  const schur_scaled_t* ss = (const schur_scaled_t*)c;
  int nu = ss->s->d.n_u;
  for (int i = 0; i < nu; ++i) ss->tmp[i] = ss->w[i] * x[i];
  oracle_schur_apply(ss->s, ss->tmp, ss->tmp2);
  for (int i = 0; i < nu; ++i) y[i] = ss->w[i] * ss->tmp2[i];
}

int oracle_pcg_schur(const oracle_schur* s, const double* ds, const double* r, double* u,
                     const double* v0, const oracle_options* opt, oracle_stats* st) {
  int nu = s->d.n_u;
  double* w = (double*)malloc(sizeof(double) * (size_t)nu);
  double* rh = (double*)malloc(sizeof(double) * (size_t)nu);
  double* uh = (double*)malloc(sizeof(double) * (size_t)nu);
  double* rho = (double*)malloc(sizeof(double) * (size_t)(opt->k + 1));
  schur_scaled_t ss = {s, w, (double*)malloc(sizeof(double) * (size_t)nu),
                       (double*)malloc(sizeof(double) * (size_t)nu)};
  int rc = 0;
  for (int i = 0; i < nu; ++i) {
    if (!(ds[i] > 0.0)) rc = -2;
    w[i] = 1.0 / sqrt(ds[i]);
  }
  if (rc == 0) {
    op_t A = {schur_scaled_apply, &ss, nu};
    for (int i = 0; i < nu; ++i) rh[i] = w[i] * r[i];
    for (int i = 0; i < nu; ++i) uh[i] = u[i] / w[i];
    double alpha = 0.0, beta = 0.0, xi = 0.0;
    double* Vown = NULL;
    cheb_t P;
    rc = setup_prec(&A, v0, opt, &P, rho, &alpha, &beta, &xi, &Vown);
    if (rc == 0) {
      rc = pcg_op(&A, &P, rh, uh, opt->flexible, opt->maxit, opt->rtol, st);
      if (st) {
        st->alpha_hat = alpha;
        st->beta_hat = beta;
        st->xi = xi;
      }
      for (int i = 0; i < nu; ++i) u[i] = w[i] * uh[i];
      if (st) {
        double* t = (double*)malloc(sizeof(double) * (size_t)nu);
        oracle_schur_apply(s, u, t);
        double num = 0.0, bn = 0.0;
        for (int i = 0; i < nu; ++i) {
          num += (r[i] - t[i]) * (r[i] - t[i]);
          bn += r[i] * r[i];
        }
        st->true_rel_res = bn > 0.0 ? sqrt(num / bn) : 0.0;
        free(t);
      }
    }
    free(P.lr.L);
    free(Vown);
  }
  if (st) st->status = rc;
  free(w);
  free(rh);
  free(uh);
  free(rho);
  free(ss.tmp);
  free(ss.tmp2);
  return rc;
}

/* z = p_k(A) r + V (V^T A V)^{-1} V^T r (Section 3.1) for a CSR matrix. */
int oracle_lowrank_apply(int n, const int* rowptr, const int* col, const double* val,
                         double alpha, double beta, double xi, int k, int p, const double* V,
                         const double* r, double* z) {
  if (p < 0) return -1;
  double tb, d, sb;
  double* rho = (double*)malloc(sizeof(double) * (size_t)(k + 1));
  int rc = oracle_cheb_coeffs(alpha, beta, xi, k, &tb, &d, &sb, rho);
  if (rc == 0) {
    csr_t a = {n, rowptr, col, val};
    op_t op = {csr_apply, &a, n};
    cheb_t P;
    P.m = k;
    P.theta_bar = tb;
    P.delta = d;
    P.sigma_bar = sb;
    P.rho = rho;
    rc = lowrank_setup(&op, p, V, &P.lr);
    long long mvp = 0, dots = 0;
    if (rc == 0) rc = prec_apply(&op, &P, r, z, &mvp, &dots);
    free(P.lr.L);
  }
  free(rho);
  return rc;
}
