/*
 * Plain FP64 CPU oracle for the polynomial-preconditioned CG method of
 * Bergamaschi, Ferronato, Isotton, Janna & Martinez (arXiv 2208.01339).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load or call this library.
 * It shares no code with the CUDA path (paper_2208_01339_gb300/csrc):
 * no kernels, headers, helpers or coefficient generators.
 *
 * Every routine is a direct, unblocked restatement of the paper's
 * definitions and algorithms, in the paper's order and notation:
 *   oracle_cheb_coeffs     Section 2.2 (theta, delta, sigma), Eq. thetamod
 *                          (xi-modified theta), Eq. rhocheb (rho_k)
 *   oracle_cheb_poly       Eq. polycheb, scalar p_k(x)
 *   oracle_cheb_apply      Algorithm 2 (ChebAlg), r_hat = P_m r
 *   oracle_newton_apply    Algorithm 1 (NewtAlg) with Eq. zetaNewt, Eq. newrec0
 *   oracle_spmv            y = A x (CSR)
 *   oracle_jacobi_scale    Section 3: A_hat = W^T A W with W = diag(A)^{-1/2}
 *   oracle_lanczos         plain Lanczos tridiagonalisation (the interval
 *                          estimator used instead of the paper's DACG)
 *   oracle_tridiag_extremes  Sturm-sequence bisection on T_m
 *   oracle_lanczos_basis   Lanczos keeping its (fully reorthogonalised) basis
 *   oracle_tridiag_eig     eigenpair of T_m: bisection + inverse iteration
 *   oracle_lowrank_vectors leftmost eigenvectors by Lanczos on p_k(A) A
 *   oracle_lowrank_apply   Section 3.1: P = P_0 + V (V^T A V)^{-1} V^T
 *   oracle_pcg_csr         PCG (Section 1) with P = W p_k(A_hat) W^T, or
 *                          flexible CG, FCG(1) or truncated FCG(m)
 *   oracle_fcg_dense       FCG(m) with any dense preconditioner (pins)
 *   oracle_schur_*         Section 4.2: Algorithm 3 (y = S_u r), Algorithm 4
 *                          (D_S = diag S_u), the right-hand side
 *                          r = W^T M^{-1} f_1 and the recovery of h and p,
 *                          with A^{-1} by banded Cholesky per fracture
 *   oracle_pcg_schur       PCG on the D_S-scaled Schur complement
 *
 * Return codes: 0 ok, 1 maxit reached, -1 bad argument, -2 breakdown
 * (non-positive curvature), -3 non-finite value.
 */
#ifndef PP_ORACLE_H
#define PP_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int iterations;
  long long mvp;        /* operator applications (A or S_u)              */
  long long dots;       /* inner products counted as in Table 4          */
  double rel_res;       /* recursive ||r||/||b|| at exit                   */
  double true_rel_res;  /* ||b - A x|| / ||b|| recomputed at exit          */
  double alpha_hat, beta_hat, xi;
  int status;
} oracle_stats;

int oracle_cheb_coeffs(double alpha, double beta, double xi, int k, double* theta_bar,
                       double* delta, double* sigma_bar, double* rho);
double oracle_cheb_poly(double x, double alpha, double beta, double xi, int k);

void oracle_spmv(int n, const int* rowptr, const int* col, const double* val, const double* x,
                 double* y);
int oracle_cheb_apply(int n, const int* rowptr, const int* col, const double* val, double alpha,
                      double beta, double xi, int k, const double* r, double* z);
int oracle_newton_apply(int n, const int* rowptr, const int* col, const double* val,
                        double alpha, double beta, double xi, int nlev, const double* r,
                        double* z);
int oracle_jacobi_scale(int n, const int* rowptr, const int* col, const double* val,
                        double* val_hat, double* w);
int oracle_lanczos(int n, const int* rowptr, const int* col, const double* val,
                   const double* v0, int m, double* a, double* b);
int oracle_tridiag_extremes(int m, const double* a, const double* b, double* lmin,
                            double* lmax);

/* Section 3.1: Lanczos keeping its basis Q (n x m, full reorthogonalisation;
 * b[m-1] = beta_m), the i-th smallest eigenpair of T_m, and the corrected
 * preconditioner z = p_k(A) r + V (V^T A V)^{-1} V^T r (V: n x p, column i
 * at V + i n). */
int oracle_lanczos_basis(int n, const int* rowptr, const int* col, const double* val,
                         const double* v0, int m, double* a, double* b, double* Q);
int oracle_tridiag_eig(int m, const double* a, const double* b, int i, double* lambda,
                       double* y);
int oracle_lowrank_vectors(int n, const int* rowptr, const int* col, const double* val,
                           const double* v0, double alpha, double beta, double xi, int k, int p,
                           int m, double* V, double* theta);
int oracle_lowrank_apply(int n, const int* rowptr, const int* col, const double* val,
                         double alpha, double beta, double xi, int k, int p, const double* V,
                         const double* r, double* z);

/* Options of the full solve.  interval: 0 = Lanczos on A_hat from v0,
 * 1 = given (alpha, beta).  xi < 0 selects xi = clip(10 alpha/beta, 1e-6, 1e-2).
 * seed_scaling: 0 none, 1 Jacobi.  flexible: 0 plain PCG, 1 flexible CG
 * (FCG(1)), m >= 2 truncated flexible CG FCG(m) (A-orthogonal to the last
 * m directions; alpha = (r, p)/(p, A p)).
 * lowrank = p > 0 adds the Section 3.1 correction V (V^T A_hat V)^{-1} V^T
 * with V = lr_V (n x p, seed-scaled space) or, when lr_V is NULL, the Ritz
 * vectors of the p smallest Ritz values of lowrank_steps (0: 30) Lanczos
 * steps with full reorthogonalisation from v0 on p_k(A_hat) A_hat; the
 * interval is not changed by the correction. */
typedef struct {
  int k;
  double xi;
  int interval;
  double alpha, beta;
  int lanczos_steps;
  int seed_scaling;
  int flexible;
  int maxit;
  double rtol;
  int lowrank;
  int lowrank_steps;
  const double* lr_V;
} oracle_options;

/* FCG(m), m >= 2, on dense row-major A (n x n) with the dense operator M as
 * the (possibly nonsymmetric) preconditioner; dirs (may be NULL, n x
 * (maxit + 1)) receives the search directions. */
int oracle_fcg_dense(int n, const double* A, const double* M, const double* b, double* x, int m,
                     int maxit, double rtol, double* dirs, oracle_stats* st);

int oracle_pcg_csr(int n, const int* rowptr, const int* col, const double* val,
                   const double* b, double* x, const double* v0, const oracle_options* opt,
                   oracle_stats* st);

/* Fracture network: A is given as the global block-diagonal CSR plus the
 * fracture offsets; the other blocks are CSR (C, B: n_h x n_u; CT, BT:
 * n_u x n_h; Gh: n_h x n_h; Gu: n_u x n_u). */
typedef struct {
  int n_f, n_h, n_u;
  const long long* offset; /* n_f + 1 */
  const int *A_rowptr, *A_col; const double* A_val;
  const int *C_rowptr, *C_col; const double* C_val;
  const int *B_rowptr, *B_col; const double* B_val;
  const int *CT_rowptr, *CT_col; const double* CT_val;
  const int *BT_rowptr, *BT_col; const double* BT_val;
  const int *Gh_rowptr, *Gh_col; const double* Gh_val;
  const int *Gu_rowptr, *Gu_col; const double* Gu_val;
  double alpha_reg;
} oracle_dfn;

typedef struct oracle_schur oracle_schur;
oracle_schur* oracle_schur_create(const oracle_dfn* d);
void oracle_schur_free(oracle_schur* s);
int oracle_ainv(const oracle_schur* s, const double* v, double* y);
int oracle_schur_apply(const oracle_schur* s, const double* r, double* y);
int oracle_schur_diag(const oracle_schur* s, double* ds);
int oracle_schur_rhs(const oracle_schur* s, const double* q, double* r);
int oracle_schur_recover(const oracle_schur* s, const double* q, const double* u, double* h,
                         double* p);
int oracle_pcg_schur(const oracle_schur* s, const double* ds, const double* r, double* u,
                     const double* v0, const oracle_options* opt, oracle_stats* st);

#ifdef __cplusplus
}
#endif
#endif
