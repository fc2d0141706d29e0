/*
 * polyprec -- GB300 (sm_103a) polynomial-preconditioned Conjugate Gradient.
 *
 * C ABI of libpolyprec.so.  Method: Bergamaschi, Ferronato, Isotton, Janna &
 * Martinez, "Parallel matrix-free polynomial preconditioners with application
 * to flow simulations in discrete fracture networks" (arXiv 2208.01339).
 *
 * The library solves A x = b, A sparse SPD (Section 1), by PCG with the
 * preconditioner P = W p_k(W^T A W) W^T (Section 3), where W is the seed
 * preconditioner (identity or diag(A)^{-1/2}) and p_k is the xi-modified
 * Chebyshev polynomial of degree k (Section 2.2, Eq. polycheb, Eq. rhocheb,
 * Eq. thetamod) applied by the three-term recurrence of Algorithm 2.  The
 * same solver runs on the matrix-free Schur complement S_u of the fracture-
 * network system (Section 4.2, Eq. schur, Algorithm 3) with the diagonal
 * seed D_S = diag(S_u) of Algorithm 4.
 *
 * Conventions shared by every entry point
 *  - Device pointers are CUDA device addresses owned by the caller; the
 *    library never allocates device memory.  Scratch memory comes from one
 *    caller-allocated workspace of the size the *_workspace_size query
 *    returns; it must stay allocated, untouched, until pp_destroy().
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is ordered on that stream.  Calls on one context must
 *    not overlap (they share the workspace).
 *  - Host pointers are marked "host".  Vectors are dense FP64 with unit
 *    stride; a block of nrhs vectors is column-major (vector j starts at
 *    j*n).
 *  - Every call returns a status (PP_OK = 0).  After a failure the message
 *    is available from pp_last_error(ctx) (or pp_last_error(NULL) when no
 *    context exists).  Invalid arguments are reported before any work is
 *    enqueued; CUDA launch failures are returned as PP_ECUDA.
 */
#ifndef POLYPREC_H
#define POLYPREC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define PP_OK 0
#define PP_MAXIT 1          /* not converged within maxit; result valid      */
#define PP_EINVAL (-1)      /* invalid argument                               */
#define PP_EBREAKDOWN (-2)  /* (p,Ap) <= 0 or (r,z) <= 0: operator/precond.
                               not SPD (e.g. lambda_max >= 2 theta_bar)      */
#define PP_ENONFINITE (-3)  /* NaN/Inf met in a reduction                     */
#define PP_ECUDA (-4)       /* CUDA runtime error                             */
#define PP_ETIMEOUT (-5)    /* bounded device wait expired (reported by the
                               next pcg_solve on the context)                */
#define PP_EUNSUPPORTED (-6)/* unsupported format / precision / shape         */

/* ---- enums ------------------------------------------------------------ */
#define PP_INTERVAL_LANCZOS 0 /* [alpha,beta] = extreme Ritz values of
                                 lanczos_steps Lanczos steps on W^T A W       */
#define PP_INTERVAL_GIVEN 1   /* [alpha,beta] taken from the options          */
#define PP_SEED_NONE 0        /* W = I                                         */
#define PP_SEED_JACOBI 1      /* W = diag(A)^{-1/2}; D_S^{-1/2} for S_u        */
#define PP_FMT_AUTO 0
#define PP_FMT_CSR 1          /* CSR kernel (row groups of lanes)              */
#define PP_FMT_SELL 2         /* SELL-C-sigma kernel (warp per slice)          */
#define PP_FMT_DIA 3          /* symmetric diagonal storage without column
                                 indices (banded / structured-grid matrices with
                                 at most 16 distinct upper offsets and
                                 symmetric values); PP_EUNSUPPORTED otherwise */
#define PP_POLY_CHEB 0        /* Algorithm 2 (three-term recurrence)           */
#define PP_POLY_NEWTON 1      /* Algorithm 1 (Newton form, degree 2^nlev - 1)  */
#define PP_PREC_F64 0         /* p_k applied in FP64                           */
#define PP_PREC_F32 1         /* p_k applied with FP32 values and vectors      */
#define PP_PREC_BF16 2        /* p_k applied with BF16 values, FP32 vectors    */

typedef struct pp_ctx pp_ctx; /* opaque; host memory + the caller's workspace */

/* Square sparse matrix in CSR on the device: row i holds entries
 * [rowptr[i], rowptr[i+1]) of col/val; int32 indices; the diagonal entry of
 * every row must be present when seed_scaling = PP_SEED_JACOBI. */
typedef struct {
  int n;
  long long nnz;
  const int* rowptr; /* device, n+1 */
  const int* col;    /* device, nnz */
  const double* val; /* device, nnz */
} pp_csr;

typedef struct {
  int k;              /* polynomial degree (number of products by A in P)  */
  double xi;          /* Eq. thetamod scaling; < 0: xi = clip(10 a/b, 1e-6, 1e-2) */
  int interval;       /* PP_INTERVAL_*                                      */
  double alpha, beta; /* spectral interval of W^T A W when interval = GIVEN */
  int lanczos_steps;  /* steps of the Lanczos estimate (default 10)         */
  unsigned long long seed; /* seed of the Lanczos start vector (SplitMix64,
                              stream 3, U[-1,1) in the caller's row order)  */
  int seed_scaling;   /* PP_SEED_*                                          */
  int format;         /* PP_FMT_*                                           */
  int sell_C;         /* SELL chunk (rows per slice): 32, 64 or 128; 0: 64  */
  int sell_sigma;     /* sort window (multiple of sell_C); 0 or C: no sort  */
  int apply_prec;     /* PP_PREC_*                                          */
  int flexible;       /* 1: flexible CG (beta = -(z,q)/(p,q)), FCG(1)       */
  int maxit;          /* PCG iteration limit                                */
  double rtol;        /* stop when ||r||/||b|| <= rtol (seed-scaled system) */
  int zero_guess;     /* 1: x is ignored on input and the solve starts at 0 */
  int check_every;    /* PCG iterations enqueued between host convergence
                         reads (>= 1); results do not depend on it          */
  int use_graphs;     /* 1: replay each block of check_every iterations as
                         one captured CUDA graph                            */
  int sell_variant;   /* load path of the streaming step kernels: 0 auto,
                         1 direct global loads, 2 staged in shared memory by
                         bulk copies (TMA) completing on mbarriers -- SELL
                         slices, and the FP32/BF16 steps on a Jacobi-scaled
                         3-diagonal (7-point) DIA matrix; 3 (DIA FP32/BF16
                         on an Nx x Ny x Nz grid, Nx even) walks z through
                         tiles of grid columns, keeping the z-neighbours in
                         registers.  Auto stages SELL slices and walks z
                         for FP32/BF16 DIA where the grid allows it (direct
                         loads otherwise); pp_autotune tries them all      */
  int lowrank;        /* p in [0, 32]: low-rank acceleration of Section 3.1,
                         P_hat = p_k(A_hat) + V (V^T A_hat V)^{-1} V^T with V
                         the Ritz vectors of the p smallest Ritz values of
                         lowrank_steps Lanczos steps (full
                         reorthogonalisation, start vector as for the
                         interval) on p_k(A_hat) A_hat, a polynomial in
                         A_hat with its eigenvectors and a far smaller
                         condition number.  The interval is not changed.
                         Workspace: (lowrank_steps + 1 + p) n doubles
                         more.  0: no correction                           */
  int lowrank_steps;  /* Lanczos steps for those vectors, >= lowrank; 0: 30 */
  int poly;           /* PP_POLY_CHEB: the three-term recurrence of
                         Algorithm 2; PP_POLY_NEWTON: the Newton form of
                         Algorithm 1 (k = 2^nlev - 1, FP64 apply only;
                         2 nlev n doubles more workspace)                  */
  int max_blocks;     /* > 0: at most this many thread blocks per launch of
                         the step and vector kernels (the grid-stride loops
                         then take more rounds), e.g. to leave SMs to other
                         streams; 0: grids sized by the device            */
} pp_options;

typedef struct {
  int iterations;
  long long mvp;      /* products by the operator (Table 4 convention)     */
  long long dots;     /* inner products, 3 per iteration (Table 4)         */
  double rel_res;     /* recursive ||r||/||b|| of the scaled system at exit */
  double alpha_hat, beta_hat, xi, theta_bar, delta, sigma_bar;
  double t_solve_ms;  /* device time of the whole solve (CUDA events)      */
  double t_apply_ms;  /* device time spent inside p_k applications         */
  long long apply_launches; /* recurrence-step launches inside those       */
  long long kernel_launches; /* all kernel launches the solve enqueued
                                (including those that returned at once
                                after convergence)                         */
  int status;
} pp_stats;

typedef struct {
  int n;              /* operator size                                     */
  int format;         /* PP_FMT_CSR / PP_FMT_SELL / PP_FMT_DIA actually used */
  int sell_C, sell_sigma;
  long long nnz, nnz_padded;
  double alpha_hat, beta_hat, xi, theta_bar, delta, sigma_bar;
  int k, apply_prec, lanczos_steps_done;
  double t_setup_ms;
  int grid_blocks;    /* blocks of the persistent step kernels             */
  int ndiag;          /* DIA: stored diagonals (main + upper); else 0      */
  int lowrank;        /* vectors of the low-rank correction in use         */
  int lowrank_steps_done; /* Lanczos steps run for them at setup           */
  double ritz_resid;  /* max over them of ||A_hat v - theta v|| / theta,
                         theta = v^T A_hat v (0 for caller vectors)        */
  double theta_min;   /* smallest Rayleigh quotient theta of the vectors   */
  int band_max;       /* Schur context with general blocks: largest
                         half-bandwidth of the fracture factors; else 0   */
  long long band_elems; /* doubles of band storage of those factors       */
  double t_factor_ms; /* device time of the band factorisation          */
  double t_trace_ms;  /* device time of the trace blocks M_f built from
                         the factors (both part of t_setup_ms)             */
} pp_info;

/* Fill *opt with defaults: k=20, xi=-1 (auto), Lanczos with 10 steps, seed 0,
 * Jacobi seed, automatic format, FP64 apply, plain PCG, maxit 10000,
 * rtol 1e-8, zero_guess 1, check_every 4, use_graphs 0, lowrank 0. */
void pp_options_default(pp_options* opt);

/* Chebyshev coefficients (host, pure).  Section 2.2 and Eq. thetamod:
 * theta = (beta+alpha)/2, delta = (beta-alpha)/2, theta_bar = theta (1+xi),
 * sigma_bar = theta_bar/delta (delta kept: the xi-shift moves the interval
 * to [theta_bar - delta, theta_bar + delta]); Eq. rhocheb: rho_0 =
 * 1/sigma_bar, rho_j = 1/(2 sigma_bar - rho_{j-1}), j = 1..k.
 * rho (host) has k+1 entries (may be NULL).  PP_EINVAL unless
 * 0 < alpha < beta, xi >= 0, k >= 0. */
int polyprec_coeffs(double alpha, double beta, double xi, int k, double* theta_bar,
                    double* delta, double* sigma_bar, double* rho);

/* Workspace bytes pcg_setup needs for A under opt (reads A->rowptr from the
 * device to plan the SELL layout; synchronous). */
int pp_workspace_size(const pp_csr* A, const pp_options* opt, size_t* bytes);

/* Build a solver context: seed scaling (Section 3), the scaled matrix in the
 * chosen format inside the workspace, the spectral interval (Lanczos or
 * given), xi and the coefficients.  A may be freed after it returns.
 * workspace: device, >= pp_workspace_size bytes, 256-byte aligned.
 * Synchronous with respect to the host. */
int pcg_setup(pp_ctx** ctx, const pp_csr* A, const pp_options* opt, void* workspace,
              size_t ws_bytes, void* stream);

/* z = P r for nrhs vectors (device, n x nrhs column-major), P = W p_k(A_hat)
 * W^T by Algorithm 2: k products by A_hat, each fused with its recurrence
 * update into one pass over the matrix.  With a low-rank correction in use
 * (Section 3.1) P = W (p_k(A_hat) + V (V^T A_hat V)^{-1} V^T) W^T.
 * Asynchronous. */
int polyprec_apply(pp_ctx* ctx, const double* r, double* z, int nrhs, void* stream);

/* y = A x with the operator of the context (unscaled A, or S_u for a Schur
 * context), nrhs columns.  Asynchronous. */
int pp_operator_apply(pp_ctx* ctx, const double* x, double* y, int nrhs, void* stream);

/* Solve A x = b (or S_u u = r for a Schur context) by PCG (Section 1) with
 * P = W p_k(A_hat) W^T: standard Hestenes-Stiefel PCG on the seed-scaled
 * system, 1 + k operator products and 3 inner products per iteration (3 + p
 * with a rank-p correction, Section 3.1 and Table 4), stop
 * when ||r_hat||/||b_hat|| <= rtol.  b, x: device, n.  x is read as the
 * initial guess unless zero_guess.  stats: host, may be NULL.  Returns
 * PP_OK, PP_MAXIT, PP_EBREAKDOWN or PP_ENONFINITE (x holds the last
 * iterate).  Synchronous with respect to the host. */
int pcg_solve(pp_ctx* ctx, const double* b, double* x, pp_stats* stats, void* stream);

/* Replace the low-rank correction (Section 3.1) by p caller vectors U
 * (device, n x p column-major, leading dimension ldu >= n, caller row order,
 * in the space of the unscaled operator): the preconditioner becomes
 * P = W p_k(A_hat) W^T + U (U^T A U)^{-1} U^T, i.e. V = W^{-1} U in the
 * seed-scaled space.  U^T A U is formed here (p operator products) and
 * inverted on the host.  p must not exceed opt.lowrank of the setup (the
 * workspace reserved); p = 0 removes the correction.  PP_EBREAKDOWN if
 * U^T A U is not positive definite (then no correction is in use);
 * PP_EUNSUPPORTED for batch contexts.  Synchronous. */
int pp_set_lowrank(pp_ctx* ctx, const double* U, int p, long long ldu, void* stream);

/* ---- autotuner of the step storage -------------------------------------- */

/* One layout the autotuner tried: format (PP_FMT_CSR / _SELL / _DIA), SELL
 * chunk C (32, 64 or 128 rows per slice = 1, 2 or 4 rows per lane; 0 for
 * CSR), sort window sigma (0: none), sell_variant (1 direct loads, 2
 * TMA-staged slices), the measured device time of one fused degree step
 * in microseconds, and PP_OK or why the layout was skipped (PP_EINVAL: it
 * does not fit in the workspace; PP_EUNSUPPORTED: DIA does not apply). */
typedef struct {
  int format, sell_C, sell_sigma, sell_variant;
  double us_per_step;
  int status;
} pp_tune_entry;

/* Workspace bytes pp_autotune needs to try every layout (the largest
 * pp_workspace_size over the candidates). */
int pp_autotune_workspace_size(const pp_csr* A, const pp_options* opt, size_t* bytes);

/* Choose the storage of the fused degree step (Algorithm 2) for A: build
 * the seed-scaled matrix in each candidate layout (CSR; DIA when the matrix
 * is symmetric-banded -- for FP32/BF16 applies with direct or TMA-staged
 * loads; SELL-C-sigma with C in {32, 64, 128}, sigma in {none, 1024},
 * direct or TMA-staged loads) that fits in the workspace, time
 * min(k, 8)-step applications of p_k in opt->apply_prec with CUDA events
 * (one warm-up, 5 timed), and write the fastest layout into opt (timings
 * within 3% of the fastest count as a tie, won by the first in the order
 * DIA, SELL C = 32 .. 128, CSR) (format, sell_C, sell_sigma, sell_variant;
 * the rest of opt is unchanged).  The method is unchanged by the choice.
 * workspace: device scratch, 256-byte aligned.  entries (host, may be
 * NULL) receives up to max_entries results in trial order; *count (may be
 * NULL) the number of layouts tried.  PP_EINVAL if none fits.
 * Synchronous. */
int pp_autotune(const pp_csr* A, pp_options* opt, void* workspace, size_t ws_bytes,
                pp_tune_entry* entries, int max_entries, int* count, void* stream);

/* Context facts (host struct). */
int pp_get_info(const pp_ctx* ctx, pp_info* info);

/* Release the context (host memory only; the workspace stays the caller's). */
int pp_destroy(pp_ctx* ctx);

/* Last error message of ctx (or of the calling thread when ctx is NULL). */
const char* pp_last_error(const pp_ctx* ctx);

/* ---- fracture-network Schur complement (Section 4.2) ------------------- */

/* Blocks of the saddle-point system Eq. sys.  A is block diagonal, fracture
 * f owning the unknowns [offset[f], offset[f+1]).  Two forms of A:
 *  - rectangles (A_rowptr == NULL): A_f = T[f] * (2-D 5-point Laplacian,
 *    Dirichlet on all four sides) on an nx[f] x ny[f] grid of interior
 *    nodes (x fastest); A_f^{-1} restricted to the trace nodes is built in
 *    closed form and full solves use fast diagonalisation;
 *  - general blocks (A_rowptr != NULL): A is the caller's SPD matrix as
 *    device CSR (n_h rows, global numbering, every entry inside its
 *    fracture's rows, exactly symmetric, diagonal present, no repeated
 *    entries); nx, ny, T are ignored and may be NULL.  As the paper does
 *    (Section 4.2: the exact Cholesky factor of A), each block is factored
 *    exactly: reordered on the host by reverse Cuthill-McKee (or kept in the
 *    caller's numbering when that band is narrower) and factored on the GPU
 *    as a band matrix.  PP_EUNSUPPORTED if a block's half-bandwidth after
 *    reordering exceeds 768; PP_EBREAKDOWN if a block is not positive
 *    definite; PP_EINVAL if A is not block diagonal or not symmetric.
 *    Workspace: the band factors (sum over fractures of n_f (w_f + 1)
 *    doubles) plus min(2 x SM count, 8 GiB / (max n_f x 256 B)) x max n_f x
 *    32 doubles of solve scratch.
 * C, B: n_h x n_u CSR; CT, BT: their transposes (n_u x n_h); Gh: n_h x n_h;
 * Gu: n_u x n_u.  nx, ny, T, offset are host arrays; all CSR arrays are
 * device arrays; C..Gu must stay valid until pp_destroy, A only during
 * schur_setup. */
typedef struct {
  int n_f, n_h, n_u;
  const int* nx;            /* host, n_f */
  const int* ny;            /* host, n_f */
  const double* T;          /* host, n_f */
  const long long* offset;  /* host, n_f + 1 */
  const int *C_rowptr, *C_col; const double* C_val;
  const int *B_rowptr, *B_col; const double* B_val;
  const int *CT_rowptr, *CT_col; const double* CT_val;
  const int *BT_rowptr, *BT_col; const double* BT_val;
  const int *Gh_rowptr, *Gh_col; const double* Gh_val;
  const int *Gu_rowptr, *Gu_col; const double* Gu_val;
  double alpha_reg;         /* regularisation parameter alpha of Eq. func_psi */
  const int *A_rowptr, *A_col; const double* A_val;  /* general blocks, or NULL */
} pp_dfn;

int pp_schur_workspace_size(const pp_dfn* d, const pp_options* opt, size_t* bytes);

/* Schur context: D_S = diag(S_u) by Algorithm 4 (restricted to the trace
 * rows that C, B and G^h touch), the scaling S_hat = D_S^{-1/2} S_u
 * D_S^{-1/2}, the Lanczos interval of S_hat and the coefficients.
 * apply_prec = PP_PREC_F32 applies p_k(S_hat) with an FP32 copy of the
 * trace blocks and FP32 vectors (use flexible >= 1); the outer products,
 * D_S and the interval stay FP64.  BF16 is PP_EUNSUPPORTED.  Synchronous. */
int schur_setup(pp_ctx** ctx, const pp_dfn* d, const pp_options* opt, void* workspace,
                size_t ws_bytes, void* stream);

/* y = S_u r (Algorithm 3; r, y device n_u; unscaled).  Algorithm 3's
 * three applications of A^{-1} become two: A^{-1} B r and A^{-1} G^h t
 * (t = A^{-1} C r) enter S_u r only through C^T (A^{-1} G^h t - alpha
 * A^{-1} B r), which by linearity is one application, to G^h t - alpha B r.
 * Each application is a product with the trace blocks of A^{-1}.
 * Asynchronous. */
int schur_apply(pp_ctx* ctx, const double* r, double* y, void* stream);

/* ds (device, n_u) = diag(S_u) computed at setup (Algorithm 4). */
int schur_diag(pp_ctx* ctx, double* ds, void* stream);

/* Right-hand side of Eq. schur: r = W^T M^{-1} [q; 0] =
 * alpha B^T A^{-1} q - C^T A^{-1} G^h A^{-1} q (q device n_h, r device n_u). */
int schur_rhs(pp_ctx* ctx, const double* q, double* r, void* stream);

/* Recovery of h and p from u (Section 4.2): h = A^{-1}(q + C u),
 * p = A^{-1}(alpha B u - G^h h).  Device arrays. */
int schur_recover(pp_ctx* ctx, const double* q, const double* u, double* h, double* p,
                  void* stream);

/* y = A^{-1} v for the block-diagonal fracture matrix (device, n_h). */
int schur_ainv(pp_ctx* ctx, const double* v, double* y, void* stream);

/* Band layout that schur_setup would use for general fracture blocks
 * (Section 4.2, the exact Cholesky factor of A), computed on the host
 * without a GPU: A as HOST CSR (offset[n_f] rows, global numbering) with
 * the same requirements as pp_dfn.A_*.  w_out[f] (host, n_f) receives the
 * half-bandwidth of block f after reordering, rcm_out[f] (host, n_f, may be
 * NULL) 1 where reverse Cuthill-McKee beat the given numbering.  Returns the
 * status schur_setup's planning would return (PP_EINVAL, PP_EBREAKDOWN for a
 * non-positive diagonal, PP_EUNSUPPORTED for a band wider than 768). */
int pp_fracture_bands(int n_f, const long long* offset, const int* rowptr, const int* col,
                      const double* val, int* w_out, int* rcm_out);

/* ---- batched solves (many instances, many right-hand sides) ------------- */

/* One SPD instance of a batch: CSR on the device (kept valid during
 * pp_batch_setup only) and its number of right-hand sides (1..8). */
typedef struct {
  int n;
  long long nnz;
  const int* rowptr;
  const int* col;
  const double* val;
  int nrhs;
} pp_batch_item;

#define PP_BATCH_NFEAT 8 /* features per instance from pp_batch_features */

int pp_batch_workspace_size(const pp_batch_item* items, int count, const pp_options* opt,
                            size_t* bytes);

/* Batch context: every instance in SELL-32 with the Jacobi seed (Section 3),
 * all instances' slices in one global list walked by single persistent
 * launches, right-hand sides of one instance sharing each matrix load.
 * Interval per instance: interval = LANCZOS runs opt->lanczos_steps Lanczos
 * steps on every instance (start vector SplitMix64 seed opt->seed + i,
 * stream 3, U[-1,1), for instance i); GIVEN uses opt->alpha/beta for all.
 * xi < 0 selects clip(10 alpha/beta, 1e-6, 1e-2) per instance.  apply_prec
 * F64 or F32 (FP32 values and vectors); the outer CG is FP64.  Synchronous. */
int pp_batch_setup(pp_ctx** ctx, const pp_batch_item* items, int count, const pp_options* opt,
                   void* workspace, size_t ws_bytes, void* stream);

/* Read (abx_out) and/or replace (abx_in) the spectral interval and xi of
 * every global column: 3 doubles (alpha, beta, xi) per column, columns of
 * instance i first, in right-hand-side order.  Host arrays; either may be
 * NULL.  Replacing recomputes every column's coefficients (Eq. thetamod,
 * Eq. rhocheb). */
int pp_batch_intervals(pp_ctx* ctx, double* abx_out, const double* abx_in);

/* PP_BATCH_NFEAT cheap statistics per instance (host array count x 8):
 * log10 n, mean and std of log diag(A), Gershgorin upper and lower bounds of
 * the seed-scaled matrix, log10 of the Lanczos extreme Ritz values and of
 * their ratio (zeros when the interval was given). */
int pp_batch_features(const pp_ctx* ctx, double* feat);

/* Solve every instance for all its right-hand sides by PCG with its own
 * p_k: b, x device arrays, instance i's block of n_i x nrhs_i values in
 * row-major [row][rhs] order, blocks concatenated in item order.  iters,
 * status: host arrays with one entry per global column (may be NULL).
 * Returns the worst status.  Synchronous. */
int pp_batch_solve(pp_ctx* ctx, const double* b, double* x, int* iters, int* status,
                   pp_stats* stats, void* stream);

/* Device time of one degree step of p_k (Algorithm 2) over every column of
 * the batch, in the context's apply precision: one warm-up application of
 * the k steps, then `reps` (1..1000) applications timed with CUDA events on
 * `stream`, on the batch's current residuals (every column active).
 * *us_per_step = microseconds per step.  Overwrites the recurrence vectors;
 * call it between solves.  Synchronous.  No counterpart in the paper. */
int pp_batch_time_step(pp_ctx* ctx, int reps, double* us_per_step, void* stream);

/* Workspace bytes pp_batch_autotune needs (the largest candidate). */
int pp_batch_autotune_workspace_size(const pp_batch_item* items, int count, const pp_options* opt,
                                     size_t* bytes);

/* Choose the storage of the batch's degree step by timing it: every
 * candidate layout that applies and fits in the workspace -- per-instance
 * symmetric DIA (stencil instances) and the global SELL-32 slice list -- is
 * set up with a given interval and timed by pp_batch_time_step in
 * opt->apply_prec with min(k, 8) steps; the fastest is written to
 * opt->format (timings within 3% are a tie, won by DIA).  entries (host,
 * may be NULL) receives up to max_entries results in trial order, *tried
 * (may be NULL) the number of candidates.  PP_EINVAL if none fits.  The
 * method is unchanged by the choice.  Synchronous.  No counterpart in the
 * paper. */
int pp_batch_autotune(const pp_batch_item* items, int count, pp_options* opt, void* workspace,
                      size_t ws_bytes, pp_tune_entry* entries, int max_entries, int* tried,
                      void* stream);

/* ---- learned interval predictor --------------------------------------- */

/* A 3-layer MLP (PP_MLP_NIN -> 128 -> 128 -> PP_MLP_NOUT, ReLU) that maps
 * the cheap instance statistics of pp_batch_features to the multipliers of
 * the Lanczos interval and to xi.  The paper chooses xi by hand sweeps
 * (Section 6); this predictor has no counterpart there.  BF16 weights and
 * activations with FP32 accumulation on the tensor cores, FP32 master
 * parameters, Adam.  Parameter layout (FP32, PP_MLP_NPARAM): W1 [128 x 16]
 * (columns >= 8 zero), b1 [128], W2 [128 x 128], b2 [128], W3 [8 x 128]
 * (rows >= 3 zero), b3 [8] (entries >= 3 zero).  x, y, t: device FP32,
 * row-major [batch x 8], [batch x 3], [batch x 3]. */
#define PP_MLP_NIN 8
#define PP_MLP_NHID 128
#define PP_MLP_NOUT 3
#define PP_MLP_NPARAM 19720
typedef struct pp_mlp pp_mlp;
int pp_mlp_workspace_size(int max_batch, size_t* bytes);
/* He-uniform weights from SplitMix64 (seed, stream 7), zero biases. */
int pp_mlp_create(pp_mlp** mlp, int max_batch, unsigned long long seed, void* workspace,
                  size_t ws_bytes);
/* Copy the FP32 master parameters out (get_host) and/or in (set_host). */
int pp_mlp_params(pp_mlp* mlp, float* get_host, const float* set_host);
/* y = MLP(x) for batch rows.  Synchronous.  The products run on tcgen05
 * tensor cores (accumulators in tensor memory); every wait of those kernels
 * is bounded, and an expired one is returned as PP_ETIMEOUT by this call,
 * pp_mlp_grad or a pp_mlp_train_step given loss_host. */
int pp_mlp_forward(pp_mlp* mlp, const float* x, float* y, int batch, void* stream);
/* Loss (1/(2 batch)) sum ||y - t||^2 and its gradient (host, PP_MLP_NPARAM),
 * parameters unchanged.  Synchronous. */
int pp_mlp_grad(pp_mlp* mlp, const float* x, const float* t, int batch, float* loss_host,
                float* grad_host, void* stream);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) on the same loss. */
int pp_mlp_train_step(pp_mlp* mlp, const float* x, const float* t, int batch, float lr,
                      float* loss_host, void* stream);
int pp_mlp_destroy(pp_mlp* mlp);

/* ---- measurement (no counterpart in the paper) ------------------------- */

/* The FP64 fused multiply-add rate of the current device in TFLOP/s (2
 * flops per FMA), for the arithmetic roofline of the FP64 step kernels:
 * 4 or 8 blocks of 256 threads per SM, each thread 8 or 16 independent
 * chains of 2,048 FMAs; for each of these four shapes one warm-up launch
 * and `reps` (1..100) launches timed with CUDA events on `stream`; the
 * fastest launch counts.  sink: device, 1 double,
 * never written in practice (it keeps the loop from being removed).
 * Synchronous.  PP_EINVAL on a NULL pointer or reps out of range. */
int pp_fp64_fma_rate(double* sink, int reps, double* tflops, void* stream);

/* ---- workspace-free apply (no counterpart in the paper) ---------------- */

/* z = p_k(A) r for a CSR matrix on the device, without a workspace and
 * without allocating anything.  For callers that may not call cudaMalloc:
 * a component running inside a host application that owns every device
 * allocation (its device memory comes only from the host's own pool), or a
 * latency-critical loop where the device synchronization an allocation can
 * cause is not allowed.  The caller passes only inputs and outputs (rowptr,
 * col, val, r: device, read; z: device, n, written); the two rotating
 * vectors of the recurrence live in one static device array of
 * 2 x 262,144 doubles (4 MiB) that every GPU using the library keeps until
 * the process exits.  The polynomial is the one polyprec_apply uses with
 * seed_scaling = PP_SEED_NONE, format = PP_FMT_CSR and a given interval:
 * coefficients from polyprec_coeffs(alpha, beta, xi, k), k products by A.
 * z must not overlap r (for k mod 3 == 1 the first step writes z while
 * later steps still read r); an overlap returns PP_EINVAL.
 * n > 262,144 returns PP_EINVAL with a message; so do other bad arguments.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls on one device share the array:
 * calls that overlap on the GPU (other streams, other host threads) race
 * and corrupt each other's results, so serialize them.  The array keeps
 * the previous call's contents; every entry a call reads it writes first.
 * Asynchronous on `stream`. */
int polyprec_apply_csr_static(int n, long long nnz, const int* rowptr, const int* col,
                              const double* val, double alpha, double beta, double xi, int k,
                              const double* r, double* z, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* POLYPREC_H */
