// Host-side driver state shared by the C-ABI translation units (internal).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/polyprec.h"
#include "kernels.cuh"

struct pp_batch_state;  // batched.cu

namespace pp {

constexpr int kMaxGrid = 4096;      // upper bound on blocks of any reducing kernel (16 per SM up to 256 SMs)
constexpr int kMaxCheck = 64;        // upper bound on iterations per host check

struct SellPlan {
  int C = 32, sigma = 32;
  long long nslices = 0, n_pad = 0, nnz_pad = 0;
  bool has_perm = false;
  std::vector<long long> sptr;
  std::vector<int> perm;
};

struct SchurImpl;  // schur.cu

int fail(pp_ctx* c, int code, const std::string& msg);
int cuda_fail(pp_ctx* c, cudaError_t e, const char* where);
double auto_xi(double a, double b);
void tridiag_extremes_jacobi(const std::vector<double>& a, const std::vector<double>& b, double* lmin,
                             double* lmax);
int validate_options(pp_ctx* c, const pp_options* o);

// solve.cu
int setup_interval_and_coeffs(pp_ctx* c, cudaStream_t s);
// y = p_k(A_hat) A_hat x on FP64 vectors (the polynomial in the apply precision)
cudaError_t prec_op_apply(pp_ctx* c, const double* x, double* y, cudaStream_t s);
int time_internal_apply(pp_ctx* c, int reps, cudaStream_t s, float* ms_per_apply);
cudaError_t op_step(pp_ctx* c, bool apply_matrix, const StepParams& p, const Scalars* skip, unsigned int* counter,
                    cudaStream_t s);
void destroy_ctx_resources(pp_ctx* c);

// batched.cu
void batch_free(pp_batch_state* b);

// newton.cu: Algorithm 1 (Newton form of the polynomial)
int newton_levels(int k);  // nlev with k = 2^nlev - 1, or -1
void newton_coeffs(pp_ctx* c);
long long newton_launches(const pp_ctx* c);
cudaError_t newton_apply(pp_ctx* c, const Scalars* skip, const double* r, double* z, cudaStream_t s);
cudaError_t newton_dots(pp_ctx* c, const Scalars* skip, const double* z, const double* r, const double* q,
                        double* rz_out, double* zq_out, cudaStream_t s);

// fcg.cu: FCG(m) window products and direction update
cudaError_t fcg_dots(pp_ctx* c, int s_cur, cudaStream_t s);
cudaError_t fcg_update_p(pp_ctx* c, int s_cur, int s_new, int first, cudaStream_t s);

// lowrank.cu (Section 3.1)
size_t lowrank_bytes(int cap, int m, long long n_pad, int grid_max);
void lowrank_carve(pp_ctx* c, void* base);
int lowrank_lanczos(pp_ctx* c, cudaStream_t s);
int lowrank_build_G(pp_ctx* c, int p, bool unit_cols, cudaStream_t s);
cudaError_t lowrank_coefs(pp_ctx* c, const Scalars* skip, const double* r, cudaStream_t s);
cudaError_t lowrank_update(pp_ctx* c, const Scalars* skip, double* z, const double* r, const double* q,
                           double* rz_out, double* zq_out, cudaStream_t s);

// schur.cu
// lp = true: the FP32 operator (the preconditioner's degree steps, FP32 vectors)
cudaError_t schur_scaled_step(pp_ctx* c, bool lp, const StepParams& p, const Scalars* skip, unsigned int* counter,
                              cudaStream_t s);
void schur_free(SchurImpl* s);

}  // namespace pp

struct pp_ctx {
  int kind = 0;  // 0: sparse matrix, 1: fracture-network Schur complement
  pp_options opt{};
  int n = 0;
  long long n_pad = 0, nnz = 0, nnz_pad = 0;
  pp::MatDesc A64{};  // seed-scaled operator in FP64 (outer products, FP64 apply)
  pp::MatDesc Ap{};   // same layout in the apply precision
  bool mixed = false;
  void* mixed_val = nullptr;
  double* w = nullptr;  // internal seed weights (W, or D_S^{-1/2})
  int* perm = nullptr;  // internal row i = caller row perm[i] (SELL sorting)
  int* iperm = nullptr;
  double *xh = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *t1 = nullptr, *t2 = nullptr,
         *bh = nullptr;
  float *r32 = nullptr, *u32 = nullptr, *v32 = nullptr, *z32 = nullptr;
  void* vec_begin = nullptr;
  void* vec_end = nullptr;
  pp::Scalars* sc = nullptr;
  double* partials = nullptr;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  int num_sms = 0, grid_step = 1, grid_vec = 1;
  int grid_step_lp = 1;  // blocks of the step kernels on the apply-precision matrix (mixed)
  double alpha_hat = 0, beta_hat = 0, xi = 0, theta_bar = 0, delta = 0, sigma_bar = 0;
  std::vector<double> rho;
  int lanczos_steps_done = 0;
  double t_setup_ms = 0;
  // Schur context with general blocks: banded Cholesky factors
  int band_max = 0;
  long long band_elems = 0;
  double t_band_ms = 0, t_trace_ms = 0;
  std::string err;
  std::vector<cudaEvent_t> events;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  int graph_block = 0;
  pp::SchurImpl* schur = nullptr;
  pp_batch_state* batch = nullptr;
  int op_launches = 1;  // kernel launches per operator step (1 for a matrix)
  // low-rank correction (Section 3.1): capacity (opt.lowrank), Lanczos steps
  // kept for it, vectors in use; V and the Lanczos basis Q hold n_pad rows
  int lr_cap = 0, lr_m = 0, lr_p = 0;
  pp::LowRankState* lr = nullptr;
  double *V = nullptr, *Q = nullptr, *lr_Y = nullptr, *lr_part = nullptr;
  void* lr_base = nullptr;
  int lr_steps_done = 0;
  // truncated flexible CG, FCG(m) for m = opt.flexible >= 2: ring of the last
  // m directions P and their products Q = A P (slot j at j * n_pad)
  int fcg_m = 0;
  // Newton form (Algorithm 1): zeta_0..zeta_nlev and 2 nlev level vectors
  std::vector<double> zeta;
  double* newton_buf = nullptr;
  double *Pring = nullptr, *Qring = nullptr, *fcg_part = nullptr;
  double lr_ritz_resid = 0;
  std::vector<double> lr_theta;  // Rayleigh quotients v^T A_hat v of the vectors
};
