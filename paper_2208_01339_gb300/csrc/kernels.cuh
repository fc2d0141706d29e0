// Internal launch interface between the C-ABI driver (api.cu) and the
// kernel translation units.  Nothing here is exported from the library.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "common.cuh"

namespace pp {

enum Prec { kF64 = 0, kF32 = 1, kBF16 = 2 };

// Streaming multiprocessors of the current device (grid sizing), and the
// current device's ordinal clamped to [0, kMaxDevices) for per-device
// caches of launch attributes and occupancy (api.cu).
constexpr int kMaxDevices = 64;
int num_sms();
int current_device();

// One fused pass of a degree step (or a plain product) over the matrix:
//   kSpmv    y = A x
//   kResid   y = r - A x
//   kCheb1   y = ca r + cb (A r)                       (Algorithm 2, step 3; x = r)
//   kCheb2   y = ca x + cb r + cc (r - A x)            (first loop pass, x_old = r/theta)
//   kChebK   y = ca x + cb x_old + cc (r - A x)        (Algorithm 2 loop body)
//   kLanczos y = A x - sqrt(*dev_coef) x_old           (Lanczos three-term step)
// The Chebyshev coefficients arrive folded (cheb_step_coeffs), so an update
// costs one multiply and three fused multiply-adds per row.
// Optional fused inner products (ndot = 0, 1 or 2), written by the last block:
//   kSpmv: (x, y)   kResid: (y, y), (r, r)   kCheb*: (r, y), (aux, y)   kLanczos: (y, x)
enum StepMode { kSpmv = 0, kResid = 1, kCheb1 = 2, kCheb2 = 3, kChebK = 4, kLanczos = 5 };

constexpr int kMaxDiag = 16;  // stored diagonals of the symmetric DIA format

struct MatDesc {
  int format;  // 1 CSR, 2 SELL, 3 DIA
  int n;
  long long n_pad;
  // SELL-C-sigma: slice s holds rows [s*C, (s+1)*C), C = 32*VW; entry j of
  // row s*C + e*32 + l (lane l, e < VW) sits at slice_ptr[s] + j*C + l*VW + e.
  int C;
  long long nslices;
  const long long* slice_ptr;
  const int* col;        // SELL or CSR column indices
  const void* val;       // values in `prec`
  const int* rowptr;     // CSR only
  int csr_group;         // CSR: lanes per row (1, 8, 32)
  int prec;
  int tma;               // SELL: stage slices through shared memory with cp.async.bulk;
                         // DIA FP32/BF16: 2 TMA-staged tiles, 3 plane marching
  // DIA (symmetric; rows in natural order): the stored diagonals t =
  // 0..ndiag-1 at offsets doff[t] -- the main diagonal (doff[0] = 0) and the
  // upper ones, or, with dia_unit = 1 (Jacobi-scaled matrix, whose diagonal
  // is 1 by construction), the upper ones only.  Entry (i, i + doff[t]) sits
  // at val[t * dstride + dpad + i]; positions -dpad..-1 and entries outside
  // the matrix hold 0.  Row i takes its lower entries (i, i - doff[t]) from
  // val[t * dstride + dpad + i - doff[t]].
  int ndiag;
  int dia_unit;
  int doff[kMaxDiag];
  long long dstride, dpad;
};

// Folded coefficients of degree step j of Algorithm 2 (j >= 1): with
// rho_j, 2 sigma_bar, 2/delta and 1/theta_bar, the step
//   x_j = rho_j (2 sigma x_{j-1} - rho_{j-1} x_{j-2} + (2/delta)(r - A x_{j-1}))
// (x_0 = r/theta, and x_1 = (2 rho_1/delta)(2 r - A r/theta)) becomes
//   j = 1: ca = 4 rho_1/delta,        cb = -2 rho_1/(delta theta)
//   j = 2: ca = 2 sigma rho_2, cb = -rho_2 rho_1/theta, cc = 2 rho_2/delta
//   j > 2: ca = 2 sigma rho_j, cb = -rho_j rho_{j-1},   cc = 2 rho_j/delta
struct StepCoeffs {
  double ca, cb, cc;
};
inline StepCoeffs cheb_step_coeffs(int j, const double* rho, double theta_bar, double delta, double sigma_bar) {
  if (j == 1) return {4.0 * rho[1] / delta, -2.0 * rho[1] / (delta * theta_bar), 0.0};
  if (j == 2) return {2.0 * sigma_bar * rho[2], -rho[2] * rho[1] / theta_bar, 2.0 * rho[2] / delta};
  return {2.0 * sigma_bar * rho[j], -rho[j] * rho[j - 1], 2.0 * rho[j] / delta};
}

struct StepParams {
  int mode = kSpmv;
  int ndot = 0;
  const void* x = nullptr;
  const void* xold = nullptr;
  const void* r = nullptr;
  void* y = nullptr;
  const double* aux = nullptr;
  const double* dev_coef = nullptr;
  double ca = 0, cb = 0, cc = 0, cd = 0, ce = 0;
  double* dot_out0 = nullptr;
  double* dot_out1 = nullptr;
  int* err = nullptr;  // set to 1 when a bounded device wait expires
};

// Launchers (step.cu).  grid = number of blocks (persistent, grid-stride);
// partials must hold 2*grid doubles.
cudaError_t launch_step(const MatDesc& A, const StepParams& p, const Scalars* sc, double* partials,
                        unsigned int* counter, int grid, cudaStream_t s);
int step_max_blocks_per_sm(const MatDesc& A, int mode, int ndot);

// Vector kernels (vec.cu).  All use grid-stride loops over a fixed grid.
struct VecLaunch {
  int grid;
  double* partials;
  cudaStream_t s;
};
// out[i] = w[i] * in[perm ? perm[i] : i] (i < n), 0 for n <= i < n_pad; out FP64 or FP32.
// Optional ||out||^2 -> *dot_out.
cudaError_t vec_scale_in(const VecLaunch& L, long long n, long long n_pad, const double* w, const int* perm,
                         const double* in, void* out, int out_prec, double* dot_out, unsigned int* counter);
// out[perm ? perm[i] : i] = w[i] * in[i] (divide = 0) or in[i] / w[i] (divide = 1); in FP64 or FP32.
cudaError_t vec_scale_out(const VecLaunch& L, long long n, const double* w, const int* perm, const void* in,
                          int in_prec, double* out, int divide);
// xh[i] = x[perm ? perm[i] : i] / w[i]
cudaError_t vec_unscale_in(const VecLaunch& L, long long n, long long n_pad, const double* w, const int* perm,
                           const double* x, double* xh);
// PCG updates (device scalars in sc).  vec_update_xr with x = nullptr
// updates r only and leaves x += alpha p to vec_update_p (given x), which
// reads p anyway; x_pending is set when the solve stops in between, and
// vec_finish_x applies that pending update.
cudaError_t vec_update_xr(const VecLaunch& L, long long n, Scalars* sc, double* x, double* r, const double* p,
                          const double* q);
cudaError_t vec_finish_x(const VecLaunch& L, long long n, const Scalars* sc, double* x, const double* p);
cudaError_t vec_update_p(const VecLaunch& L, long long n, Scalars* sc, const double* z, double* p, int first,
                         double* x = nullptr);
cudaError_t pcg_init(Scalars* sc, double rtol, int maxit, int flexible, cudaStream_t s);
// z = double(z32); (r, z) -> sc->rz_new, (q, z) -> sc->zq when q != nullptr.
cudaError_t vec_from32_dot(const VecLaunch& L, long long n, const Scalars* skip, const float* z32, double* z,
                           const double* r, const double* q, double* rz_out, double* zq_out, unsigned int* counter);
// z = r * inv_theta (degree 0), optional dots as above; prec of r/z FP64 or FP32.
cudaError_t vec_scale_dot(const VecLaunch& L, long long n, const Scalars* skip, const void* r, void* z, int prec,
                          double inv_theta, const double* rd, const double* q, double* rz_out, double* zq_out,
                          unsigned int* counter);
cudaError_t vec_convert(const VecLaunch& L, long long n, const void* in, int in_prec, void* out, int out_prec,
                        const Scalars* skip = nullptr);
// Lanczos helpers.
cudaError_t lanczos_start(const VecLaunch& L, long long n, long long n_pad, uint64_t key, const int* perm,
                          double* v, double* nrm2_out, unsigned int* counter);
cudaError_t vec_scale_by_rsqrt(const VecLaunch& L, long long n, double* v, const double* nrm2);
// w -= a v, ||w||^2 -> b2_out
cudaError_t lanczos_orth(const VecLaunch& L, long long n, double* w, const double* v, const double* a,
                         double* b2_out, unsigned int* counter);
cudaError_t vec_dot(const VecLaunch& L, long long n, const double* x, const double* y, double* out,
                    unsigned int* counter);
cudaError_t vec_axpby(const VecLaunch& L, long long n, double a, const double* x, double b, double* y);
// w_int[i] = w_orig ? w_orig[perm ? perm[i] : i] : 1 for i < n, 1 on the padding.
cudaError_t gather_weights(const VecLaunch& L, long long n, long long n_pad, const double* w_orig, const int* perm,
                           double* w_int);

// Setup kernels (setup.cu).
cudaError_t csr_jacobi_weights(int n, const int* rowptr, const int* col, const double* val, double* w,
                               int* bad_row, cudaStream_t s);
cudaError_t sell_fill(const MatDesc& dst, const int* perm, const int* iperm, const int* rowptr, const int* col,
                      const double* val, const double* w, void* out_val, int out_prec, cudaStream_t s);
cudaError_t csr_fill(int n, const int* rowptr, const int* col, const double* val, const double* w, int* out_rowptr,
                     int* out_col, void* out_val, int out_prec, long long nnz, cudaStream_t s);
cudaError_t sell_convert_values(long long nnz_pad, const double* in, void* out, int out_prec, cudaStream_t s);
// DIA fill from CSR (entries with col >= row): val[t * dstride + dpad + row] = w_row a w_col (w may be null).
cudaError_t dia_fill(const MatDesc& dst, const int* rowptr, const int* col, const double* val, const double* w,
                     cudaStream_t s);

// DIA planning on the device (setup.cu); dia_plan() is synchronous and
// copies the finished table to the host struct *out.
constexpr int kDiaSlots = 64;
enum DiaPlanError {
  kDiaOk = 0,
  kDiaBadRowptr = 1,
  kDiaBadCol = 2,
  kDiaRepeated = 3,
  kDiaNoDiagonal = 4,
  kDiaUnsymmetric = 5,
  kDiaTooMany = 6
};
struct DiaPlanTable {
  unsigned long long slot[kDiaSlots];  // upper offset + 1, 0 = empty
  int count;                           // distinct upper offsets
  int pad_;
  unsigned long long err;              // (row << 8) | DiaPlanError of the first error; ~0: none
};
cudaError_t dia_plan(int n, long long nnz, const int* rowptr, const int* col, const double* val, DiaPlanTable* t,
                     cudaStream_t s);

// DIA step kernels (step_dia.cu).
cudaError_t launch_step_dia(const MatDesc& A, const StepParams& p, const Scalars* sc, double* partials,
                            unsigned int* counter, int grid, cudaStream_t s);
int step_blocks_per_sm_dia(const MatDesc& A);

}  // namespace pp
