// Shared by the DIA step translation units (step_dia.cu, step_dia_tma.cu):
// the kernel-side view of a symmetric DIA matrix.  Internal header.
#pragma once

#include "step_impl.cuh"

namespace pp {

struct DiaArgs {
  int nd;
  int unit;  // 1: the main diagonal is 1 and not stored
  int doff[kMaxDiag];
  long long dstride, dpad, n_pad;
};

inline DiaArgs dia_args(const MatDesc& A) {
  DiaArgs d;
  d.nd = A.ndiag;
  d.unit = A.dia_unit;
  for (int t = 0; t < kMaxDiag; ++t) d.doff[t] = t < A.ndiag ? A.doff[t] : 0;
  d.dstride = A.dstride;
  d.dpad = A.dpad;
  d.n_pad = A.n_pad;
  return d;
}

// The TMA-staged FP32/BF16 step (step_dia_tma.cu) applies to the Jacobi-
// scaled matrix with 3 stored upper diagonals, increasing offsets and a
// middle offset of at most kDiaTmaMaxMid rows.
constexpr int kDiaTmaMaxMid = 512;
inline bool dia_tma_applies(const MatDesc& A) {
  return A.ndiag == 3 && A.dia_unit && A.doff[0] < A.doff[1] && A.doff[1] < A.doff[2] &&
         A.doff[1] <= kDiaTmaMaxMid && A.prec != kF64;
}
// One degree step (kCheb1, kCheb2, kChebK) of the FP32/BF16 matrix A with
// FP32 vectors, TMA-staged; A must satisfy dia_tma_applies.
cudaError_t launch_step_dia_tma(const MatDesc& A, const StepParams& p, const Scalars* sc, int grid, cudaStream_t s);

// The plane-marching FP32/BF16 step (step_dia_z.cu) applies to the Jacobi-
// scaled matrix of a structured Nx x Ny x Nz grid: upper offsets 1, Nx and
// Nx*Ny with Nx even, and n = Nx*Ny*Nz.
inline bool dia_z_applies(const MatDesc& A) {
  if (A.ndiag != 3 || !A.dia_unit || A.prec == kF64 || A.doff[0] != 1 || A.doff[1] < 2 || (A.doff[1] & 1)) return false;
  if (A.doff[2] % A.doff[1] != 0 || A.doff[2] <= A.doff[1]) return false;
  return (long long)A.n % A.doff[2] == 0 && (long long)A.n / A.doff[2] >= 1;
}
// One degree step (kCheb1, kCheb2, kChebK) by plane marching; A must
// satisfy dia_z_applies; grid_cap > 0 caps the blocks of the launch.
cudaError_t launch_step_dia_z(const MatDesc& A, const StepParams& p, const Scalars* sc, int grid_cap,
                              cudaStream_t s);

}  // namespace pp
