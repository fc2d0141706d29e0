// Launch entry of the fused step kernels; the instantiations live in
// step_f64.cu and step_lp.cu so that they compile in parallel.
#include "kernels.cuh"

namespace pp {

cudaError_t launch_step_f64(const MatDesc& A, const StepParams& p, const Scalars* sc, double* partials,
                            unsigned int* counter, int grid, cudaStream_t s);
cudaError_t launch_step_lp(const MatDesc& A, const StepParams& p, const Scalars* sc, double* partials,
                           unsigned int* counter, int grid, cudaStream_t s);
int step_blocks_per_sm_f64(const MatDesc& A);

cudaError_t launch_step(const MatDesc& A, const StepParams& p, const Scalars* sc, double* partials,
                        unsigned int* counter, int grid, cudaStream_t s) {
  if (grid <= 0) return cudaErrorInvalidConfiguration;
  if (p.ndot == 2 && p.mode != kResid && p.aux == nullptr) return cudaErrorInvalidValue;
  if (A.format == 3) return launch_step_dia(A, p, sc, partials, counter, grid, s);
  if (A.prec == kF64) return launch_step_f64(A, p, sc, partials, counter, grid, s);
  return launch_step_lp(A, p, sc, partials, counter, grid, s);
}

int step_max_blocks_per_sm(const MatDesc& A, int mode, int ndot) {
  (void)mode;
  (void)ndot;
  if (A.format == 3) return step_blocks_per_sm_dia(A);
  return step_blocks_per_sm_f64(A);  // SELL/CSR: the FP64 kernel's occupancy for every precision
}

}  // namespace pp
