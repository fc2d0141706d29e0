// FP32 / BF16-value instantiations of the fused step kernels (the
// preconditioner of the mixed-precision solver; see step_impl.cuh).
#include "step_impl.cuh"

namespace pp {

cudaError_t launch_step_lp(const MatDesc& A, const StepParams& p, const Scalars* sc, double* partials,
                           unsigned int* counter, int grid, cudaStream_t s) {
  if (A.prec == kF32) return dispatch_mode<float, float>(A, p, sc, partials, counter, grid, s);
  if (A.prec == kBF16) return dispatch_mode<__nv_bfloat16, float>(A, p, sc, partials, counter, grid, s);
  return cudaErrorInvalidValue;
}

}  // namespace pp
