// FP64 instantiations of the fused step kernels (see step_impl.cuh).
#include "step_impl.cuh"

namespace pp {

cudaError_t launch_step_f64(const MatDesc& A, const StepParams& p, const Scalars* sc, double* partials,
                            unsigned int* counter, int grid, cudaStream_t s) {
  return dispatch_mode<double, double>(A, p, sc, partials, counter, grid, s);
}

int step_blocks_per_sm_f64(const MatDesc& A) {
  int nb = 0;
  cudaError_t e;
  if (A.format == 2 && A.tma) {
    if (A.C == 128) {
      using S = TmaStage<double, double, 4, kChebK>;
      auto k = sell_step_tma_kernel<double, double, 4, kChebK, 0>;
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBlockBytes);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kBlock, S::kBlockBytes);
    } else if (A.C == 64) {
      using S = TmaStage<double, double, 2, kChebK>;
      auto k = sell_step_tma_kernel<double, double, 2, kChebK, 0>;
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBlockBytes);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kBlock, S::kBlockBytes);
    } else {
      using S = TmaStage<double, double, 1, kChebK>;
      auto k = sell_step_tma_kernel<double, double, 1, kChebK, 0>;
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBlockBytes);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kBlock, S::kBlockBytes);
    }
  } else if (A.format == 2 && A.C == 128) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sell_step_kernel<double, double, 4, kChebK, 0>, kBlock, 0);
  } else if (A.format == 2 && A.C == 64) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sell_step_kernel<double, double, 2, kChebK, 0>, kBlock, 0);
  } else if (A.format == 2) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sell_step_kernel<double, double, 1, kChebK, 0>, kBlock, 0);
  } else {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, csr_step_kernel<double, double, 8, kChebK, 0>, kBlock, 0);
  }
  return (e == cudaSuccess && nb > 0) ? nb : 2;
}

}  // namespace pp
