// pp_fp64_fma_rate: the FP64 fused multiply-add rate of the current device,
// measured with CUDA events (the denominator of the arithmetic roofline of
// the FP64 step kernels).  Every thread runs 8 or 16 independent FMA chains,
// so the FP64 pipe, not the chain latency, bounds the loop; the grid fills
// every SM with 4 or 8 blocks; the fastest shape counts.
#include <cuda_runtime.h>

#include <algorithm>

#include "driver.cuh"

using namespace pp;

namespace {

constexpr int kIters = 2048;
constexpr int kPeakBlock = 256;

// kChains independent chains per thread; the loop body is unrolled 4 times
// so that loop control is a small share of the issue slots.
template <int kChains>
__global__ void __launch_bounds__(kPeakBlock) fma_rate_kernel(double* sink, double m, double c) {
  double a[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) a[j] = 1.0 + 1e-3 * (double)(threadIdx.x + j);
#pragma unroll 4
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) a[j] = fma(a[j], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += a[j];
  // never true for the values used (|a| stays near 1); keeps the loop live
  if (s == -1.0) *sink = s;
}

}  // namespace

namespace {

// Best rate (FMA/s) of one launch shape over `reps` timed launches after a warm-up.
template <int kChains>
cudaError_t time_shape(int blocks_per_sm, int reps, double* sink, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1,
                       double* best_rate) {
  const int grid = num_sms() * blocks_per_sm;
  const double fmas = (double)grid * kPeakBlock * kIters * kChains;
  cudaError_t e = cudaSuccess;
  for (int r = -1; r < reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
      fma_rate_kernel<kChains><<<grid, kPeakBlock, 0, s>>>(sink, 0.9999999, 1e-7);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r >= 0 && ms > 0.f) *best_rate = std::max(*best_rate, fmas / (ms * 1e-3));
  }
  return e;
}

}  // namespace

extern "C" int pp_fp64_fma_rate(double* sink, int reps, double* tflops, void* stream) {
  if (!sink || !tflops || reps < 1 || reps > 100) return fail(nullptr, PP_EINVAL, "pp_fp64_fma_rate: invalid argument");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best = 0.0;
  // the best of a few shapes: 8 or 16 chains per thread, 4 or 8 blocks of
  // 256 threads per SM
  for (int bps : {4, 8}) {
    if (e == cudaSuccess) e = time_shape<8>(bps, reps, sink, s, e0, e1, &best);
    if (e == cudaSuccess) e = time_shape<16>(bps, reps, sink, s, e0, e1, &best);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "pp_fp64_fma_rate");
  *tflops = 2.0 * best / 1e12;
  return PP_OK;
}
