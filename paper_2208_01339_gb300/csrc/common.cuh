// Shared device-side definitions of libpolyprec (internal header).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace pp {

constexpr int kMaxDots = 3;        // values reduced by one fused kernel
constexpr int kMaxLanczos = 512;   // Lanczos steps kept on the device
constexpr int kBlock = 256;        // threads per block of the streaming kernels
constexpr int kMaxLowRank = 32;    // vectors of the low-rank correction (Section 3.1)
constexpr int kMaxFcg = 8;         // window of truncated flexible CG, FCG(m)

// PCG / Lanczos state kept on the device so that a block of iterations can
// run (or be replayed as a CUDA graph) without host round trips.  Kernels
// read `done` on entry and return at once when it is set.
struct Scalars {
  double bb;       // ||b_hat||^2
  double rtol2;    // rtol^2 * bb
  double rz;       // (r, z) of the current search direction
  double rz_new;   // (r, z) of the latest preconditioned residual
  double pq;       // (p, A p)
  double zq;       // (z_new, q) for flexible CG
  double rr;       // ||r||^2 after the latest update
  double vv;       // scratch norm (Lanczos start vector)
  int done;        // 1: stop enqueued work (converged / breakdown / maxit)
  int status;      // PP_* status of the solve
  int iter;        // completed PCG iterations
  int maxit;
  int flexible;
  int lan_steps;   // Lanczos steps completed without breakdown
  int dev_error;   // 1: a bounded wait inside a kernel expired (PP_ETIMEOUT)
  int x_pending;   // 1: the solve stopped after an r update whose x update (fused
                   // into the next first degree step) did not run
  unsigned int counters[8];
  double fcg_pq[kMaxFcg];  // FCG(m): (p_j, A p_j) of the directions in the window, by ring slot
  double fcg_zq[kMaxFcg];  // FCG(m): (z, A p_j) of the latest preconditioned residual, by ring slot
  double lan_a[kMaxLanczos];
  double lan_b2[kMaxLanczos];
};

// Counter slots (one per kernel family so that consecutive kernels never
// share a counter).
enum CounterSlot { kCntStep = 0, kCntUpdXR = 1, kCntUpdP = 2, kCntVec = 3, kCntLan = 4, kCntSchur = 5, kCntLr = 6 };

// Device state of the low-rank correction: G^{-1} = (V^T A V)^{-1} (row
// stride kMaxLowRank), the coefficients c = G^{-1} V^T r of the latest
// application, and the Gram-Schmidt coefficients of the Lanczos run.
struct LowRankState {
  double Ginv[kMaxLowRank * kMaxLowRank];
  double c[kMaxLowRank];
  double h[kMaxLanczos + 8];
};

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// Sum NV values over the block; the result is valid in every thread.
// Fixed order (lane, then warp), so the result is deterministic.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    double x = warp_sum(v[i]);
    if (lane == 0) sh[i][wid] = x;
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double x = lane < nw ? sh[i][lane] : 0.0;
      x = warp_sum(x);
      if (lane == 0) sh[i][0] = x;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = sh[i][0];
  __syncthreads();
}

// Grid-wide deterministic reduction: every block stores its partial sums,
// the last block to arrive adds the partials in block order and returns
// true (in all of its threads) with the totals in v.  The counter is reset
// by the last block, so consecutive launches can reuse it.
template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], double* partials, unsigned int* counter) {
  __shared__ bool last;
  block_sum<NV>(v);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) partials[i * gridDim.x + blockIdx.x] = v[i];
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double acc[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) {
    acc[i] = 0.0;
    for (unsigned int j = threadIdx.x; j < gridDim.x; j += blockDim.x) acc[i] += __ldcg(&partials[i * gridDim.x + j]);
  }
  block_sum<NV>(acc);
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = acc[i];
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// True in the last block of the grid to reach this point (counter reset).
__device__ __forceinline__ bool grid_last(unsigned int* counter) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int t = atomicAdd(counter, 1u);
    last = (t == gridDim.x - 1);
    if (last) *counter = 0u;
  }
  __syncthreads();
  return last;
}

__device__ __forceinline__ int load_done(const Scalars* sc) {
  return *reinterpret_cast<const volatile int*>(&sc->done);
}

// SplitMix64 (Steele, Lea & Flood 2014) as a counter-based stream:
// key = mix(seed ^ mix(stream + C0)), value_i = mix(key + (i+1) * GOLDEN).
__host__ __device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t splitmix_key(uint64_t seed, uint64_t stream) {
  return splitmix_mix(seed ^ splitmix_mix(stream + 0x632BE59BD9B4E019ull));
}
__host__ __device__ __forceinline__ double splitmix_uniform(uint64_t key, uint64_t i) {
  uint64_t v = splitmix_mix(key + (i + 1) * 0x9E3779B97F4A7C15ull);
  return (double)(v >> 11) * 0x1.0p-53;
}

}  // namespace pp
