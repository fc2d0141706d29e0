// Fused degree-step kernels: one pass over the matrix computes A x and the
// Chebyshev three-term update of Algorithm 2 (or a plain product, a
// residual, a Lanczos step), with optional fused inner products.
//
// SELL-C-sigma layout (C = 32*VW rows per slice): lane l of the warp that
// owns slice s handles rows s*C + e*32 + l, e = 0..VW-1, and entry j of
// those VW rows is stored contiguously at slice_ptr[s] + j*C + l*VW + e.
// Matrix loads are therefore 8*VW-byte (16-byte for FP64 VW=2) per lane and
// contiguous across the warp, while gathers and vector accesses of one e
// touch 32 consecutive rows.
//
// Two SELL kernels:
//  * sell_step_kernel      -- matrix loads straight from global memory
//                             (evict-first), gathers through the read-only
//                             path;
//  * sell_step_tma_kernel  -- each warp double-buffers its next slice (values,
//                             column indices and the r / x_old rows it
//                             needs) into shared memory with cp.async.bulk
//                             completing on an mbarrier, with an evict-first
//                             L2 policy for the matrix stream, so the load
//                             units only serve the x gathers.  Slices wider
//                             than kTmaWmax fall back to direct loads.
// CSR: G lanes per row, strided over the row, reduced by warp shuffles.
#pragma once

#include <type_traits>

#include "kernels.cuh"

namespace pp {
namespace {

constexpr int kTmaWmax = 7;           // widest slice staged through shared memory
constexpr int kTmaStages = 2;         // per-warp pipeline depth
constexpr long long kSpinLimit = 1LL << 22;  // bounded mbarrier waits

// ---------------------------------------------------------------- loads ----
template <typename TV, int VW, typename TA>
struct ValLd;
template <typename TA>
struct ValLd<double, 1, TA> {
  __device__ static void ld(const double* p, TA (&o)[1]) { o[0] = (TA)__ldcs(p); }
  __device__ static void lds(const double* p, TA (&o)[1]) { o[0] = (TA)*p; }
};
template <typename TA>
struct ValLd<double, 2, TA> {
  __device__ static void ld(const double* p, TA (&o)[2]) {
    double2 t = __ldcs(reinterpret_cast<const double2*>(p));
    o[0] = (TA)t.x;
    o[1] = (TA)t.y;
  }
  __device__ static void lds(const double* p, TA (&o)[2]) {
    double2 t = *reinterpret_cast<const double2*>(p);
    o[0] = (TA)t.x;
    o[1] = (TA)t.y;
  }
};
template <typename TA>
struct ValLd<double, 4, TA> {
  __device__ static void ld(const double* p, TA (&o)[4]) {
    double2 t0 = __ldcs(reinterpret_cast<const double2*>(p));
    double2 t1 = __ldcs(reinterpret_cast<const double2*>(p) + 1);
    o[0] = (TA)t0.x;
    o[1] = (TA)t0.y;
    o[2] = (TA)t1.x;
    o[3] = (TA)t1.y;
  }
  __device__ static void lds(const double* p, TA (&o)[4]) {
    double2 t0 = *reinterpret_cast<const double2*>(p);
    double2 t1 = *(reinterpret_cast<const double2*>(p) + 1);
    o[0] = (TA)t0.x;
    o[1] = (TA)t0.y;
    o[2] = (TA)t1.x;
    o[3] = (TA)t1.y;
  }
};
template <typename TA>
struct ValLd<float, 1, TA> {
  __device__ static void ld(const float* p, TA (&o)[1]) { o[0] = (TA)__ldcs(p); }
  __device__ static void lds(const float* p, TA (&o)[1]) { o[0] = (TA)*p; }
};
template <typename TA>
struct ValLd<float, 2, TA> {
  __device__ static void ld(const float* p, TA (&o)[2]) {
    float2 t = __ldcs(reinterpret_cast<const float2*>(p));
    o[0] = (TA)t.x;
    o[1] = (TA)t.y;
  }
  __device__ static void lds(const float* p, TA (&o)[2]) {
    float2 t = *reinterpret_cast<const float2*>(p);
    o[0] = (TA)t.x;
    o[1] = (TA)t.y;
  }
};
template <typename TA>
struct ValLd<float, 4, TA> {
  __device__ static void ld(const float* p, TA (&o)[4]) {
    float4 t = __ldcs(reinterpret_cast<const float4*>(p));
    o[0] = (TA)t.x;
    o[1] = (TA)t.y;
    o[2] = (TA)t.z;
    o[3] = (TA)t.w;
  }
  __device__ static void lds(const float* p, TA (&o)[4]) {
    float4 t = *reinterpret_cast<const float4*>(p);
    o[0] = (TA)t.x;
    o[1] = (TA)t.y;
    o[2] = (TA)t.z;
    o[3] = (TA)t.w;
  }
};
__device__ __forceinline__ float bf16_lo(unsigned int u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(unsigned int u) { return __uint_as_float(u & 0xffff0000u); }
template <typename TA>
struct ValLd<__nv_bfloat16, 1, TA> {
  __device__ static void ld(const __nv_bfloat16* p, TA (&o)[1]) {
    unsigned short u = __ldcs(reinterpret_cast<const unsigned short*>(p));
    o[0] = (TA)__uint_as_float(((unsigned int)u) << 16);
  }
  __device__ static void lds(const __nv_bfloat16* p, TA (&o)[1]) {
    unsigned short u = *reinterpret_cast<const unsigned short*>(p);
    o[0] = (TA)__uint_as_float(((unsigned int)u) << 16);
  }
};
template <typename TA>
struct ValLd<__nv_bfloat16, 2, TA> {
  __device__ static void ld(const __nv_bfloat16* p, TA (&o)[2]) {
    unsigned int u = __ldcs(reinterpret_cast<const unsigned int*>(p));
    o[0] = (TA)bf16_lo(u);
    o[1] = (TA)bf16_hi(u);
  }
  __device__ static void lds(const __nv_bfloat16* p, TA (&o)[2]) {
    unsigned int u = *reinterpret_cast<const unsigned int*>(p);
    o[0] = (TA)bf16_lo(u);
    o[1] = (TA)bf16_hi(u);
  }
};
template <typename TA>
struct ValLd<__nv_bfloat16, 4, TA> {
  __device__ static void ld(const __nv_bfloat16* p, TA (&o)[4]) {
    uint2 u = __ldcs(reinterpret_cast<const uint2*>(p));
    o[0] = (TA)bf16_lo(u.x);
    o[1] = (TA)bf16_hi(u.x);
    o[2] = (TA)bf16_lo(u.y);
    o[3] = (TA)bf16_hi(u.y);
  }
  __device__ static void lds(const __nv_bfloat16* p, TA (&o)[4]) {
    uint2 u = *reinterpret_cast<const uint2*>(p);
    o[0] = (TA)bf16_lo(u.x);
    o[1] = (TA)bf16_hi(u.x);
    o[2] = (TA)bf16_lo(u.y);
    o[3] = (TA)bf16_hi(u.y);
  }
};

template <int VW>
struct ColLd;
template <>
struct ColLd<1> {
  __device__ static void ld(const int* p, int (&o)[1]) { o[0] = __ldcs(p); }
  __device__ static void lds(const int* p, int (&o)[1]) { o[0] = *p; }
};
template <>
struct ColLd<2> {
  __device__ static void ld(const int* p, int (&o)[2]) {
    int2 t = __ldcs(reinterpret_cast<const int2*>(p));
    o[0] = t.x;
    o[1] = t.y;
  }
  __device__ static void lds(const int* p, int (&o)[2]) {
    int2 t = *reinterpret_cast<const int2*>(p);
    o[0] = t.x;
    o[1] = t.y;
  }
};
template <>
struct ColLd<4> {
  __device__ static void ld(const int* p, int (&o)[4]) {
    int4 t = __ldcs(reinterpret_cast<const int4*>(p));
    o[0] = t.x;
    o[1] = t.y;
    o[2] = t.z;
    o[3] = t.w;
  }
  __device__ static void lds(const int* p, int (&o)[4]) {
    int4 t = *reinterpret_cast<const int4*>(p);
    o[0] = t.x;
    o[1] = t.y;
    o[2] = t.z;
    o[3] = t.w;
  }
};

template <typename TX>
struct StepArgs {
  const TX* x;
  const TX* xold;
  const TX* r;
  TX* y;
  const double* aux;
  const double* dev_coef;
  TX ca, cb, cc, cd, ce;
  double* out0;
  double* out1;
  int* err;
};

template <int MODE>
__host__ __device__ constexpr bool mode_needs_r() {
  return MODE == kResid || MODE == kCheb1 || MODE == kCheb2 || MODE == kChebK;
}
template <int MODE>
__host__ __device__ constexpr bool mode_needs_xold() {
  return MODE == kChebK || MODE == kLanczos;
}
template <int MODE, int NDOT>
__host__ __device__ constexpr bool mode_needs_xown() {
  return MODE == kCheb2 || MODE == kChebK || ((MODE == kSpmv || MODE == kLanczos) && NDOT > 0);
}

// Value of one output row from acc = (A x)_row and the row's own entries.
template <typename TX, int MODE>
__device__ __forceinline__ TX row_value(const StepArgs<TX>& a, TX acc, TX xs, TX rs, TX xo, TX lan_coef) {
  if constexpr (MODE == kSpmv) {
    return acc;
  } else if constexpr (MODE == kResid) {
    return rs - acc;
  } else if constexpr (MODE == kCheb1) {
    return fma(a.cb, acc, a.ca * rs);
  } else if constexpr (MODE == kCheb2) {
    return fma(a.cc, rs - acc, fma(a.cb, rs, a.ca * xs));
  } else if constexpr (MODE == kChebK) {
    return fma(a.cc, rs - acc, fma(a.cb, xo, a.ca * xs));
  } else {
    return acc - lan_coef * xo;
  }
}

template <typename TX, int MODE, int NDOT>
__device__ __forceinline__ void row_dots(const StepArgs<TX>& a, long long row, TX y, TX xs, TX rs,
                                         double (&dot)[NDOT > 0 ? NDOT : 1]) {
  if constexpr (NDOT > 0) {
    const double yd = (double)y;
    if constexpr (MODE == kSpmv || MODE == kLanczos) {
      dot[0] += (double)xs * yd;
    } else if constexpr (MODE == kResid) {
      dot[0] += yd * yd;
      if constexpr (NDOT > 1) dot[1] += (double)rs * (double)rs;
    } else {
      dot[0] += (double)rs * yd;
      if constexpr (NDOT > 1) dot[1] += __ldg(a.aux + row) * yd;
    }
  }
}

template <typename TX, int NDOT>
__device__ __forceinline__ void finish_dots(const StepArgs<TX>& a, double (&dot)[NDOT > 0 ? NDOT : 1],
                                            double* partials, unsigned int* counter) {
  if constexpr (NDOT > 0) {
    double v[NDOT];
#pragma unroll
    for (int i = 0; i < NDOT; ++i) v[i] = dot[i];
    if (grid_sum<NDOT>(v, partials, counter) && threadIdx.x == 0) {
      a.out0[0] = v[0];
      if constexpr (NDOT > 1) a.out1[0] = v[1];
    }
  }
}

template <typename TX, int MODE>
__device__ __forceinline__ TX lanczos_coef(const StepArgs<TX>& a) {
  if constexpr (MODE == kLanczos) {
    if (a.dev_coef) return (TX)sqrt(*a.dev_coef);
  }
  return (TX)0;
}

// Row sums of one slice for the VW rows of this lane; matrix entries come
// from `vals`/`cols` (global or shared) with stride C between entries.
// Slices up to 8 wide (every 7-point stencil slice) run as straight-line
// code: all value/index loads of the slice, then all gathers, then the FMAs
// in entry order.
template <typename TV, typename TX, int VW, bool SMEM, int W>
__device__ __forceinline__ void rowsums_fixed(const TV* vals, const int* cols, const TX* __restrict__ x,
                                              TX (&acc)[VW]) {
  constexpr int C = 32 * VW;
  TX v[W][VW];
  int c[W][VW];
#pragma unroll
  for (int u = 0; u < W; ++u) {
    if constexpr (SMEM) {
      ValLd<TV, VW, TX>::lds(vals + u * C, v[u]);
      ColLd<VW>::lds(cols + u * C, c[u]);
    } else {
      ValLd<TV, VW, TX>::ld(vals + (long long)u * C, v[u]);
      ColLd<VW>::ld(cols + (long long)u * C, c[u]);
    }
  }
  TX xv[W][VW];
#pragma unroll
  for (int u = 0; u < W; ++u)
#pragma unroll
    for (int e = 0; e < VW; ++e) xv[u][e] = __ldg(x + c[u][e]);
#pragma unroll
  for (int e = 0; e < VW; ++e) acc[e] = (TX)0;
#pragma unroll
  for (int u = 0; u < W; ++u)
#pragma unroll
    for (int e = 0; e < VW; ++e) acc[e] = fma(v[u][e], xv[u][e], acc[e]);
}

template <typename TV, typename TX, int VW, bool SMEM>
__device__ __forceinline__ void slice_rowsums(const TV* vals, const int* cols, int w, const TX* __restrict__ x,
                                              TX (&acc)[VW]) {
  constexpr int C = 32 * VW;
  switch (w) {
    case 1: rowsums_fixed<TV, TX, VW, SMEM, 1>(vals, cols, x, acc); return;
    case 2: rowsums_fixed<TV, TX, VW, SMEM, 2>(vals, cols, x, acc); return;
    case 3: rowsums_fixed<TV, TX, VW, SMEM, 3>(vals, cols, x, acc); return;
    case 4: rowsums_fixed<TV, TX, VW, SMEM, 4>(vals, cols, x, acc); return;
    case 5: rowsums_fixed<TV, TX, VW, SMEM, 5>(vals, cols, x, acc); return;
    case 6: rowsums_fixed<TV, TX, VW, SMEM, 6>(vals, cols, x, acc); return;
    case 7: rowsums_fixed<TV, TX, VW, SMEM, 7>(vals, cols, x, acc); return;
    case 8: rowsums_fixed<TV, TX, VW, SMEM, 8>(vals, cols, x, acc); return;
    default: break;
  }
#pragma unroll
  for (int e = 0; e < VW; ++e) acc[e] = (TX)0;
  constexpr int CH = 4;
  for (int j0 = 0; j0 < w; j0 += CH) {
    TX v[CH][VW];
    int c[CH][VW];
#pragma unroll
    for (int u = 0; u < CH; ++u) {
      if (j0 + u < w) {
        if constexpr (SMEM) {
          ValLd<TV, VW, TX>::lds(vals + (j0 + u) * C, v[u]);
          ColLd<VW>::lds(cols + (j0 + u) * C, c[u]);
        } else {
          ValLd<TV, VW, TX>::ld(vals + (long long)(j0 + u) * C, v[u]);
          ColLd<VW>::ld(cols + (long long)(j0 + u) * C, c[u]);
        }
      } else {
#pragma unroll
        for (int e = 0; e < VW; ++e) {
          v[u][e] = (TX)0;
          c[u][e] = 0;
        }
      }
    }
    TX xv[CH][VW];
#pragma unroll
    for (int u = 0; u < CH; ++u)
#pragma unroll
      for (int e = 0; e < VW; ++e) xv[u][e] = (j0 + u < w) ? __ldg(x + c[u][e]) : (TX)0;
#pragma unroll
    for (int u = 0; u < CH; ++u)
#pragma unroll
      for (int e = 0; e < VW; ++e) acc[e] = fma(v[u][e], xv[u][e], acc[e]);
  }
}

template <typename TV, typename TX, int VW, int MODE, int NDOT>
__global__ void __launch_bounds__(kBlock) sell_step_kernel(int n, long long nslices, const long long* __restrict__ sptr,
                                                           const int* __restrict__ col, const TV* __restrict__ val,
                                                           StepArgs<TX> a, const Scalars* sc, double* partials,
                                                           unsigned int* counter) {
  if (sc && load_done(sc)) return;
  constexpr int C = 32 * VW;
  const int lane = threadIdx.x & 31;
  const long long wpb = blockDim.x >> 5;
  const long long gw = (long long)blockIdx.x * wpb + (threadIdx.x >> 5);
  const long long nw = (long long)gridDim.x * wpb;
  double dot[NDOT > 0 ? NDOT : 1];
#pragma unroll
  for (int i = 0; i < (NDOT > 0 ? NDOT : 1); ++i) dot[i] = 0.0;
  const TX lan = lanczos_coef<TX, MODE>(a);
  for (long long s = gw; s < nslices; s += nw) {
    const long long base = sptr[s];
    const int w = (int)((sptr[s + 1] - base) / C);
    TX acc[VW];
    slice_rowsums<TV, TX, VW, false>(val + base + lane * VW, col + base + lane * VW, w, a.x, acc);
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const long long row = s * C + e * 32 + lane;
      TX xs = (TX)0, rs = (TX)0, xo = (TX)0;
      if constexpr (mode_needs_xown<MODE, NDOT>()) xs = __ldg(a.x + row);
      if constexpr (mode_needs_r<MODE>()) rs = a.r[row];
      if constexpr (mode_needs_xold<MODE>()) {
        if (MODE == kChebK || a.xold) xo = a.xold[row];
      }
      const TX y = row_value<TX, MODE>(a, acc[e], xs, rs, xo, lan);
      a.y[row] = y;
      if (row < n) row_dots<TX, MODE, NDOT>(a, row, y, xs, rs, dot);
    }
  }
  finish_dots<TX, NDOT>(a, dot, partials, counter);
}

// ------------------------------------------------------ TMA bulk staging ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: false when the copy did not land within kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < kSpinLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
// global -> shared bulk copy (16-byte aligned, size multiple of 16) that
// completes `bytes` of transaction count on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
      : "memory");
}

template <typename TV, typename TX, int VW, int MODE>
struct TmaStage {
  static constexpr int C = 32 * VW;
  static constexpr int kVal = kTmaWmax * C * (int)sizeof(TV);
  static constexpr int kCol = kTmaWmax * C * 4;
  static constexpr int kR = mode_needs_r<MODE>() ? C * (int)sizeof(TX) : 0;
  static constexpr int kXo = mode_needs_xold<MODE>() ? C * (int)sizeof(TX) : 0;
  static constexpr int kBytes = ((kVal + kCol + kR + kXo + 127) / 128) * 128;
  static constexpr int kBlockBytes = kBytes * kTmaStages * (kBlock / 32);
};

template <typename TV, typename TX, int VW, int MODE, int NDOT>
__global__ void __launch_bounds__(kBlock) sell_step_tma_kernel(int n, long long nslices,
                                                               const long long* __restrict__ sptr,
                                                               const int* __restrict__ col,
                                                               const TV* __restrict__ val, StepArgs<TX> a,
                                                               const Scalars* sc, double* partials,
                                                               unsigned int* counter) {
  using S = TmaStage<TV, TX, VW, MODE>;
  constexpr int C = S::C;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kBlock / 32][kTmaStages];
  if (sc && load_done(sc)) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned char* wsm = smem_raw + (size_t)wid * kTmaStages * S::kBytes;
  if (lane == 0) {
#pragma unroll
    for (int b = 0; b < kTmaStages; ++b) mbar_init(&bars[wid][b], 1);
    mbar_fence_init();
  }
  __syncwarp();
  const long long wpb = blockDim.x >> 5;
  const long long gw = (long long)blockIdx.x * wpb + wid;
  const long long nw = (long long)gridDim.x * wpb;
  const uint64_t pol_stream = policy_evict_first();
  const uint64_t pol_keep = policy_evict_last();
  const bool has_xo = mode_needs_xold<MODE>() && (MODE == kChebK || a.xold != nullptr);

  // Stage slice s into buffer b; returns false (nothing issued) when the
  // slice is wider than the staging buffer.
  auto issue = [&](long long s, int b) -> bool {
    const long long base = sptr[s];
    const int w = (int)((sptr[s + 1] - base) / C);
    if (w > kTmaWmax) return false;
    if (lane == 0) {
      unsigned char* st = wsm + b * S::kBytes;
      uint32_t bytes = (uint32_t)(w * C * (int)(sizeof(TV) + 4));
      if constexpr (S::kR > 0) bytes += S::kR;
      if (has_xo) bytes += S::kXo;
      // order this warp's earlier generic reads of buffer b before the
      // async-proxy writes that refill it
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive_expect_tx(&bars[wid][b], bytes);
      if (w > 0) {
        bulk_g2s(st, val + base, (uint32_t)(w * C * (int)sizeof(TV)), &bars[wid][b], pol_stream);
        bulk_g2s(st + S::kVal, col + base, (uint32_t)(w * C * 4), &bars[wid][b], pol_stream);
      }
      if constexpr (S::kR > 0) bulk_g2s(st + S::kVal + S::kCol, a.r + s * C, S::kR, &bars[wid][b], pol_keep);
      if constexpr (S::kXo > 0) {
        if (has_xo) bulk_g2s(st + S::kVal + S::kCol + S::kR, a.xold + s * C, S::kXo, &bars[wid][b], pol_stream);
      }
    }
    return true;
  };

  double dot[NDOT > 0 ? NDOT : 1];
#pragma unroll
  for (int i = 0; i < (NDOT > 0 ? NDOT : 1); ++i) dot[i] = 0.0;
  const TX lan = lanczos_coef<TX, MODE>(a);
  uint32_t phase = 0u;     // bit b: parity of the next completion of buffer b
  uint32_t inflight = 0u;  // bit b: buffer b has a copy in flight
  int b = 0;
  bool ok = true;
  long long s = gw;
  if (s < nslices && issue(s, 0)) inflight |= 1u;
  bool staged_cur = (inflight & 1u) != 0;
  for (; s < nslices && ok; s += nw) {
    const long long sn = s + nw;
    bool staged_next = false;
    if (sn < nslices) {
      staged_next = issue(sn, b ^ 1);
      if (staged_next) inflight |= 1u << (b ^ 1);
    }
    const long long base = sptr[s];
    const int w = (int)((sptr[s + 1] - base) / C);
    unsigned char* st = wsm + b * S::kBytes;
    TX acc[VW];
    if (staged_cur) {
      if (!mbar_wait_bounded(&bars[wid][b], (phase >> b) & 1u)) {
        ok = false;
        break;
      }
      phase ^= 1u << b;
      inflight &= ~(1u << b);
      slice_rowsums<TV, TX, VW, true>(reinterpret_cast<const TV*>(st) + lane * VW,
                                      reinterpret_cast<const int*>(st + S::kVal) + lane * VW, w, a.x, acc);
    } else {
      slice_rowsums<TV, TX, VW, false>(val + base + lane * VW, col + base + lane * VW, w, a.x, acc);
    }
    const TX* r_s = reinterpret_cast<const TX*>(st + S::kVal + S::kCol);
    const TX* xo_s = reinterpret_cast<const TX*>(st + S::kVal + S::kCol + S::kR);
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      const int lr = e * 32 + lane;
      const long long row = s * C + lr;
      TX xs = (TX)0, rs = (TX)0, xo = (TX)0;
      if constexpr (mode_needs_xown<MODE, NDOT>()) xs = __ldg(a.x + row);
      if constexpr (mode_needs_r<MODE>()) rs = staged_cur ? r_s[lr] : a.r[row];
      if constexpr (mode_needs_xold<MODE>()) {
        if (has_xo) xo = staged_cur ? xo_s[lr] : a.xold[row];
      }
      const TX y = row_value<TX, MODE>(a, acc[e], xs, rs, xo, lan);
      a.y[row] = y;
      if (row < n) row_dots<TX, MODE, NDOT>(a, row, y, xs, rs, dot);
    }
    __syncwarp();
    b ^= 1;
    staged_cur = staged_next;
  }
  if (!ok) {
    // A staged copy did not arrive in time: record it, wait (bounded) for
    // this warp's copies still in flight so none lands after exit, and still
    // take part in the grid reduction below.
    if (lane == 0 && a.err) atomicExch(a.err, 1);
    for (int bb = 0; bb < kTmaStages; ++bb)
      if ((inflight >> bb) & 1u) mbar_wait_bounded(&bars[wid][bb], (phase >> bb) & 1u);
  }
  finish_dots<TX, NDOT>(a, dot, partials, counter);
}

template <typename TV, typename TX, int G, int MODE, int NDOT>
__global__ void __launch_bounds__(kBlock) csr_step_kernel(int n, const int* __restrict__ rowptr,
                                                          const int* __restrict__ col, const TV* __restrict__ val,
                                                          StepArgs<TX> a, const Scalars* sc, double* partials,
                                                          unsigned int* counter) {
  if (sc && load_done(sc)) return;
  const int sub = threadIdx.x % G;
  const long long rows_per_block = blockDim.x / G;
  double dot[NDOT > 0 ? NDOT : 1];
#pragma unroll
  for (int i = 0; i < (NDOT > 0 ? NDOT : 1); ++i) dot[i] = 0.0;
  const TX lan = lanczos_coef<TX, MODE>(a);
  for (long long rb = (long long)blockIdx.x * rows_per_block; rb < n; rb += (long long)gridDim.x * rows_per_block) {
    const long long row = rb + threadIdx.x / G;
    TX acc = (TX)0;
    if (row < n) {
      const int beg = rowptr[row], end = rowptr[row + 1];
      for (int p = beg + sub; p < end; p += G) {
        TX v[1];
        ValLd<TV, 1, TX>::ld(val + p, v);
        acc = fma(v[0], __ldg(a.x + __ldcs(col + p)), acc);
      }
    }
    if constexpr (G > 1) {
      // fixed-order tree over the G lanes of the row group
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o, G);
    }
    if (sub == 0 && row < n) {
      TX xs = (TX)0, rs = (TX)0, xo = (TX)0;
      if constexpr (mode_needs_xown<MODE, NDOT>()) xs = __ldg(a.x + row);
      if constexpr (mode_needs_r<MODE>()) rs = a.r[row];
      if constexpr (mode_needs_xold<MODE>()) {
        if (MODE == kChebK || a.xold) xo = a.xold[row];
      }
      const TX y = row_value<TX, MODE>(a, acc, xs, rs, xo, lan);
      a.y[row] = y;
      row_dots<TX, MODE, NDOT>(a, row, y, xs, rs, dot);
    }
  }
  finish_dots<TX, NDOT>(a, dot, partials, counter);
}

template <typename TX>
StepArgs<TX> make_args(const StepParams& p) {
  StepArgs<TX> a;
  a.x = static_cast<const TX*>(p.x);
  a.xold = static_cast<const TX*>(p.xold);
  a.r = static_cast<const TX*>(p.r);
  a.y = static_cast<TX*>(p.y);
  a.aux = p.aux;
  a.dev_coef = p.dev_coef;
  a.ca = (TX)p.ca;
  a.cb = (TX)p.cb;
  a.cc = (TX)p.cc;
  a.cd = (TX)p.cd;
  a.ce = (TX)p.ce;
  a.out0 = p.dot_out0;
  a.out1 = p.dot_out1;
  a.err = p.err;
  return a;
}

template <typename TV, typename TX, int VW, int MODE, int NDOT>
cudaError_t go_sell(const MatDesc& A, const StepParams& p, const Scalars* sc, double* partials, unsigned int* cnt,
                    int grid, cudaStream_t s) {
  if (A.tma) {
    using S = TmaStage<TV, TX, VW, MODE>;
    auto kern = sell_step_tma_kernel<TV, TX, VW, MODE, NDOT>;
    // the attribute belongs to the function on one device: set it once per
    // instantiation and device
    static bool attr_set[kMaxDevices] = {false};
    const int dev = current_device();
    if (!attr_set[dev]) {
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, S::kBlockBytes);
      if (e != cudaSuccess) return e;
      attr_set[dev] = true;
    }
    kern<<<grid, kBlock, S::kBlockBytes, s>>>(A.n, A.nslices, A.slice_ptr, A.col, static_cast<const TV*>(A.val),
                                             make_args<TX>(p), sc, partials, cnt);
  } else {
    sell_step_kernel<TV, TX, VW, MODE, NDOT><<<grid, kBlock, 0, s>>>(
        A.n, A.nslices, A.slice_ptr, A.col, static_cast<const TV*>(A.val), make_args<TX>(p), sc, partials, cnt);
  }
  return cudaGetLastError();
}

template <typename TV, typename TX, int G, int MODE, int NDOT>
cudaError_t go_csr(const MatDesc& A, const StepParams& p, const Scalars* sc, double* partials, unsigned int* cnt,
                   int grid, cudaStream_t s) {
  csr_step_kernel<TV, TX, G, MODE, NDOT><<<grid, kBlock, 0, s>>>(A.n, A.rowptr, A.col, static_cast<const TV*>(A.val),
                                                                 make_args<TX>(p), sc, partials, cnt);
  return cudaGetLastError();
}

// Only the (mode, ndot) pairs the driver uses are instantiated; FP32/BF16
// matrices serve the preconditioner steps only.
template <typename TX, int MODE, int NDOT>
__host__ __device__ constexpr bool step_variant_used() {
  if constexpr (std::is_same<TX, double>::value) {
    if (MODE == kSpmv) return NDOT <= 1;
    if (MODE == kResid || MODE == kLanczos) return NDOT == 1;
    return true;
  } else {
    return (MODE == kCheb1 || MODE == kCheb2 || MODE == kChebK) && NDOT == 0;
  }
}

template <typename TV, typename TX, int MODE, int NDOT>
cudaError_t dispatch_fmt(const MatDesc& A, const StepParams& p, const Scalars* sc, double* partials, unsigned int* cnt,
                         int grid, cudaStream_t s) {
  if constexpr (!step_variant_used<TX, MODE, NDOT>()) {
    return cudaErrorNotSupported;
  } else {
    if (A.format == 2) {
      const int vw = A.C / 32;
      if (vw == 1) return go_sell<TV, TX, 1, MODE, NDOT>(A, p, sc, partials, cnt, grid, s);
      if (vw == 2) return go_sell<TV, TX, 2, MODE, NDOT>(A, p, sc, partials, cnt, grid, s);
      if (vw == 4) return go_sell<TV, TX, 4, MODE, NDOT>(A, p, sc, partials, cnt, grid, s);
      return cudaErrorInvalidValue;
    }
    switch (A.csr_group) {
      case 1: return go_csr<TV, TX, 1, MODE, NDOT>(A, p, sc, partials, cnt, grid, s);
      case 8: return go_csr<TV, TX, 8, MODE, NDOT>(A, p, sc, partials, cnt, grid, s);
      case 32: return go_csr<TV, TX, 32, MODE, NDOT>(A, p, sc, partials, cnt, grid, s);
      default: return cudaErrorInvalidValue;
    }
  }
}

template <typename TV, typename TX, int MODE>
cudaError_t dispatch_ndot(const MatDesc& A, const StepParams& p, const Scalars* sc, double* partials,
                          unsigned int* cnt, int grid, cudaStream_t s) {
  switch (p.ndot) {
    case 0: return dispatch_fmt<TV, TX, MODE, 0>(A, p, sc, partials, cnt, grid, s);
    case 1: return dispatch_fmt<TV, TX, MODE, 1>(A, p, sc, partials, cnt, grid, s);
    case 2: return dispatch_fmt<TV, TX, MODE, 2>(A, p, sc, partials, cnt, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename TV, typename TX>
cudaError_t dispatch_mode(const MatDesc& A, const StepParams& p, const Scalars* sc, double* partials,
                          unsigned int* cnt, int grid, cudaStream_t s) {
  switch (p.mode) {
    case kSpmv: return dispatch_ndot<TV, TX, kSpmv>(A, p, sc, partials, cnt, grid, s);
    case kResid: return dispatch_ndot<TV, TX, kResid>(A, p, sc, partials, cnt, grid, s);
    case kCheb1: return dispatch_ndot<TV, TX, kCheb1>(A, p, sc, partials, cnt, grid, s);
    case kCheb2: return dispatch_ndot<TV, TX, kCheb2>(A, p, sc, partials, cnt, grid, s);
    case kChebK: return dispatch_ndot<TV, TX, kChebK>(A, p, sc, partials, cnt, grid, s);
    case kLanczos: return dispatch_ndot<TV, TX, kLanczos>(A, p, sc, partials, cnt, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace pp
