// Fused degree-step kernels: one pass over the matrix computes A x and the
// Chebyshev three-term update of Algorithm 2 (or a plain product, a
// residual, a Lanczos step), with optional fused inner products.
//
// SELL-C-sigma: one warp per slice of C = 32*VW rows; lane l owns rows
// l*VW .. l*VW+VW-1 of the slice, so every matrix load of the warp is one
// contiguous 32*VW-element segment (16-byte loads for FP64 VW=2 / FP32 VW=4).
// Matrix streams use evict-first loads; the gathered vector goes through the
// read-only path and is expected to hit in L2.
//
// CSR: G lanes per row, strided over the row, reduced by warp shuffles.
#pragma once

#include <type_traits>

#include "kernels.cuh"

namespace pp {
namespace {

// ---------------------------------------------------------------- loads ----
template <typename TV, int VW, typename TA>
struct ValLd;
template <typename TA>
struct ValLd<double, 1, TA> {
  __device__ static void ld(const double* p, TA (&o)[1]) { o[0] = (TA)__ldcs(p); }
};
template <typename TA>
struct ValLd<double, 2, TA> {
  __device__ static void ld(const double* p, TA (&o)[2]) {
    double2 t = __ldcs(reinterpret_cast<const double2*>(p));
    o[0] = (TA)t.x;
    o[1] = (TA)t.y;
  }
};
template <typename TA>
struct ValLd<float, 1, TA> {
  __device__ static void ld(const float* p, TA (&o)[1]) { o[0] = (TA)__ldcs(p); }
};
template <typename TA>
struct ValLd<float, 2, TA> {
  __device__ static void ld(const float* p, TA (&o)[2]) {
    float2 t = __ldcs(reinterpret_cast<const float2*>(p));
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
};
__device__ __forceinline__ float bf16_lo(unsigned int u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16_hi(unsigned int u) { return __uint_as_float(u & 0xffff0000u); }
template <typename TA>
struct ValLd<__nv_bfloat16, 1, TA> {
  __device__ static void ld(const __nv_bfloat16* p, TA (&o)[1]) {
    unsigned short u = __ldcs(reinterpret_cast<const unsigned short*>(p));
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
};

template <int VW>
__device__ __forceinline__ void col_ld(const int* p, int (&o)[VW]);
template <>
__device__ __forceinline__ void col_ld<1>(const int* p, int (&o)[1]) { o[0] = __ldcs(p); }
template <>
__device__ __forceinline__ void col_ld<2>(const int* p, int (&o)[2]) {
  int2 t = __ldcs(reinterpret_cast<const int2*>(p));
  o[0] = t.x;
  o[1] = t.y;
}
template <>
__device__ __forceinline__ void col_ld<4>(const int* p, int (&o)[4]) {
  int4 t = __ldcs(reinterpret_cast<const int4*>(p));
  o[0] = t.x;
  o[1] = t.y;
  o[2] = t.z;
  o[3] = t.w;
}

// VW consecutive vector entries (aligned: rows are multiples of VW).
template <typename TX, int VW>
struct VecLd;
template <int VW>
struct VecLd<double, VW> {
  __device__ static void ld(const double* p, double (&o)[VW]) {
    if constexpr (VW == 1) {
      o[0] = __ldcs(p);
    } else {
      double2 t = __ldcs(reinterpret_cast<const double2*>(p));
      o[0] = t.x;
      o[1] = t.y;
    }
  }
  __device__ static void st(double* p, const double (&v)[VW]) {
    if constexpr (VW == 1) {
      p[0] = v[0];
    } else {
      *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    }
  }
};
template <int VW>
struct VecLd<float, VW> {
  __device__ static void ld(const float* p, float (&o)[VW]) {
    if constexpr (VW == 1) {
      o[0] = __ldcs(p);
    } else if constexpr (VW == 2) {
      float2 t = __ldcs(reinterpret_cast<const float2*>(p));
      o[0] = t.x;
      o[1] = t.y;
    } else {
      float4 t = __ldcs(reinterpret_cast<const float4*>(p));
      o[0] = t.x;
      o[1] = t.y;
      o[2] = t.z;
      o[3] = t.w;
    }
  }
  __device__ static void st(float* p, const float (&v)[VW]) {
    if constexpr (VW == 1) {
      p[0] = v[0];
    } else if constexpr (VW == 2) {
      *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
    } else {
      *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
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
};

// Epilogue shared by both formats: acc = (A x)_row for VW rows at row0.
template <typename TX, int VW, int MODE, int NDOT>
__device__ __forceinline__ void epilogue(const StepArgs<TX>& a, long long row0, int n, const TX (&acc)[VW],
                                         TX lan_coef, double (&dot)[NDOT > 0 ? NDOT : 1]) {
  TX y[VW];
  TX xs[VW], rs[VW], xo[VW];
  if constexpr (MODE == kSpmv) {
#pragma unroll
    for (int e = 0; e < VW; ++e) y[e] = acc[e];
    if constexpr (NDOT > 0) VecLd<TX, VW>::ld(a.x + row0, xs);
  } else if constexpr (MODE == kResid) {
    VecLd<TX, VW>::ld(a.r + row0, rs);
#pragma unroll
    for (int e = 0; e < VW; ++e) y[e] = rs[e] - acc[e];
  } else if constexpr (MODE == kCheb1) {
    VecLd<TX, VW>::ld(a.r + row0, rs);
#pragma unroll
    for (int e = 0; e < VW; ++e) y[e] = a.ca * ((TX)2 * rs[e] - acc[e] * a.ce);
  } else if constexpr (MODE == kCheb2) {
    VecLd<TX, VW>::ld(a.x + row0, xs);
    VecLd<TX, VW>::ld(a.r + row0, rs);
#pragma unroll
    for (int e = 0; e < VW; ++e)
      y[e] = a.ca * (a.cb * xs[e] - a.cc * (rs[e] * a.ce) + a.cd * (rs[e] - acc[e]));
  } else if constexpr (MODE == kChebK) {
    VecLd<TX, VW>::ld(a.x + row0, xs);
    VecLd<TX, VW>::ld(a.xold + row0, xo);
    VecLd<TX, VW>::ld(a.r + row0, rs);
#pragma unroll
    for (int e = 0; e < VW; ++e) y[e] = a.ca * (a.cb * xs[e] - a.cc * xo[e] + a.cd * (rs[e] - acc[e]));
  } else {  // kLanczos
    VecLd<TX, VW>::ld(a.x + row0, xs);
    if (a.xold) {
      VecLd<TX, VW>::ld(a.xold + row0, xo);
    } else {
#pragma unroll
      for (int e = 0; e < VW; ++e) xo[e] = (TX)0;
    }
#pragma unroll
    for (int e = 0; e < VW; ++e) y[e] = acc[e] - lan_coef * xo[e];
  }
  VecLd<TX, VW>::st(a.y + row0, y);
  if constexpr (NDOT > 0) {
#pragma unroll
    for (int e = 0; e < VW; ++e) {
      if (row0 + e < n) {
        double yd = (double)y[e];
        if constexpr (MODE == kSpmv || MODE == kLanczos) {
          dot[0] += (double)xs[e] * yd;
        } else if constexpr (MODE == kResid) {
          dot[0] += yd * yd;
          if constexpr (NDOT > 1) dot[1] += (double)rs[e] * (double)rs[e];
        } else {
          dot[0] += (double)rs[e] * yd;
          if constexpr (NDOT > 1) dot[1] += __ldg(a.aux + row0 + e) * yd;
        }
      }
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

template <typename TV, typename TX, int VW, int MODE, int NDOT>
__global__ void __launch_bounds__(kBlock) sell_step_kernel(int n, long long nslices, const long long* __restrict__ sptr,
                                                           const int* __restrict__ col, const TV* __restrict__ val,
                                                           StepArgs<TX> a, const Scalars* sc, double* partials,
                                                           unsigned int* counter) {
  if (sc && load_done(sc)) return;
  constexpr int C = 32 * VW;
  constexpr int CH = VW == 1 ? 8 : 4;  // matrix entries per row loaded per batch
  const int lane = threadIdx.x & 31;
  const long long wpb = blockDim.x >> 5;
  const long long gw = (long long)blockIdx.x * wpb + (threadIdx.x >> 5);
  const long long nw = (long long)gridDim.x * wpb;
  double dot[NDOT > 0 ? NDOT : 1];
#pragma unroll
  for (int i = 0; i < (NDOT > 0 ? NDOT : 1); ++i) dot[i] = 0.0;
  TX lan_coef = (TX)0;
  if constexpr (MODE == kLanczos) {
    if (a.dev_coef) lan_coef = (TX)sqrt(*a.dev_coef);
  }
  const TX* __restrict__ x = a.x;
  for (long long s = gw; s < nslices; s += nw) {
    const long long base = sptr[s];
    const int w = (int)((sptr[s + 1] - base) / C);
    const long long row0 = s * C + lane * VW;
    TX acc[VW];
#pragma unroll
    for (int e = 0; e < VW; ++e) acc[e] = (TX)0;
    const long long off0 = base + lane * VW;
    for (int j0 = 0; j0 < w; j0 += CH) {
      TX v[CH][VW];
      int c[CH][VW];
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        if (j0 + u < w) {
          ValLd<TV, VW, TX>::ld(val + off0 + (long long)(j0 + u) * C, v[u]);
          col_ld<VW>(col + off0 + (long long)(j0 + u) * C, c[u]);
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
    epilogue<TX, VW, MODE, NDOT>(a, row0, n, acc, lan_coef, dot);
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
  TX lan_coef = (TX)0;
  if constexpr (MODE == kLanczos) {
    if (a.dev_coef) lan_coef = (TX)sqrt(*a.dev_coef);
  }
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
      TX accv[1] = {acc};
      epilogue<TX, 1, MODE, NDOT>(a, row, n, accv, lan_coef, dot);
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
  return a;
}

template <typename TV, typename TX, int VW, int MODE, int NDOT>
cudaError_t go_sell(const MatDesc& A, const StepParams& p, const Scalars* sc, double* partials, unsigned int* cnt,
                    int grid, cudaStream_t s) {
  sell_step_kernel<TV, TX, VW, MODE, NDOT><<<grid, kBlock, 0, s>>>(
      A.n, A.nslices, A.slice_ptr, A.col, static_cast<const TV*>(A.val), make_args<TX>(p), sc, partials, cnt);
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
constexpr bool step_variant_used() {
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
    if constexpr (!std::is_same<TX, double>::value) {
      if (vw == 4) return go_sell<TV, TX, 4, MODE, NDOT>(A, p, sc, partials, cnt, grid, s);
    }
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
