// Fused degree-step kernels on the symmetric diagonal (DIA) storage: the
// same modes and fused inner products as the SELL/CSR kernels
// (step_impl.cuh), for matrices whose nonzeros lie on a few diagonals --
// the 7-point stencil of a structured 3-D grid has 4 stored diagonals
// (offsets 0, 1, N, N^2).  No column indices are stored, and of each pair
// of symmetric off-diagonals only the upper one: row i reads its upper
// entries at position i of each diagonal and its lower entries at position
// i - offset, which another thread of the same sweep has just read, so the
// second read is served by L2.  Consecutive row groups on consecutive
// lanes: every stream is coalesced.
#include "step_dia.cuh"

namespace pp {
namespace {

template <typename TV, typename TX>
__device__ __forceinline__ TX ldv(const TV* p) {
  if constexpr (std::is_same<TV, __nv_bfloat16>::value) {
    const unsigned short u = __ldg(reinterpret_cast<const unsigned short*>(p));
    return (TX)__uint_as_float(((unsigned int)u) << 16);
  } else {
    return (TX)__ldg(p);
  }
}

// R consecutive rows per thread (R = 4 for FP64, 2 for FP32/BF16, the
// fastest of R in {2, 4, 8} at 192^3): the
// aligned streams (the stored diagonals at the thread's rows, its own x, r,
// x_old and y) move as one vector access each, and the thread keeps R times
// more loads in flight.  (Aligned vector loads of the partners at offsets
// that are multiples of R, and lane shuffles for offset 1, measured slower:
// they doubled the registers per thread and cost occupancy.)  Rows run over [0, n_pad): padding rows have zero
// entries and zero vectors, so they produce y = 0 and add nothing to the
// inner products.
template <typename T, int R>
struct Vec;
template <>
struct Vec<double, 2> {
  __device__ static void ld(const double* p, double (&o)[2]) {
    const double2 t = __ldg(reinterpret_cast<const double2*>(p));
    o[0] = t.x;
    o[1] = t.y;
  }
  __device__ static void st(double* p, const double (&v)[2]) { *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]); }
};
template <>
struct Vec<double, 4> {
  __device__ static void ld(const double* p, double (&o)[4]) {
    const double2 t0 = __ldg(reinterpret_cast<const double2*>(p));
    const double2 t1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
    o[0] = t0.x;
    o[1] = t0.y;
    o[2] = t1.x;
    o[3] = t1.y;
  }
  __device__ static void st(double* p, const double (&v)[4]) {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
};
template <>
struct Vec<float, 2> {
  __device__ static void ld(const float* p, float (&o)[2]) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    o[0] = t.x;
    o[1] = t.y;
  }
  __device__ static void st(float* p, const float (&v)[2]) { *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]); }
};
template <>
struct Vec<float, 8> {
  __device__ static void ld(const float* p, float (&o)[8]) {
    const float4 t0 = __ldg(reinterpret_cast<const float4*>(p));
    const float4 t1 = __ldg(reinterpret_cast<const float4*>(p) + 1);
    o[0] = t0.x;
    o[1] = t0.y;
    o[2] = t0.z;
    o[3] = t0.w;
    o[4] = t1.x;
    o[5] = t1.y;
    o[6] = t1.z;
    o[7] = t1.w;
  }
  __device__ static void st(float* p, const float (&v)[8]) {
    reinterpret_cast<float4*>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
    reinterpret_cast<float4*>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
  }
};
template <>
struct Vec<float, 4> {
  __device__ static void ld(const float* p, float (&o)[4]) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = t.x;
    o[1] = t.y;
    o[2] = t.z;
    o[3] = t.w;
  }
  __device__ static void st(float* p, const float (&v)[4]) {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <typename TV, typename TX, int R>
__device__ __forceinline__ void ldvals(const TV* p, TX (&o)[R]) {
  if constexpr (std::is_same<TV, __nv_bfloat16>::value) {
    if constexpr (R == 2) {
      const unsigned int u = __ldg(reinterpret_cast<const unsigned int*>(p));
      o[0] = (TX)bf16_lo(u);
      o[1] = (TX)bf16_hi(u);
    } else if constexpr (R == 4) {
      const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
      o[0] = (TX)bf16_lo(u.x);
      o[1] = (TX)bf16_hi(u.x);
      o[2] = (TX)bf16_lo(u.y);
      o[3] = (TX)bf16_hi(u.y);
    } else {
      const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
      const unsigned int w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        o[2 * q] = (TX)bf16_lo(w[q]);
        o[2 * q + 1] = (TX)bf16_hi(w[q]);
      }
    }
  } else {
    Vec<TX, R>::ld(p, o);
  }
}

// Loads with an L2 eviction priority, for the FP32/BF16 steps (2 rows per
// thread): the stored diagonals stream through once per step (evict first),
// while r is read by every step of an application and x, x_old are the two
// previous steps' outputs, so the vectors stay in L2 between steps when the
// matrix does not push them out.
template <typename TV>
__device__ __forceinline__ void ld2_hint(const TV* p, float (&o)[2], uint64_t pol) {
  if constexpr (std::is_same<TV, __nv_bfloat16>::value) {
    unsigned int u;
    asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(u) : "l"(p), "l"(pol));
    o[0] = bf16_lo(u);
    o[1] = bf16_hi(u);
  } else {
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(o[0]), "=f"(o[1]) : "l"(p), "l"(pol));
  }
}
template <typename TV>
__device__ __forceinline__ float ld1_hint(const TV* p, uint64_t pol) {
  if constexpr (std::is_same<TV, __nv_bfloat16>::value) {
    unsigned short u;
    asm("ld.global.nc.L2::cache_hint.b16 %0, [%1], %2;" : "=h"(u) : "l"(p), "l"(pol));
    return __uint_as_float(((unsigned int)u) << 16);
  } else {
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
  }
}

// ND > 0: that many stored diagonals, unrolled, the main one first unless
// UNIT; ND = 0: d.nd and d.unit at run time.  UNIT (the Jacobi-scaled matrix,
// whose diagonal is 1 by construction) starts each row sum from x_i and
// saves one multiply per row and one stored diagonal.
template <typename TV, typename TX, int R, int ND, int MODE, int NDOT, bool UNIT = false>
__global__ void __launch_bounds__(kBlock) dia_step_kernel(DiaArgs d, const TV* __restrict__ val, StepArgs<TX> a,
                                                          const Scalars* sc, double* partials,
                                                          unsigned int* counter) {
  if (sc && load_done(sc)) return;
  double dot[NDOT > 0 ? NDOT : 1];
#pragma unroll
  for (int i = 0; i < (NDOT > 0 ? NDOT : 1); ++i) dot[i] = 0.0;
  const TX lan = lanczos_coef<TX, MODE>(a);
  const int nd = ND > 0 ? ND : d.nd;
  const long long last = d.n_pad - 1;
  const TV* base = val + d.dpad;
  // Folded form of the recurrence steps with the unit diagonal:
  //   kChebK  y = ca x + cb x_old + cc (r - x - S x) = cc (u - S x),
  //           u = r + (ca/cc - 1) x + (cb/cc) x_old;
  //   kCheb2  y = ca x + cb r + cc (r - x - S x) = cc (u - S x),
  //           u = (ca/cc - 1) x + (cb/cc + 1) r,
  // S the off-diagonal part (a.cd, a.ce hold the folded ratios).  The row
  // sum starts from u, so a row costs 2 + 2 nd + 1 FP64 operations (9 for
  // the 7-point stencil) instead of 2 nd + 4.
  constexpr bool kFold = ND > 0 && UNIT && (MODE == kChebK || MODE == kCheb2);
  constexpr bool kHint = std::is_same<TX, float>::value && R == 2;  // L2 priorities (see ld2_hint)
  uint64_t pol_first = 0, pol_last = 0;
  if constexpr (kHint) {
    pol_first = policy_evict_first();
    pol_last = policy_evict_last();
  }
  for (long long i0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * R; i0 < d.n_pad;
       i0 += (long long)gridDim.x * blockDim.x * R) {
    TX xs[R], acc[R], u[R];
    Vec<TX, R>::ld(a.x + i0, xs);
    if constexpr (kFold) {
      TX rs[R], xo[R], y[R];
      if constexpr (kHint)
        ld2_hint<float>(reinterpret_cast<const float*>(a.r + i0), reinterpret_cast<float(&)[2]>(rs), pol_last);
      else
        Vec<TX, R>::ld(a.r + i0, rs);
      if constexpr (MODE == kChebK) {
        Vec<TX, R>::ld(a.xold + i0, xo);
#pragma unroll
        for (int e = 0; e < R; ++e) acc[e] = fma(a.ce, xo[e], fma(a.cd, xs[e], rs[e]));
      } else {
#pragma unroll
        for (int e = 0; e < R; ++e) acc[e] = fma(a.cd, xs[e], a.ce * rs[e]);
      }
#pragma unroll
      for (int t = 0; t < ND; ++t) {
        const long long o = d.doff[t];
        const TV* vt = base + (long long)t * d.dstride;
        if constexpr (kHint)
          ld2_hint<TV>(vt + i0, reinterpret_cast<float(&)[2]>(u), pol_first);
        else
          ldvals<TV, TX, R>(vt + i0, u);
#pragma unroll
        for (int e = 0; e < R; ++e) {
          const long long i = i0 + e;
          TX lo;
          if constexpr (kHint)
            lo = ld1_hint<TV>(vt + i - o, pol_first);
          else
            lo = ldv<TV, TX>(vt + i - o);
          const long long ju = i + o < last ? i + o : last;
          const long long jl = i - o > 0 ? i - o : 0;
          acc[e] = fma(-u[e], __ldg(a.x + ju), acc[e]);
          acc[e] = fma(-lo, __ldg(a.x + jl), acc[e]);
        }
      }
#pragma unroll
      for (int e = 0; e < R; ++e) {
        y[e] = a.cc * acc[e];
        row_dots<TX, MODE, NDOT>(a, i0 + e, y[e], xs[e], rs[e], dot);
      }
      Vec<TX, R>::st(a.y + i0, y);
      continue;
    }
    const bool unit = ND > 0 ? UNIT : (d.unit != 0);
    if (unit) {
#pragma unroll
      for (int e = 0; e < R; ++e) acc[e] = xs[e];
    } else {
      ldvals<TV, TX, R>(base + i0, u);
#pragma unroll
      for (int e = 0; e < R; ++e) acc[e] = u[e] * xs[e];
    }
#pragma unroll
    for (int t = (ND > 0 ? (UNIT ? 0 : 1) : 0); t < (ND > 0 ? ND : kMaxDiag); ++t) {
      if (ND == 0 && (t >= nd || (t == 0 && !unit))) {
        if (t >= nd) break;
        continue;
      }
      const long long o = d.doff[t];
      const TV* vt = base + (long long)t * d.dstride;
      if constexpr (kHint)  // a(i, i + o); 0 past the last row
        ld2_hint<TV>(vt + i0, reinterpret_cast<float(&)[2]>(u), pol_first);
      else
        ldvals<TV, TX, R>(vt + i0, u);
#pragma unroll
      for (int e = 0; e < R; ++e) {
        const long long i = i0 + e;
        TX lo;  // a(i - o, i) = a(i, i - o); 0 in the front pad
        if constexpr (kHint)
          lo = ld1_hint<TV>(vt + i - o, pol_first);
        else
          lo = ldv<TV, TX>(vt + i - o);
        const long long ju = i + o < last ? i + o : last;
        const long long jl = i - o > 0 ? i - o : 0;
        acc[e] = fma(u[e], __ldg(a.x + ju), acc[e]);
        acc[e] = fma(lo, __ldg(a.x + jl), acc[e]);
      }
    }
    TX rs[R], xo[R], y[R];
#pragma unroll
    for (int e = 0; e < R; ++e) rs[e] = xo[e] = (TX)0;
    if constexpr (mode_needs_r<MODE>()) {
      if constexpr (kHint)
        ld2_hint<float>(reinterpret_cast<const float*>(a.r + i0), reinterpret_cast<float(&)[2]>(rs), pol_last);
      else
        Vec<TX, R>::ld(a.r + i0, rs);
    }
    if constexpr (mode_needs_xold<MODE>()) {
      if (MODE == kChebK || a.xold) Vec<TX, R>::ld(a.xold + i0, xo);
    }
#pragma unroll
    for (int e = 0; e < R; ++e) {
      y[e] = row_value<TX, MODE>(a, acc[e], xs[e], rs[e], xo[e], lan);
      row_dots<TX, MODE, NDOT>(a, i0 + e, y[e], xs[e], rs[e], dot);
    }
    Vec<TX, R>::st(a.y + i0, y);
  }
  finish_dots<TX, NDOT>(a, dot, partials, counter);
}

// Whole resident waves per launch: the grid-stride loops split the rows evenly
// over the blocks, so a grid that is not a whole number of waves leaves a
// partly filled last wave.  The variants differ in registers (the ones that
// reduce inner products hold more), hence in resident blocks per SM, so the
// grid is taken per instantiation, capped by the caller's grid.
constexpr int kWaves = 2;  // resident waves per launch (measured: 2 beats 1 and equals 3)

template <typename TV, typename TX, int R, int ND, int MODE, int NDOT, bool UNIT = false>
int wave_grid(int cap) {
  static int blocks[kMaxDevices] = {0};  // per kernel instantiation and device
  const int dev = current_device();
  if (blocks[dev] == 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dia_step_kernel<TV, TX, R, ND, MODE, NDOT, UNIT>,
                                                      kBlock, 0) != cudaSuccess ||
        per_sm <= 0)
      per_sm = 1;
    blocks[dev] = num_sms() * per_sm * kWaves;
  }
  return blocks[dev] < cap ? blocks[dev] : cap;
}


template <typename TV, typename TX, int MODE, int NDOT>
cudaError_t go_dia(const MatDesc& A, const StepParams& p, const Scalars* sc, double* partials, unsigned int* cnt,
                   int grid, cudaStream_t s) {
  if constexpr (!step_variant_used<TX, MODE, NDOT>()) {
    return cudaErrorNotSupported;
  } else {
    if constexpr (std::is_same<TX, float>::value && NDOT == 0 &&
                  (MODE == kCheb1 || MODE == kCheb2 || MODE == kChebK)) {
      if (A.tma == 2 && dia_tma_applies(A)) return launch_step_dia_tma(A, p, sc, grid, s);
      if (A.tma == 3 && dia_z_applies(A)) return launch_step_dia_z(A, p, sc, grid, s);
    }
    constexpr int R = std::is_same<TX, double>::value ? 4 : 2;
    const TV* v = static_cast<const TV*>(A.val);
    if (A.ndiag == 3 && A.dia_unit) {  // Jacobi-scaled 7-point stencil
      StepArgs<TX> args = make_args<TX>(p);
      if (MODE == kChebK || MODE == kCheb2) {  // folded coefficients (see dia_step_kernel)
        args.cd = (TX)(p.ca / p.cc - 1.0);
        args.ce = (TX)(MODE == kChebK ? p.cb / p.cc : p.cb / p.cc + 1.0);
      }
      dia_step_kernel<TV, TX, R, 3, MODE, NDOT, true><<<wave_grid<TV, TX, R, 3, MODE, NDOT, true>(grid), kBlock, 0,
                                                         s>>>(dia_args(A), v, args, sc, partials, cnt);
    }
    else if (A.ndiag == 4 && !A.dia_unit)
      dia_step_kernel<TV, TX, R, 4, MODE, NDOT><<<wave_grid<TV, TX, R, 4, MODE, NDOT>(grid), kBlock, 0, s>>>(
          dia_args(A), v, make_args<TX>(p), sc, partials, cnt);
    else
      dia_step_kernel<TV, TX, R, 0, MODE, NDOT><<<wave_grid<TV, TX, R, 0, MODE, NDOT>(grid), kBlock, 0, s>>>(
          dia_args(A), v, make_args<TX>(p), sc, partials, cnt);
    return cudaGetLastError();
  }
}

template <typename TV, typename TX, int MODE>
cudaError_t dia_ndot(const MatDesc& A, const StepParams& p, const Scalars* sc, double* partials, unsigned int* cnt,
                     int grid, cudaStream_t s) {
  switch (p.ndot) {
    case 0: return go_dia<TV, TX, MODE, 0>(A, p, sc, partials, cnt, grid, s);
    case 1: return go_dia<TV, TX, MODE, 1>(A, p, sc, partials, cnt, grid, s);
    case 2: return go_dia<TV, TX, MODE, 2>(A, p, sc, partials, cnt, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename TV, typename TX>
cudaError_t dia_mode(const MatDesc& A, const StepParams& p, const Scalars* sc, double* partials, unsigned int* cnt,
                     int grid, cudaStream_t s) {
  switch (p.mode) {
    case kSpmv: return dia_ndot<TV, TX, kSpmv>(A, p, sc, partials, cnt, grid, s);
    case kResid: return dia_ndot<TV, TX, kResid>(A, p, sc, partials, cnt, grid, s);
    case kCheb1: return dia_ndot<TV, TX, kCheb1>(A, p, sc, partials, cnt, grid, s);
    case kCheb2: return dia_ndot<TV, TX, kCheb2>(A, p, sc, partials, cnt, grid, s);
    case kChebK: return dia_ndot<TV, TX, kChebK>(A, p, sc, partials, cnt, grid, s);
    case kLanczos: return dia_ndot<TV, TX, kLanczos>(A, p, sc, partials, cnt, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_step_dia(const MatDesc& A, const StepParams& p, const Scalars* sc, double* partials,
                            unsigned int* counter, int grid, cudaStream_t s) {
  if (A.ndiag < 0 || A.ndiag > kMaxDiag || (A.ndiag == 0 && !A.dia_unit)) return cudaErrorInvalidValue;
  if (A.prec == kF64) return dia_mode<double, double>(A, p, sc, partials, counter, grid, s);
  if (A.prec == kF32) return dia_mode<float, float>(A, p, sc, partials, counter, grid, s);
  return dia_mode<__nv_bfloat16, float>(A, p, sc, partials, counter, grid, s);
}

// DIA launches size their own grid per variant (wave_grid); the caller's grid
// is only the cap, so no occupancy figure is needed here.
int step_blocks_per_sm_dia(const MatDesc& A) {
  (void)A;
  return 16;
}

}  // namespace pp
