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
#include "step_impl.cuh"

namespace pp {
namespace {

struct DiaArgs {
  int nd;
  int unit;  // 1: the main diagonal is 1 and not stored
  int doff[kMaxDiag];
  long long dstride, dpad, n_pad;
};

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
  for (long long i0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) * R; i0 < d.n_pad;
       i0 += (long long)gridDim.x * blockDim.x * R) {
    TX xs[R], acc[R], u[R];
    Vec<TX, R>::ld(a.x + i0, xs);
    if constexpr (kFold) {
      TX rs[R], xo[R], y[R];
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
        ldvals<TV, TX, R>(vt + i0, u);
#pragma unroll
        for (int e = 0; e < R; ++e) {
          const long long i = i0 + e;
          const TX lo = ldv<TV, TX>(vt + i - o);
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
      ldvals<TV, TX, R>(vt + i0, u);  // a(i, i + o); 0 past the last row
#pragma unroll
      for (int e = 0; e < R; ++e) {
        const long long i = i0 + e;
        const TX lo = ldv<TV, TX>(vt + i - o);  // a(i - o, i) = a(i, i - o); 0 in the front pad
        const long long ju = i + o < last ? i + o : last;
        const long long jl = i - o > 0 ? i - o : 0;
        acc[e] = fma(u[e], __ldg(a.x + ju), acc[e]);
        acc[e] = fma(lo, __ldg(a.x + jl), acc[e]);
      }
    }
    TX rs[R], xo[R], y[R];
#pragma unroll
    for (int e = 0; e < R; ++e) rs[e] = xo[e] = (TX)0;
    if constexpr (mode_needs_r<MODE>()) Vec<TX, R>::ld(a.r + i0, rs);
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

// ------------------------------------------ TMA-staged low-precision step ----
// The FP32/BF16 steps move few bytes per row and have little arithmetic, so
// the load latency, not the bandwidth, limits the direct kernel above.  Here
// every stream of a tile of kDT consecutive rows is a contiguous range --
// the 3 stored diagonals at the tile's rows (upper entries) and at the rows
// shifted by -offset (lower entries), x at the tile's rows and shifted by
// +-offset, r and x_old -- so one thread per CTA moves them into shared
// memory with cp.async.bulk (completing on an mbarrier), kDStages tiles
// ahead, and the CTA's threads compute rows from shared memory.  The shifted
// ranges were (or soon will be) read by the tiles they belong to, so they
// come from L2.  Starts are rounded down to 16 bytes (the copy's alignment
// rule) and the vector ranges are clipped to [0, n_pad); a row's neighbour
// index is clipped the same way, where the matrix entry is 0.  The Jacobi-
// scaled 7-point stencil only: 3 upper diagonals, unit main diagonal.
constexpr int kDT = 1024;     // rows per tile
constexpr int kDStages = 3;   // tiles in flight per CTA
constexpr int kDThreads = 256;
constexpr int kDRanges = 15;  // 3 upper + 3 lower value ranges, 7 x ranges, r, x_old

template <typename TV>
struct DiaTma {
  static constexpr int kAV = 16 / (int)sizeof(TV);  // alignment unit of the value ranges (elements)
  static constexpr int kAX = 4;                     // of the FP32 vector ranges
  static constexpr int kUpB = kDT * (int)sizeof(TV);
  // a shifted range of kDT rows spans at most kDT + 2 (alignment unit) - 2
  // elements once its ends are rounded out to 16 bytes
  static constexpr int kLoB = (((kDT + 2 * kAV) * (int)sizeof(TV)) + 127) / 128 * 128;
  static constexpr int kXB = (((kDT + 2 * kAX) * 4) + 127) / 128 * 128;
  static constexpr int kVB = kDT * 4;
  static constexpr int kOffLo = 3 * kUpB;
  static constexpr int kOffX = kOffLo + 3 * kLoB;
  static constexpr int kOffR = kOffX + 7 * kXB;
  static constexpr int kOffXo = kOffR + kVB;
  static constexpr int kStage = kOffXo + kVB;
  static constexpr int kSmem = kStage * kDStages;
};

__device__ __forceinline__ void bulk_g2s_plain(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}

template <typename TV>
__device__ __forceinline__ float smem_val(const unsigned char* p, long long k) {
  if constexpr (std::is_same<TV, __nv_bfloat16>::value)
    return __uint_as_float(((unsigned int)reinterpret_cast<const unsigned short*>(p)[k]) << 16);
  else
    return reinterpret_cast<const float*>(p)[k];
}

template <typename TV, int MODE>
__global__ void __launch_bounds__(kDThreads, 1) dia_step_tma_kernel(DiaArgs d, const TV* __restrict__ val,
                                                                    StepArgs<float> a, const Scalars* sc) {
  using L = DiaTma<TV>;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ __align__(8) uint64_t bars[kDStages];
  __shared__ long long rstart[kDStages][kDRanges];  // row coordinate of each range's first staged element
  if (sc && load_done(sc)) return;
  const long long n_pad = d.n_pad;
  const long long ntiles = (n_pad + kDT - 1) / kDT;
  if (threadIdx.x == 0) {
    for (int b = 0; b < kDStages; ++b) mbar_init(&bars[b], 1);
    mbar_fence_init();
  }
  __syncthreads();
  const bool has_xo = MODE == kChebK;

  // Stage tile `tile` into buffer b (thread 0 only).
  auto issue = [&](long long tile, int b) {
    unsigned char* st = dsm + (size_t)b * L::kStage;
    const long long i0 = tile * kDT;
    const long long len = (n_pad - i0 < kDT) ? n_pad - i0 : kDT;
    const char* vbase = reinterpret_cast<const char*>(val);
    long long src[kDRanges];
    int dst[kDRanges];
    uint32_t nb[kDRanges];
    int nr = 0;
    // upper entries a(i, i + o_t): rows [i0, i0 + len) of diagonal t
    for (int t = 0; t < 3; ++t) {
      const long long e0 = (long long)t * d.dstride + d.dpad + i0;
      src[nr] = e0 * (long long)sizeof(TV);
      dst[nr] = t * L::kUpB;
      nb[nr] = (uint32_t)(len * (long long)sizeof(TV));
      rstart[b][nr++] = i0;
    }
    // lower entries a(i, i - o_t) = a(i - o_t, i): positions [i0 - o_t, i0 - o_t + len)
    for (int t = 0; t < 3; ++t) {
      const long long o = d.doff[t];
      const long long dbeg = (long long)t * d.dstride;  // diagonal t's storage (front pad included)
      const long long dend = dbeg + d.dpad + n_pad;
      long long e0 = dbeg + d.dpad + i0 - o;
      const long long sh = e0 % L::kAV;
      e0 -= sh;
      long long e1 = dbeg + d.dpad + i0 - o + len;
      e1 = (e1 + L::kAV - 1) / L::kAV * L::kAV;
      if (e1 > dend) e1 = dend;
      src[nr] = e0 * (long long)sizeof(TV);
      dst[nr] = L::kOffLo + t * L::kLoB;
      nb[nr] = (uint32_t)((e1 - e0) * (long long)sizeof(TV));
      rstart[b][nr++] = i0 - o - sh;
    }
    // x at the tile's rows and shifted by +-o_t, clipped to [0, n_pad)
    for (int q = 0; q < 7; ++q) {
      const long long sft = q == 0 ? 0 : (q & 1 ? (long long)d.doff[(q - 1) / 2] : -(long long)d.doff[(q - 1) / 2]);
      long long r0 = i0 + sft, r1 = i0 + sft + len;
      if (r0 < 0) r0 = 0;
      if (r1 > n_pad) r1 = n_pad;
      if (r1 <= r0) {  // the whole range lies outside: stage one aligned group at the nearest end
        r0 = sft < 0 ? 0 : n_pad - L::kAX;
        r1 = r0 + L::kAX;
      }
      r0 = r0 / L::kAX * L::kAX;
      r1 = (r1 + L::kAX - 1) / L::kAX * L::kAX;
      src[nr] = -1 - q;  // vector range, resolved below
      dst[nr] = L::kOffX + q * L::kXB;
      nb[nr] = (uint32_t)((r1 - r0) * 4);
      rstart[b][nr++] = r0;
    }
    uint32_t total = 0;
    for (int k = 0; k < nr; ++k) total += nb[k];
    total += (uint32_t)(len * 4);
    if (has_xo) total += (uint32_t)(len * 4);
    // order this CTA's earlier generic reads of buffer b before the refill
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_arrive_expect_tx(&bars[b], total);
    for (int k = 0; k < nr; ++k) {
      const void* g = src[k] >= 0 ? (const void*)(vbase + src[k]) : (const void*)(a.x + rstart[b][k]);
      bulk_g2s_plain(st + dst[k], g, nb[k], &bars[b]);
    }
    bulk_g2s_plain(st + L::kOffR, a.r + i0, (uint32_t)(len * 4), &bars[b]);
    if (has_xo) bulk_g2s_plain(st + L::kOffXo, a.xold + i0, (uint32_t)(len * 4), &bars[b]);
  };

  const long long g = gridDim.x;
  uint32_t inflight = 0u;  // bit b: stage b has a copy in flight (the same in every thread)
  uint32_t phase = 0u;     // bit b: parity of stage b's next completion
  for (int p = 0; p < kDStages - 1; ++p) {
    const long long tl = blockIdx.x + p * g;
    if (tl < ntiles) {
      if (threadIdx.x == 0) issue(tl, p);
      inflight |= 1u << p;
    }
  }
  bool ok = true;
  long long k = 0;
  for (long long tile = blockIdx.x; tile < ntiles; tile += g, ++k) {
    const int b = (int)(k % kDStages);
    {
      const long long nxt = tile + (long long)(kDStages - 1) * g;
      const int bn = (int)((k + kDStages - 1) % kDStages);
      if (nxt < ntiles) {
        if (threadIdx.x == 0) issue(nxt, bn);
        inflight |= 1u << bn;
      }
    }
    const bool arrived = mbar_wait_bounded(&bars[b], (phase >> b) & 1u);
    if (!__syncthreads_and(arrived)) {
      ok = false;
      break;
    }
    inflight &= ~(1u << b);
    phase ^= 1u << b;
    const unsigned char* st = dsm + (size_t)b * L::kStage;
    const long long i0 = tile * kDT;
    const int len = (int)((n_pad - i0 < kDT) ? n_pad - i0 : kDT);
    // per tile: index of row i0's entry in each staged range, and the
    // clipping bounds of the neighbour indices (in staged-range units)
    int clo[3], cxp[3], cxm[3], hip[3], lom[3];
    const int cx0 = (int)(i0 - rstart[b][6]);
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const long long o = d.doff[t];
      clo[t] = (int)(i0 - o - rstart[b][3 + t]);
      cxp[t] = (int)(i0 + o - rstart[b][7 + 2 * t]);
      cxm[t] = (int)(i0 - o - rstart[b][8 + 2 * t]);
      hip[t] = (int)(n_pad - 1 - rstart[b][7 + 2 * t]);  // x[n_pad - 1]
      lom[t] = (int)(-rstart[b][8 + 2 * t]);             // x[0]
    }
    const float* xsm = reinterpret_cast<const float*>(st + L::kOffX);
    const float* rsm = reinterpret_cast<const float*>(st + L::kOffR);
    const float* xosm = reinterpret_cast<const float*>(st + L::kOffXo);
    float* yg = a.y + i0;
    for (int li = threadIdx.x; li < len; li += kDThreads) {
      const float xs = xsm[li + cx0];
      const float rs = rsm[li];
      float acc;
      if constexpr (MODE == kChebK) {
        acc = fmaf(a.ce, xosm[li], fmaf(a.cd, xs, rs));
      } else if constexpr (MODE == kCheb2) {
        acc = fmaf(a.cd, xs, a.ce * rs);
      } else {
        acc = xs;  // kCheb1: x = r and A x = x + S x
      }
#pragma unroll
      for (int t = 0; t < 3; ++t) {
        const float up = smem_val<TV>(st + t * L::kUpB, li);
        const float lo = smem_val<TV>(st + L::kOffLo + t * L::kLoB, li + clo[t]);
        const int jp = min(li + cxp[t], hip[t]);
        const int jm = max(li + cxm[t], lom[t]);
        const float xp = reinterpret_cast<const float*>(st + L::kOffX + (1 + 2 * t) * L::kXB)[jp];
        const float xm = reinterpret_cast<const float*>(st + L::kOffX + (2 + 2 * t) * L::kXB)[jm];
        if constexpr (MODE == kCheb1) {
          acc = fmaf(up, xp, acc);
          acc = fmaf(lo, xm, acc);
        } else {
          acc = fmaf(-up, xp, acc);
          acc = fmaf(-lo, xm, acc);
        }
      }
      yg[li] = MODE == kCheb1 ? fmaf(a.cb, acc, a.ca * rs) : a.cc * acc;
    }
    __syncthreads();  // stage b is read; it may be refilled
  }
  if (!ok) {
    // a staged copy did not arrive in time: record it, and wait (bounded)
    // for this CTA's copies still in flight so that none lands after exit
    if (threadIdx.x == 0 && a.err) atomicExch(a.err, 1);
    for (int b = 0; b < kDStages; ++b)
      if ((inflight >> b) & 1u) mbar_wait_bounded(&bars[b], (phase >> b) & 1u);
  }
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

DiaArgs dia_args(const MatDesc& A) {
  DiaArgs d;
  d.nd = A.ndiag;
  d.unit = A.dia_unit;
  for (int t = 0; t < kMaxDiag; ++t) d.doff[t] = t < A.ndiag ? A.doff[t] : 0;
  d.dstride = A.dstride;
  d.dpad = A.dpad;
  d.n_pad = A.n_pad;
  return d;
}

// TMA-staged launch: one CTA per SM (the stages take most of its shared
// memory), capped by the caller's grid and the number of tiles.
template <typename TV, int MODE>
cudaError_t go_dia_tma(const MatDesc& A, const StepParams& p, const Scalars* sc, int grid, cudaStream_t s) {
  using L = DiaTma<TV>;
  auto kern = dia_step_tma_kernel<TV, MODE>;
  static bool attr_set[kMaxDevices] = {false};
  static int per_sm[kMaxDevices] = {0};
  const int dev = current_device();
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kSmem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kDThreads, L::kSmem);
    if (e != cudaSuccess) return e;
    per_sm[dev] = nb > 0 ? nb : 1;
    attr_set[dev] = true;
  }
  StepArgs<float> args = make_args<float>(p);
  if (MODE == kChebK || MODE == kCheb2) {  // folded coefficients, as in dia_step_kernel
    args.cd = (float)(p.ca / p.cc - 1.0);
    args.ce = (float)(MODE == kChebK ? p.cb / p.cc : p.cb / p.cc + 1.0);
  }
  const long long tiles = (A.n_pad + kDT - 1) / kDT;
  long long g = (long long)num_sms() * per_sm[dev];
  if (g > tiles) g = tiles;
  if (g > grid) g = grid;
  if (g < 1) g = 1;
  kern<<<(int)g, kDThreads, L::kSmem, s>>>(dia_args(A), static_cast<const TV*>(A.val), args, sc);
  return cudaGetLastError();
}

template <typename TV, typename TX, int MODE, int NDOT>
cudaError_t go_dia(const MatDesc& A, const StepParams& p, const Scalars* sc, double* partials, unsigned int* cnt,
                   int grid, cudaStream_t s) {
  if constexpr (!step_variant_used<TX, MODE, NDOT>()) {
    return cudaErrorNotSupported;
  } else {
    if constexpr (std::is_same<TX, float>::value && NDOT == 0 &&
                  (MODE == kCheb1 || MODE == kCheb2 || MODE == kChebK)) {
      if (A.tma && A.ndiag == 3 && A.dia_unit) return go_dia_tma<TV, MODE>(A, p, sc, grid, s);
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
