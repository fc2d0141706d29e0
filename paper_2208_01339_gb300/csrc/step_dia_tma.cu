// TMA-staged degree step of the FP32/BF16 DIA matrix (see step_dia.cuh).
#include "step_dia.cuh"

namespace pp {
namespace {

// ------------------------------------------ TMA-staged low-precision step ----
// The FP32/BF16 steps move few bytes per row and do little arithmetic, so
// their cost is set by how many bytes are in flight.  Here every stream of a
// tile of kDT consecutive rows is a contiguous range, moved into shared
// memory with cp.async.bulk by a producer warp up to kDStages tiles ahead,
// while kDConsumers warps compute the rows from shared memory.  With the
// stored upper offsets o0 < o1 < o2 (1, N, N^2 for the 7-point stencil):
//   XM   x over [i0 - o1, i0 + len + o1)  (own, +-o0, +-o1 neighbours)
//   XP2  x over [i0 + o2, ...), XM2  x over [i0 - o2, ...)
//   V0   diagonal 0 over positions [i0 - o0, i0 + len) (upper and lower)
//   V1   diagonal 1 over [i0 - o1, i0 + len)
//   V2U  diagonal 2 over [i0, i0 + len), V2L over [i0 - o2, ...)
//   R, XO  r and x_old over [i0, i0 + len)
// Starts are rounded down to 16 bytes (the copy's alignment rule), vector
// ranges are clipped to [0, n_pad), and a neighbour index is clipped the
// same way (its matrix entry is 0 there).  A stage is refilled once every
// consumer warp has released it (one "empty" mbarrier per stage).  Applies
// to the Jacobi-scaled matrix with 3 upper diagonals and o1 <= kDMaxMid.
constexpr int kDT = 1024;         // rows per tile
constexpr int kDStages = 4;       // tiles in flight per CTA
constexpr int kDConsumers = 8;    // consumer warps
constexpr int kDThreads = (kDConsumers + 1) * 32;
constexpr int kDMaxMid = kDiaTmaMaxMid;  // largest o1 the merged ranges hold

template <typename TV>
struct DiaTma {
  static constexpr int kAV = 16 / (int)sizeof(TV);  // alignment unit of the value ranges (elements)
  static constexpr int kAX = 4;                     // of the FP32 vector ranges
  static constexpr int r128(int b) { return (b + 127) / 128 * 128; }
  static constexpr int kXMB = r128((kDT + 2 * kDMaxMid + 2 * kAX) * 4);
  static constexpr int kX2B = r128((kDT + 2 * kAX) * 4);
  static constexpr int kV01B = r128((kDT + kDMaxMid + 2 * kAV) * (int)sizeof(TV));
  static constexpr int kV2UB = r128(kDT * (int)sizeof(TV));
  static constexpr int kV2LB = r128((kDT + 2 * kAV) * (int)sizeof(TV));
  static constexpr int kVecB = kDT * 4;
  static constexpr int kOffXP2 = kXMB;
  static constexpr int kOffXM2 = kOffXP2 + kX2B;
  static constexpr int kOffV0 = kOffXM2 + kX2B;
  static constexpr int kOffV1 = kOffV0 + kV01B;
  static constexpr int kOffV2U = kOffV1 + kV01B;
  static constexpr int kOffV2L = kOffV2U + kV2UB;
  static constexpr int kOffR = kOffV2L + kV2LB;
  static constexpr int kOffXO = kOffR + kVecB;
  static constexpr int kStage = kOffXO + kVecB;
  static constexpr int kSmem = kStage * kDStages;
};

// Row coordinates of the staged ranges of one tile: staged element k of
// range q holds global index start[q] + k (diagonal positions for V0, V1,
// V2L).  Ranges: 0 XM, 1 XP2, 2 XM2, 3 V0, 4 V1, 5 V2L.
struct DiaTile {
  long long i0;
  long long start[6];
  int len;
  int pad_;
};

__device__ __forceinline__ void bulk_g2s_plain(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_plain(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

template <typename TV>
__device__ __forceinline__ float smem_val(const unsigned char* p, int k) {
  if constexpr (std::is_same<TV, __nv_bfloat16>::value)
    return __uint_as_float(((unsigned int)reinterpret_cast<const unsigned short*>(p)[k]) << 16);
  else
    return reinterpret_cast<const float*>(p)[k];
}

template <typename TV, int MODE>
__global__ void __launch_bounds__(kDThreads, 1) dia_step_tma_kernel(DiaArgs d, const TV* __restrict__ val,
                                                                    StepArgs<float> a, const Scalars* sc, int* err) {
  using L = DiaTma<TV>;
  constexpr int AV = L::kAV, AX = L::kAX;
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ __align__(8) uint64_t full[kDStages], empty[kDStages];
  __shared__ DiaTile tiles[kDStages];
  __shared__ int filled[kDStages], drained[kDStages];
  if (sc && load_done(sc)) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const long long n_pad = d.n_pad;
  const long long ntiles = (n_pad + kDT - 1) / kDT;
  const long long g = gridDim.x;
  const long long o0 = d.doff[0], o1 = d.doff[1], o2 = d.doff[2];
  if (threadIdx.x == 0) {
    for (int b = 0; b < kDStages; ++b) {
      mbar_init(&full[b], 1);
      mbar_init(&empty[b], kDConsumers);
      filled[b] = 0;
      drained[b] = 0x7fffffff;
    }
    mbar_fence_init();
  }
  __syncthreads();
  if (wid == kDConsumers) {
    // ---- producer warp: lane 0 stages the CTA's tiles in order ----
    if (lane == 0) {
      const char* vb = reinterpret_cast<const char*>(val);
      // L2 priorities: the stored diagonals stream through once per step, r
      // is read by every step of an application
      const uint64_t pol_first = policy_evict_first(), pol_last = policy_evict_last();
      long long k = 0;
      for (long long tile = blockIdx.x; tile < ntiles; tile += g, ++k) {
        const int b = (int)(k % kDStages);
        if (k >= kDStages && !mbar_wait_bounded(&empty[b], (uint32_t)(((k / kDStages) - 1) & 1))) {
          if (err) atomicExch(err, 1);
          break;
        }
        unsigned char* st = dsm + (size_t)b * L::kStage;
        const long long i0 = tile * kDT;
        const long long len = (n_pad - i0 < kDT) ? n_pad - i0 : kDT;
        DiaTile& T = tiles[b];
        T.i0 = i0;
        T.len = (int)len;
        // vector range [r0, r1) of x, clipped to [0, n_pad) and rounded out to 16 bytes
        auto xr = [&](long long r0, long long r1, bool low_end, long long* s0) -> uint32_t {
          if (r0 < 0) r0 = 0;
          if (r1 > n_pad) r1 = n_pad;
          if (r1 <= r0) {  // entirely outside: one aligned group at the nearest end
            r0 = low_end ? 0 : n_pad - AX;
            r1 = r0 + AX;
          }
          r0 = r0 / AX * AX;
          r1 = (r1 + AX - 1) / AX * AX;
          *s0 = r0;
          return (uint32_t)((r1 - r0) * 4);
        };
        // diagonal t's positions [p0, p1) (relative to its row 0), rounded out and clipped to its storage
        auto vr = [&](int t, long long p0, long long p1, long long* s0, long long* e0) -> uint32_t {
          const long long dbeg = (long long)t * d.dstride, dend = dbeg + d.dpad + n_pad;
          long long a0 = dbeg + d.dpad + p0, a1 = dbeg + d.dpad + p1;
          const long long sh = a0 % AV;
          a0 -= sh;
          a1 = (a1 + AV - 1) / AV * AV;
          if (a1 > dend) a1 = dend;
          *s0 = p0 - sh;
          *e0 = a0;
          return (uint32_t)((a1 - a0) * (long long)sizeof(TV));
        };
        long long e0v, e1v, e2v;
        const uint32_t bxm = xr(i0 - o1, i0 + len + o1, true, &T.start[0]);
        const uint32_t bxp = xr(i0 + o2, i0 + len + o2, false, &T.start[1]);
        const uint32_t bxq = xr(i0 - o2, i0 + len - o2, true, &T.start[2]);
        const uint32_t bv0 = vr(0, i0 - o0, i0 + len, &T.start[3], &e0v);
        const uint32_t bv1 = vr(1, i0 - o1, i0 + len, &T.start[4], &e1v);
        const uint32_t bv2 = vr(2, i0 - o2, i0 - o2 + len, &T.start[5], &e2v);
        const uint32_t bv2u = (uint32_t)(len * (long long)sizeof(TV));
        const uint32_t bvec = (uint32_t)(len * 4);
        const uint32_t total = bxm + bxp + bxq + bv0 + bv1 + bv2 + bv2u + bvec + (MODE == kChebK ? bvec : 0u);
        // the consumers' generic reads of stage b are ordered (empty barrier)
        // before this asynchronous refill
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&full[b], total);
        bulk_g2s_plain(st, a.x + T.start[0], bxm, &full[b]);
        bulk_g2s_plain(st + L::kOffXP2, a.x + T.start[1], bxp, &full[b]);
        bulk_g2s_plain(st + L::kOffXM2, a.x + T.start[2], bxq, &full[b]);
        bulk_g2s(st + L::kOffV0, vb + e0v * (long long)sizeof(TV), bv0, &full[b], pol_first);
        bulk_g2s(st + L::kOffV1, vb + e1v * (long long)sizeof(TV), bv1, &full[b], pol_first);
        bulk_g2s(st + L::kOffV2U, vb + (2 * d.dstride + d.dpad + i0) * (long long)sizeof(TV), bv2u, &full[b],
                 pol_first);
        bulk_g2s(st + L::kOffV2L, vb + e2v * (long long)sizeof(TV), bv2, &full[b], pol_first);
        bulk_g2s(st + L::kOffR, a.r + i0, bvec, &full[b], pol_last);
        if (MODE == kChebK) bulk_g2s_plain(st + L::kOffXO, a.xold + i0, bvec, &full[b]);
        filled[b] += 1;
      }
    }
  } else {
    // ---- consumer warps: rows of the staged tiles ----
    long long k = 0;  // tiles consumed by this warp
    for (long long tile = blockIdx.x; tile < ntiles; tile += g, ++k) {
      const int b = (int)(k % kDStages);
      if (!mbar_wait_bounded(&full[b], (uint32_t)((k / kDStages) & 1))) {
        if (lane == 0 && err) atomicExch(err, 1);
        break;
      }
      const unsigned char* st = dsm + (size_t)b * L::kStage;
      const DiaTile& T = tiles[b];
      const long long i0 = T.i0;
      const int len = T.len;
      // staged index of row i0 in each range, and the staged indices of
      // global rows 0 and n_pad - 1 (the clipping bounds of neighbours)
      const int cm = (int)(i0 - T.start[0]), cp2 = (int)(i0 + o2 - T.start[1]), cq2 = (int)(i0 - o2 - T.start[2]);
      const int c0 = (int)(i0 - T.start[3]), c1 = (int)(i0 - T.start[4]), c2 = (int)(i0 - o2 - T.start[5]);
      const int lo_m = (int)(-T.start[0]), hi_m = (int)(n_pad - 1 - T.start[0]);
      const int hi_p = (int)(n_pad - 1 - T.start[1]), lo_q = (int)(-T.start[2]);
      const int io0 = (int)o0, io1 = (int)o1;
      const float* xm = reinterpret_cast<const float*>(st);
      const float* xp2 = reinterpret_cast<const float*>(st + L::kOffXP2);
      const float* xq2 = reinterpret_cast<const float*>(st + L::kOffXM2);
      const float* rsm = reinterpret_cast<const float*>(st + L::kOffR);
      const float* xosm = reinterpret_cast<const float*>(st + L::kOffXO);
      float* yg = a.y + i0;
      for (int li = threadIdx.x; li < len; li += kDConsumers * 32) {
        const int im = li + cm;
        const float xs = xm[im];
        const float rs = rsm[li];
        float acc;
        if constexpr (MODE == kChebK) {
          acc = fmaf(a.ce, xosm[li], fmaf(a.cd, xs, rs));
        } else if constexpr (MODE == kCheb2) {
          acc = fmaf(a.cd, xs, a.ce * rs);
        } else {
          acc = xs;  // kCheb1: x = r and A x = x + S x
        }
        const float u0 = smem_val<TV>(st + L::kOffV0, li + c0), l0 = smem_val<TV>(st + L::kOffV0, li + c0 - io0);
        const float u1 = smem_val<TV>(st + L::kOffV1, li + c1), l1 = smem_val<TV>(st + L::kOffV1, li + c1 - io1);
        const float u2 = smem_val<TV>(st + L::kOffV2U, li), l2 = smem_val<TV>(st + L::kOffV2L, li + c2);
        const float xp0 = xm[min(im + io0, hi_m)], xq0 = xm[max(im - io0, lo_m)];
        const float xp1 = xm[min(im + io1, hi_m)], xq1 = xm[max(im - io1, lo_m)];
        const float xpp = xp2[min(li + cp2, hi_p)], xqq = xq2[max(li + cq2, lo_q)];
        if constexpr (MODE == kCheb1) {
          acc = fmaf(u0, xp0, acc);
          acc = fmaf(l0, xq0, acc);
          acc = fmaf(u1, xp1, acc);
          acc = fmaf(l1, xq1, acc);
          acc = fmaf(u2, xpp, acc);
          acc = fmaf(l2, xqq, acc);
          yg[li] = fmaf(a.cb, acc, a.ca * rs);
        } else {
          acc = fmaf(-u0, xp0, acc);
          acc = fmaf(-l0, xq0, acc);
          acc = fmaf(-u1, xp1, acc);
          acc = fmaf(-l1, xq1, acc);
          acc = fmaf(-u2, xpp, acc);
          acc = fmaf(-l2, xqq, acc);
          yg[li] = a.cc * acc;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive_plain(&empty[b]);
    }
    // uses of each stage this warp has drained; the slowest warp counts
    if (lane == 0)
      for (int b = 0; b < kDStages; ++b) atomicMin(&drained[b], k > b ? (int)((k - b - 1) / kDStages) + 1 : 0);
  }
  __syncthreads();
  // a stage filled more often than its slowest consumer drained it has a copy
  // in flight (only after a timeout): wait for it, bounded, before exit
  if (threadIdx.x == 0)
    for (int b = 0; b < kDStages; ++b) {
      const int dd = drained[b];
      if (filled[b] > dd) mbar_wait_bounded(&full[b], (uint32_t)(dd & 1));
    }
}

// TMA-staged launch: one CTA per SM (the stages take most of its shared
// memory), capped by the caller's grid and the number of tiles.
template <typename TV, int MODE>
cudaError_t go_dia_tma(const MatDesc& A, const StepParams& p, const Scalars* sc, int grid, cudaStream_t s) {
  using L = DiaTma<TV>;
  auto kern = dia_step_tma_kernel<TV, MODE>;
  static bool attr_set[kMaxDevices] = {false};
  const int dev = current_device();
  if (!attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, L::kSmem);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  StepArgs<float> args = make_args<float>(p);
  if (MODE == kChebK || MODE == kCheb2) {  // folded coefficients, as in dia_step_kernel
    args.cd = (float)(p.ca / p.cc - 1.0);
    args.ce = (float)(MODE == kChebK ? p.cb / p.cc : p.cb / p.cc + 1.0);
  }
  // one CTA per SM (the stages take most of its shared memory)
  const long long tiles = (A.n_pad + kDT - 1) / kDT;
  long long g = num_sms();
  if (g > tiles) g = tiles;
  if (g > grid) g = grid;
  if (g < 1) g = 1;
  kern<<<(int)g, kDThreads, L::kSmem, s>>>(dia_args(A), static_cast<const TV*>(A.val), args, sc, p.err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step_dia_tma(const MatDesc& A, const StepParams& p, const Scalars* sc, int grid, cudaStream_t s) {
  if (!dia_tma_applies(A) || p.ndot != 0) return cudaErrorInvalidValue;
  if (A.prec == kF32) {
    switch (p.mode) {
      case kCheb1: return go_dia_tma<float, kCheb1>(A, p, sc, grid, s);
      case kCheb2: return go_dia_tma<float, kCheb2>(A, p, sc, grid, s);
      case kChebK: return go_dia_tma<float, kChebK>(A, p, sc, grid, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (p.mode) {
    case kCheb1: return go_dia_tma<__nv_bfloat16, kCheb1>(A, p, sc, grid, s);
    case kCheb2: return go_dia_tma<__nv_bfloat16, kCheb2>(A, p, sc, grid, s);
    case kChebK: return go_dia_tma<__nv_bfloat16, kChebK>(A, p, sc, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pp
