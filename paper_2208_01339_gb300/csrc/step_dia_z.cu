// Plane-marching degree step of the FP32/BF16 DIA matrix of a structured
// 3-D grid (see step_dia.cuh): offsets 1, Nx, Nx*Ny and n = Nx*Ny*Nz.
//
// The direct kernel (step_dia.cu) reads the two z-neighbours x[i +- Nx*Ny]
// and the lower z-entry a(i, i - Nx*Ny) of every row from L2: they were
// loaded by rows one plane away, far outside the SM's L1.  Here a thread owns
// C adjacent grid columns (x .. x+C-1 at one y) of a 64-wide tile and walks z
// through a chunk of planes, so those three values come from registers: x at
// z-1 and z+1 around the current plane, and the upper z-entry of the
// previous plane, which is the lower one of this plane.  The in-plane
// neighbours (x +- 1, y +- 1) were loaded by neighbouring threads of the
// same CTA at the same step and come from L1.  Per row the DRAM streams are
// the three stored diagonals, x, r, x_old and y, as in the direct kernel.
// Neighbour indices are clipped to [0, n_pad) like the direct kernel's;
// their matrix entries are 0 there.
//
// C = 4 (16-byte FP32 / 8-byte BF16 loads, 64 x 16 tiles) when Nx is a
// multiple of 4, else C = 2 (64 x 8 tiles).  The (tile, z chunk) work items
// are sized so that one resident wave covers them (at least kZMinPlanes
// planes per chunk); a capped grid walks them with a grid stride.
#include <atomic>

#include "step_dia.cuh"

namespace pp {
namespace {

constexpr int kZTileX = 64;     // grid columns in x per tile
constexpr int kZMinPlanes = 4;  // planes per z chunk, at least

template <int C>
struct ZVec {
  float v[C];
};

// C consecutive stored values (FP32 or BF16) with an L2 priority
template <typename TV, int C>
__device__ __forceinline__ ZVec<C> zld(const TV* p, uint64_t pol) {
  ZVec<C> o;
  if constexpr (std::is_same<TV, __nv_bfloat16>::value) {
    if constexpr (C == 2) {
      unsigned int u;
      asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(u) : "l"(p), "l"(pol));
      o.v[0] = __uint_as_float(u << 16);
      o.v[1] = __uint_as_float(u & 0xffff0000u);
    } else {
      unsigned int u0, u1;
      asm("ld.global.nc.L2::cache_hint.v2.b32 {%0, %1}, [%2], %3;" : "=r"(u0), "=r"(u1) : "l"(p), "l"(pol));
      o.v[0] = __uint_as_float(u0 << 16);
      o.v[1] = __uint_as_float(u0 & 0xffff0000u);
      o.v[2] = __uint_as_float(u1 << 16);
      o.v[3] = __uint_as_float(u1 & 0xffff0000u);
    }
  } else {
    if constexpr (C == 2)
      asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(o.v[0]), "=f"(o.v[1]) : "l"(p), "l"(pol));
    else
      asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
          : "=f"(o.v[0]), "=f"(o.v[1]), "=f"(o.v[2]), "=f"(o.v[3])
          : "l"(p), "l"(pol));
  }
  return o;
}
template <typename TV>
__device__ __forceinline__ float zld1(const TV* p) {
  if constexpr (std::is_same<TV, __nv_bfloat16>::value)
    return __uint_as_float(((unsigned int)__ldg(reinterpret_cast<const unsigned short*>(p))) << 16);
  else
    return __ldg(p);
}
// C consecutive FP32 vector entries through the read-only path
template <int C>
__device__ __forceinline__ ZVec<C> xld(const float* p) {
  ZVec<C> o;
  if constexpr (C == 2) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    o.v[0] = t.x;
    o.v[1] = t.y;
  } else {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    o.v[0] = t.x;
    o.v[1] = t.y;
    o.v[2] = t.z;
    o.v[3] = t.w;
  }
  return o;
}

// One work item: the thread's C grid columns of tile (bx, by) through z
// chunk cz.
template <typename TV, int MODE, int C>
__device__ __forceinline__ void z_item(const DiaArgs& d, int Nx, int Ny, int Nz, int zchunk, int bx, int by, int cz,
                                       const TV* __restrict__ val, const StepArgs<float>& a) {
  constexpr int kLanes = kZTileX / C;   // threads per tile row
  constexpr int kRows = kBlock / kLanes;  // tile rows in y
  const long long nxy = (long long)Nx * Ny;
  const long long hi = d.n_pad - C;  // last C-aligned index
  const TV* v0 = val + d.dpad;
  const TV* v1 = v0 + d.dstride;
  const TV* v2 = v1 + d.dstride;
  const uint64_t pol_first = policy_evict_first(), pol_last = policy_evict_last();
  const float* X = a.x;
  auto clip = [&](long long j) { return j < 0 ? 0LL : (j > hi ? hi : j); };
  {
    const int x = bx * kZTileX + (int)(threadIdx.x % kLanes) * C, y = by * kRows + (int)(threadIdx.x / kLanes);
    const int z0 = cz * zchunk, z1 = min(Nz, z0 + zchunk);
    if (x >= Nx || y >= Ny || z0 >= z1) return;
    long long i = x + (long long)Nx * y + nxy * z0;  // a multiple of C: Nx and x are
    ZVec<C> xm = xld<C>(X + clip(i - nxy));
    ZVec<C> xc = xld<C>(X + i);
    ZVec<C> l2 = zld<TV, C>(v2 + i - nxy, pol_first);  // a(i - nxy, i); 0 in the front pad below plane 0
#pragma unroll 1
    for (int z = z0; z < z1; ++z, i += nxy) {
      const ZVec<C> xp = xld<C>(X + clip(i + nxy));
      const ZVec<C> u0 = zld<TV, C>(v0 + i, pol_first);
      const ZVec<C> u1 = zld<TV, C>(v1 + i, pol_first);
      const ZVec<C> u2 = zld<TV, C>(v2 + i, pol_first);
      const float l0 = zld1<TV>(v0 + i - 1);  // a(i - 1, i); the later rows' are in u0
      const ZVec<C> l1 = zld<TV, C>(v1 + i - Nx, pol_first);
      const float xw = __ldg(X + (i > 0 ? i - 1 : 0));
      const float xe = __ldg(X + (i + C <= d.n_pad - 1 ? i + C : d.n_pad - 1));
      const ZVec<C> xs = xld<C>(X + clip(i - Nx));
      const ZVec<C> xn = xld<C>(X + clip(i + Nx));
      ZVec<C> rs;
      if constexpr (C == 2)
        asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
            : "=f"(rs.v[0]), "=f"(rs.v[1])
            : "l"(a.r + i), "l"(pol_last));
      else
        asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
            : "=f"(rs.v[0]), "=f"(rs.v[1]), "=f"(rs.v[2]), "=f"(rs.v[3])
            : "l"(a.r + i), "l"(pol_last));
      ZVec<C> xo;
      if constexpr (MODE == kChebK) xo = xld<C>(a.xold + i);
      ZVec<C> yv;
#pragma unroll
      for (int e = 0; e < C; ++e) {
        float acc;
        if constexpr (MODE == kChebK)
          acc = fmaf(a.ce, xo.v[e], fmaf(a.cd, xc.v[e], rs.v[e]));
        else if constexpr (MODE == kCheb2)
          acc = fmaf(a.cd, xc.v[e], a.ce * rs.v[e]);
        else  // kCheb1: x = r and A x = x + S x
          acc = xc.v[e];
        // the six off-diagonal entries of the row: x +- 1, y +- 1, z +- 1
        const float right = e + 1 < C ? xc.v[e + 1 < C ? e + 1 : e] : xe;
        const float lc = e > 0 ? u0.v[e > 0 ? e - 1 : 0] : l0;
        const float lx = e > 0 ? xc.v[e > 0 ? e - 1 : 0] : xw;
        const float se = fmaf(u0.v[e], right,
                              fmaf(lc, lx, fmaf(u1.v[e], xn.v[e], fmaf(l1.v[e], xs.v[e],
                                                                          fmaf(u2.v[e], xp.v[e], l2.v[e] * xm.v[e])))));
        if constexpr (MODE == kCheb1)
          yv.v[e] = fmaf(a.cb, acc + se, a.ca * rs.v[e]);
        else
          yv.v[e] = a.cc * (acc - se);
      }
      if constexpr (C == 2)
        *reinterpret_cast<float2*>(a.y + i) = make_float2(yv.v[0], yv.v[1]);
      else
        *reinterpret_cast<float4*>(a.y + i) = make_float4(yv.v[0], yv.v[1], yv.v[2], yv.v[3]);
      xm = xc;
      xc = xp;
      l2 = u2;
    }
  }
}

// An uncapped launch takes one item per block on a 2-D grid (x: tile, y:
// z chunk); with STRIDE a capped 1-D grid walks the items (tile-major) with a
// grid stride.  No barriers: threads outside the grid skip their items.
template <typename TV, int MODE, int C, bool STRIDE>
__global__ void __launch_bounds__(kBlock) dia_step_z_kernel(DiaArgs d, int Nx, int Ny, int Nz, int zchunk,
                                                            int chunks, long long items,
                                                            const TV* __restrict__ val, StepArgs<float> a,
                                                            const Scalars* sc) {
  if (sc && load_done(sc)) return;
  const int tiles_x = (Nx + kZTileX - 1) / kZTileX;
  if constexpr (STRIDE) {
    for (long long item = blockIdx.x; item < items; item += gridDim.x) {
      const long long tile = item / chunks;
      z_item<TV, MODE, C>(d, Nx, Ny, Nz, zchunk, (int)(tile % tiles_x), (int)(tile / tiles_x),
                          (int)(item - tile * chunks), val, a);
    }
  } else {
    z_item<TV, MODE, C>(d, Nx, Ny, Nz, zchunk, (int)(blockIdx.x % tiles_x), (int)(blockIdx.x / tiles_x),
                        (int)blockIdx.y, val, a);
  }
}

// Resident CTAs per SM of one kernel instance, per device.
template <typename TV, int MODE, int C>
int z_resident() {
  static std::atomic<int> per_sm[kMaxDevices];
  const int dev = current_device();
  int v = per_sm[dev].load(std::memory_order_relaxed);
  if (v <= 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, dia_step_z_kernel<TV, MODE, C, false>, kBlock, 0) != cudaSuccess ||
        v <= 0)
      v = 1;
    per_sm[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

template <typename TV, int MODE, int C>
cudaError_t go_dia_z(const MatDesc& A, const StepParams& p, const Scalars* sc, int grid_cap, cudaStream_t s) {
  const int Nx = A.doff[1], Ny = A.doff[2] / A.doff[1], Nz = (int)((long long)A.n / A.doff[2]);
  StepArgs<float> args = make_args<float>(p);
  if (MODE == kChebK || MODE == kCheb2) {  // folded coefficients, as in dia_step_kernel
    args.cd = (float)(p.ca / p.cc - 1.0);
    args.ce = (float)(MODE == kChebK ? p.cb / p.cc : p.cb / p.cc + 1.0);
  }
  constexpr int kRows = kBlock / (kZTileX / C);
  const long long tiles = (long long)((Nx + kZTileX - 1) / kZTileX) * ((Ny + kRows - 1) / kRows);
  // z chunks: as many as one resident wave holds, at least kZMinPlanes planes each
  const long long slots = (long long)z_resident<TV, MODE, C>() * num_sms();
  int chunks = (int)std::max(1LL, std::min<long long>(slots / tiles, (Nz + kZMinPlanes - 1) / kZMinPlanes));
  const int zchunk = (Nz + chunks - 1) / chunks;
  chunks = (Nz + zchunk - 1) / zchunk;
  const long long items = tiles * chunks;
  if (grid_cap > 0 && grid_cap < items) {
    dia_step_z_kernel<TV, MODE, C, true><<<(unsigned)grid_cap, kBlock, 0, s>>>(
        dia_args(A), Nx, Ny, Nz, zchunk, chunks, items, static_cast<const TV*>(A.val), args, sc);
  } else {
    if (tiles > 0x7fffffffLL || chunks > 65535) return cudaErrorInvalidConfiguration;
    dia_step_z_kernel<TV, MODE, C, false><<<dim3((unsigned)tiles, (unsigned)chunks), kBlock, 0, s>>>(
        dia_args(A), Nx, Ny, Nz, zchunk, chunks, items, static_cast<const TV*>(A.val), args, sc);
  }
  return cudaGetLastError();
}

template <typename TV, int MODE>
cudaError_t go_dia_z_c(const MatDesc& A, const StepParams& p, const Scalars* sc, int grid_cap, cudaStream_t s) {
  if (A.doff[1] % 4 == 0) return go_dia_z<TV, MODE, 4>(A, p, sc, grid_cap, s);
  return go_dia_z<TV, MODE, 2>(A, p, sc, grid_cap, s);
}

}  // namespace

cudaError_t launch_step_dia_z(const MatDesc& A, const StepParams& p, const Scalars* sc, int grid_cap, cudaStream_t s) {
  if (!dia_z_applies(A) || p.ndot != 0) return cudaErrorInvalidValue;
  if (A.prec == kF32) {
    switch (p.mode) {
      case kCheb1: return go_dia_z_c<float, kCheb1>(A, p, sc, grid_cap, s);
      case kCheb2: return go_dia_z_c<float, kCheb2>(A, p, sc, grid_cap, s);
      case kChebK: return go_dia_z_c<float, kChebK>(A, p, sc, grid_cap, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (p.mode) {
    case kCheb1: return go_dia_z_c<__nv_bfloat16, kCheb1>(A, p, sc, grid_cap, s);
    case kCheb2: return go_dia_z_c<__nv_bfloat16, kCheb2>(A, p, sc, grid_cap, s);
    case kChebK: return go_dia_z_c<__nv_bfloat16, kChebK>(A, p, sc, grid_cap, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pp
