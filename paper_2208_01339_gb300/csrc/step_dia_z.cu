// Plane-marching degree step of the FP32/BF16 DIA matrix of a structured
// 3-D grid (see step_dia.cuh): offsets 1, Nx, Nx*Ny and n = Nx*Ny*Nz.
//
// The direct kernel (step_dia.cu) reads the two z-neighbours x[i +- Nx*Ny]
// and the lower z-entry a(i, i - Nx*Ny) of every row from L2: they were
// loaded by rows one plane away, far outside the SM's L1.  Here a thread owns
// two adjacent grid columns (x, x+1 at one y) of a 64 x 8 tile and walks z
// through a chunk of planes, so those three values come from registers: x at
// z-1 and z+1 around the current plane, and the upper z-entry of the
// previous plane, which is the lower one of this plane.  The in-plane
// neighbours (x +- 1, y +- 1) were loaded by neighbouring threads of the
// same CTA at the same step and come from L1.  Per row the DRAM streams are
// the three stored diagonals, x, r, x_old and y, as in the direct kernel.
// Neighbour indices are clipped to [0, n_pad) like the direct kernel's;
// their matrix entries are 0 there.
#include "step_dia.cuh"

namespace pp {
namespace {

constexpr int kZTileX = 64;  // grid columns in x per tile (2 per thread)
constexpr int kZTileY = 8;   // rows of the tile in y (one warp each)

template <typename TV>
__device__ __forceinline__ float2 zld2(const TV* p, uint64_t pol) {
  if constexpr (std::is_same<TV, __nv_bfloat16>::value) {
    unsigned int u;
    asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(u) : "l"(p), "l"(pol));
    return make_float2(__uint_as_float(u << 16), __uint_as_float(u & 0xffff0000u));
  } else {
    float2 v;
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(v.x), "=f"(v.y) : "l"(p), "l"(pol));
    return v;
  }
}
template <typename TV>
__device__ __forceinline__ float zld1(const TV* p) {
  if constexpr (std::is_same<TV, __nv_bfloat16>::value)
    return __uint_as_float(((unsigned int)__ldg(reinterpret_cast<const unsigned short*>(p))) << 16);
  else
    return __ldg(p);
}
__device__ __forceinline__ float2 xld2(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }

template <typename TV, int MODE>
__global__ void __launch_bounds__(kBlock) dia_step_z_kernel(DiaArgs d, int Nx, int Ny, int Nz, int zchunk,
                                                            const TV* __restrict__ val, StepArgs<float> a,
                                                            const Scalars* sc) {
  if (sc && load_done(sc)) return;
  const int tiles_x = (Nx + kZTileX - 1) / kZTileX;
  const int bx = blockIdx.x % tiles_x, by = blockIdx.x / tiles_x;
  const int x = bx * kZTileX + (threadIdx.x & 31) * 2, y = by * kZTileY + (threadIdx.x >> 5);
  const int z0 = blockIdx.y * zchunk, z1 = min(Nz, z0 + zchunk);
  if (x >= Nx || y >= Ny || z0 >= z1) return;  // no barriers below: idle threads may leave
  const long long nxy = (long long)Nx * Ny;
  const long long hi = d.n_pad - 2;  // last even index (pairs are loaded at even indices)
  const TV* v0 = val + d.dpad;
  const TV* v1 = v0 + d.dstride;
  const TV* v2 = v1 + d.dstride;
  const uint64_t pol_first = policy_evict_first(), pol_last = policy_evict_last();
  const float* X = a.x;
  long long i = x + (long long)Nx * y + nxy * z0;  // even: Nx and x are even
  auto clip = [&](long long j) { return j < 0 ? 0LL : (j > hi ? hi : j); };
  float2 xm = xld2(X + clip(i - nxy));
  float2 xc = xld2(X + i);
  float2 l2 = zld2<TV>(v2 + i - nxy, pol_first);  // a(i - nxy, i); 0 in the front pad below plane 0
#pragma unroll 2
  for (int z = z0; z < z1; ++z, i += nxy) {
    const float2 xp = xld2(X + clip(i + nxy));
    const float2 u0 = zld2<TV>(v0 + i, pol_first);
    const float2 u1 = zld2<TV>(v1 + i, pol_first);
    const float2 u2 = zld2<TV>(v2 + i, pol_first);
    const float l0 = zld1<TV>(v0 + i - 1);  // a(i, i - 1); the second row's is u0.x
    const float2 l1 = zld2<TV>(v1 + i - Nx, pol_first);
    const float xw = __ldg(X + (i > 0 ? i - 1 : 0));
    const float xe = __ldg(X + (i + 2 <= d.n_pad - 1 ? i + 2 : d.n_pad - 1));
    const float2 xs = xld2(X + clip(i - Nx));
    const float2 xn = xld2(X + clip(i + Nx));
    float2 rs;
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(rs.x), "=f"(rs.y) : "l"(a.r + i), "l"(pol_last));
    float acc0, acc1;
    if constexpr (MODE == kChebK) {
      const float2 xo = xld2(a.xold + i);
      acc0 = fmaf(a.ce, xo.x, fmaf(a.cd, xc.x, rs.x));
      acc1 = fmaf(a.ce, xo.y, fmaf(a.cd, xc.y, rs.y));
    } else if constexpr (MODE == kCheb2) {
      acc0 = fmaf(a.cd, xc.x, a.ce * rs.x);
      acc1 = fmaf(a.cd, xc.y, a.ce * rs.y);
    } else {  // kCheb1: x = r and A x = x + S x
      acc0 = xc.x;
      acc1 = xc.y;
    }
    // the six off-diagonal entries of each row: x +- 1, y +- 1, z +- 1
    const float s0 = fmaf(u0.x, xc.y, fmaf(l0, xw, fmaf(u1.x, xn.x, fmaf(l1.x, xs.x, fmaf(u2.x, xp.x, l2.x * xm.x)))));
    const float s1 = fmaf(u0.y, xe, fmaf(u0.x, xc.x, fmaf(u1.y, xn.y, fmaf(l1.y, xs.y, fmaf(u2.y, xp.y, l2.y * xm.y)))));
    float2 yv;
    if constexpr (MODE == kCheb1) {
      yv.x = fmaf(a.cb, acc0 + s0, a.ca * rs.x);
      yv.y = fmaf(a.cb, acc1 + s1, a.ca * rs.y);
    } else {
      yv.x = a.cc * (acc0 - s0);
      yv.y = a.cc * (acc1 - s1);
    }
    *reinterpret_cast<float2*>(a.y + i) = yv;
    xm = xc;
    xc = xp;
    l2 = u2;
  }
}

template <typename TV, int MODE>
cudaError_t go_dia_z(const MatDesc& A, const StepParams& p, const Scalars* sc, cudaStream_t s) {
  const int Nx = A.doff[1], Ny = A.doff[2] / A.doff[1], Nz = (int)((long long)A.n / A.doff[2]);
  StepArgs<float> args = make_args<float>(p);
  if (MODE == kChebK || MODE == kCheb2) {  // folded coefficients, as in dia_step_kernel
    args.cd = (float)(p.ca / p.cc - 1.0);
    args.ce = (float)(MODE == kChebK ? p.cb / p.cc : p.cb / p.cc + 1.0);
  }
  const long long tiles = (long long)((Nx + kZTileX - 1) / kZTileX) * ((Ny + kZTileY - 1) / kZTileY);
  // z chunks: about 8 resident CTAs per SM in all, at least 4 planes per chunk
  const long long want = 8LL * num_sms();
  int chunks = (int)std::max(1LL, std::min<long long>((want + tiles - 1) / tiles, (Nz + 3) / 4));
  const int zchunk = (Nz + chunks - 1) / chunks;
  chunks = (Nz + zchunk - 1) / zchunk;
  if (tiles > 0x7fffffffLL || chunks > 65535) return cudaErrorInvalidConfiguration;
  dia_step_z_kernel<TV, MODE><<<dim3((unsigned)tiles, (unsigned)chunks), kBlock, 0, s>>>(
      dia_args(A), Nx, Ny, Nz, zchunk, static_cast<const TV*>(A.val), args, sc);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step_dia_z(const MatDesc& A, const StepParams& p, const Scalars* sc, cudaStream_t s) {
  if (!dia_z_applies(A) || p.ndot != 0) return cudaErrorInvalidValue;
  if (A.prec == kF32) {
    switch (p.mode) {
      case kCheb1: return go_dia_z<float, kCheb1>(A, p, sc, s);
      case kCheb2: return go_dia_z<float, kCheb2>(A, p, sc, s);
      case kChebK: return go_dia_z<float, kChebK>(A, p, sc, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (p.mode) {
    case kCheb1: return go_dia_z<__nv_bfloat16, kCheb1>(A, p, sc, s);
    case kCheb2: return go_dia_z<__nv_bfloat16, kCheb2>(A, p, sc, s);
    case kChebK: return go_dia_z<__nv_bfloat16, kChebK>(A, p, sc, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pp
