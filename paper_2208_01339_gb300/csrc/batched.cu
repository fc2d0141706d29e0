// Batched polynomial-preconditioned CG: many independent SPD instances of
// uneven size, each with 1..8 right-hand sides, solved together.
//
// Layout.  Every instance is stored in SELL-32 (one warp per 32-row slice,
// lane = row), and the slices of all instances form one global list, so a
// single persistent launch per Chebyshev step walks every instance
// (work item = slice).  Vectors of instance i are row-major [row][rhs] at
// voff[i], so one matrix entry is loaded once and applied to all the
// instance's right-hand sides (SpMM-style reuse).  Each global column
// g = cbase[i] + r has its own Chebyshev coefficients (theta_bar, delta,
// sigma_bar, rho_0..rho_k) and its own PCG scalars; converged columns are
// masked, and slices of fully converged instances are skipped.
//
// Reductions are deterministic: every slice stores per-column partial sums,
// then one block per global column adds its instance's partials in slice
// order (b_seg_reduce), and its epilogue updates that column's scalars.
// Iterations therefore run without host round trips and a block of them can
// be replayed as one captured CUDA graph until no column is active.
//
// The preconditioner p_k (Algorithm 2) is applied in FP64 or in FP32 (FP32
// values and vectors, FP32 accumulate); the outer CG is always FP64.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "driver.cuh"

namespace pp {

constexpr int kBR = 8;     // maximum right-hand sides per instance
constexpr int kBDiag = 8;  // DIA mode: stored upper diagonals per instance

// One plane-marching work item: a 32 x 8 tile (x0, y0) of instance inst's
// grid through planes [z0, z1).
struct BZItem {
  int inst, x0, y0;
  unsigned short z0, z1;
};
constexpr int kBZTileX = 32, kBZTileY = 8;
constexpr int kBZPlanes = 32;  // planes per item, at most

struct BatchDev {
  int nb = 0;             // instances
  int ncols = 0;          // global columns
  long long nslices = 0;  // global slices
  int k = 0;
  const int* s_inst = nullptr;      // instance of each slice
  const long long* s_row0 = nullptr;  // instance-local first row of each slice
  const long long* sptr = nullptr;  // global entry offsets
  const int* col = nullptr;         // instance-local column indices
  const double* val64 = nullptr;
  const float* val32 = nullptr;
  const int* n = nullptr;           // rows per instance
  const int* R = nullptr;           // right-hand sides per instance
  const long long* voff = nullptr;  // vector offset (elements) per instance
  const long long* uoff = nullptr;  // offset of the instance in the caller's b / x
  const int* cbase = nullptr;       // first global column per instance
  const long long* sbase = nullptr; // first global slice per instance (nb+1)
  const int* ccol_inst = nullptr;   // instance of each global column
  const double* w = nullptr;        // Jacobi seed weights, per instance row (voff1 layout)
  const long long* woff = nullptr;  // weight offset per instance
  // DIA mode (format = PP_FMT_DIA): every instance symmetric-banded; with the
  // Jacobi seed its diagonal is 1 and only the upper diagonals are stored:
  // entry (row, row + dia_off[i][t]) at dval[dia_base[i] + t * dia_stride[i]
  // + dia_pad[i] + row], zero-padded in front (dia_pad >= largest offset) and
  // over the padded rows of the instance's last slice.
  int dia = 0;
  const int* dia_nd = nullptr;
  const int* dia_off = nullptr;  // [nb][kBDiag]
  const long long* dia_base = nullptr;
  const long long* dia_stride = nullptr;
  const long long* dia_pad = nullptr;
  const double* dval64 = nullptr;
  const float* dval32 = nullptr;
  // DIA instances of a structured Nx x Ny x Nz grid (upper offsets 1, Nx,
  // Nx*Ny; zmode[i] = 1) take the FP32 plane-marching step over zitem
  // (b_cheb_z_kernel); the others the slice kernel
  const int* zmode = nullptr;
  const BZItem* zitem = nullptr;
  long long nzitems = 0;
  // per-column coefficients
  const double* theta_bar = nullptr;
  const double* delta = nullptr;
  const double* sigma_bar = nullptr;
  const double* rho = nullptr;      // [g][k+1]
};

struct BatchCols {
  double *rz, *rz_new, *pq, *zq, *rr, *bb, *rtol2;
  double *al, *be;  // alpha = (r,z)/(p,q) and beta per column, formed once by the reductions
  int *done, *iter, *status;
  int* n_active;
  int maxit, flexible;
  double rtol;
};

}  // namespace pp

struct pp_batch_state {
  pp::BatchDev d;
  pp::BatchCols c;
  std::vector<int> n_h, R_h, cbase_h;
  std::vector<long long> voff_h, woff_h;
  long long vec_elems = 0, rows_pad = 0;
  int apply_prec = 0;
  // vectors (elements = vec_elems)
  double *x = nullptr, *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *t1 = nullptr, *t2 = nullptr;
  float *r32 = nullptr, *u32 = nullptr, *v32 = nullptr, *z32 = nullptr;
  double* part0 = nullptr;  // [slice][kBR]
  double* part1 = nullptr;
  double* lan_a = nullptr;   // [inst][m]
  double* lan_b2 = nullptr;  // [inst][m]
  double* nrm = nullptr;     // [inst]
  double *theta_bar = nullptr, *delta = nullptr, *sigma_bar = nullptr, *rho = nullptr;
  double* coefT = nullptr;   // [j][column][3] folded step coefficients (cheb_step_coeffs)
  double* feat = nullptr;    // [inst][4] device feature sums
  std::vector<double> abx;   // host (alpha, beta, xi) per column
  std::vector<double> ritz;  // host: per instance, lanczos Ritz extremes and more
  int lanczos_steps = 0;
  int nz_inst = 0;  // instances stepped by plane marching
  long long zclass[4] = {0, 0, 0, 0};  // their item offsets per register class
  cudaGraphExec_t graph = nullptr;
  cudaStream_t cap = nullptr;
  int graph_block = 0;
  // the plane-marching register classes run as concurrent branches: two side
  // streams forked from and joined back into the solver's stream by events
  cudaStream_t zs[2] = {nullptr, nullptr};
  cudaEvent_t zfork = nullptr, zjoin[2] = {nullptr, nullptr};
};

namespace pp {
namespace {

__device__ __forceinline__ long long bgw() { return ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ long long bnw() { return ((long long)gridDim.x * blockDim.x) >> 5; }

template <typename T>
__device__ __forceinline__ T ldv(const T* p) {
  return *p;
}

// ------------------------------------------------------------- products ---
// R consecutive vector entries of one row (the instance's right-hand sides).
template <typename T, int R>
struct RowVec {
  T v[R];
  __device__ __forceinline__ void load(const T* p) {
    if constexpr (sizeof(T) * R % 16 == 0) {
#pragma unroll
      for (int q = 0; q < (int)(sizeof(T) * R / 16); ++q) {
        const uint4 u = __ldg(reinterpret_cast<const uint4*>(p) + q);
        const T* t = reinterpret_cast<const T*>(&u);
#pragma unroll
        for (int e = 0; e < (int)(16 / sizeof(T)); ++e) v[q * (16 / sizeof(T)) + e] = t[e];
      }
    } else if constexpr (sizeof(T) * R == 8) {
      const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
      const T* t = reinterpret_cast<const T*>(&u);
#pragma unroll
      for (int e = 0; e < R; ++e) v[e] = t[e];
    } else {
#pragma unroll
      for (int e = 0; e < R; ++e) v[e] = __ldg(p + e);
    }
  }
  // plain (cached) load, for vectors the same kernel also writes
  __device__ __forceinline__ void load_rw(const T* p) {
    if constexpr (sizeof(T) * R % 16 == 0) {
#pragma unroll
      for (int q = 0; q < (int)(sizeof(T) * R / 16); ++q) {
        const uint4 u = reinterpret_cast<const uint4*>(p)[q];
        const T* t = reinterpret_cast<const T*>(&u);
#pragma unroll
        for (int e = 0; e < (int)(16 / sizeof(T)); ++e) v[q * (16 / sizeof(T)) + e] = t[e];
      }
    } else if constexpr (sizeof(T) * R == 8) {
      const uint2 u = *reinterpret_cast<const uint2*>(p);
      const T* t = reinterpret_cast<const T*>(&u);
#pragma unroll
      for (int e = 0; e < R; ++e) v[e] = t[e];
    } else {
#pragma unroll
      for (int e = 0; e < R; ++e) v[e] = p[e];
    }
  }
  __device__ __forceinline__ void store(T* p) const {
    if constexpr (sizeof(T) * R % 16 == 0) {
#pragma unroll
      for (int q = 0; q < (int)(sizeof(T) * R / 16); ++q) {
        uint4 u;
        T* t = reinterpret_cast<T*>(&u);
#pragma unroll
        for (int e = 0; e < (int)(16 / sizeof(T)); ++e) t[e] = v[q * (16 / sizeof(T)) + e];
        reinterpret_cast<uint4*>(p)[q] = u;
      }
    } else if constexpr (sizeof(T) * R == 8) {
      uint2 u;
      T* t = reinterpret_cast<T*>(&u);
#pragma unroll
      for (int e = 0; e < R; ++e) t[e] = v[e];
      *reinterpret_cast<uint2*>(p) = u;
    } else {
#pragma unroll
      for (int e = 0; e < R; ++e) p[e] = v[e];
    }
  }
};

// DIA mode: row sums of the instance's seed-scaled matrix for R right-hand
// sides ([row][rhs] vectors; stride RS with R = 1 for the Lanczos view):
// the unit diagonal, then each stored diagonal and its mirror.
template <typename TV, typename TX, int R>
__device__ __forceinline__ void b_dia_rowsum(const BatchDev& d, int i, long long row, const TV* __restrict__ dval,
                                             const TX* __restrict__ xi, int RS, TX (&acc)[R]) {
  if (R == 1 && RS != 1) {
    acc[0] = xi[row * RS];
  } else {
    RowVec<TX, R> xs;
    xs.load(xi + row * R);
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = xs.v[r];
  }
  const int nd = d.dia_nd[i];
  const long long base = d.dia_base[i] + d.dia_pad[i];
  const long long str = d.dia_stride[i];
  const long long last = (d.sbase[i + 1] - d.sbase[i]) * 32 - 1;
  for (int t = 0; t < nd; ++t) {
    const long long o = d.dia_off[i * kBDiag + t];
    const TV* U = dval + base + t * str;
    const TX up = (TX)U[row];      // a(row, row + o); 0 past the instance's last row
    const TX lo = (TX)U[row - o];  // a(row - o, row); 0 in the front pad
    const long long ju = row + o < last ? row + o : last;
    const long long jl = row - o > 0 ? row - o : 0;
    if (R == 1 && RS != 1) {
      acc[0] = fma(up, xi[ju * RS], fma(lo, xi[jl * RS], acc[0]));
    } else {
      RowVec<TX, R> xu, xl;
      xu.load(xi + ju * R);
      xl.load(xi + jl * R);
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = fma(up, xu.v[r], fma(lo, xl.v[r], acc[r]));
    }
  }
}

__device__ __forceinline__ unsigned active_mask(const int* done, int g0, int R) {
  unsigned m = 0;
  for (int r = 0; r < R; ++r)
    if (!done[g0 + r]) m |= 1u << r;
  return m;
}

// Column sums of one slice: lane l holds row l's R values v[0..R-1]; the sum
// of each column over the 32 lanes is written to out[0..R-1] by the lanes
// whose low bits are zero.  Recursive halving: each exchange with the lane
// 16, 8, ... apart halves the columns a lane keeps (it adds the half it
// keeps to the partner's copy of it), so a lane does (Rp - 1) + (5 - log2 Rp)
// FP64 additions (Rp = R rounded up to a power of 2) instead of 5 per column
// -- FP64 additions are scarce on this GPU.  The order of the additions is
// fixed, so the sums are deterministic.
template <int R>
__device__ __forceinline__ void slice_col_sums(const double (&v)[R], double* out, int lane) {
  constexpr int Rp = R <= 1 ? 1 : (R <= 2 ? 2 : (R <= 4 ? 4 : 8));
  constexpr int L = Rp == 1 ? 0 : (Rp == 2 ? 1 : (Rp == 4 ? 2 : 3));
  double w[Rp];
#pragma unroll
  for (int c = 0; c < Rp; ++c) w[c] = c < R ? v[c] : 0.0;
  int col = 0;
#pragma unroll
  for (int st = 0; st < L; ++st) {
    const int off = 16 >> st, h = Rp >> (st + 1);
    const bool up = (lane & off) != 0;
#pragma unroll
    for (int c = 0; c < h; ++c) {
      const double keep = up ? w[c + h] : w[c];
      const double send = up ? w[c] : w[c + h];
      w[c] = keep + __shfl_xor_sync(0xffffffffu, send, off);
    }
    if (up) col += h;
  }
  double t = w[0];
#pragma unroll
  for (int off = 16 >> L; off >= 1; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  if ((lane & ((32 >> L) - 1)) == 0 && col < R) out[col] = t;
}

// FP64 product of one slice for R right-hand sides: y = A x with partials
// (x, y) (kSpmv), or the Lanczos step on column 0 (R = 1 view).
template <int R, int MODE>
__device__ __forceinline__ void b_spmv_slice(const BatchDev& d, long long s, int i, int RS, const double* x,
                                             const double* xold, double* y, double coef, unsigned act,
                                             double* part) {
  const int lane = threadIdx.x & 31;
  const long long row = d.s_row0[s] + lane;
  const bool in = row < d.n[i];
  const double* xi = x + d.voff[i];
  double acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = 0.0;
  if (d.dia) {
    b_dia_rowsum<double, double, R>(d, i, row, d.dval64, xi, MODE == kLanczos ? RS : R, acc);
  } else {
    const long long base = d.sptr[s];
    const int w = (int)((d.sptr[s + 1] - base) / 32);
    for (int j = 0; j < w; ++j) {
      const double v = __ldcs(d.val64 + base + (long long)j * 32 + lane);
      const long long c = __ldcs(d.col + base + (long long)j * 32 + lane);
      RowVec<double, R> xv;
      if (MODE == kLanczos) xv.v[0] = __ldg(xi + c * RS); else xv.load(xi + c * R);
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = fma(v, xv.v[r], acc[r]);
    }
  }
  double pr[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    pr[r] = 0.0;
    const long long e = d.voff[i] + row * RS + r;
    if ((act >> r) & 1u) {
      double yv = acc[r];
      if (MODE == kLanczos && xold) yv -= coef * xold[e];
      y[e] = yv;
      if (in) pr[r] = x[e] * yv;
    }
  }
  slice_col_sums<R>(pr, part + s * kBR, lane);
}

template <int MODE>
__global__ void __launch_bounds__(kBlock) b_spmv64_kernel(BatchDev d, const double* __restrict__ x,
                                                          const double* __restrict__ xold, double* __restrict__ y,
                                                          const int* __restrict__ done, const double* b2prev, int lan_j,
                                                          double* __restrict__ part) {
  for (long long s = bgw(); s < d.nslices; s += bnw()) {
    const int i = d.s_inst[s];
    const int RS = d.R[i];
    if (MODE == kLanczos) {
      const double coef = lan_j > 0 ? sqrt(b2prev[(long long)i * kMaxLanczos + lan_j - 1]) : 0.0;
      b_spmv_slice<1, kLanczos>(d, s, i, RS, x, lan_j > 0 ? xold : nullptr, y, coef, 1u, part);
      continue;
    }
    const unsigned act = active_mask(done, d.cbase[i], RS);
    if (!act) continue;
    switch (RS) {
      case 1: b_spmv_slice<1, kSpmv>(d, s, i, RS, x, nullptr, y, 0.0, act, part); break;
      case 2: b_spmv_slice<2, kSpmv>(d, s, i, RS, x, nullptr, y, 0.0, act, part); break;
      case 3: b_spmv_slice<3, kSpmv>(d, s, i, RS, x, nullptr, y, 0.0, act, part); break;
      case 4: b_spmv_slice<4, kSpmv>(d, s, i, RS, x, nullptr, y, 0.0, act, part); break;
      case 5: b_spmv_slice<5, kSpmv>(d, s, i, RS, x, nullptr, y, 0.0, act, part); break;
      case 6: b_spmv_slice<6, kSpmv>(d, s, i, RS, x, nullptr, y, 0.0, act, part); break;
      case 7: b_spmv_slice<7, kSpmv>(d, s, i, RS, x, nullptr, y, 0.0, act, part); break;
      default: b_spmv_slice<8, kSpmv>(d, s, i, RS, x, nullptr, y, 0.0, act, part); break;
    }
  }
}

// Chebyshev degree step of one slice for R right-hand sides, with the folded
// per-column coefficients (ca, cb, cc) of this step (see cheb_step_coeffs):
//   kCheb1 y = ca r + cb (A r); kCheb2 y = ca x + cb r + cc (r - A x);
//   kChebK y = ca x + cb x_old + cc (r - A x).
template <typename TV, typename TX, int R, int MODE>
__device__ __forceinline__ void b_cheb_slice(const BatchDev& d, long long s, int i, const TV* val, const TX* x,
                                             const TX* xold, const TX* rin, TX* y, const double* coef, unsigned act) {
  const int lane = threadIdx.x & 31;
  const long long row = d.s_row0[s] + lane;
  const TX* xi = x + d.voff[i];
  TX acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = (TX)0;
  if (d.dia) {
    b_dia_rowsum<TV, TX, R>(d, i, row, val, xi, R, acc);  // val: the DIA values in this precision
  } else {
    const long long base = d.sptr[s];
    const int w = (int)((d.sptr[s + 1] - base) / 32);
    for (int jj = 0; jj < w; ++jj) {
      const TX v = (TX)__ldcs(val + base + (long long)jj * 32 + lane);
      const long long c = __ldcs(d.col + base + (long long)jj * 32 + lane);
      RowVec<TX, R> xv;
      xv.load(xi + c * R);
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = fma(v, xv.v[r], acc[r]);
    }
  }
  const long long e0 = d.voff[i] + row * R;
  RowVec<TX, R> rs, xs, xo;
  rs.load(rin + e0);
  if (MODE != kCheb1) xs.load(x + e0);
  if (MODE == kChebK) xo.load(xold + e0);
  const int g0 = d.cbase[i];
  TX out[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const double* cf = coef + (long long)(g0 + r) * 3;
    const TX ca = (TX)cf[0], cb = (TX)cf[1], cc = (TX)cf[2];
    if (MODE == kCheb1)
      out[r] = fma(cb, acc[r], ca * rs.v[r]);
    else if (MODE == kCheb2)
      out[r] = fma(cc, rs.v[r] - acc[r], fma(cb, rs.v[r], ca * xs.v[r]));
    else
      out[r] = fma(cc, rs.v[r] - acc[r], fma(cb, xo.v[r], ca * xs.v[r]));
  }
#pragma unroll
  for (int r = 0; r < R; ++r)
    if ((act >> r) & 1u) y[e0 + r] = out[r];
}

// DIA mode with 3 stored diagonals (the 7-point stencil), kBChunk slices of
// one instance per warp work item: the instance's metadata and column
// coefficients are read once per item instead of once per slice, and each
// lane walks kBChunk rows (row0 + lane + 32 q).  Stored diagonals stream with
// an evict-first L2 priority, r (read by every step) with evict-last.
constexpr int kBChunk = 4;

__device__ __forceinline__ uint64_t b_policy(bool last) {
  uint64_t pol;
  if (last)
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  else
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

template <typename T>
__device__ __forceinline__ T ld_pol(const T* p, uint64_t pol) {
  if constexpr (std::is_same<T, double>::value) {
    double v;
    asm("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(v) : "l"(p), "l"(pol));
    return v;
  } else {
    float v;
    asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(p), "l"(pol));
    return v;
  }
}

// R consecutive floats of a row vector with an L2 cache hint, as 16- or
// 8-byte accesses where the row allows (the RowVec rule: a multiple of 16
// bytes per row from a 32-element aligned base; 8 bytes for R = 2).
template <int R>
__device__ __forceinline__ void ld_pol_row(const float* p, uint64_t pol, float (&o)[R]) {
  if constexpr (R % 4 == 0) {
#pragma unroll
    for (int q = 0; q < R / 4; ++q)
      asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
          : "=f"(o[4 * q]), "=f"(o[4 * q + 1]), "=f"(o[4 * q + 2]), "=f"(o[4 * q + 3])
          : "l"(p + 4 * q), "l"(pol));
  } else if constexpr (R == 2) {
    asm("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;" : "=f"(o[0]), "=f"(o[1]) : "l"(p), "l"(pol));
  } else {
#pragma unroll
    for (int r = 0; r < R; ++r) o[r] = ld_pol<float>(p + r, pol);
  }
}

template <typename TV, typename TX, int R, int MODE>
__device__ __forceinline__ void b_cheb_dia3_chunk(const BatchDev& d, int i, long long row0, const TV* val,
                                                  const TX* x, const TX* xold, const TX* rin, TX* y,
                                                  const double* coef, unsigned act, uint64_t pol_first,
                                                  uint64_t pol_last) {
  const int lane = threadIdx.x & 31;
  const long long vo = d.voff[i];
  const TX* xi = x + vo;
  const long long base = d.dia_base[i] + d.dia_pad[i];
  const long long str = d.dia_stride[i];
  const long long last = (d.sbase[i + 1] - d.sbase[i]) * 32 - 1;
  const long long o[3] = {d.dia_off[i * kBDiag], d.dia_off[i * kBDiag + 1], d.dia_off[i * kBDiag + 2]};
  const double* cf0 = coef + (long long)d.cbase[i] * 3;
#pragma unroll 1
  for (int q = 0; q < kBChunk; ++q) {
    const long long row = row0 + lane + 32 * q;
    TX acc[R];
    {
      RowVec<TX, R> xs0;
      xs0.load(xi + row * R);
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = xs0.v[r];  // the unit diagonal
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const TV* U = val + base + t * str;
      const TX up = (TX)ld_pol<TV>(U + row, pol_first);
      const TX lo = (TX)ld_pol<TV>(U + row - o[t], pol_first);
      const long long ju = row + o[t] < last ? row + o[t] : last;
      const long long jl = row - o[t] > 0 ? row - o[t] : 0;
      RowVec<TX, R> xu, xl;
      xu.load(xi + ju * R);
      xl.load(xi + jl * R);
#pragma unroll
      for (int r = 0; r < R; ++r) acc[r] = fma(up, xu.v[r], fma(lo, xl.v[r], acc[r]));
    }
    const long long e0 = vo + row * R;
    TX rs[R];
#pragma unroll
    for (int r = 0; r < R; ++r) rs[r] = ld_pol<TX>(rin + e0 + r, pol_last);
    RowVec<TX, R> xs, xo;
    if (MODE != kCheb1) xs.load(x + e0);
    if (MODE == kChebK) xo.load(xold + e0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const TX ca = (TX)__ldg(cf0 + 3 * r), cb = (TX)__ldg(cf0 + 3 * r + 1), cc = (TX)__ldg(cf0 + 3 * r + 2);
      TX out;
      if (MODE == kCheb1)
        out = fma(cb, acc[r], ca * rs[r]);
      else if (MODE == kCheb2)
        out = fma(cc, rs[r] - acc[r], fma(cb, rs[r], ca * xs.v[r]));
      else
        out = fma(cc, rs[r] - acc[r], fma(cb, xo.v[r], ca * xs.v[r]));
      if ((act >> r) & 1u) y[e0 + r] = out;
    }
  }
}

// TZ: some instances are stepped by b_cheb_z_kernel and skipped here.
template <typename TV, typename TX, int MODE, bool TZ>
__global__ void __launch_bounds__(kBlock, std::is_same<TX, float>::value ? 3 : 2) b_cheb_dia3_kernel(BatchDev d, const TV* __restrict__ val,
                                                             const TX* __restrict__ x, const TX* __restrict__ xold,
                                                             const TX* __restrict__ rin, TX* __restrict__ y,
                                                             const int* __restrict__ done,
                                                             const double* __restrict__ coef) {
  const uint64_t pol_first = b_policy(false), pol_last = b_policy(true);
  const long long nchunks = (d.nslices + kBChunk - 1) / kBChunk;
  for (long long c = bgw(); c < nchunks; c += bnw()) {
    const long long s0 = c * kBChunk;
    const long long s1 = s0 + kBChunk <= d.nslices ? s0 + kBChunk : d.nslices;
    const int i = d.s_inst[s0];
    const int R = d.R[i];
    const unsigned act = active_mask(done, d.cbase[i], R);
    const bool whole = s1 - s0 == kBChunk && d.s_inst[s1 - 1] == i && d.dia_nd[i] == 3;
    if (!whole) {  // an item that spans instances (or is short): slice by slice
      for (long long s = s0; s < s1; ++s) {
        const int is = d.s_inst[s];
        if (TZ && d.zmode[is]) continue;  // stepped by b_cheb_z_kernel
        const int Rs = d.R[is];
        const unsigned as = active_mask(done, d.cbase[is], Rs);
        if (!as) continue;
        switch (Rs) {
          case 1: b_cheb_slice<TV, TX, 1, MODE>(d, s, is, val, x, xold, rin, y, coef, as); break;
          case 2: b_cheb_slice<TV, TX, 2, MODE>(d, s, is, val, x, xold, rin, y, coef, as); break;
          case 3: b_cheb_slice<TV, TX, 3, MODE>(d, s, is, val, x, xold, rin, y, coef, as); break;
          case 4: b_cheb_slice<TV, TX, 4, MODE>(d, s, is, val, x, xold, rin, y, coef, as); break;
          case 5: b_cheb_slice<TV, TX, 5, MODE>(d, s, is, val, x, xold, rin, y, coef, as); break;
          case 6: b_cheb_slice<TV, TX, 6, MODE>(d, s, is, val, x, xold, rin, y, coef, as); break;
          case 7: b_cheb_slice<TV, TX, 7, MODE>(d, s, is, val, x, xold, rin, y, coef, as); break;
          default: b_cheb_slice<TV, TX, 8, MODE>(d, s, is, val, x, xold, rin, y, coef, as); break;
        }
      }
      continue;
    }
    if (!act || (TZ && d.zmode[i])) continue;
    const long long row0 = d.s_row0[s0];
    switch (R) {
      case 1: b_cheb_dia3_chunk<TV, TX, 1, MODE>(d, i, row0, val, x, xold, rin, y, coef, act, pol_first, pol_last); break;
      case 2: b_cheb_dia3_chunk<TV, TX, 2, MODE>(d, i, row0, val, x, xold, rin, y, coef, act, pol_first, pol_last); break;
      case 3: b_cheb_dia3_chunk<TV, TX, 3, MODE>(d, i, row0, val, x, xold, rin, y, coef, act, pol_first, pol_last); break;
      case 4: b_cheb_dia3_chunk<TV, TX, 4, MODE>(d, i, row0, val, x, xold, rin, y, coef, act, pol_first, pol_last); break;
      case 5: b_cheb_dia3_chunk<TV, TX, 5, MODE>(d, i, row0, val, x, xold, rin, y, coef, act, pol_first, pol_last); break;
      case 6: b_cheb_dia3_chunk<TV, TX, 6, MODE>(d, i, row0, val, x, xold, rin, y, coef, act, pol_first, pol_last); break;
      case 7: b_cheb_dia3_chunk<TV, TX, 7, MODE>(d, i, row0, val, x, xold, rin, y, coef, act, pol_first, pol_last); break;
      default: b_cheb_dia3_chunk<TV, TX, 8, MODE>(d, i, row0, val, x, xold, rin, y, coef, act, pol_first, pol_last); break;
    }
  }
}

// Plane marching for the instances of a structured grid (FP32 values and
// vectors): a thread owns one grid column (x, y) of a 32 x 8 tile with all R
// right-hand sides and walks z through the item's planes, so the z-neighbours
// x(z - 1), x(z + 1) and the lower z-entry come from registers (the planes it
// loaded before) and the in-plane neighbours from L1 (loaded by the
// neighbouring threads of the same step); the slice kernel reads those from
// L2.  Neighbour rows are clipped to the instance's padded rows like the
// slice kernel's; their matrix entries are 0.  The same sums as the slice
// kernel: A x = x + sum over the three diagonals of (upper, lower) terms.
template <int R, int MODE>
__device__ __forceinline__ void b_z_item(const BatchDev& d, const BZItem it, const float* __restrict__ val,
                                         const float* __restrict__ x, const float* __restrict__ xold,
                                         const float* __restrict__ rin, float* __restrict__ y,
                                         const double* __restrict__ coef, unsigned act, uint64_t pol_first,
                                         uint64_t pol_last) {
  const int i = it.inst;
  const int Nx = d.dia_off[i * kBDiag + 1];
  const long long nxy = d.dia_off[i * kBDiag + 2];
  const int Ny = (int)(nxy / Nx);
  const int xx = it.x0 + (int)(threadIdx.x & 31), yy = it.y0 + (int)(threadIdx.x >> 5);
  if (xx >= Nx || yy >= Ny) return;
  const long long vo = d.voff[i];
  const float* X = x + vo;
  const long long last = (d.sbase[i + 1] - d.sbase[i]) * 32 - 1;
  const long long str = d.dia_stride[i];
  const float* U0 = val + d.dia_base[i] + d.dia_pad[i];
  const float* U1 = U0 + str;
  const float* U2 = U1 + str;
  float ca[R], cb[R], cc[R];
  const double* cf0 = coef + (long long)d.cbase[i] * 3;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    ca[r] = (float)__ldg(cf0 + 3 * r);
    cb[r] = (float)__ldg(cf0 + 3 * r + 1);
    cc[r] = (float)__ldg(cf0 + 3 * r + 2);
  }
  auto clip = [&](long long j) { return j < 0 ? 0LL : (j > last ? last : j); };
  long long row = xx + (long long)Nx * yy + nxy * it.z0;
  RowVec<float, R> xm, xc;
  xm.load(X + clip(row - nxy) * R);
  xc.load(X + row * R);
  float l2 = ld_pol<float>(U2 + row - nxy, pol_first);  // a(row - nxy, row); 0 in the front pad
#pragma unroll 1
  for (int z = it.z0; z < it.z1; ++z, row += nxy) {
    RowVec<float, R> xp, xw, xe, xs, xn;
    xp.load(X + clip(row + nxy) * R);
    const float u0 = ld_pol<float>(U0 + row, pol_first);
    const float u1 = ld_pol<float>(U1 + row, pol_first);
    const float u2 = ld_pol<float>(U2 + row, pol_first);
    const float l0 = __ldg(U0 + row - 1);
    const float l1 = __ldg(U1 + row - Nx);
    xw.load(X + clip(row - 1) * R);
    xe.load(X + clip(row + 1) * R);
    xs.load(X + clip(row - Nx) * R);
    xn.load(X + clip(row + Nx) * R);
    const long long e0 = vo + row * R;
    float rs[R];
    ld_pol_row<R>(rin + e0, pol_last, rs);
    RowVec<float, R> xo;
    if (MODE == kChebK) xo.load(xold + e0);
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float acc = xc.v[r];
      acc = fmaf(u0, xe.v[r], fmaf(l0, xw.v[r], acc));
      acc = fmaf(u1, xn.v[r], fmaf(l1, xs.v[r], acc));
      acc = fmaf(u2, xp.v[r], fmaf(l2, xm.v[r], acc));
      float out;
      if (MODE == kCheb1)
        out = fmaf(cb[r], acc, ca[r] * rs[r]);
      else if (MODE == kCheb2)
        out = fmaf(cc[r], rs[r] - acc, fmaf(cb[r], rs[r], ca[r] * xc.v[r]));
      else
        out = fmaf(cc[r], rs[r] - acc, fmaf(cb[r], xo.v[r], ca[r] * xc.v[r]));
      if ((act >> r) & 1u) y[e0 + r] = out;
    }
    xm = xc;
    xc = xp;
    l2 = u2;
  }
}

// One plane-marching item per block, items item0 + blockIdx.x of the
// instances with RLO..RHI right-hand sides (one launch per register class:
// the R = 8 path needs three times the registers of R = 1).  Within a class
// the items are ordered by decreasing work, so the block scheduler hands the
// large ones out first.  No barriers.
template <int RLO, int RHI, int MODE>
__global__ void __launch_bounds__(kBlock) b_cheb_z_kernel(BatchDev d, long long item0, const float* __restrict__ val,
                                                          const float* __restrict__ x,
                                                          const float* __restrict__ xold,
                                                          const float* __restrict__ rin, float* __restrict__ y,
                                                          const int* __restrict__ done,
                                                          const double* __restrict__ coef) {
  const BZItem it = d.zitem[item0 + blockIdx.x];
  const int R = d.R[it.inst];
  const unsigned act = active_mask(done, d.cbase[it.inst], R);
  if (!act || R < RLO || R > RHI) return;
  const uint64_t pol_first = b_policy(false), pol_last = b_policy(true);
#define PP_BZ_CASE(RR)                                                                           \
  case RR:                                                                                       \
    if constexpr (RR >= RLO && RR <= RHI)                                                        \
      b_z_item<RR, MODE>(d, it, val, x, xold, rin, y, coef, act, pol_first, pol_last);           \
    break;
  switch (R) {
    PP_BZ_CASE(1)
    PP_BZ_CASE(2)
    PP_BZ_CASE(3)
    PP_BZ_CASE(4)
    PP_BZ_CASE(5)
    PP_BZ_CASE(6)
    PP_BZ_CASE(7)
    PP_BZ_CASE(8)
    default: break;
  }
#undef PP_BZ_CASE
}

// The register classes of the plane-marching step: R in [kBZClass[c], kBZClass[c + 1]).
constexpr int kBZClasses = 3;
constexpr int kBZClass[kBZClasses + 1] = {1, 3, 5, kBR + 1};

template <typename TV, typename TX, int MODE>
__global__ void __launch_bounds__(kBlock) b_cheb_kernel(BatchDev d, const TV* __restrict__ val, const TX* __restrict__ x,
                                                        const TX* __restrict__ xold, const TX* __restrict__ rin,
                                                        TX* __restrict__ y, const int* __restrict__ done,
                                                        const double* __restrict__ coef) {
  for (long long s = bgw(); s < d.nslices; s += bnw()) {
    const int i = d.s_inst[s];
    const int R = d.R[i];
    const unsigned act = active_mask(done, d.cbase[i], R);
    if (!act) continue;
    switch (R) {
      case 1: b_cheb_slice<TV, TX, 1, MODE>(d, s, i, val, x, xold, rin, y, coef, act); break;
      case 2: b_cheb_slice<TV, TX, 2, MODE>(d, s, i, val, x, xold, rin, y, coef, act); break;
      case 3: b_cheb_slice<TV, TX, 3, MODE>(d, s, i, val, x, xold, rin, y, coef, act); break;
      case 4: b_cheb_slice<TV, TX, 4, MODE>(d, s, i, val, x, xold, rin, y, coef, act); break;
      case 5: b_cheb_slice<TV, TX, 5, MODE>(d, s, i, val, x, xold, rin, y, coef, act); break;
      case 6: b_cheb_slice<TV, TX, 6, MODE>(d, s, i, val, x, xold, rin, y, coef, act); break;
      case 7: b_cheb_slice<TV, TX, 7, MODE>(d, s, i, val, x, xold, rin, y, coef, act); break;
      default: b_cheb_slice<TV, TX, 8, MODE>(d, s, i, val, x, xold, rin, y, coef, act); break;
    }
  }
}

// ------------------------------------------------------------ vectors -----
// Per-element loops walk slices too (lane = row, r < R) so that partial sums
// line up with the product kernels.
// With the FP32 preconditioner the iteration uses the fused forms: kBUpdXR32
// also writes r32 (no separate kBTo32 pass), kBDots32 forms (r, z) and (q, z)
// from z32 without storing z in FP64, and kBUpdP32 reads z32.
enum BVec { kBScaleIn = 0, kBUpdXR = 1, kBTo32 = 2, kBFrom32 = 3, kBUpdP = 4, kBScaleOut = 5, kBZtoP = 6,
            kBDeg0 = 7, kBUpdXR32 = 8, kBDots32 = 9, kBUpdP32 = 10 };

// ns consecutive slices s0.. of instance i (lane = row): every row's R
// entries of a vector are loaded and stored as one row vector (16-byte
// accesses where R allows), and the per-column partial sums of all ns slices
// are accumulated per lane and reduced once (slice_col_sums) into the
// chunk's first slice; the other slices of the chunk get zeros, so the
// segmented reduction's sum over the instance's slices is unchanged.
template <int OP, int R>
__device__ __forceinline__ void b_vec_rows(const BatchDev& d, const BatchCols& cc, long long s0, int ns, int i,
                                           unsigned act, const double* bin, double* xout, double* x, double* r,
                                           double* z, double* p, const double* q, float* r32, const float* z32,
                                           double* part0, double* part1, int first) {
  constexpr bool sums = OP == kBScaleIn || OP == kBUpdXR || OP == kBUpdXR32 || OP == kBFrom32 || OP == kBDots32 ||
                        OP == kBZtoP || OP == kBDeg0;
  constexpr bool two = OP == kBFrom32 || OP == kBDots32 || OP == kBZtoP || OP == kBDeg0;
  const int lane = threadIdx.x & 31;
  const int g0 = d.cbase[i];
  double p0[R], p1[R];
  double al[R], be[R];
  bool ok[R];
#pragma unroll
  for (int rr = 0; rr < R; ++rr) {
    p0[rr] = 0.0;
    p1[rr] = 0.0;
    const bool a = (OP == kBScaleIn || OP == kBScaleOut) || ((act >> rr) & 1u);
    ok[rr] = a;
    al[rr] = 0.0;
    be[rr] = 0.0;
    if (OP == kBUpdXR || OP == kBUpdXR32) {
      const double pq = cc.pq[g0 + rr];
      ok[rr] = a && pq > 0.0 && isfinite(pq);
      al[rr] = cc.al[g0 + rr];  // (r, z) / (p, q), formed by the reduction
    }
    if ((OP == kBUpdP || OP == kBUpdP32) && !first) be[rr] = cc.be[g0 + rr];
  }
  for (int j = 0; j < ns; ++j) {
    const long long s = s0 + j;
    const long long row = d.s_row0[s] + lane;
    const bool in = row < d.n[i];
    const long long e0 = d.voff[i] + row * R;
    if (OP == kBScaleIn) {
      const double wr = in ? d.w[d.woff[i] + row] : 1.0;
      RowVec<double, R> rv, xv;
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        const double v = in ? wr * bin[d.uoff[i] + row * R + rr] : 0.0;
        rv.v[rr] = v;
        xv.v[rr] = 0.0;
        p0[rr] += v * v;
      }
      rv.store(r + e0);
      xv.store(x + e0);
    } else if (OP == kBScaleOut) {
      if (in) {
        const double wr = d.w[d.woff[i] + row];
        RowVec<double, R> xv;
        xv.load_rw(x + e0);
#pragma unroll
        for (int rr = 0; rr < R; ++rr) xout[d.uoff[i] + row * R + rr] = wr * xv.v[rr];
      }
    } else if (OP == kBUpdXR || OP == kBUpdXR32) {
      RowVec<double, R> xv, pv, rv, qv;
      xv.load_rw(x + e0);
      pv.load_rw(p + e0);
      rv.load_rw(r + e0);
      qv.load_rw(q + e0);
#pragma unroll
      for (int rr = 0; rr < R; ++rr) {
        if (!ok[rr]) continue;
        xv.v[rr] = fma(al[rr], pv.v[rr], xv.v[rr]);
        rv.v[rr] = fma(-al[rr], qv.v[rr], rv.v[rr]);
        if (in) p0[rr] = fma(rv.v[rr], rv.v[rr], p0[rr]);
      }
      xv.store(x + e0);
      rv.store(r + e0);
      if (OP == kBUpdXR32) {
        RowVec<float, R> r3;
#pragma unroll
        for (int rr = 0; rr < R; ++rr) r3.v[rr] = (float)rv.v[rr];
        r3.store(r32 + e0);
      }
    } else if (OP == kBTo32) {
      RowVec<double, R> rv;
      rv.load_rw(r + e0);
      RowVec<float, R> r3;
#pragma unroll
      for (int rr = 0; rr < R; ++rr) r3.v[rr] = (float)rv.v[rr];
      r3.store(r32 + e0);
    } else if (OP == kBFrom32 || OP == kBDots32 || OP == kBZtoP || OP == kBDeg0) {
      RowVec<double, R> rv, qv, zv;
      rv.load_rw(r + e0);
      qv.load_rw(q + e0);
      if (OP == kBFrom32 || OP == kBDots32) {
        RowVec<float, R> z3;
        z3.load_rw(z32 + e0);
#pragma unroll
        for (int rr = 0; rr < R; ++rr) zv.v[rr] = (double)z3.v[rr];
      } else if (OP == kBZtoP) {
        zv.load_rw(z + e0);
      } else {
#pragma unroll
        for (int rr = 0; rr < R; ++rr) zv.v[rr] = rv.v[rr] / d.theta_bar[g0 + rr];
      }
      if (OP == kBFrom32 || OP == kBDeg0) zv.store(z + e0);
      if (in) {
#pragma unroll
        for (int rr = 0; rr < R; ++rr) {
          if (!ok[rr]) continue;
          p0[rr] = fma(rv.v[rr], zv.v[rr], p0[rr]);
          p1[rr] = fma(qv.v[rr], zv.v[rr], p1[rr]);
        }
      }
    } else if (OP == kBUpdP || OP == kBUpdP32) {
      RowVec<double, R> pv, zv;
      pv.load_rw(p + e0);
      if (OP == kBUpdP32) {
        RowVec<float, R> z3;
        z3.load_rw(z32 + e0);
#pragma unroll
        for (int rr = 0; rr < R; ++rr) zv.v[rr] = (double)z3.v[rr];
      } else {
        zv.load_rw(z + e0);
      }
#pragma unroll
      for (int rr = 0; rr < R; ++rr)
        if (ok[rr]) pv.v[rr] = fma(be[rr], pv.v[rr], zv.v[rr]);
      pv.store(p + e0);
    }
  }
  if (sums) {
    slice_col_sums<R>(p0, part0 + s0 * kBR, lane);
    if (two && part1) slice_col_sums<R>(p1, part1 + s0 * kBR, lane);
    if (lane < R) {
      for (int j = 1; j < ns; ++j) {
        part0[(s0 + j) * kBR + lane] = 0.0;
        if (two && part1) part1[(s0 + j) * kBR + lane] = 0.0;
      }
    }
  }
}

// Work items of kBChunk slices; an item that spans instances (or is short)
// goes slice by slice.
template <int OP>
__global__ void __launch_bounds__(kBlock) b_vec_kernel(BatchDev d, BatchCols cc, const double* __restrict__ bin,
                                                       double* __restrict__ xout, double* x, double* r, double* z,
                                                       double* p, const double* q, float* r32, const float* z32,
                                                       double* __restrict__ part0, double* __restrict__ part1,
                                                       int first) {
  const long long nchunks = (d.nslices + kBChunk - 1) / kBChunk;
  for (long long c = bgw(); c < nchunks; c += bnw()) {
    const long long c0 = c * kBChunk;
    const long long c1 = c0 + kBChunk <= d.nslices ? c0 + kBChunk : d.nslices;
    const bool whole = c1 - c0 == kBChunk && d.s_inst[c0] == d.s_inst[c1 - 1];
    for (long long s = c0; s < c1; s += whole ? kBChunk : 1) {
      const int ns = whole ? kBChunk : 1;
      const int i = d.s_inst[s];
      const int R = d.R[i];
      const unsigned act = (OP == kBScaleIn || OP == kBScaleOut) ? 0xffu : active_mask(cc.done, d.cbase[i], R);
      if (!act) continue;
#define PP_BV(RR)                                                                                          \
  b_vec_rows<OP, RR>(d, cc, s, ns, i, act, bin, xout, x, r, z, p, q, r32, z32, part0, part1, first); \
  break;
      switch (R) {
        case 1: PP_BV(1)
        case 2: PP_BV(2)
        case 3: PP_BV(3)
        case 4: PP_BV(4)
        case 5: PP_BV(5)
        case 6: PP_BV(6)
        case 7: PP_BV(7)
        default: PP_BV(8)
      }
#undef PP_BV
    }
  }
}

// ------------------------------------------------------ segmented reduce --
enum BRed { kRedBB = 0, kRedPQ = 1, kRedRR = 2, kRedRZ = 3, kRedLanA = 4, kRedLanB = 5, kRedNrm = 6 };

// One block per global column (or per instance for the Lanczos values):
// adds the partials of the instance's slices in slice order.
template <int OP>
__global__ void __launch_bounds__(kBlock) b_reduce_kernel(BatchDev d, BatchCols cc, const double* __restrict__ part0,
                                                          const double* __restrict__ part1, double* lan_out,
                                                          int lan_j) {
  const int nitems = (OP == kRedLanA || OP == kRedLanB || OP == kRedNrm) ? d.nb : d.ncols;
  for (int g = blockIdx.x; g < nitems; g += gridDim.x) {
    int i, r;
    if (OP == kRedLanA || OP == kRedLanB || OP == kRedNrm) {
      i = g;
      r = 0;
    } else {
      i = d.ccol_inst[g];
      r = g - d.cbase[i];
    }
    if (OP != kRedBB && OP != kRedLanA && OP != kRedLanB && OP != kRedNrm && cc.done[g]) continue;
    const long long s0 = d.sbase[i], s1 = d.sbase[i + 1];
    double v[2] = {0.0, 0.0};
    for (long long s = s0 + threadIdx.x; s < s1; s += blockDim.x) {
      v[0] += part0[s * kBR + r];
      if (OP == kRedRZ) v[1] += part1[s * kBR + r];
    }
    block_sum<2>(v);
    if (threadIdx.x == 0) {
      if (OP == kRedBB) {
        cc.bb[g] = v[0];
        cc.rr[g] = v[0];
        cc.rtol2[g] = cc.rtol * cc.rtol * v[0];
        cc.iter[g] = 0;
        cc.status[g] = 1;
        cc.done[g] = 0;
        if (!isfinite(v[0])) {
          cc.status[g] = -3;
          cc.done[g] = 1;
        } else if (v[0] == 0.0) {
          cc.status[g] = 0;
          cc.done[g] = 1;
        }
        if (cc.done[g]) atomicSub(cc.n_active, 1);
      } else if (OP == kRedPQ) {
        cc.rz[g] = cc.rz_new[g];
        cc.pq[g] = v[0];
        cc.al[g] = (v[0] > 0.0 && isfinite(v[0])) ? cc.rz[g] / v[0] : 0.0;
        if (!(v[0] > 0.0)) {
          cc.status[g] = isfinite(v[0]) ? -2 : -3;
          cc.done[g] = 1;
          atomicSub(cc.n_active, 1);
        }
      } else if (OP == kRedRR) {
        cc.rr[g] = v[0];
        cc.iter[g] += 1;
        int st = 1;
        bool fin = false;
        if (!isfinite(v[0])) {
          st = -3;
          fin = true;
        } else if (v[0] <= cc.rtol2[g]) {
          st = 0;
          fin = true;
        } else if (cc.iter[g] >= cc.maxit) {
          st = 1;
          fin = true;
        }
        if (fin) {
          cc.status[g] = st;
          cc.done[g] = 1;
          atomicSub(cc.n_active, 1);
        }
      } else if (OP == kRedRZ) {
        cc.rz_new[g] = v[0];
        cc.zq[g] = v[1];
        // beta of the next direction update (unused by the first one)
        cc.be[g] = cc.flexible ? -v[1] / cc.pq[g] : v[0] / cc.rz[g];
        if (!(v[0] > 0.0)) {
          cc.status[g] = isfinite(v[0]) ? -2 : -3;
          cc.done[g] = 1;
          atomicSub(cc.n_active, 1);
        }
      } else {
        lan_out[(long long)i * kMaxLanczos + lan_j] = v[0];
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ Lanczos -----
__global__ void __launch_bounds__(kBlock) b_lan_start_kernel(BatchDev d, unsigned long long seed, double* v,
                                                             double* part) {
  const int lane = threadIdx.x & 31;
  for (long long s = bgw(); s < d.nslices; s += bnw()) {
    const int i = d.s_inst[s];
    const int R = d.R[i];
    const long long row = d.s_row0[s] + lane;
    const bool in = row < d.n[i];
    const uint64_t key = splitmix_key(seed + (unsigned long long)i, 3);
    const double x = in ? 2.0 * splitmix_uniform(key, (uint64_t)row) - 1.0 : 0.0;
    v[d.voff[i] + row * R] = x;
    const double pr = warp_sum(x * x);
    if (lane == 0) part[s * kBR] = pr;
  }
}

// OP 0: v /= sqrt(nrm[i]); OP 1: w -= a_j v with partial ||w||^2
template <int OP>
__global__ void __launch_bounds__(kBlock) b_lan_vec_kernel(BatchDev d, double* a, const double* v, const double* coef,
                                                           int j, double* part) {
  const int lane = threadIdx.x & 31;
  for (long long s = bgw(); s < d.nslices; s += bnw()) {
    const int i = d.s_inst[s];
    const int R = d.R[i];
    const long long row = d.s_row0[s] + lane;
    const bool in = row < d.n[i];
    const long long e = d.voff[i] + row * R;
    double pr = 0.0;
    if (OP == 0) {
      const double nv = sqrt(coef[(long long)i * kMaxLanczos + j]);
      if (in) a[e] = a[e] / nv;
    } else {
      if (in) {
        const double wv = a[e] - coef[(long long)i * kMaxLanczos + j] * v[e];
        a[e] = wv;
        pr = wv * wv;
      }
      pr = warp_sum(pr);
      if (lane == 0) part[s * kBR] = pr;
    }
  }
}

// Per-instance feature sums of the seed-scaled matrix: sum log diag(A),
// sum (log diag)^2, Gershgorin max of row sums of |A_hat|, min of
// (A_hat_ii - off-diagonal sum).
__global__ void __launch_bounds__(kBlock) b_feature_kernel(BatchDev d, const double* __restrict__ diag_log,
                                                           double* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  for (long long s = bgw(); s < d.nslices; s += bnw()) {
    const int i = d.s_inst[s];
    const long long row = d.s_row0[s] + lane;
    const bool in = row < d.n[i];
    double off = 0.0, dg = 0.0;
    if (d.dia) {
      dg = 1.0;
      const long long b0 = d.dia_base[i] + d.dia_pad[i];
      for (int t = 0; t < d.dia_nd[i]; ++t) {
        const double* U = d.dval64 + b0 + t * d.dia_stride[i];
        off += fabs(U[row]) + fabs(U[row - d.dia_off[i * kBDiag + t]]);
      }
    } else {
      const long long base = d.sptr[s];
      const int w = (int)((d.sptr[s + 1] - base) / 32);
      for (int j = 0; j < w; ++j) {
        const double v = d.val64[base + (long long)j * 32 + lane];
        const long long c = d.col[base + (long long)j * 32 + lane];
        if (c == row) dg += v; else off += fabs(v);
      }
    }
    const double dl = in ? diag_log[d.woff[i] + row] : 0.0;
    double a0 = warp_sum(dl), a1 = warp_sum(dl * dl);
    double mx = in ? dg + off : 0.0, mn = in ? dg - off : 1e300;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, o));
      mn = fmin(mn, __shfl_down_sync(0xffffffffu, mn, o));
    }
    if (lane == 0) {
      part[s * kBR + 0] = a0;
      part[s * kBR + 1] = a1;
      part[s * kBR + 2] = mx;
      part[s * kBR + 3] = mn;
    }
  }
}

__global__ void b_feature_reduce_kernel(BatchDev d, const double* part, double* feat) {
  for (int i = blockIdx.x; i < d.nb; i += gridDim.x) {
    if (threadIdx.x != 0) continue;
    double a0 = 0, a1 = 0, mx = 0, mn = 1e300;
    for (long long s = d.sbase[i]; s < d.sbase[i + 1]; ++s) {
      a0 += part[s * kBR + 0];
      a1 += part[s * kBR + 1];
      mx = fmax(mx, part[s * kBR + 2]);
      mn = fmin(mn, part[s * kBR + 3]);
    }
    feat[i * 4 + 0] = a0;
    feat[i * 4 + 1] = a1;
    feat[i * 4 + 2] = mx;
    feat[i * 4 + 3] = mn;
  }
}

// ------------------------------------------------------------- setup ------
__global__ void b_fill_kernel(BatchDev d, const int* const* rowptrs, const int* const* cols,
                              const double* const* vals, double* __restrict__ w, double* __restrict__ diag_log,
                              int* __restrict__ ocol, double* __restrict__ oval, int* bad) {
  const int lane = threadIdx.x & 31;
  for (long long s = bgw(); s < d.nslices; s += bnw()) {
    const int i = d.s_inst[s];
    const long long row = d.s_row0[s] + lane;
    const bool in = row < d.n[i];
    if (ocol) {  // SELL mode
      const long long base = d.sptr[s];
      const int wd = (int)((d.sptr[s + 1] - base) / 32);
      int j = 0;
      if (in) {
        const int* rp = rowptrs[i];
        const int* ci = cols[i];
        const double* va = vals[i];
        for (int p = rp[row]; p < rp[row + 1]; ++p, ++j) {
          ocol[base + (long long)j * 32 + lane] = ci[p];
          oval[base + (long long)j * 32 + lane] = va[p];
        }
      }
      for (; j < wd; ++j) {
        ocol[base + (long long)j * 32 + lane] = in ? (int)row : 0;
        oval[base + (long long)j * 32 + lane] = 0.0;
      }
    }
    if (in) {
      double dg = 0.0;
      const int* rp = rowptrs[i];
      for (int p = rp[row]; p < rp[row + 1]; ++p)
        if (cols[i][p] == row) dg += vals[i][p];
      if (!(dg > 0.0)) atomicExch(bad, 1);
      w[d.woff[i] + row] = dg > 0.0 ? 1.0 / sqrt(dg) : 1.0;
      diag_log[d.woff[i] + row] = dg > 0.0 ? log(dg) : 0.0;
    }
  }
}

// DIA mode: every entry of instance i lies on one of its offsets (or their
// mirrors) and a(c, row) == a(row, c) exactly; otherwise bad[i] = 1.
__global__ void b_dia_check_kernel(BatchDev d, const int* const* rowptrs, const int* const* cols,
                                   const double* const* vals, int* __restrict__ bad) {
  const int lane = threadIdx.x & 31;
  for (long long s = bgw(); s < d.nslices; s += bnw()) {
    const int i = d.s_inst[s];
    const long long row = d.s_row0[s] + lane;
    if (row >= d.n[i]) continue;
    const int* rp = rowptrs[i];
    const int* ci = cols[i];
    const double* va = vals[i];
    bool ok = true;
    for (int p = rp[row]; p < rp[row + 1] && ok; ++p) {
      const long long c = ci[p];
      const long long o = c > row ? c - row : row - c;
      if (o == 0) continue;
      bool on = false;
      for (int t = 0; t < d.dia_nd[i]; ++t) on = on || (d.dia_off[i * kBDiag + t] == o);
      bool mirror = false;
      for (int q = rp[c]; q < rp[c + 1]; ++q)
        if (ci[q] == row) {
          mirror = va[q] == va[p];
          break;
        }
      ok = on && mirror;
    }
    if (!ok) atomicExch(bad + i, 1);
  }
}

// DIA mode: the seed-scaled upper entries w_row a w_col into their diagonals.
__global__ void b_dia_fill_kernel(BatchDev d, const int* const* rowptrs, const int* const* cols,
                                  const double* const* vals, double* __restrict__ dval64, float* __restrict__ dval32) {
  const int lane = threadIdx.x & 31;
  for (long long s = bgw(); s < d.nslices; s += bnw()) {
    const int i = d.s_inst[s];
    const long long row = d.s_row0[s] + lane;
    if (row >= d.n[i]) continue;
    const int* rp = rowptrs[i];
    const int* ci = cols[i];
    const double* va = vals[i];
    const double wr = d.w[d.woff[i] + row];
    for (int p = rp[row]; p < rp[row + 1]; ++p) {
      const long long c = ci[p];
      if (c <= row) continue;
      for (int t = 0; t < d.dia_nd[i]; ++t)
        if (d.dia_off[i * kBDiag + t] == c - row) {
          const long long e = d.dia_base[i] + t * d.dia_stride[i] + d.dia_pad[i] + row;
          const double v = (wr * va[p]) * d.w[d.woff[i] + c];
          dval64[e] = v;
          if (dval32) dval32[e] = (float)v;
          break;
        }
    }
  }
}

// A_hat = W A W in place (needs all weights of the instance first).
__global__ void b_scale_kernel(BatchDev d, double* __restrict__ oval, float* __restrict__ val32) {
  const int lane = threadIdx.x & 31;
  for (long long s = bgw(); s < d.nslices; s += bnw()) {
    const int i = d.s_inst[s];
    const long long row = d.s_row0[s] + lane;
    const bool in = row < d.n[i];
    const long long base = d.sptr[s];
    const int wd = (int)((d.sptr[s + 1] - base) / 32);
    const double wr = in ? d.w[d.woff[i] + row] : 1.0;
    for (int j = 0; j < wd; ++j) {
      const long long e = base + (long long)j * 32 + lane;
      const double v = in ? (wr * oval[e]) * d.w[d.woff[i] + d.col[e]] : 0.0;
      oval[e] = v;
      if (val32) val32[e] = (float)v;
    }
  }
}

int grid_b(long long nslices) {
  long long g = (nslices * 32 + kBlock - 1) / kBlock;
  return (int)std::max(1LL, std::min<long long>(g, 8LL * num_sms()));
}

}  // namespace
}  // namespace pp

// ===========================================================================
// host side
// ===========================================================================
namespace pp {
namespace {

struct BBump {
  uintptr_t base, off = 0;
  explicit BBump(void* b) : base((uintptr_t)b) {}
  template <typename T>
  T* take(long long count) {
    off = (off + 255) & ~(uintptr_t)255;
    T* p = reinterpret_cast<T*>(base + off);
    off += (uintptr_t)(count > 0 ? count : 1) * sizeof(T);
    return p;
  }
};

struct BPlan {
  int nb = 0, ncols = 0;
  long long nslices = 0, nnz_pad = 0, vec_elems = 0, rows_pad = 0;
  std::vector<int> s_inst, n, R, cbase, ccol_inst;
  std::vector<long long> s_row0, sptr, voff, woff, uoff, sbase;
  // DIA mode
  bool dia = false;
  long long dia_total = 0;
  std::vector<int> dia_nd, dia_off;
  std::vector<long long> dia_base, dia_stride, dia_pad;
  std::vector<int> zmode;
  std::vector<BZItem> zitems;
  std::vector<long long> zclass;  // item offsets of the register classes
  int nz_inst = 0;
};

// Plane-marching items (FP32 apply, DIA): every instance whose upper offsets
// are 1, Nx, Nx*Ny with n = Nx*Ny*Nz (a structured grid in natural order) is
// cut into 32 x 8 tiles and z chunks of at most kBZPlanes planes; the items
// are sorted by decreasing work so that one block per item balances.
void plan_z_items(BPlan& P) {
  P.zmode.assign(P.nb, 0);
  std::vector<std::pair<double, BZItem>> it;
  for (int i = 0; i < P.nb; ++i) {
    if (P.dia_nd[i] != 3) continue;
    const long long o0 = P.dia_off[(size_t)i * kBDiag], o1 = P.dia_off[(size_t)i * kBDiag + 1],
                    o2 = P.dia_off[(size_t)i * kBDiag + 2];
    if (o0 != 1 || o1 < 2 || o2 <= o1 || o2 % o1 != 0 || P.n[i] % o2 != 0) continue;
    const long long Nx = o1, Ny = o2 / o1, Nz = P.n[i] / o2;
    if (Nz > 65535) continue;
    P.zmode[i] = 1;
    P.nz_inst += 1;
    const long long chunks = (Nz + kBZPlanes - 1) / kBZPlanes;
    const long long zc = (Nz + chunks - 1) / chunks;
    for (long long y0 = 0; y0 < Ny; y0 += kBZTileY)
      for (long long x0 = 0; x0 < Nx; x0 += kBZTileX)
        for (long long z0 = 0; z0 < Nz; z0 += zc) {
          const long long z1 = std::min(Nz, z0 + zc);
          BZItem b{i, (int)x0, (int)y0, (unsigned short)z0, (unsigned short)z1};
          const double rows = (double)std::min<long long>(kBZTileX, Nx - x0) *
                              std::min<long long>(kBZTileY, Ny - y0) * (z1 - z0);
          it.push_back({rows * (12.0 + 16.0 * P.R[i]), b});
        }
  }
  auto cls = [&](const BZItem& b) {
    int c = 0;
    while (c + 1 < kBZClasses && P.R[b.inst] >= kBZClass[c + 1]) ++c;
    return c;
  };
  std::stable_sort(it.begin(), it.end(), [&](const auto& a, const auto& b) {
    const int ca = cls(a.second), cb = cls(b.second);
    return ca != cb ? ca < cb : a.first > b.first;
  });
  P.zitems.clear();
  P.zclass.assign(kBZClasses + 1, 0);
  for (const auto& e : it) {
    P.zitems.push_back(e.second);
    P.zclass[cls(e.second) + 1] += 1;
  }
  for (int c = 0; c < kBZClasses; ++c) P.zclass[c + 1] += P.zclass[c];
}

// DIA mode: the upper offsets of instance i are those of its first row
// (for a Dirichlet stencil every offset occurs there); pp_batch_setup then
// checks every entry against them on the device.
int plan_dia_instance(const pp_batch_item& it, int i, long long ns, BPlan& P, cudaStream_t s) {
  int r0[2];
  cudaError_t e = cudaMemcpyAsync(r0, it.rowptr, sizeof(int) * 2, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "pp_batch: reading rowptr");
  const int len = r0[1] - r0[0];
  std::vector<int> c0((size_t)std::max(len, 1));
  if (len > 0) e = cudaMemcpyAsync(c0.data(), it.col + r0[0], sizeof(int) * len, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "pp_batch: reading row 0");
  std::vector<int> offs;
  for (int q = 0; q < len; ++q)
    if (c0[q] > 0) offs.push_back(c0[q]);
  std::sort(offs.begin(), offs.end());
  offs.erase(std::unique(offs.begin(), offs.end()), offs.end());
  if ((int)offs.size() > kBDiag)
    return fail(nullptr, PP_EUNSUPPORTED, "pp_batch DIA: more than 8 upper diagonals (item " + std::to_string(i) + ")");
  const long long pad = offs.empty() ? 0 : ((long long)offs.back() + 31) / 32 * 32;
  P.dia_nd.push_back((int)offs.size());
  for (int t = 0; t < kBDiag; ++t) P.dia_off.push_back(t < (int)offs.size() ? offs[t] : 0);
  P.dia_pad.push_back(pad);
  P.dia_stride.push_back(pad + ns * 32);
  P.dia_base.push_back(P.dia_total);
  P.dia_total += (long long)offs.size() * (pad + ns * 32);
  return PP_OK;
}

int plan_batch(const pp_batch_item* items, int count, BPlan& P, cudaStream_t s, bool dia) {
  P.dia = dia;
  P.nb = count;
  P.sbase.assign(count + 1, 0);
  P.sptr.push_back(0);
  long long vo = 0, wo = 0, uo = 0;
  int cb = 0;
  for (int i = 0; i < count; ++i) {
    const pp_batch_item& it = items[i];
    std::vector<int> rp((size_t)it.n + 1);
    cudaError_t e = cudaMemcpyAsync(rp.data(), it.rowptr, sizeof(int) * (it.n + 1), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "pp_batch: reading rowptr");
    if (rp[0] != 0 || rp[it.n] != it.nnz) return fail(nullptr, PP_EINVAL, "pp_batch: rowptr[0] != 0 or rowptr[n] != nnz");
    const long long ns = ((long long)it.n + 31) / 32;
    for (long long sl = 0; sl < ns; ++sl) {
      int wmax = 0;
      for (long long r = sl * 32; r < std::min<long long>(it.n, sl * 32 + 32); ++r) wmax = std::max(wmax, rp[r + 1] - rp[r]);
      P.s_inst.push_back(i);
      P.s_row0.push_back(sl * 32);
      P.sptr.push_back(P.sptr.back() + (long long)wmax * 32);
    }
    P.sbase[i + 1] = P.sbase[i] + ns;
    if (dia) {
      const int rc = plan_dia_instance(it, i, ns, P, s);
      if (rc) return rc;
    }
    P.n.push_back(it.n);
    P.R.push_back(it.nrhs);
    P.cbase.push_back(cb);
    for (int r = 0; r < it.nrhs; ++r) P.ccol_inst.push_back(i);
    cb += it.nrhs;
    P.voff.push_back(vo);
    P.woff.push_back(wo);
    P.uoff.push_back(uo);
    vo += ns * 32 * it.nrhs;
    wo += ns * 32;
    uo += (long long)it.n * it.nrhs;
  }
  P.ncols = cb;
  P.nslices = (long long)P.s_inst.size();
  P.nnz_pad = P.sptr.back();
  P.vec_elems = vo;
  P.rows_pad = wo;
  if (dia) plan_z_items(P);
  return PP_OK;
}

size_t layout_batch(pp_ctx* c, pp_batch_state* B, const BPlan& P, void* base) {
  BBump M(base);
  const int k = c->opt.k;
  c->sc = M.take<Scalars>(1);
  BatchDev& d = B->d;
  d.nb = P.nb;
  d.ncols = P.ncols;
  d.nslices = P.nslices;
  d.k = k;
  d.s_inst = M.take<int>(P.nslices);
  d.s_row0 = M.take<long long>(P.nslices);
  d.sptr = M.take<long long>(P.nslices + 1);
  d.dia = P.dia ? 1 : 0;
  if (P.dia) {
    d.col = nullptr;
    d.val64 = nullptr;
    d.val32 = nullptr;
    d.dia_nd = M.take<int>(P.nb);
    d.dia_off = M.take<int>((long long)P.nb * kBDiag);
    d.dia_base = M.take<long long>(P.nb);
    d.dia_stride = M.take<long long>(P.nb);
    d.dia_pad = M.take<long long>(P.nb);
    d.dval64 = M.take<double>(P.dia_total);
    d.dval32 = B->apply_prec == PP_PREC_F32 ? M.take<float>(P.dia_total) : nullptr;
    d.zmode = M.take<int>(P.nb);
    d.zitem = M.take<BZItem>((long long)P.zitems.size());
    // the plane-marching step is FP32 only
    d.nzitems = B->apply_prec == PP_PREC_F32 ? (long long)P.zitems.size() : 0;
  } else {
    d.col = M.take<int>(P.nnz_pad);
    d.val64 = M.take<double>(P.nnz_pad);
    d.val32 = B->apply_prec == PP_PREC_F32 ? M.take<float>(P.nnz_pad) : nullptr;
  }
  d.n = M.take<int>(P.nb);
  d.R = M.take<int>(P.nb);
  d.voff = M.take<long long>(P.nb);
  d.uoff = M.take<long long>(P.nb);
  d.cbase = M.take<int>(P.nb);
  d.sbase = M.take<long long>(P.nb + 1);
  d.ccol_inst = M.take<int>(P.ncols);
  d.w = M.take<double>(P.rows_pad);
  d.woff = M.take<long long>(P.nb);
  B->theta_bar = M.take<double>(P.ncols);
  B->delta = M.take<double>(P.ncols);
  B->sigma_bar = M.take<double>(P.ncols);
  B->rho = M.take<double>((long long)P.ncols * (k + 1));
  B->coefT = M.take<double>((long long)(k + 1) * P.ncols * 3);
  d.theta_bar = B->theta_bar;
  d.delta = B->delta;
  d.sigma_bar = B->sigma_bar;
  d.rho = B->rho;
  BatchCols& cc = B->c;
  cc.rz = M.take<double>(P.ncols);
  cc.rz_new = M.take<double>(P.ncols);
  cc.pq = M.take<double>(P.ncols);
  cc.zq = M.take<double>(P.ncols);
  cc.rr = M.take<double>(P.ncols);
  cc.bb = M.take<double>(P.ncols);
  cc.rtol2 = M.take<double>(P.ncols);
  cc.al = M.take<double>(P.ncols);
  cc.be = M.take<double>(P.ncols);
  cc.done = M.take<int>(P.ncols);
  cc.iter = M.take<int>(P.ncols);
  cc.status = M.take<int>(P.ncols);
  cc.n_active = M.take<int>(1);
  B->part0 = M.take<double>(P.nslices * kBR);
  B->part1 = M.take<double>(P.nslices * kBR);
  B->lan_a = M.take<double>((long long)P.nb * kMaxLanczos);
  B->lan_b2 = M.take<double>((long long)P.nb * kMaxLanczos);
  B->nrm = M.take<double>((long long)P.nb * kMaxLanczos);
  B->feat = M.take<double>((long long)P.nb * 4);
  B->x = M.take<double>(P.vec_elems);
  B->r = M.take<double>(P.vec_elems);
  B->z = M.take<double>(P.vec_elems);
  B->p = M.take<double>(P.vec_elems);
  B->q = M.take<double>(P.vec_elems);
  B->t1 = M.take<double>(P.vec_elems);
  B->t2 = M.take<double>(P.vec_elems);
  if (B->apply_prec == PP_PREC_F32) {
    B->r32 = M.take<float>(P.vec_elems);
    B->u32 = M.take<float>(P.vec_elems);
    B->v32 = M.take<float>(P.vec_elems);
    B->z32 = M.take<float>(P.vec_elems);
  }
  c->partials = M.take<double>(P.rows_pad);  // diag logs during setup
  return M.off + 256;
}

struct BLaunch {
  int grid;
  cudaStream_t s;
};

cudaError_t b_reduce(pp_batch_state* B, int op, double* lan_out, int j, cudaStream_t s) {
  const BatchDev& d = B->d;
  const int items = (op == kRedLanA || op == kRedLanB || op == kRedNrm) ? d.nb : d.ncols;
  const int g = std::max(1, std::min(items, 8 * num_sms()));
  switch (op) {
    case kRedBB: b_reduce_kernel<kRedBB><<<g, kBlock, 0, s>>>(d, B->c, B->part0, B->part1, lan_out, j); break;
    case kRedPQ: b_reduce_kernel<kRedPQ><<<g, kBlock, 0, s>>>(d, B->c, B->part0, B->part1, lan_out, j); break;
    case kRedRR: b_reduce_kernel<kRedRR><<<g, kBlock, 0, s>>>(d, B->c, B->part0, B->part1, lan_out, j); break;
    case kRedRZ: b_reduce_kernel<kRedRZ><<<g, kBlock, 0, s>>>(d, B->c, B->part0, B->part1, lan_out, j); break;
    case kRedLanA: b_reduce_kernel<kRedLanA><<<g, kBlock, 0, s>>>(d, B->c, B->part0, B->part1, lan_out, j); break;
    case kRedLanB: b_reduce_kernel<kRedLanB><<<g, kBlock, 0, s>>>(d, B->c, B->part0, B->part1, lan_out, j); break;
    default: b_reduce_kernel<kRedNrm><<<g, kBlock, 0, s>>>(d, B->c, B->part0, B->part1, lan_out, j); break;
  }
  return cudaGetLastError();
}

template <int OP>
cudaError_t b_vec(pp_batch_state* B, const double* bin, double* xout, int first, cudaStream_t s) {
  b_vec_kernel<OP><<<grid_b((B->d.nslices + kBChunk - 1) / kBChunk), kBlock, 0, s>>>(B->d, B->c, bin, xout, B->x, B->r, B->z, B->p, B->q,
                                                          B->r32, B->z32, B->part0, B->part1, first);
  return cudaGetLastError();
}

// The k degree steps of Algorithm 2 for every active column: from r (or
// r32) into z (or z32), in the apply precision.
cudaError_t b_cheb_steps(pp_batch_state* B, cudaStream_t s) {
  const BatchDev& d = B->d;
  const int k = d.k;
  // DIA: work items of kBChunk slices; SELL: one slice per warp
  const int g = d.dia ? grid_b((d.nslices + kBChunk - 1) / kBChunk) : grid_b(d.nslices);
  cudaError_t e = cudaSuccess;
  auto step = [&](auto tv, auto tx, const auto* val, const auto* xin, const auto* xo, const auto* rin, auto* yout,
                  int mode, const double* cj) {
    using TV = std::remove_cv_t<std::remove_pointer_t<decltype(tv)>>;
    using TX = std::remove_cv_t<std::remove_pointer_t<decltype(tx)>>;
    const TV* v = reinterpret_cast<const TV*>(val);
    if (d.dia) {
      bool tz = false;  // plane-marching instances present (FP32 only)
      if constexpr (std::is_same<TX, float>::value) {
        if (d.nzitems > 0) {
          tz = true;
          // the classes touch disjoint instances: the largest runs on s, the
          // others on the side streams, so a small class does not leave the
          // GPU part-empty for a launch of its own
          int nonempty = 0;
          for (int c = 0; c < 3; ++c) nonempty += B->zclass[c + 1] > B->zclass[c] ? 1 : 0;
          const bool fork = nonempty > 1 && B->zs[0] && B->zs[1];
          cudaError_t fe = cudaSuccess;
          if (fork) {
            fe = cudaEventRecord(B->zfork, s);
            for (int q = 0; q < 2 && fe == cudaSuccess; ++q) fe = cudaStreamWaitEvent(B->zs[q], B->zfork, 0);
            if (fe != cudaSuccess) return fe;
          }
          auto zl = [&](auto lo, auto hi, int c, cudaStream_t ls) {
            constexpr int RLO = decltype(lo)::value, RHI = decltype(hi)::value;
            const long long i0 = B->zclass[c], cnt = B->zclass[c + 1] - i0;
            if (cnt <= 0) return;
            const unsigned gz = (unsigned)cnt;
            if (mode == kCheb1)
              b_cheb_z_kernel<RLO, RHI, kCheb1><<<gz, kBlock, 0, ls>>>(d, i0, v, xin, xo, rin, yout, B->c.done, cj);
            else if (mode == kCheb2)
              b_cheb_z_kernel<RLO, RHI, kCheb2><<<gz, kBlock, 0, ls>>>(d, i0, v, xin, xo, rin, yout, B->c.done, cj);
            else
              b_cheb_z_kernel<RLO, RHI, kChebK><<<gz, kBlock, 0, ls>>>(d, i0, v, xin, xo, rin, yout, B->c.done, cj);
          };
          zl(std::integral_constant<int, kBZClass[2]>(), std::integral_constant<int, kBZClass[3] - 1>(), 2, s);
          zl(std::integral_constant<int, kBZClass[1]>(), std::integral_constant<int, kBZClass[2] - 1>(), 1,
             fork ? B->zs[0] : s);
          zl(std::integral_constant<int, kBZClass[0]>(), std::integral_constant<int, kBZClass[1] - 1>(), 0,
             fork ? B->zs[1] : s);
          if (fork) {
            // join before anything else reads the step's output
            for (int q = 0; q < 2 && fe == cudaSuccess; ++q) {
              fe = cudaEventRecord(B->zjoin[q], B->zs[q]);
              if (fe == cudaSuccess) fe = cudaStreamWaitEvent(s, B->zjoin[q], 0);
            }
            if (fe != cudaSuccess) return fe;
          }
          if (B->nz_inst == d.nb) return cudaGetLastError();  // every instance plane-marched
        }
      }
      if (tz) {
        if (mode == kCheb1) b_cheb_dia3_kernel<TV, TX, kCheb1, true><<<g, kBlock, 0, s>>>(d, v, xin, xo, rin, yout, B->c.done, cj);
        else if (mode == kCheb2) b_cheb_dia3_kernel<TV, TX, kCheb2, true><<<g, kBlock, 0, s>>>(d, v, xin, xo, rin, yout, B->c.done, cj);
        else b_cheb_dia3_kernel<TV, TX, kChebK, true><<<g, kBlock, 0, s>>>(d, v, xin, xo, rin, yout, B->c.done, cj);
      } else {
        if (mode == kCheb1) b_cheb_dia3_kernel<TV, TX, kCheb1, false><<<g, kBlock, 0, s>>>(d, v, xin, xo, rin, yout, B->c.done, cj);
        else if (mode == kCheb2) b_cheb_dia3_kernel<TV, TX, kCheb2, false><<<g, kBlock, 0, s>>>(d, v, xin, xo, rin, yout, B->c.done, cj);
        else b_cheb_dia3_kernel<TV, TX, kChebK, false><<<g, kBlock, 0, s>>>(d, v, xin, xo, rin, yout, B->c.done, cj);
      }
    } else {
      if (mode == kCheb1) b_cheb_kernel<TV, TX, kCheb1><<<g, kBlock, 0, s>>>(d, v, xin, xo, rin, yout, B->c.done, cj);
      else if (mode == kCheb2) b_cheb_kernel<TV, TX, kCheb2><<<g, kBlock, 0, s>>>(d, v, xin, xo, rin, yout, B->c.done, cj);
      else b_cheb_kernel<TV, TX, kChebK><<<g, kBlock, 0, s>>>(d, v, xin, xo, rin, yout, B->c.done, cj);
    }
    return cudaGetLastError();
  };
  if (B->apply_prec == PP_PREC_F32) {
    float* buf[3] = {B->u32, B->v32, B->z32};
    const int off = ((2 - k) % 3 + 3) % 3;
    auto Y = [&](int j) { return buf[(j + off) % 3]; };
    const float* val = d.dia ? d.dval32 : d.val32;
    for (int j = 1; j <= k && e == cudaSuccess; ++j) {
      const double* cj = B->coefT + (size_t)j * d.ncols * 3;
      if (j == 1) e = step((float*)nullptr, (float*)nullptr, val, B->r32, (const float*)nullptr, B->r32, Y(1), kCheb1, cj);
      else if (j == 2) e = step((float*)nullptr, (float*)nullptr, val, Y(1), (const float*)nullptr, B->r32, Y(2), kCheb2, cj);
      else e = step((float*)nullptr, (float*)nullptr, val, Y(j - 1), Y(j - 2), B->r32, Y(j), kChebK, cj);
    }
  } else {
    double* buf[3] = {B->t1, B->t2, B->z};
    const int off = ((2 - k) % 3 + 3) % 3;
    auto Y = [&](int j) { return buf[(j + off) % 3]; };
    const double* val = d.dia ? d.dval64 : d.val64;
    for (int j = 1; j <= k && e == cudaSuccess; ++j) {
      const double* cj = B->coefT + (size_t)j * d.ncols * 3;
      if (j == 1) e = step((double*)nullptr, (double*)nullptr, val, B->r, (const double*)nullptr, B->r, Y(1), kCheb1, cj);
      else if (j == 2) e = step((double*)nullptr, (double*)nullptr, val, Y(1), (const double*)nullptr, B->r, Y(2), kCheb2, cj);
      else e = step((double*)nullptr, (double*)nullptr, val, Y(j - 1), Y(j - 2), B->r, Y(j), kChebK, cj);
    }
  }
  return e;
}

// z = p_k(A_hat) r for every active column, then (r,z), (q,z) -> rz_new, zq.
// FP32 preconditioner: z stays in z32 (the p update reads it there); r32 is
// written here unless the r update already wrote it (r32_ready).
cudaError_t b_precond(pp_batch_state* B, cudaStream_t s, bool r32_ready) {
  const int k = B->d.k;
  cudaError_t e = cudaSuccess;
  if (k == 0) {
    e = b_vec<kBDeg0>(B, nullptr, nullptr, 0, s);
    return e == cudaSuccess ? b_reduce(B, kRedRZ, nullptr, 0, s) : e;
  }
  if (B->apply_prec == PP_PREC_F32) {
    if (!r32_ready) e = b_vec<kBTo32>(B, nullptr, nullptr, 0, s);
    if (e == cudaSuccess) e = b_cheb_steps(B, s);
    if (e == cudaSuccess) e = b_vec<kBDots32>(B, nullptr, nullptr, 0, s);
  } else {
    e = b_cheb_steps(B, s);
    if (e == cudaSuccess) e = b_vec<kBZtoP>(B, nullptr, nullptr, 0, s);
  }
  return e == cudaSuccess ? b_reduce(B, kRedRZ, nullptr, 0, s) : e;
}

cudaError_t b_iteration(pp_batch_state* B, cudaStream_t s) {
  const BatchDev& d = B->d;
  b_spmv64_kernel<kSpmv><<<grid_b(d.nslices), kBlock, 0, s>>>(d, B->p, nullptr, B->q, B->c.done, nullptr, 0, B->part0);
  cudaError_t e = cudaGetLastError();
  const bool lp = B->apply_prec == PP_PREC_F32 && B->d.k > 0;
  if (e == cudaSuccess) e = b_reduce(B, kRedPQ, nullptr, 0, s);
  if (e == cudaSuccess) e = lp ? b_vec<kBUpdXR32>(B, nullptr, nullptr, 0, s) : b_vec<kBUpdXR>(B, nullptr, nullptr, 0, s);
  if (e == cudaSuccess) e = b_reduce(B, kRedRR, nullptr, 0, s);
  if (e == cudaSuccess) e = b_precond(B, s, lp);
  if (e == cudaSuccess) e = lp ? b_vec<kBUpdP32>(B, nullptr, nullptr, 0, s) : b_vec<kBUpdP>(B, nullptr, nullptr, 0, s);
  return e;
}

void set_coeffs(pp_batch_state* B, int k) {
  const int nc = B->d.ncols;
  std::vector<double> tb(nc), dl(nc), sb(nc), rho((size_t)nc * (k + 1));
  for (int g = 0; g < nc; ++g)
    polyprec_coeffs(B->abx[3 * g], B->abx[3 * g + 1], B->abx[3 * g + 2], k, &tb[g], &dl[g], &sb[g],
                    &rho[(size_t)g * (k + 1)]);
  cudaMemcpy(B->theta_bar, tb.data(), sizeof(double) * nc, cudaMemcpyHostToDevice);
  cudaMemcpy(B->delta, dl.data(), sizeof(double) * nc, cudaMemcpyHostToDevice);
  cudaMemcpy(B->sigma_bar, sb.data(), sizeof(double) * nc, cudaMemcpyHostToDevice);
  cudaMemcpy(B->rho, rho.data(), sizeof(double) * rho.size(), cudaMemcpyHostToDevice);
  std::vector<double> ct((size_t)(k + 1) * nc * 3, 0.0);
  for (int j = 1; j <= k; ++j)
    for (int g = 0; g < nc; ++g) {
      const StepCoeffs cf = cheb_step_coeffs(j, &rho[(size_t)g * (k + 1)], tb[g], dl[g], sb[g]);
      double* o = &ct[((size_t)j * nc + g) * 3];
      o[0] = cf.ca;
      o[1] = cf.cb;
      o[2] = cf.cc;
    }
  cudaMemcpy(B->coefT, ct.data(), sizeof(double) * ct.size(), cudaMemcpyHostToDevice);
}

int b_lanczos(pp_ctx* c, pp_batch_state* B, cudaStream_t s) {
  const BatchDev& d = B->d;
  const int m = c->opt.lanczos_steps;
  const int g = grid_b(d.nslices);
  double* buf[3] = {B->t1, B->t2, B->z};
  b_lan_start_kernel<<<g, kBlock, 0, s>>>(d, c->opt.seed, buf[0], B->part0);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = b_reduce(B, kRedNrm, B->nrm, 0, s);
  if (e == cudaSuccess) {
    b_lan_vec_kernel<0><<<g, kBlock, 0, s>>>(d, buf[0], nullptr, B->nrm, 0, nullptr);
    e = cudaGetLastError();
  }
  int iv = 0, ivp = -1, iw = 1;
  for (int j = 0; j < m && e == cudaSuccess; ++j) {
    b_spmv64_kernel<kLanczos><<<g, kBlock, 0, s>>>(d, buf[iv], ivp >= 0 ? buf[ivp] : nullptr, buf[iw], B->c.done,
                                                   B->lan_b2, j, B->part0);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = b_reduce(B, kRedLanA, B->lan_a, j, s);
    if (e == cudaSuccess) {
      b_lan_vec_kernel<1><<<g, kBlock, 0, s>>>(d, buf[iw], buf[iv], B->lan_a, j, B->part0);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = b_reduce(B, kRedLanB, B->lan_b2, j, s);
    if (e == cudaSuccess && j < m - 1) {
      b_lan_vec_kernel<0><<<g, kBlock, 0, s>>>(d, buf[iw], nullptr, B->lan_b2, j, nullptr);
      e = cudaGetLastError();
      const int spare = ivp >= 0 ? ivp : 2;
      ivp = iv;
      iv = iw;
      iw = spare;
    }
  }
  std::vector<double> ha((size_t)d.nb * kMaxLanczos), hb((size_t)d.nb * kMaxLanczos);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ha.data(), B->lan_a, sizeof(double) * ha.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data(), B->lan_b2, sizeof(double) * hb.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "pp_batch: Lanczos");
  B->ritz.assign((size_t)d.nb * 5, 0.0);
  std::vector<double> alpha(d.nb), beta(d.nb);
  for (int i = 0; i < d.nb; ++i) {
    std::vector<double> ta, tb;
    for (int j = 0; j < m; ++j) {
      ta.push_back(ha[(size_t)i * kMaxLanczos + j]);
      if (j == m - 1) break;
      const double bj = std::sqrt(hb[(size_t)i * kMaxLanczos + j]);
      if (!(bj > 1e-300)) break;
      tb.push_back(bj);
    }
    double lo, hi;
    tridiag_extremes_jacobi(ta, tb, &lo, &hi);
    if (!(lo > 0.0)) return fail(c, PP_EBREAKDOWN, "pp_batch: instance " + std::to_string(i) + " is not SPD");
    alpha[i] = lo;
    beta[i] = hi > lo ? hi : lo * (1.0 + 1e-12);
    B->ritz[(size_t)i * 5 + 0] = lo;
    B->ritz[(size_t)i * 5 + 1] = hi;
  }
  B->abx.assign((size_t)d.ncols * 3, 0.0);
  for (int i = 0; i < d.nb; ++i)
    for (int r = 0; r < B->R_h[i]; ++r) {
      const int gg = B->cbase_h[i] + r;
      B->abx[3 * gg] = alpha[i];
      B->abx[3 * gg + 1] = beta[i];
      B->abx[3 * gg + 2] = c->opt.xi >= 0.0 ? c->opt.xi : auto_xi(alpha[i], beta[i]);
    }
  B->lanczos_steps = m;
  return PP_OK;
}

}  // namespace

void batch_free(pp_batch_state* B) {
  if (!B) return;
  if (B->graph) cudaGraphExecDestroy(B->graph);
  if (B->cap) cudaStreamDestroy(B->cap);
  for (int q = 0; q < 2; ++q) {
    if (B->zs[q]) cudaStreamDestroy(B->zs[q]);
    if (B->zjoin[q]) cudaEventDestroy(B->zjoin[q]);
  }
  if (B->zfork) cudaEventDestroy(B->zfork);
  delete B;
}

}  // namespace pp

using namespace pp;

namespace {

int check_items(const pp_batch_item* items, int count) {
  if (!items || count <= 0) return fail(nullptr, PP_EINVAL, "pp_batch: no items");
  for (int i = 0; i < count; ++i) {
    const pp_batch_item& it = items[i];
    if (it.n <= 0 || it.nnz < 0 || it.nnz > 2147483647LL || !it.rowptr || !it.col || !it.val)
      return fail(nullptr, PP_EINVAL, "pp_batch: invalid matrix " + std::to_string(i));
    if (it.nrhs < 1 || it.nrhs > kBR)
      return fail(nullptr, PP_EINVAL, "pp_batch: nrhs must be in [1, 8] (item " + std::to_string(i) + ")");
  }
  return PP_OK;
}

int check_batch_opts(const pp_options* o) {
  int rc = validate_options(nullptr, o);
  if (rc == PP_OK && o->lowrank != 0)
    rc = fail(nullptr, PP_EUNSUPPORTED, "the low-rank correction is not available for batch contexts");
  if (rc == PP_OK && o->poly != PP_POLY_CHEB)
    rc = fail(nullptr, PP_EUNSUPPORTED, "pp_batch: the Chebyshev recurrence only");
  if (rc == PP_OK && o->flexible > 1)
    rc = fail(nullptr, PP_EUNSUPPORTED, "pp_batch: flexible must be 0 or 1 (FCG(1))");
  if (rc) return rc;
  if (o->apply_prec == PP_PREC_BF16) return fail(nullptr, PP_EUNSUPPORTED, "pp_batch: apply_prec must be F64 or F32");
  if (o->seed_scaling != PP_SEED_JACOBI) return fail(nullptr, PP_EUNSUPPORTED, "pp_batch: Jacobi seed only");
  return PP_OK;
}

}  // namespace

extern "C" int pp_batch_workspace_size(const pp_batch_item* items, int count, const pp_options* opt, size_t* bytes) {
  int rc = check_items(items, count);
  if (rc) return rc;
  if ((rc = check_batch_opts(opt))) return rc;
  if (!bytes) return fail(nullptr, PP_EINVAL, "bytes is NULL");
  BPlan P;
  if ((rc = plan_batch(items, count, P, nullptr, opt->format == PP_FMT_DIA))) return rc;
  pp_ctx tmp;
  tmp.opt = *opt;
  pp_batch_state B;
  B.apply_prec = opt->apply_prec;
  *bytes = layout_batch(&tmp, &B, P, nullptr);
  return PP_OK;
}

extern "C" int pp_batch_setup(pp_ctx** out, const pp_batch_item* items, int count, const pp_options* opt, void* ws,
                              size_t ws_bytes, void* stream) {
  if (!out) return fail(nullptr, PP_EINVAL, "ctx pointer is NULL");
  *out = nullptr;
  int rc = check_items(items, count);
  if (rc) return rc;
  if ((rc = check_batch_opts(opt))) return rc;
  if (!ws || ((uintptr_t)ws & 255)) return fail(nullptr, PP_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  pp_ctx* c = new pp_ctx();
  c->kind = 2;
  c->opt = *opt;
  if (c->opt.check_every <= 0) c->opt.check_every = 4;
  pp_batch_state* B = new pp_batch_state();
  c->batch = B;
  B->apply_prec = opt->apply_prec;
  auto bail = [&](int code) {
    std::string m = c->err;
    destroy_ctx_resources(c);
    delete c;
    if (!m.empty()) fail(nullptr, code, m);
    return code;
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  BPlan P;
  if ((rc = plan_batch(items, count, P, s, opt->format == PP_FMT_DIA))) return bail(rc);
  const size_t need = layout_batch(c, B, P, nullptr);
  if (ws_bytes < need) return bail(fail(c, PP_EINVAL, "workspace too small: need " + std::to_string(need) + " bytes"));
  layout_batch(c, B, P, ws);
  c->ws = ws;
  c->ws_bytes = ws_bytes;
  c->n = P.ncols;
  c->nnz = 0;
  for (int i = 0; i < count; ++i) c->nnz += items[i].nnz;
  c->nnz_pad = P.nnz_pad;
  B->n_h = P.n;
  B->R_h = P.R;
  B->cbase_h = P.cbase;
  B->voff_h = P.voff;
  B->woff_h = P.woff;
  B->vec_elems = P.vec_elems;
  B->rows_pad = P.rows_pad;
  B->nz_inst = B->d.nzitems > 0 ? P.nz_inst : 0;
  for (int q = 0; q < 4 && q < (int)P.zclass.size(); ++q) B->zclass[q] = P.zclass[q];
  if (B->d.nzitems > 0) {
    cudaError_t se = cudaEventCreateWithFlags(&B->zfork, cudaEventDisableTiming);
    for (int q = 0; q < 2 && se == cudaSuccess; ++q) {
      se = cudaStreamCreateWithFlags(&B->zs[q], cudaStreamNonBlocking);
      if (se == cudaSuccess) se = cudaEventCreateWithFlags(&B->zjoin[q], cudaEventDisableTiming);
    }
    if (se != cudaSuccess) return bail(cuda_fail(c, se, "pp_batch_setup: side streams"));
  }
  BatchDev& d = B->d;
  B->c.maxit = opt->maxit;
  B->c.flexible = opt->flexible;
  B->c.rtol = opt->rtol;
  // upload the plan (and the instance pointer tables, kept in t1 for the fill)
  std::vector<const int*> rps(count), cis(count);
  std::vector<const double*> vas(count);
  for (int i = 0; i < count; ++i) {
    rps[i] = items[i].rowptr;
    cis[i] = items[i].col;
    vas[i] = items[i].val;
  }
  const int** d_rp = reinterpret_cast<const int**>(B->t1);
  const int** d_ci = d_rp + count;
  const double** d_va = reinterpret_cast<const double**>(d_ci + count);
  struct Up {
    const void* dst;
    const void* src;
    size_t n;
  } ups[] = {{d.s_inst, P.s_inst.data(), sizeof(int) * P.s_inst.size()},
             {d.s_row0, P.s_row0.data(), sizeof(long long) * P.s_row0.size()},
             {d.sptr, P.sptr.data(), sizeof(long long) * P.sptr.size()},
             {d.n, P.n.data(), sizeof(int) * P.n.size()},
             {d.R, P.R.data(), sizeof(int) * P.R.size()},
             {d.voff, P.voff.data(), sizeof(long long) * P.voff.size()},
             {d.uoff, P.uoff.data(), sizeof(long long) * P.uoff.size()},
             {d.cbase, P.cbase.data(), sizeof(int) * P.cbase.size()},
             {d.sbase, P.sbase.data(), sizeof(long long) * P.sbase.size()},
             {d.ccol_inst, P.ccol_inst.data(), sizeof(int) * P.ccol_inst.size()},
             {d.woff, P.woff.data(), sizeof(long long) * P.woff.size()},
             {d.dia_nd, P.dia_nd.data(), sizeof(int) * P.dia_nd.size()},
             {d.dia_off, P.dia_off.data(), sizeof(int) * P.dia_off.size()},
             {d.dia_base, P.dia_base.data(), sizeof(long long) * P.dia_base.size()},
             {d.dia_stride, P.dia_stride.data(), sizeof(long long) * P.dia_stride.size()},
             {d.dia_pad, P.dia_pad.data(), sizeof(long long) * P.dia_pad.size()},
             {d_rp, rps.data(), sizeof(void*) * count},
             {d_ci, cis.data(), sizeof(void*) * count},
             {d.zmode, P.zmode.data(), sizeof(int) * P.zmode.size()},
             {d.zitem, P.zitems.data(), sizeof(BZItem) * P.zitems.size()},
             {d_va, vas.data(), sizeof(void*) * count}};
  cudaError_t e = cudaSuccess;
  for (const Up& u : ups)
    if (e == cudaSuccess && u.n) e = cudaMemcpyAsync(const_cast<void*>(u.dst), u.src, u.n, cudaMemcpyHostToDevice, s);
  int* d_bad = B->c.n_active;
  if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(int), s);
  double* diag_log = c->partials;
  if (e == cudaSuccess) {
    b_fill_kernel<<<grid_b(d.nslices), kBlock, 0, s>>>(d, d_rp, d_ci, d_va, const_cast<double*>(d.w), diag_log,
                                                        const_cast<int*>(d.col), const_cast<double*>(d.val64), d_bad);
    e = cudaGetLastError();
  }
  int dia_bad = 0;
  if (d.dia) {
    // weights first (above), then the scaled upper entries; every entry is
    // checked to lie on the planned diagonals with a symmetric partner
    int* d_dbad = reinterpret_cast<int*>(B->t2);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_dbad, 0, sizeof(int) * count, s);
    if (e == cudaSuccess && P.dia_total > 0)
      e = cudaMemsetAsync(const_cast<double*>(d.dval64), 0, sizeof(double) * (size_t)P.dia_total, s);
    if (e == cudaSuccess && d.dval32 && P.dia_total > 0)
      e = cudaMemsetAsync(const_cast<float*>(d.dval32), 0, sizeof(float) * (size_t)P.dia_total, s);
    if (e == cudaSuccess) {
      b_dia_check_kernel<<<grid_b(d.nslices), kBlock, 0, s>>>(d, d_rp, d_ci, d_va, d_dbad);
      b_dia_fill_kernel<<<grid_b(d.nslices), kBlock, 0, s>>>(d, d_rp, d_ci, d_va, const_cast<double*>(d.dval64),
                                                              const_cast<float*>(d.dval32));
      e = cudaGetLastError();
    }
    std::vector<int> hb(count, 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data(), d_dbad, sizeof(int) * count, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    for (int i = 0; i < count && e == cudaSuccess; ++i) dia_bad |= hb[i];
  } else if (e == cudaSuccess) {
    b_scale_kernel<<<grid_b(d.nslices), kBlock, 0, s>>>(d, const_cast<double*>(d.val64), const_cast<float*>(d.val32));
    e = cudaGetLastError();
  }
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  // clear vectors and column state
  const size_t vb = sizeof(double) * (size_t)P.vec_elems;
  for (double* v : {B->x, B->r, B->z, B->p, B->q, B->t1, B->t2})
    if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, vb, s);
  if (B->apply_prec == PP_PREC_F32)
    for (float* v : {B->r32, B->u32, B->v32, B->z32})
      if (e == cudaSuccess) e = cudaMemsetAsync(v, 0, sizeof(float) * (size_t)P.vec_elems, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(B->c.done, 0, sizeof(int) * P.ncols, s);
  // features: sums of log diag(A) and Gershgorin bounds of A_hat
  if (e == cudaSuccess) {
    b_feature_kernel<<<grid_b(d.nslices), kBlock, 0, s>>>(d, diag_log, B->part0);
    b_feature_reduce_kernel<<<std::min(d.nb, 1024), 32, 0, s>>>(d, B->part0, B->feat);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "pp_batch setup"));
  if (bad) return bail(fail(c, PP_EINVAL, "pp_batch: non-positive diagonal"));
  if (dia_bad)
    return bail(fail(c, PP_EUNSUPPORTED, "pp_batch DIA: an instance is not symmetric-banded on its first row's offsets"));
  if (opt->interval == PP_INTERVAL_GIVEN) {
    B->abx.assign((size_t)P.ncols * 3, 0.0);
    for (int g = 0; g < P.ncols; ++g) {
      B->abx[3 * g] = opt->alpha;
      B->abx[3 * g + 1] = opt->beta;
      B->abx[3 * g + 2] = opt->xi >= 0.0 ? opt->xi : auto_xi(opt->alpha, opt->beta);
    }
    B->ritz.assign((size_t)P.nb * 5, 0.0);
  } else if ((rc = b_lanczos(c, B, s))) {
    return bail(rc);
  }
  set_coeffs(B, opt->k);
  cudaEventRecord(e1, s);
  e = cudaEventSynchronize(e1);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "pp_batch setup"));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->t_setup_ms = ms;
  *out = c;
  return PP_OK;
}

extern "C" int pp_batch_intervals(pp_ctx* c, double* abx_out, const double* abx_in) {
  if (!c || c->kind != 2) return fail(c, PP_EINVAL, "not a batch context");
  pp_batch_state* B = c->batch;
  if (abx_out) std::memcpy(abx_out, B->abx.data(), sizeof(double) * B->abx.size());
  if (abx_in) {
    for (int g = 0; g < B->d.ncols; ++g)
      if (!(abx_in[3 * g] > 0.0 && abx_in[3 * g + 1] > abx_in[3 * g] && abx_in[3 * g + 2] >= 0.0))
        return fail(c, PP_EINVAL, "pp_batch_intervals: need 0 < alpha < beta and xi >= 0 for column " +
                                      std::to_string(g));
    std::memcpy(B->abx.data(), abx_in, sizeof(double) * B->abx.size());
    set_coeffs(B, c->opt.k);
  }
  return PP_OK;
}

extern "C" int pp_batch_features(const pp_ctx* c, double* feat) {
  if (!c || c->kind != 2 || !feat) return fail(nullptr, PP_EINVAL, "pp_batch_features: bad argument");
  pp_batch_state* B = c->batch;
  const int nb = B->d.nb;
  std::vector<double> f4((size_t)nb * 4);
  if (cudaMemcpy(f4.data(), B->feat, sizeof(double) * f4.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(nullptr, PP_ECUDA, "pp_batch_features: copy");
  for (int i = 0; i < nb; ++i) {
    const double n = B->n_h[i];
    const double mean = f4[i * 4] / n;
    const double var = std::max(0.0, f4[i * 4 + 1] / n - mean * mean);
    double* o = feat + (size_t)i * PP_BATCH_NFEAT;
    const double lo = B->ritz[(size_t)i * 5], hi = B->ritz[(size_t)i * 5 + 1];
    o[0] = std::log10(n);
    o[1] = mean;
    o[2] = std::sqrt(var);
    o[3] = f4[i * 4 + 2];
    o[4] = f4[i * 4 + 3];
    o[5] = lo > 0 ? std::log10(lo) : 0.0;
    o[6] = hi > 0 ? std::log10(hi) : 0.0;
    o[7] = (lo > 0 && hi > 0) ? std::log10(hi / lo) : 0.0;
  }
  return PP_OK;
}

extern "C" int pp_batch_solve(pp_ctx* c, const double* b, double* x, int* iters, int* status, pp_stats* st,
                              void* stream) {
  if (!c || c->kind != 2) return fail(c, PP_EINVAL, "not a batch context");
  if (!b || !x) return fail(c, PP_EINVAL, "vector argument is NULL");
  pp_batch_state* B = c->batch;
  BatchDev& d = B->d;
  cudaStream_t s = (cudaStream_t)stream;
  const int Bk = std::max(1, std::min(c->opt.check_every, kMaxCheck));
  const bool graphs = c->opt.use_graphs != 0;
  if (c->events.size() < 2) {
    for (int i = 0; i < 2; ++i) {
      cudaEvent_t ev;
      cudaEventCreate(&ev);
      c->events.push_back(ev);
    }
  }
  if (graphs && (!B->graph || B->graph_block != Bk)) {
    if (B->graph) cudaGraphExecDestroy(B->graph);
    B->graph = nullptr;
    cudaError_t e = cudaSuccess;
    if (!B->cap) e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(c, e, "pp_batch: capture");
    cudaError_t e2 = cudaSuccess;
    for (int i = 0; i < Bk && e2 == cudaSuccess; ++i) e2 = b_iteration(B, B->cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(B->cap, &g);
    if (e2 != cudaSuccess || e != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(c, e2 != cudaSuccess ? e2 : e, "pp_batch: capture");
    }
    e = cudaGraphInstantiate(&B->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(c, e, "pp_batch: graph instantiate");
    B->graph_block = Bk;
  }
  const int nc = d.ncols;
  cudaError_t e = cudaEventRecord(c->events[0], s);
  int act = nc;
  if (e == cudaSuccess) e = cudaMemcpyAsync(B->c.n_active, &act, sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(B->c.done, 0, sizeof(int) * nc, s);
  if (e == cudaSuccess) e = b_vec<kBScaleIn>(B, b, nullptr, 0, s);
  if (e == cudaSuccess) e = b_reduce(B, kRedBB, nullptr, 0, s);
  const bool lp = B->apply_prec == PP_PREC_F32 && d.k > 0;
  if (e == cudaSuccess) e = b_precond(B, s, false);
  if (e == cudaSuccess) e = lp ? b_vec<kBUpdP32>(B, nullptr, nullptr, 1, s) : b_vec<kBUpdP>(B, nullptr, nullptr, 1, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "pp_batch_solve start");
  // kernel launches: every degree step launches one kernel per non-empty
  // plane-marching class plus the slice kernel when other instances remain
  long long per_step = 1;
  if (d.dia && B->apply_prec == PP_PREC_F32 && d.nzitems > 0) {
    per_step = B->nz_inst < d.nb ? 1 : 0;
    for (int q = 0; q < 3; ++q) per_step += B->zclass[q + 1] > B->zclass[q] ? 1 : 0;
  }
  long long launches = 0;
  const long long k = c->opt.k;
  // preconditioner: k steps, the dots (and the r32 copy at the start), the reduction
  const long long pre = k == 0 ? 2 : k * per_step + 2;
  const long long per_it = 5 + pre;
  launches += 3 + pre + (lp ? 1 : 0) + 1;
  for (int guard = 0;; ++guard) {
    if (graphs) {
      e = cudaGraphLaunch(B->graph, s);
    } else {
      for (int i = 0; i < Bk && e == cudaSuccess; ++i) e = b_iteration(B, s);
    }
    launches += per_it * Bk;
    int host_act = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&host_act, B->c.n_active, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "pp_batch_solve iteration");
    if (host_act <= 0) break;
    if ((long long)guard * Bk > (long long)c->opt.maxit + 2LL * Bk) break;  // every column hits maxit before this
  }
  if (e == cudaSuccess) e = b_vec<kBScaleOut>(B, nullptr, x, 0, s);
  launches += 1;
  if (e == cudaSuccess) e = cudaEventRecord(c->events[1], s);
  std::vector<int> hi(nc), hs(nc);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hi.data(), B->c.iter, sizeof(int) * nc, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), B->c.status, sizeof(int) * nc, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "pp_batch_solve finish");
  if (iters) std::memcpy(iters, hi.data(), sizeof(int) * nc);
  if (status) std::memcpy(status, hs.data(), sizeof(int) * nc);
  int worst = PP_OK, maxit = 0;
  for (int g = 0; g < nc; ++g) {
    maxit = std::max(maxit, hi[g]);
    if (hs[g] < 0) worst = std::min(worst, hs[g]);
    else if (hs[g] == PP_MAXIT && worst == PP_OK) worst = PP_MAXIT;
  }
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->iterations = maxit;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->events[0], c->events[1]);
    st->t_solve_ms = ms;
    st->kernel_launches = launches;
    st->status = worst;
  }
  return worst;
}

// ---------------------------------------------------------------------------
// timing and storage choice of the batched degree step
// ---------------------------------------------------------------------------
extern "C" int pp_batch_time_step(pp_ctx* c, int reps, double* us_per_step, void* stream) {
  if (!c || c->kind != 2 || !us_per_step || reps < 1 || reps > 1000)
    return fail(c, PP_EINVAL, "pp_batch_time_step: bad argument");
  pp_batch_state* B = c->batch;
  if (B->d.k < 1) return fail(c, PP_EINVAL, "pp_batch_time_step: the degree k must be >= 1");
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  // every column active; the steps run on the current residuals (the values
  // do not change the work)
  if (e == cudaSuccess) e = cudaMemsetAsync(B->c.done, 0, sizeof(int) * B->d.ncols, s);
  if (e == cudaSuccess) e = b_cheb_steps(B, s);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0, s);
  for (int r = 0; r < reps && e == cudaSuccess; ++r) e = b_cheb_steps(B, s);
  if (e == cudaSuccess) e = cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_fail(c, e, "pp_batch_time_step");
  *us_per_step = 1e3 * (double)ms / ((double)reps * B->d.k);
  return PP_OK;
}

namespace {

// candidate layouts in preference order for ties (fewest bytes first)
const int kBatchFormats[2] = {PP_FMT_DIA, PP_FMT_SELL};

pp_options batch_candidate(const pp_options& base, int fmt) {
  pp_options o = base;
  o.format = fmt;
  o.interval = PP_INTERVAL_GIVEN;  // the timing needs valid coefficients only
  o.alpha = 1e-2;
  o.beta = 2.0;
  o.xi = 0.0;
  o.k = std::max(1, std::min(base.k, 8));
  o.use_graphs = 0;
  return o;
}

}  // namespace

extern "C" int pp_batch_autotune_workspace_size(const pp_batch_item* items, int count, const pp_options* opt,
                                                size_t* bytes) {
  if (!opt || !bytes) return fail(nullptr, PP_EINVAL, "NULL argument");
  size_t most = 0;
  for (int fmt : kBatchFormats) {
    pp_options o = batch_candidate(*opt, fmt);
    size_t b = 0;
    const int rc = pp_batch_workspace_size(items, count, &o, &b);
    if (rc == PP_EUNSUPPORTED) continue;  // layout not applicable to these instances
    if (rc) return rc;
    most = std::max(most, b);
  }
  *bytes = most;
  return PP_OK;
}

extern "C" int pp_batch_autotune(const pp_batch_item* items, int count, pp_options* opt, void* ws, size_t ws_bytes,
                                 pp_tune_entry* entries, int max_entries, int* tried_out, void* stream) {
  if (!opt) return fail(nullptr, PP_EINVAL, "NULL argument");
  if (!ws || ((uintptr_t)ws & 255)) return fail(nullptr, PP_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (max_entries < 0) return fail(nullptr, PP_EINVAL, "max_entries must be >= 0");
  int rc = check_items(items, count);
  if (rc) return rc;
  if ((rc = check_batch_opts(opt))) return rc;
  std::vector<pp_tune_entry> res;
  int best = -1;
  for (int fmt : kBatchFormats) {
    pp_options o = batch_candidate(*opt, fmt);
    pp_tune_entry e{};
    e.format = fmt;
    e.sell_C = fmt == PP_FMT_SELL ? 32 : 0;
    size_t need = 0;
    e.status = pp_batch_workspace_size(items, count, &o, &need);
    if (e.status == PP_OK && need > ws_bytes) e.status = PP_EINVAL;  // does not fit: skipped
    if (e.status == PP_OK) {
      pp_ctx* c = nullptr;
      e.status = pp_batch_setup(&c, items, count, &o, ws, ws_bytes, stream);
      if (e.status == PP_OK) {
        e.status = pp_batch_time_step(c, 5, &e.us_per_step, stream);
        pp_destroy(c);
      }
      if (e.status == PP_ECUDA) {
        res.push_back(e);
        for (int i = 0; entries && i < (int)res.size() && i < max_entries; ++i) entries[i] = res[i];
        if (tried_out) *tried_out = (int)res.size();
        return PP_ECUDA;  // the device is in an unknown state: stop
      }
    }
    if (e.status == PP_OK && (best < 0 || e.us_per_step < res[best].us_per_step)) best = (int)res.size();
    res.push_back(e);
  }
  for (int i = 0; entries && i < (int)res.size() && i < max_entries; ++i) entries[i] = res[i];
  if (tried_out) *tried_out = (int)res.size();
  if (best < 0) return fail(nullptr, PP_EINVAL, "pp_batch_autotune: no candidate layout fits in the workspace");
  // timings within 3% of the fastest are a tie, won by the first in order
  const double fastest = res[best].us_per_step;
  for (int i = 0; i < (int)res.size(); ++i)
    if (res[i].status == PP_OK && res[i].us_per_step <= 1.03 * fastest) {
      best = i;
      break;
    }
  opt->format = res[best].format;
  return PP_OK;
}
