// Fracture-network Schur complement on the GPU (Section 4.2).
//
// S_u(alpha) = G^u - alpha B^T A^{-1} C - alpha C^T A^{-1} B + C^T A^{-1} G^h A^{-1} C
// (the expansion below Eq. schur), applied matrix-free as in Algorithm 3.
//
// GB300 design.  Every A^{-1} of Algorithm 3 acts on a vector that is
// nonzero only at trace nodes (rows touched by C, B, G^h) and is read back
// only at trace nodes, so S_u needs only M = (A^{-1}) restricted to trace
// rows and columns: one dense symmetric block per fracture.  M is built once
// at setup, exactly (up to rounding), from the separable structure of the
// uniform Dirichlet rectangles A_f = T_f (I (x) K_x + K_y (x) I):
//   A_f^{-1}[(i,j),(i',j')] = (1/T_f) sum_m S[i][m] S[i'][m] G_m[j][j'],
// with S the orthonormal sine eigenvectors of K_x (eigenvalues lambda_m) and
// G_m = (K_y + lambda_m I)^{-1}, whose entries are U_{j<}(c) U_{ny-1-j>}(c) /
// U_{ny}(c), c = 1 + lambda_m/2, U_k the Chebyshev polynomials of the second
// kind (inverse of a symmetric tridiagonal Toeplitz matrix).  One S_u apply
// is then 5 launches: the CSR gathers into trace space, a block-dense
// product with M (t = A^{-1} C x), the trace-space combination
// g = G^h t - alpha B x, a second product with M (A^{-1} g: Algorithm 3's
// A^{-1} B x and A^{-1} G^h t enter the result only through the combination
// C^T (A^{-1} G^h t - alpha A^{-1} B x), so by linearity one application
// serves both), and the final sparse products fused with the caller's step
// epilogue (Chebyshev recurrence, Lanczos, dots).
// Algorithm 4 (D_S) uses the same M.  Full-vector solves with A (right-hand
// side, recovery of h and p) use fast diagonalisation: sine transform along
// x, a Thomas solve along y per mode, inverse transform.
//
// Fractures of any other shape or coefficients are given as the caller's
// block-diagonal CSR A; M and the full solves then come from a banded
// Cholesky factor of each block (band.cu), and everything downstream of M
// is shared.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "band.cuh"
#include "driver.cuh"
#include "step_impl.cuh"

using namespace pp;

namespace pp {

struct DCsr {  // device CSR view
  int nrows = 0;
  const int* rowptr = nullptr;
  const int* col = nullptr;
  const double* val = nullptr;
};

struct SchurImpl {
  int n_f = 0, n_h = 0, n_u = 0, n_T = 0, max_t = 0, max_nx = 0;
  long long m_elems = 0, s_elems = 0, u_elems = 0, rows_y = 0;
  double alpha = 0.0;
  // general blocks: banded Cholesky factors instead of the closed form
  bool general = false;
  long long band_elems = 0;
  BandDev band;
  // fracture metadata (device)
  int *nx = nullptr, *ny = nullptr;
  double* T = nullptr;
  long long *off = nullptr, *toff = nullptr, *moff = nullptr, *soff = nullptr, *loff = nullptr, *uoff = nullptr,
            *yoff = nullptr;
  // trace nodes (device): fracture and local grid index of each trace node
  int *tfrac = nullptr, *tloc = nullptr, *tnode = nullptr;
  double *M = nullptr, *S = nullptr, *lam = nullptr, *U = nullptr;
  // products restricted to trace space; CT_T/BT_T/Gu act on the u side
  DCsr C_T, B_T, Gh_T, CT_T, BT_T, Gu;
  // the caller's full blocks (for right-hand side and recovery)
  DCsr C, B, Gh, CT, BT;
  // scratch
  double *vT = nullptr, *zT = nullptr, *tT = nullptr, *gT = nullptr, *w2T = nullptr;
  // FP32 copy of M and FP32 trace-space scratch for the preconditioner applied
  // in FP32 (apply_prec = F32; the outer products stay FP64)
  float* M32 = nullptr;
  float *vT32 = nullptr, *zT32 = nullptr, *tT32 = nullptr, *gT32 = nullptr, *w2T32 = nullptr;
  double *fa = nullptr, *fb = nullptr, *fc = nullptr, *fd = nullptr;
  double* ds = nullptr;  // diag(S_u)
};

}  // namespace pp

namespace pp {
namespace {

__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

// index f with off[f] <= e < off[f+1]
__device__ __forceinline__ int find_block(const long long* off, int nf, long long e) {
  int lo = 0, hi = nf;  // invariant off[lo] <= e < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= e) lo = mid; else hi = mid;
  }
  return lo;
}

// ------------------------------------------------------------ setup --------
// S[i][m] = sqrt(2/(nx+1)) sin(pi (i+1)(m+1)/(nx+1)); lambda_m = 4 sin^2(pi (m+1)/(2(nx+1))).
__global__ void sine_tables_kernel(int nf, const int* nx, const long long* soff, const long long* loff, double* S,
                                   double* lam) {
  const long long total = soff[nf];
  for (long long e = gtid(); e < total; e += gstride()) {
    const int f = find_block(soff, nf, e);
    const int n = nx[f];
    const long long loc = e - soff[f];
    const int i = (int)(loc / n), m = (int)(loc % n);
    const long long k = ((long long)(i + 1) * (m + 1)) % (2LL * (n + 1));
    S[e] = sqrt(2.0 / (n + 1)) * sinpi((double)k / (double)(n + 1));
    if (i == 0) {
      const double sh = sinpi((double)(m + 1) / (2.0 * (n + 1)));
      lam[loff[f] + m] = 4.0 * sh * sh;
    }
  }
}

// U_k(c), k = 0..ny, for c = 1 + lambda_m / 2, one thread per (fracture, mode).
__global__ void cheb_u_kernel(int nf, const int* nx, const int* ny, const long long* loff, const long long* uoff,
                              const double* lam, double* U) {
  const long long total = loff[nf];
  for (long long e = gtid(); e < total; e += gstride()) {
    const int f = find_block(loff, nf, e);
    const int m = (int)(e - loff[f]);
    const int n = ny[f];
    const double two_c = 2.0 + lam[e];
    double* u = U + uoff[f] + (long long)m * (n + 1);
    double um1 = 1.0, u0 = two_c;
    u[0] = 1.0;
    if (n >= 1) u[1] = two_c;
    for (int k = 2; k <= n; ++k) {
      const double up = two_c * u0 - um1;
      u[k] = up;
      um1 = u0;
      u0 = up;
    }
  }
}

// M_f[a][b] = (1/T_f) sum_m S[ia][m] S[ib][m] U_{jmin} U_{ny-1-jmax} / U_{ny}.
__global__ void m_blocks_kernel(int nf, const long long* toff, const long long* moff, const int* nx, const int* ny,
                                const double* T, const long long* soff, const long long* uoff, const int* tloc,
                                const double* S, const double* U, double* M) {
  const long long total = moff[nf];
  for (long long e = gtid(); e < total; e += gstride()) {
    const int f = find_block(moff, nf, e);
    const long long t = toff[f + 1] - toff[f];
    const long long loc = e - moff[f];
    const int a = (int)(loc / t), b = (int)(loc % t);
    const int n = nx[f], nyf = ny[f];
    const int la = tloc[toff[f] + a], lb = tloc[toff[f] + b];
    const int ia = la % n, ja = la / n, ib = lb % n, jb = lb / n;
    const int jmin = ja < jb ? ja : jb, jmax = ja < jb ? jb : ja;
    const double* Sa = S + soff[f] + (long long)ia * n;
    const double* Sb = S + soff[f] + (long long)ib * n;
    const double* Uf = U + uoff[f];
    double acc = 0.0;
    for (int m = 0; m < n; ++m) {
      const double* um = Uf + (long long)m * (nyf + 1);
      acc = fma(Sa[m] * Sb[m], um[jmin] * (um[nyf - 1 - jmax] / um[nyf]), acc);
    }
    M[e] = acc / T[f];
  }
}

// Algorithm 4 restricted to trace space: one block per column i of C:
// m = M c_i (c_i lies in one fracture), D_i = G^u_ii + m^T (G^h m) - 2 alpha m^T b_i.
__global__ void schur_diag_kernel(int n_u, int nf, const long long* toff, const long long* moff, const int* tfrac,
                                  DCsr CT_T, DCsr BT_T, DCsr Gh_T, DCsr Gu, const double* M, double alpha, double* ds,
                                  int* bad) {
  extern __shared__ double mvec[];
  for (int i = blockIdx.x; i < n_u; i += gridDim.x) {
    const int p0 = CT_T.rowptr[i], p1 = CT_T.rowptr[i + 1];
    int f = -1;
    if (p1 > p0) f = tfrac[CT_T.col[p0]];
    double acc[1] = {0.0};
    if (f >= 0) {
      const long long t0 = toff[f];
      const int t = (int)(toff[f + 1] - t0);
      const double* Mf = M + moff[f];
      for (int a = threadIdx.x; a < t; a += blockDim.x) {
        double s = 0.0;
        for (int p = p0; p < p1; ++p) {
          const int tc = CT_T.col[p];
          if (tfrac[tc] != f) {
            atomicExch(bad, 1);
            continue;
          }
          s += Mf[(long long)a * t + (tc - t0)] * CT_T.val[p];
        }
        mvec[a] = s;
      }
      __syncthreads();
      for (int a = threadIdx.x; a < t; a += blockDim.x) {
        double g = 0.0;
        const long long row = t0 + a;
        for (int p = Gh_T.rowptr[row]; p < Gh_T.rowptr[row + 1]; ++p) {
          const int c = Gh_T.col[p];
          if (tfrac[c] != f) {
            atomicExch(bad, 2);
            continue;
          }
          g += Gh_T.val[p] * mvec[c - t0];
        }
        acc[0] += mvec[a] * g;
      }
      for (int p = BT_T.rowptr[i] + threadIdx.x; p < BT_T.rowptr[i + 1]; p += blockDim.x) {
        const int c = BT_T.col[p];
        if (tfrac[c] == f) acc[0] -= 2.0 * alpha * mvec[c - t0] * BT_T.val[p];
      }
    }
    block_sum<1>(acc);
    if (threadIdx.x == 0) {
      double gii = 0.0;
      for (int p = Gu.rowptr[i]; p < Gu.rowptr[i + 1]; ++p)
        if (Gu.col[p] == i) gii += Gu.val[p];
      ds[i] = gii + acc[0];
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------ apply --------
// vT = C_T (w o x), zT = B_T (w o x): trace-space gathers (thread per row).
// T is the vector type: double, or float for the FP32 preconditioner.
template <typename T>
__global__ void trace_gather_kernel(int n_T, DCsr C_T, DCsr B_T, const double* __restrict__ w,
                                    const T* __restrict__ x, T* __restrict__ vT, T* __restrict__ zT) {
  for (long long r = gtid(); r < n_T; r += gstride()) {
    T v = (T)0, z = (T)0;
    for (int p = C_T.rowptr[r]; p < C_T.rowptr[r + 1]; ++p) {
      const int c = C_T.col[p];
      v += (T)C_T.val[p] * (w ? (T)w[c] * x[c] : x[c]);
    }
    for (int p = B_T.rowptr[r]; p < B_T.rowptr[r + 1]; ++p) {
      const int c = B_T.col[p];
      z += (T)B_T.val[p] * (w ? (T)w[c] * x[c] : x[c]);
    }
    vT[r] = v;
    zT[r] = z;
  }
}

// gT = Gh_T tT - alpha zT (zT may be null: gT = Gh_T tT)
template <typename T>
__global__ void trace_gh_kernel(int n_T, DCsr Gh_T, const T* __restrict__ tT, const T* __restrict__ zT, T alpha,
                                T* __restrict__ gT) {
  for (long long r = gtid(); r < n_T; r += gstride()) {
    T g = (T)0;
    for (int p = Gh_T.rowptr[r]; p < Gh_T.rowptr[r + 1]; ++p) g += (T)Gh_T.val[p] * tT[Gh_T.col[p]];
    gT[r] = zT ? g - alpha * zT[r] : g;
  }
}

template <typename T>
__device__ __forceinline__ T warp_sum_t(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  return x;
}

// y = M x, M the dense trace blocks (fracture f's block M_f is t_f x t_f,
// row-major, at moff[f]).  A warp takes kMRows rows at a time, kMG lanes per
// row: each lane reads 16 bytes of the row per step (the kMG lanes of a row
// cover 128 contiguous bytes), so a warp-wide load fetches whole lines, and
// the row's sum needs log2(kMG) shuffle-add steps instead of 5 -- those adds
// run on the FP64 pipe, which bounds this product (one FMA per entry).  The
// row's unaligned head (before its first 16-byte boundary) is added by its
// first lane.  Partial sums are combined in a fixed order.
constexpr int kMG = 8;              // lanes per row
constexpr int kMRows = 32 / kMG;    // rows per warp pass

template <typename T>
struct MVec;
template <>
struct MVec<double> {
  static constexpr int W = 2;
  __device__ static void ld(const double* p, double (&o)[2]) {
    const double2 v = __ldcs(reinterpret_cast<const double2*>(p));
    o[0] = v.x;
    o[1] = v.y;
  }
};
template <>
struct MVec<float> {
  static constexpr int W = 4;
  __device__ static void ld(const float* p, float (&o)[4]) {
    const float4 v = __ldcs(reinterpret_cast<const float4*>(p));
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
  }
};

template <typename T>
__global__ void __launch_bounds__(kBlock, sizeof(T) == 4 ? 4 : 8) m_apply_kernel(int n_T, const long long* __restrict__ toff,
                                                         const long long* __restrict__ moff,
                                                         const int* __restrict__ tfrac, const T* __restrict__ M,
                                                         const T* __restrict__ x, T* __restrict__ y) {
  constexpr int W = MVec<T>::W;  // elements per 16 bytes
  const int lane = threadIdx.x & 31, q = lane / kMG, l = lane % kMG;
  const long long gw = gtid() >> 5, nw = gstride() >> 5;
  for (long long r0 = gw * kMRows; r0 < n_T; r0 += nw * kMRows) {
    const long long r = r0 + q;
    T a = (T)0;
    if (r < n_T) {
      const int f = tfrac[r];
      const long long t0 = toff[f];
      const int t = (int)(toff[f + 1] - t0);
      const long long e = moff[f] + (r - t0) * t;  // element index of the row's first entry
      const T* row = M + e;
      const T* xf = x + t0;
      const int head = (int)((W - e % W) % W) < t ? (int)((W - e % W) % W) : t;  // entries before alignment
      T acc0 = (T)0, acc1 = (T)0;
      if (l == 0)
        for (int j = 0; j < head; ++j) acc0 = fma(__ldcs(row + j), __ldg(xf + j), acc0);
      int j = head + l * W;
      if constexpr (sizeof(T) == 4) {
        // FP32 (bound by load latency, not by the FMAs): four 16-byte loads
        // in flight per lane per step
        for (; j + 3 * kMG * W + W <= t; j += 4 * kMG * W) {
          T m0[W], m1[W], m2[W], m3[W], x0[W], x1[W], x2[W], x3[W];
          MVec<T>::ld(row + j, m0);
          MVec<T>::ld(row + j + kMG * W, m1);
          MVec<T>::ld(row + j + 2 * kMG * W, m2);
          MVec<T>::ld(row + j + 3 * kMG * W, m3);
#pragma unroll
          for (int u = 0; u < W; ++u) {
            x0[u] = __ldg(xf + j + u);
            x1[u] = __ldg(xf + j + kMG * W + u);
            x2[u] = __ldg(xf + j + 2 * kMG * W + u);
            x3[u] = __ldg(xf + j + 3 * kMG * W + u);
          }
#pragma unroll
          for (int u = 0; u < W; ++u) {
            acc0 = fma(m0[u], x0[u], acc0);
            acc1 = fma(m1[u], x1[u], acc1);
          }
#pragma unroll
          for (int u = 0; u < W; ++u) {
            acc0 = fma(m2[u], x2[u], acc0);
            acc1 = fma(m3[u], x3[u], acc1);
          }
        }
      }
      // two 16-byte loads in flight per lane per step
      for (; j + kMG * W + W <= t; j += 2 * kMG * W) {
        T m0[W], m1[W];
        MVec<T>::ld(row + j, m0);
        MVec<T>::ld(row + j + kMG * W, m1);
#pragma unroll
        for (int u = 0; u < W; ++u) acc0 = fma(m0[u], __ldg(xf + j + u), acc0);
#pragma unroll
        for (int u = 0; u < W; ++u) acc1 = fma(m1[u], __ldg(xf + j + kMG * W + u), acc1);
      }
      for (; j + W <= t; j += kMG * W) {
        T m0[W];
        MVec<T>::ld(row + j, m0);
#pragma unroll
        for (int u = 0; u < W; ++u) acc0 = fma(m0[u], __ldg(xf + j + u), acc0);
      }
      for (int u = 0; u < W; ++u)  // the tail after the last full 16 bytes
        if (j + u < t) acc0 = fma(__ldcs(row + j + u), __ldg(xf + j + u), acc0);
      a = acc0 + acc1;
    }
#pragma unroll
    for (int o = kMG / 2; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o, kMG);
    if (r < n_T && l == 0) y[r] = a;
  }
}

// Final sparse products in u space fused with the caller's step epilogue:
// s = w o (G^u (w o x) - alpha BT_T t + CT_T w2) = (S_hat x)_row, with
// t = M C (w o x) and w2 = M (G^h t - alpha B (w o x)).
template <int MODE, int NDOT, typename T>
__global__ void __launch_bounds__(kBlock) schur_final_kernel(int n_u, DCsr Gu, DCsr BT_T, DCsr CT_T, double alpha,
                                                             const double* __restrict__ w, const T* __restrict__ tT,
                                                             const T* __restrict__ w2T,
                                                             StepArgs<T> a, const Scalars* sc, double* partials,
                                                             unsigned int* counter) {
  if (sc && load_done(sc)) return;
  double dot[NDOT > 0 ? NDOT : 1];
  for (int i = 0; i < (NDOT > 0 ? NDOT : 1); ++i) dot[i] = 0.0;
  const T lan = lanczos_coef<T, MODE>(a);
  const T al = (T)alpha;
  for (long long i = gtid(); i < n_u; i += gstride()) {
    T gu = (T)0, bt = (T)0, ct = (T)0;
    for (int p = Gu.rowptr[i]; p < Gu.rowptr[i + 1]; ++p) {
      const int c = Gu.col[p];
      gu += (T)Gu.val[p] * (w ? (T)w[c] * a.x[c] : a.x[c]);
    }
    for (int p = BT_T.rowptr[i]; p < BT_T.rowptr[i + 1]; ++p) bt += (T)BT_T.val[p] * tT[BT_T.col[p]];
    for (int p = CT_T.rowptr[i]; p < CT_T.rowptr[i + 1]; ++p) {
      const int c = CT_T.col[p];
      ct += (T)CT_T.val[p] * w2T[c];
    }
    T s = gu - al * bt + ct;
    if (w) s *= (T)w[i];
    T xs = (T)0, rs = (T)0, xo = (T)0;
    if constexpr (mode_needs_xown<MODE, NDOT>()) xs = a.x[i];
    if constexpr (mode_needs_r<MODE>()) rs = a.r[i];
    if constexpr (mode_needs_xold<MODE>()) {
      if (MODE == kChebK || a.xold) xo = a.xold[i];
    }
    const T y = row_value<T, MODE>(a, s, xs, rs, xo, lan);
    a.y[i] = y;
    row_dots<T, MODE, NDOT>(a, i, y, xs, rs, dot);
  }
  finish_dots<T, NDOT>(a, dot, partials, counter);
}

// ------------------------------------------------ fast diagonalisation ----
// out[row][m] = sum_i S[i][m] in[row][i] for every grid row (f, j): one warp
// per row, the row staged in shared memory.
__global__ void __launch_bounds__(kBlock) fd_transform_kernel(int nf, const long long* yoff, const long long* off,
                                                              const int* nx, const long long* soff, const double* S,
                                                              const double* __restrict__ in,
                                                              double* __restrict__ out, int max_nx) {
  extern __shared__ double srow[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double* buf = srow + (long long)wid * max_nx;
  const long long total = yoff[nf];
  const long long gw = gtid() >> 5, nw = gstride() >> 5;
  for (long long rr = gw; rr < total; rr += nw) {
    const int f = find_block(yoff, nf, rr);
    const int n = nx[f];
    const long long base = off[f] + (rr - yoff[f]) * n;
    for (int i = lane; i < n; i += 32) buf[i] = in[base + i];
    __syncwarp();
    const double* Sf = S + soff[f];
    for (int m0 = 0; m0 < n; m0 += 32) {
      const int m = m0 + lane;
      double acc = 0.0;
      if (m < n)
        for (int i = 0; i < n; ++i) acc = fma(Sf[(long long)i * n + m], buf[i], acc);
      if (m < n) out[base + m] = acc;
    }
    __syncwarp();
  }
}

// Thomas solve along y for each (fracture, mode): T_f (K_y + lambda_m) u = v.
__global__ void fd_thomas_kernel(int nf, const long long* loff, const long long* off, const int* nx, const int* ny,
                                 const double* T, const double* lam, const double* __restrict__ v,
                                 double* __restrict__ u, double* __restrict__ cp) {
  const long long total = loff[nf];
  for (long long e = gtid(); e < total; e += gstride()) {
    const int f = find_block(loff, nf, e);
    const int m = (int)(e - loff[f]);
    const int n = nx[f], nyf = ny[f];
    const double d = 2.0 + lam[e];
    const double it = 1.0 / T[f];
    const long long b = off[f] + m;
    // forward sweep: sub- and super-diagonal are -1
    double c_prev = -1.0 / d;
    double d_prev = v[b] * it / d;
    cp[b] = c_prev;
    u[b] = d_prev;
    for (int j = 1; j < nyf; ++j) {
      const long long idx = b + (long long)j * n;
      const double den = d + c_prev;
      c_prev = -1.0 / den;
      d_prev = (v[idx] * it + d_prev) / den;
      cp[idx] = c_prev;
      u[idx] = d_prev;
    }
    for (int j = nyf - 2; j >= 0; --j) {
      const long long idx = b + (long long)j * n;
      u[idx] = u[idx] - cp[idx] * u[idx + n];
    }
  }
}

// generic y = A x (CSR) and y = alpha * y0 + beta * (A x)
__global__ void csr_axpy_kernel(DCsr A, const double* __restrict__ x, double a0, const double* __restrict__ y0,
                                double a1, double* __restrict__ y) {
  for (long long r = gtid(); r < A.nrows; r += gstride()) {
    double s = 0.0;
    for (int p = A.rowptr[r]; p < A.rowptr[r + 1]; ++p) s += A.val[p] * x[A.col[p]];
    y[r] = (y0 ? a0 * y0[r] : 0.0) + a1 * s;
  }
}

__global__ void trace_restrict_kernel(int n_T, const int* tnode, const double* __restrict__ full,
                                      double* __restrict__ tr) {
  for (long long r = gtid(); r < n_T; r += gstride()) tr[r] = full[tnode[r]];
}

int grid_of(long long work, int per_block = kBlock) {
  long long g = (work + per_block - 1) / per_block;
  return (int)std::max(1LL, std::min<long long>(g, 16LL * num_sms()));
}

}  // namespace
}  // namespace pp

// ---------------------------------------------------------------------------
// host-side trace analysis
// ---------------------------------------------------------------------------
namespace pp {
namespace {

struct HCsr {
  int nrows = 0;
  std::vector<int> rp, col;
  std::vector<double> val;
};

struct TracePlan {
  int n_T = 0, max_t = 0, max_nx = 0;
  bool general = false;
  BandHost band;  // general blocks only
  std::vector<int> tnode;             // global node of trace index
  std::vector<int> tfrac, tloc;       // fracture, local grid index
  std::vector<long long> toff, moff, soff, loff, uoff, yoff;
  HCsr C_T, B_T, Gh_T, CT_T, BT_T;
  long long m_elems = 0;
};

int download(const int* rp, const int* ci, const double* va, int nrows, HCsr& h, cudaStream_t s) {
  h.nrows = nrows;
  h.rp.resize((size_t)nrows + 1);
  cudaError_t e = cudaMemcpyAsync(h.rp.data(), rp, sizeof(int) * (nrows + 1), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "reading a fracture-network block");
  const int nnz = h.rp[nrows];
  if (h.rp[0] != 0 || nnz < 0) return fail(nullptr, PP_EINVAL, "fracture-network block: bad rowptr");
  h.col.resize(std::max(nnz, 1));
  h.val.resize(std::max(nnz, 1));
  if (nnz > 0) {
    e = cudaMemcpyAsync(h.col.data(), ci, sizeof(int) * nnz, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.val.data(), va, sizeof(double) * nnz, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "reading a fracture-network block");
  }
  return PP_OK;
}

int check_dfn(const pp_dfn* d) {
  if (!d) return fail(nullptr, PP_EINVAL, "pp_dfn is NULL");
  if (d->n_f <= 0 || d->n_h <= 0 || d->n_u <= 0) return fail(nullptr, PP_EINVAL, "n_f, n_h, n_u must be positive");
  const bool general = d->A_rowptr != nullptr;
  if (!d->offset) return fail(nullptr, PP_EINVAL, "fracture offsets are NULL");
  if (general && (!d->A_col || !d->A_val)) return fail(nullptr, PP_EINVAL, "A_col or A_val is NULL");
  if (!general && (!d->nx || !d->ny || !d->T)) return fail(nullptr, PP_EINVAL, "fracture metadata is NULL");
  const void* ptrs[] = {d->C_rowptr, d->C_col, d->C_val, d->B_rowptr, d->B_col, d->B_val, d->CT_rowptr,
                        d->CT_col, d->CT_val, d->BT_rowptr, d->BT_col, d->BT_val, d->Gh_rowptr, d->Gh_col,
                        d->Gh_val, d->Gu_rowptr, d->Gu_col, d->Gu_val};
  for (const void* p : ptrs)
    if (!p) return fail(nullptr, PP_EINVAL, "a fracture-network CSR array is NULL");
  if (d->offset[0] != 0 || d->offset[d->n_f] != d->n_h) return fail(nullptr, PP_EINVAL, "offset must span [0, n_h]");
  for (int f = 0; f < d->n_f; ++f) {
    if (d->offset[f + 1] <= d->offset[f])
      return fail(nullptr, PP_EINVAL, "fracture " + std::to_string(f) + " has no nodes");
    if (general) continue;
    if (d->nx[f] <= 0 || d->ny[f] <= 0 || !(d->T[f] > 0.0))
      return fail(nullptr, PP_EINVAL, "fracture " + std::to_string(f) + ": nx, ny, T must be positive");
    if (d->offset[f + 1] - d->offset[f] != (long long)d->nx[f] * d->ny[f])
      return fail(nullptr, PP_EINVAL, "fracture " + std::to_string(f) + ": offset does not match nx*ny");
  }
  return PP_OK;
}

int plan_traces(const pp_dfn* d, TracePlan& P, cudaStream_t s) {
  HCsr C, B, Gh, CT, BT;
  int rc;
  if ((rc = download(d->C_rowptr, d->C_col, d->C_val, d->n_h, C, s))) return rc;
  if ((rc = download(d->B_rowptr, d->B_col, d->B_val, d->n_h, B, s))) return rc;
  if ((rc = download(d->Gh_rowptr, d->Gh_col, d->Gh_val, d->n_h, Gh, s))) return rc;
  if ((rc = download(d->CT_rowptr, d->CT_col, d->CT_val, d->n_u, CT, s))) return rc;
  if ((rc = download(d->BT_rowptr, d->BT_col, d->BT_val, d->n_u, BT, s))) return rc;
  const int nh = d->n_h, nf = d->n_f;
  std::vector<char> is_t(nh, 0);
  auto mark_rows = [&](const HCsr& X) {
    for (int r = 0; r < X.nrows; ++r)
      if (X.rp[r + 1] > X.rp[r]) is_t[r] = 1;
  };
  mark_rows(C);
  mark_rows(B);
  mark_rows(Gh);
  for (int r = 0; r < nh; ++r)
    for (int p = Gh.rp[r]; p < Gh.rp[r + 1]; ++p) {
      if (Gh.col[p] < 0 || Gh.col[p] >= nh) return fail(nullptr, PP_EINVAL, "G^h column out of range");
      is_t[Gh.col[p]] = 1;
    }
  for (const HCsr* X : {&CT, &BT})
    for (int p = 0; p < X->rp[X->nrows]; ++p) {
      if (X->col[p] < 0 || X->col[p] >= nh) return fail(nullptr, PP_EINVAL, "C^T/B^T column out of range");
      is_t[X->col[p]] = 1;
    }
  std::vector<int> tidx(nh, -1);
  P.toff.assign(nf + 1, 0);
  int f = 0;
  for (int node = 0; node < nh; ++node) {
    while (node >= d->offset[f + 1]) ++f;
    if (!is_t[node]) continue;
    tidx[node] = (int)P.tnode.size();
    P.tnode.push_back(node);
    P.tfrac.push_back(f);
    P.tloc.push_back((int)(node - d->offset[f]));
    P.toff[f + 1]++;
  }
  for (int g = 0; g < nf; ++g) P.toff[g + 1] += P.toff[g];
  P.n_T = (int)P.tnode.size();
  P.moff.assign(nf + 1, 0);
  P.soff.assign(nf + 1, 0);
  P.loff.assign(nf + 1, 0);
  P.uoff.assign(nf + 1, 0);
  P.yoff.assign(nf + 1, 0);
  P.general = d->A_rowptr != nullptr;
  for (int g = 0; g < nf; ++g) {
    const long long t = P.toff[g + 1] - P.toff[g];
    P.max_t = std::max<long long>(P.max_t, t);
    P.moff[g + 1] = P.moff[g] + t * t;
    if (P.general) continue;  // no closed-form tables
    P.max_nx = std::max(P.max_nx, d->nx[g]);
    P.soff[g + 1] = P.soff[g] + (long long)d->nx[g] * d->nx[g];
    P.loff[g + 1] = P.loff[g] + d->nx[g];
    P.uoff[g + 1] = P.uoff[g] + (long long)d->nx[g] * (d->ny[g] + 1);
    P.yoff[g + 1] = P.yoff[g] + d->ny[g];
  }
  P.m_elems = P.moff[nf];

  // restrict the row side of C, B, G^h and remap the column side of C^T, B^T, G^h
  auto restrict_rows = [&](const HCsr& X, HCsr& Y, bool remap_cols) -> int {
    Y.nrows = P.n_T;
    Y.rp.assign(P.n_T + 1, 0);
    for (int r = 0; r < P.n_T; ++r) {
      const int node = P.tnode[r];
      for (int p = X.rp[node]; p < X.rp[node + 1]; ++p) {
        int c = X.col[p];
        if (remap_cols) {
          c = tidx[c];
          if (c < 0) return fail(nullptr, PP_EINVAL, "G^h couples a non-trace node");
        }
        Y.col.push_back(c);
        Y.val.push_back(X.val[p]);
      }
      Y.rp[r + 1] = (int)Y.col.size();
    }
    return PP_OK;
  };
  if ((rc = restrict_rows(C, P.C_T, false))) return rc;
  if ((rc = restrict_rows(B, P.B_T, false))) return rc;
  if ((rc = restrict_rows(Gh, P.Gh_T, true))) return rc;
  auto remap_cols = [&](const HCsr& X, HCsr& Y) {
    Y = X;
    for (int p = 0; p < X.rp[X.nrows]; ++p) Y.col[p] = tidx[X.col[p]];
  };
  remap_cols(CT, P.CT_T);
  remap_cols(BT, P.BT_T);
  for (const HCsr* X : {&P.C_T, &P.B_T})
    for (int p = 0; p < X->rp[X->nrows]; ++p)
      if (X->col[p] < 0 || X->col[p] >= d->n_u) return fail(nullptr, PP_EINVAL, "C/B column out of range");
  if (P.general) {
    HCsr A;
    if ((rc = download(d->A_rowptr, d->A_col, d->A_val, d->n_h, A, s))) return rc;
    for (int p = 0; p < A.rp[nh]; ++p)
      if (A.col[p] < 0 || A.col[p] >= nh) return fail(nullptr, PP_EINVAL, "A column out of range");
    std::string err;
    if ((rc = band_plan(nf, nh, d->offset, A.rp, A.col, A.val, P.toff, P.tnode, P.band, err)))
      return fail(nullptr, rc, err);
  }
  return PP_OK;
}

struct Bump {
  uintptr_t base, off = 0;
  explicit Bump(void* b) : base((uintptr_t)b) {}
  template <typename T>
  T* take(long long count) {
    off = (off + 255) & ~(uintptr_t)255;
    T* p = reinterpret_cast<T*>(base + off);
    off += (uintptr_t)(count > 0 ? count : 1) * sizeof(T);
    return p;
  }
  void* here() {
    off = (off + 255) & ~(uintptr_t)255;
    return reinterpret_cast<void*>(base + off);
  }
};

template <typename T>
T* put(Bump& B, const std::vector<T>& v, std::vector<std::pair<void*, std::pair<const void*, size_t>>>* up) {
  T* p = B.take<T>((long long)v.size());
  if (up && !v.empty()) up->push_back({(void*)p, {(const void*)v.data(), v.size() * sizeof(T)}});
  return p;
}

DCsr put_csr(Bump& B, const HCsr& h, std::vector<std::pair<void*, std::pair<const void*, size_t>>>* up) {
  DCsr d;
  d.nrows = h.nrows;
  d.rowptr = put(B, h.rp, up);
  d.col = put(B, h.col, up);
  d.val = put(B, h.val, up);
  return d;
}

// Lay out the Schur context in the workspace (base may be null to size it);
// uploads are collected in `up`.
size_t layout_schur(pp_ctx* c, SchurImpl* S, const pp_dfn* d, const TracePlan& P, void* base,
                    std::vector<std::pair<void*, std::pair<const void*, size_t>>>* up,
                    std::vector<long long>* off_host, std::vector<int>* nxh, std::vector<int>* nyh,
                    std::vector<double>* Th) {
  Bump B(base);
  const long long n_pad = ((long long)d->n_u + 127) / 128 * 128;
  c->n = d->n_u;
  c->n_pad = n_pad;
  c->sc = B.take<Scalars>(1);
  c->partials = B.take<double>(2LL * kMaxGrid);
  c->w = B.take<double>(n_pad);
  S->nx = put(B, *nxh, up);
  S->ny = put(B, *nyh, up);
  S->T = put(B, *Th, up);
  S->off = put(B, *off_host, up);
  S->toff = put(B, P.toff, up);
  S->moff = put(B, P.moff, up);
  S->soff = put(B, P.soff, up);
  S->loff = put(B, P.loff, up);
  S->uoff = put(B, P.uoff, up);
  S->yoff = put(B, P.yoff, up);
  S->tfrac = put(B, P.tfrac, up);
  S->tloc = put(B, P.tloc, up);
  S->tnode = put(B, P.tnode, up);
  S->C_T = put_csr(B, P.C_T, up);
  S->B_T = put_csr(B, P.B_T, up);
  S->Gh_T = put_csr(B, P.Gh_T, up);
  S->CT_T = put_csr(B, P.CT_T, up);
  S->BT_T = put_csr(B, P.BT_T, up);
  S->M = B.take<double>(P.m_elems);
  S->general = P.general;
  if (P.general) {
    const BandHost& H = P.band;
    BandDev& D = S->band;
    D.n_f = d->n_f;
    D.max_w = H.max_w;
    D.max_n = H.max_n;
    D.n_items = H.n_items;
    D.factor_smem = H.factor_smem;
    D.off = S->off;
    D.w = put(B, H.w, up);
    D.boff = put(B, H.boff, up);
    D.gwoff = put(B, H.gwoff, up);
    D.pos = put(B, H.pos, up);
    D.perm = put(B, H.perm, up);
    D.trace_at = put(B, H.trace_at, up);
    D.order = put(B, H.order, up);
    D.tcol = put(B, H.tcol, up);
    D.tpos = put(B, H.tpos, up);
    D.tposa = put(B, H.tposa, up);
    D.items = put(B, H.items, up);
    D.L = B.take<double>(H.elems);
    D.dinv = B.take<double>(d->n_h);
    D.gwin = B.take<double>(H.gwin_elems);
    // forward-sweep scratch: max_n x 32 doubles per block of the M build,
    // at most 8 GiB in all (fewer blocks for very large fractures)
    const long long per_block = std::max(1LL, (long long)H.max_n * kBandCols * (long long)sizeof(double));
    const long long cap_blocks = std::max(1LL, (8LL << 30) / per_block);
    D.grid_trace = (int)std::max(1LL, std::min<long long>({(long long)H.n_items, 2LL * num_sms(), cap_blocks}));
    D.Z = B.take<double>((long long)D.grid_trace * H.max_n * kBandCols);
    D.flags = B.take<int>(2);
    S->band_elems = H.elems;
  }
  S->S = B.take<double>(P.soff.back());
  S->lam = B.take<double>(P.loff.back());
  S->U = B.take<double>(P.uoff.back());
  S->ds = B.take<double>(n_pad);
  S->vT = B.take<double>(P.n_T);
  S->zT = B.take<double>(P.n_T);
  S->tT = B.take<double>(P.n_T);
  S->gT = B.take<double>(P.n_T);
  S->w2T = B.take<double>(P.n_T);
  S->fa = B.take<double>(d->n_h);
  S->fb = B.take<double>(d->n_h);
  S->fc = B.take<double>(d->n_h);
  S->fd = B.take<double>(d->n_h);
  c->mixed = c->opt.apply_prec == PP_PREC_F32;
  if (c->mixed) {
    S->M32 = B.take<float>(P.m_elems);
    S->vT32 = B.take<float>(P.n_T);
    S->zT32 = B.take<float>(P.n_T);
    S->tT32 = B.take<float>(P.n_T);
    S->gT32 = B.take<float>(P.n_T);
    S->w2T32 = B.take<float>(P.n_T);
  }
  c->vec_begin = B.here();
  c->xh = B.take<double>(n_pad);
  c->r = B.take<double>(n_pad);
  c->z = B.take<double>(n_pad);
  c->p = B.take<double>(n_pad);
  c->q = B.take<double>(n_pad);
  c->t1 = B.take<double>(n_pad);
  c->t2 = B.take<double>(n_pad);
  c->bh = B.take<double>(n_pad);
  if (c->mixed) {
    c->r32 = B.take<float>(n_pad);
    c->u32 = B.take<float>(n_pad);
    c->v32 = B.take<float>(n_pad);
    c->z32 = B.take<float>(n_pad);
  }
  c->newton_buf = c->opt.poly == PP_POLY_NEWTON && newton_levels(c->opt.k) > 0
                      ? B.take<double>(2LL * newton_levels(c->opt.k) * n_pad)
                      : nullptr;
  c->fcg_m = c->opt.flexible >= 2 ? c->opt.flexible : 0;
  if (c->fcg_m) {
    c->Pring = B.take<double>((long long)c->fcg_m * n_pad);
    c->Qring = B.take<double>((long long)c->fcg_m * n_pad);
    c->fcg_part = B.take<double>((long long)kMaxFcg * kMaxGrid);
  }
  c->vec_end = reinterpret_cast<void*>(B.base + B.off);
  c->lr_cap = c->opt.lowrank;
  c->lr_m = c->lr_cap > 0 ? (c->opt.lowrank_steps > 0 ? c->opt.lowrank_steps : 30) : 0;
  c->lr_base = B.take<char>((long long)lowrank_bytes(c->lr_cap, c->lr_m, n_pad, kMaxGrid));
  lowrank_carve(c, c->lr_base);
  S->n_T = P.n_T;
  return B.off + 256;
}

// Full solve y = A^{-1} v: banded Cholesky factors for general blocks, else
// fast diagonalisation.
cudaError_t ainv_full(const SchurImpl* S, const double* v, double* y, cudaStream_t s) {
  if (S->general) return band_solve(S->band, S->n_h, v, y, S->fd, s);
  const size_t sm = (size_t)(kBlock / 32) * S->max_nx * sizeof(double);
  const int g_rows = grid_of(S->rows_y * 32);
  fd_transform_kernel<<<g_rows, kBlock, sm, s>>>(S->n_f, S->yoff, S->off, S->nx, S->soff, S->S, v, S->fc,
                                                  S->max_nx);
  fd_thomas_kernel<<<grid_of(S->u_elems), kBlock, 0, s>>>(S->n_f, S->loff, S->off, S->nx, S->ny, S->T, S->lam,
                                                          S->fc, S->fd, y);
  fd_transform_kernel<<<g_rows, kBlock, sm, s>>>(S->n_f, S->yoff, S->off, S->nx, S->soff, S->S, S->fd, y,
                                                  S->max_nx);
  return cudaGetLastError();
}

template <typename T>
cudaError_t m_apply(const SchurImpl* S, const T* M, const T* x, T* y, int* err, cudaStream_t s) {
  (void)err;  // no device waits in the product
  const int g = grid_of((long long)S->n_T * 32);
  m_apply_kernel<T><<<g, kBlock, 0, s>>>(S->n_T, S->toff, S->moff, S->tfrac, M, x, y);
  return cudaGetLastError();
}

// Trace-space scratch and M in the vector type T.
template <typename T>
struct SchurBufs;
template <>
struct SchurBufs<double> {
  static const double* M(const SchurImpl* S) { return S->M; }
  static double* v(const SchurImpl* S) { return S->vT; }
  static double* z(const SchurImpl* S) { return S->zT; }
  static double* t(const SchurImpl* S) { return S->tT; }
  static double* g(const SchurImpl* S) { return S->gT; }
  static double* w2(const SchurImpl* S) { return S->w2T; }
};
template <>
struct SchurBufs<float> {
  static const float* M(const SchurImpl* S) { return S->M32; }
  static float* v(const SchurImpl* S) { return S->vT32; }
  static float* z(const SchurImpl* S) { return S->zT32; }
  static float* t(const SchurImpl* S) { return S->tT32; }
  static float* g(const SchurImpl* S) { return S->gT32; }
  static float* w2(const SchurImpl* S) { return S->w2T32; }
};

template <int MODE, int NDOT, typename T>
cudaError_t final_go(pp_ctx* c, const double* w, const StepParams& p, const Scalars* skip, unsigned int* counter,
                     cudaStream_t s) {
  SchurImpl* S = c->schur;
  using B = SchurBufs<T>;
  StepArgs<T> a = make_args<T>(p);
  schur_final_kernel<MODE, NDOT, T><<<c->grid_vec, kBlock, 0, s>>>(S->n_u, S->Gu, S->BT_T, S->CT_T, S->alpha, w,
                                                                   B::t(S), B::w2(S), a, skip, c->partials,
                                                                   counter);
  return cudaGetLastError();
}

template <int MODE, typename T>
cudaError_t final_ndot(pp_ctx* c, const double* w, const StepParams& p, const Scalars* skip, unsigned int* counter,
                       cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    // the FP32 operator serves the preconditioner's degree steps only
    if (p.ndot != 0 || !(MODE == kCheb1 || MODE == kCheb2 || MODE == kChebK)) return cudaErrorNotSupported;
    return final_go<MODE, 0, T>(c, w, p, skip, counter, s);
  } else {
    if (p.ndot == 0) return final_go<MODE, 0, T>(c, w, p, skip, counter, s);
    if (p.ndot == 1) return final_go<MODE, 1, T>(c, w, p, skip, counter, s);
    return final_go<MODE, 2, T>(c, w, p, skip, counter, s);
  }
}

// Operator step with the (optionally scaled) Schur complement: the five
// launches described at the top of this file.  w = nullptr gives S_u itself.
// T = float runs the whole step on the FP32 copy of M (preconditioner only).
template <typename T>
cudaError_t schur_step(pp_ctx* c, const double* w, const StepParams& p, const Scalars* skip, unsigned int* counter,
                       cudaStream_t s) {
  SchurImpl* S = c->schur;
  using B = SchurBufs<T>;
  const T* x = static_cast<const T*>(p.x);
  trace_gather_kernel<T><<<grid_of(S->n_T), kBlock, 0, s>>>(S->n_T, S->C_T, S->B_T, w, x, B::v(S), B::z(S));
  int* err = &c->sc->dev_error;
  cudaError_t e = m_apply<T>(S, B::M(S), B::v(S), B::t(S), err, s);  // t = A^{-1} C x
  if (e != cudaSuccess) return e;
  // Algorithm 3 applies A^{-1} to B x and to G^h t and uses the results only
  // in C^T (A^{-1} G^h t - alpha A^{-1} B x); by linearity that is one
  // application, to g = G^h t - alpha B x
  trace_gh_kernel<T><<<grid_of(S->n_T), kBlock, 0, s>>>(S->n_T, S->Gh_T, B::t(S), B::z(S), (T)S->alpha, B::g(S));
  e = m_apply<T>(S, B::M(S), B::g(S), B::w2(S), err, s);  // w2 = A^{-1} g
  if (e != cudaSuccess) return e;
  switch (p.mode) {
    case kSpmv: return final_ndot<kSpmv, T>(c, w, p, skip, counter, s);
    case kResid: return final_ndot<kResid, T>(c, w, p, skip, counter, s);
    case kCheb1: return final_ndot<kCheb1, T>(c, w, p, skip, counter, s);
    case kCheb2: return final_ndot<kCheb2, T>(c, w, p, skip, counter, s);
    case kChebK: return final_ndot<kChebK, T>(c, w, p, skip, counter, s);
    case kLanczos: return final_ndot<kLanczos, T>(c, w, p, skip, counter, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace
}  // namespace pp

namespace pp {

cudaError_t schur_scaled_step(pp_ctx* c, bool lp, const StepParams& p, const Scalars* skip, unsigned int* counter,
                              cudaStream_t s) {
  if (lp) return schur_step<float>(c, c->w, p, skip, counter, s);
  return schur_step<double>(c, c->w, p, skip, counter, s);
}

void schur_free(SchurImpl* s) { delete s; }

}  // namespace pp

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
namespace pp {
namespace {

int prepare(pp_ctx* c, SchurImpl* S, const pp_dfn* d, TracePlan& P, void* base, bool upload, cudaStream_t s,
            size_t* bytes) {
  std::vector<long long> offh(d->offset, d->offset + d->n_f + 1);
  // general blocks carry no grid metadata (nx, ny, T may be NULL)
  std::vector<int> nxh(d->n_f, 0), nyh(d->n_f, 0);
  std::vector<double> Th(d->n_f, 0.0);
  if (!P.general) {
    nxh.assign(d->nx, d->nx + d->n_f);
    nyh.assign(d->ny, d->ny + d->n_f);
    Th.assign(d->T, d->T + d->n_f);
  }
  std::vector<std::pair<void*, std::pair<const void*, size_t>>> up;
  *bytes = layout_schur(c, S, d, P, base, upload ? &up : nullptr, &offh, &nxh, &nyh, &Th);
  if (!upload) return PP_OK;
  for (auto& u : up) {
    cudaError_t e = cudaMemcpyAsync(u.first, u.second.first, u.second.second, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(c, e, "uploading fracture-network structures");
  }
  cudaError_t e = cudaStreamSynchronize(s);  // host vectors go out of scope
  if (e != cudaSuccess) return cuda_fail(c, e, "uploading fracture-network structures");
  return PP_OK;
}

int check_schur_opts(const pp_options* o) {
  int rc = validate_options(nullptr, o);
  if (rc) return rc;
  if (o->apply_prec == PP_PREC_BF16)
    return fail(nullptr, PP_EUNSUPPORTED, "the Schur operator is applied in FP64, or in FP32 inside p_k");
  return PP_OK;
}

}  // namespace
}  // namespace pp

extern "C" int pp_schur_workspace_size(const pp_dfn* d, const pp_options* opt, size_t* bytes) {
  int rc = check_dfn(d);
  if (rc) return rc;
  if ((rc = check_schur_opts(opt))) return rc;
  if (!bytes) return fail(nullptr, PP_EINVAL, "bytes is NULL");
  TracePlan P;
  if ((rc = plan_traces(d, P, nullptr))) return rc;
  pp_ctx tmp;
  tmp.opt = *opt;
  SchurImpl S;
  return prepare(&tmp, &S, d, P, nullptr, false, nullptr, bytes);
}

extern "C" int schur_setup(pp_ctx** out, const pp_dfn* d, const pp_options* opt, void* ws, size_t ws_bytes,
                           void* stream) {
  if (!out) return fail(nullptr, PP_EINVAL, "ctx pointer is NULL");
  *out = nullptr;
  int rc = check_dfn(d);
  if (rc) return rc;
  if ((rc = check_schur_opts(opt))) return rc;
  if (!ws || ((uintptr_t)ws & 255)) return fail(nullptr, PP_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  pp_ctx* c = new pp_ctx();
  c->schur = new SchurImpl();
  auto bail = [&](int code) {
    std::string m = c->err;
    destroy_ctx_resources(c);
    delete c;
    if (!m.empty()) fail(nullptr, code, m);
    return code;
  };
  c->kind = 1;
  c->opt = *opt;
  if (c->opt.check_every <= 0) c->opt.check_every = 4;
  c->op_launches = 5;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  SchurImpl* S = c->schur;
  TracePlan P;
  if ((rc = plan_traces(d, P, s))) return bail(rc);
  size_t need = 0;
  prepare(c, S, d, P, nullptr, false, s, &need);
  if (ws_bytes < need) return bail(fail(c, PP_EINVAL, "workspace too small: need " + std::to_string(need) + " bytes"));
  if ((rc = prepare(c, S, d, P, ws, true, s, &need))) return bail(rc);
  c->ws = ws;
  c->ws_bytes = ws_bytes;
  c->num_sms = num_sms();
  S->n_f = d->n_f;
  S->n_h = d->n_h;
  S->n_u = d->n_u;
  S->max_t = P.max_t;
  S->max_nx = P.max_nx;
  S->m_elems = P.m_elems;
  S->s_elems = P.soff.back();
  S->u_elems = P.loff.back();
  S->rows_y = P.yoff.back();
  S->alpha = d->alpha_reg;
  S->Gu.nrows = d->n_u;
  S->Gu.rowptr = d->Gu_rowptr;
  S->Gu.col = d->Gu_col;
  S->Gu.val = d->Gu_val;
  S->C = DCsr{d->n_h, d->C_rowptr, d->C_col, d->C_val};
  S->B = DCsr{d->n_h, d->B_rowptr, d->B_col, d->B_val};
  S->Gh = DCsr{d->n_h, d->Gh_rowptr, d->Gh_col, d->Gh_val};
  S->CT = DCsr{d->n_u, d->CT_rowptr, d->CT_col, d->CT_val};
  S->BT = DCsr{d->n_u, d->BT_rowptr, d->BT_col, d->BT_val};
  c->nnz = P.m_elems;
  c->nnz_pad = P.m_elems;
  c->grid_vec = (int)std::max(1LL, std::min<long long>(std::min(kMaxGrid, c->num_sms * 8),
                                                       (c->n_pad / 2 + kBlock - 1) / kBlock));
  if (c->opt.max_blocks > 0) c->grid_vec = std::min(c->grid_vec, c->opt.max_blocks);
  c->grid_step = c->grid_vec;
  cudaError_t e = cudaMemsetAsync(c->vec_begin, 0, (char*)c->vec_end - (char*)c->vec_begin, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->sc, 0, sizeof(Scalars), s);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "clearing workspace"));
  if (S->general) {
    // banded Cholesky of every block, then M from band solves
    cudaEvent_t b0 = nullptr, b1 = nullptr, b2 = nullptr;
    cudaEventCreate(&b0);
    cudaEventCreate(&b1);
    cudaEventCreate(&b2);
    cudaEventRecord(b0, s);
    e = cudaMemsetAsync(S->band.L, 0, sizeof(double) * (size_t)S->band_elems, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(S->band.flags, 0, 2 * sizeof(int), s);
    if (e == cudaSuccess) e = band_fill(S->band, d->n_h, d->A_rowptr, d->A_col, d->A_val, s);
    if (e == cudaSuccess) e = band_factor(S->band, s);
    cudaEventRecord(b2, s);
    int bad_f = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad_f, S->band.flags, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      cudaEventDestroy(b0);
      cudaEventDestroy(b1);
      cudaEventDestroy(b2);
      return bail(cuda_fail(c, e, "banded Cholesky of the fracture blocks"));
    }
    if (bad_f) {
      cudaEventDestroy(b0);
      cudaEventDestroy(b1);
      cudaEventDestroy(b2);
      return bail(fail(c, PP_EBREAKDOWN,
                       "A_f of fracture " + std::to_string(bad_f - 1) + " is not positive definite"));
    }
    e = band_trace_blocks(S->band, S->toff, S->moff, S->M, s);
    cudaEventRecord(b1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(b1);
    float fms = 0.f, tms = 0.f;
    if (e == cudaSuccess) {
      cudaEventElapsedTime(&fms, b0, b2);
      cudaEventElapsedTime(&tms, b2, b1);
    }
    cudaEventDestroy(b0);
    cudaEventDestroy(b1);
    cudaEventDestroy(b2);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "trace blocks from the band factors"));
    c->band_max = P.band.max_w;
    c->band_elems = S->band_elems;
    c->t_band_ms = fms;
    c->t_trace_ms = tms;
  } else {
    // sine tables, eigenvalues, U tables, the trace blocks M
    sine_tables_kernel<<<grid_of(S->s_elems), kBlock, 0, s>>>(S->n_f, S->nx, S->soff, S->loff, S->S, S->lam);
    cheb_u_kernel<<<grid_of(S->u_elems), kBlock, 0, s>>>(S->n_f, S->nx, S->ny, S->loff, S->uoff, S->lam, S->U);
    m_blocks_kernel<<<grid_of(S->m_elems), kBlock, 0, s>>>(S->n_f, S->toff, S->moff, S->nx, S->ny, S->T, S->soff,
                                                           S->uoff, S->tloc, S->S, S->U, S->M);
  }
  // then D_S (Algorithm 4)
  if (c->mixed) e = sell_convert_values(S->m_elems, S->M, S->M32, kF32, s);  // M rounded to FP32
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "FP32 copy of M"));
  int* d_bad = reinterpret_cast<int*>(c->t1);
  e = cudaMemsetAsync(d_bad, 0, sizeof(int), s);
  const size_t dsm = (size_t)std::max(S->max_t, 1) * sizeof(double);
  if (dsm > 200 * 1024) return bail(fail(c, PP_EUNSUPPORTED, "a fracture carries more than 25600 trace nodes"));
  if (e == cudaSuccess && dsm > 48 * 1024)
    e = cudaFuncSetAttribute(schur_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dsm);
  if (e == cudaSuccess) {
    schur_diag_kernel<<<std::min(d->n_u, 16 * num_sms()), 128, dsm, s>>>(d->n_u, S->n_f, S->toff, S->moff, S->tfrac,
                                                                  S->CT_T, S->BT_T, S->Gh_T, S->Gu, S->M, S->alpha,
                                                                  S->ds, d_bad);
    e = cudaGetLastError();
  }
  int bad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "Schur setup"));
  if (bad) return bail(fail(c, PP_EUNSUPPORTED, "C columns and G^h must be fracture-local"));
  // seed: W = D_S^{-1/2} (end of Section 4.3)
  std::vector<double> dsh(d->n_u);
  e = cudaMemcpyAsync(dsh.data(), S->ds, sizeof(double) * d->n_u, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "reading D_S"));
  std::vector<double> wh(c->n_pad, 1.0);
  for (int i = 0; i < d->n_u; ++i) {
    if (!(dsh[i] > 0.0)) return bail(fail(c, PP_EBREAKDOWN, "diag(S_u) is not positive at " + std::to_string(i)));
    wh[i] = opt->seed_scaling == PP_SEED_JACOBI ? 1.0 / std::sqrt(dsh[i]) : 1.0;
  }
  e = cudaMemcpyAsync(c->w, wh.data(), sizeof(double) * c->n_pad, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "seed weights"));
  rc = setup_interval_and_coeffs(c, s);
  if (rc) return bail(rc);
  cudaEventRecord(e1, s);
  e = cudaEventSynchronize(e1);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "Schur setup"));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->t_setup_ms = ms;
  *out = c;
  return PP_OK;
}

extern "C" int schur_apply(pp_ctx* c, const double* r, double* y, void* stream) {
  if (!c || c->kind != 1) return fail(c, PP_EINVAL, "not a Schur context");
  if (!r || !y) return fail(c, PP_EINVAL, "vector argument is NULL");
  StepParams p;
  p.mode = kSpmv;
  p.x = r;
  p.y = y;
  cudaError_t e = schur_step<double>(c, nullptr, p, nullptr, &c->sc->counters[kCntSchur], (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "schur_apply");
  return PP_OK;
}

extern "C" int schur_diag(pp_ctx* c, double* ds, void* stream) {
  if (!c || c->kind != 1) return fail(c, PP_EINVAL, "not a Schur context");
  if (!ds) return fail(c, PP_EINVAL, "ds is NULL");
  cudaError_t e = cudaMemcpyAsync(ds, c->schur->ds, sizeof(double) * c->n, cudaMemcpyDeviceToDevice,
                                  (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "schur_diag");
  return PP_OK;
}

extern "C" int schur_ainv(pp_ctx* c, const double* v, double* y, void* stream) {
  if (!c || c->kind != 1) return fail(c, PP_EINVAL, "not a Schur context");
  if (!v || !y) return fail(c, PP_EINVAL, "vector argument is NULL");
  cudaError_t e = ainv_full(c->schur, v, y, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "schur_ainv");
  return PP_OK;
}

extern "C" int schur_rhs(pp_ctx* c, const double* q, double* r, void* stream) {
  if (!c || c->kind != 1) return fail(c, PP_EINVAL, "not a Schur context");
  if (!q || !r) return fail(c, PP_EINVAL, "vector argument is NULL");
  SchurImpl* S = c->schur;
  cudaStream_t s = (cudaStream_t)stream;
  // a1 = A^{-1} q (full), g = G^h a1 on trace nodes, a2 = M g (trace),
  // r = alpha B^T a1 - C^T a2
  cudaError_t e = ainv_full(S, q, S->fa, s);
  if (e == cudaSuccess) {
    trace_restrict_kernel<<<grid_of(S->n_T), kBlock, 0, s>>>(S->n_T, S->tnode, S->fa, S->tT);
    trace_gh_kernel<double><<<grid_of(S->n_T), kBlock, 0, s>>>(S->n_T, S->Gh_T, S->tT, nullptr, 0.0, S->gT);
    e = m_apply<double>(S, S->M, S->gT, S->w2T, &c->sc->dev_error, s);
  }
  if (e == cudaSuccess) {
    csr_axpy_kernel<<<grid_of(S->n_u), kBlock, 0, s>>>(S->BT_T, S->tT, 0.0, nullptr, S->alpha, c->t1);
    csr_axpy_kernel<<<grid_of(S->n_u), kBlock, 0, s>>>(S->CT_T, S->w2T, 1.0, c->t1, -1.0, r);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "schur_rhs");
  return PP_OK;
}

extern "C" int schur_recover(pp_ctx* c, const double* q, const double* u, double* h, double* p, void* stream) {
  if (!c || c->kind != 1) return fail(c, PP_EINVAL, "not a Schur context");
  if (!q || !u || !h || !p) return fail(c, PP_EINVAL, "vector argument is NULL");
  SchurImpl* S = c->schur;
  cudaStream_t s = (cudaStream_t)stream;
  // h = A^{-1}(q + C u); p = A^{-1}(alpha B u - G^h h)
  csr_axpy_kernel<<<grid_of(S->n_h), kBlock, 0, s>>>(S->C, u, 1.0, q, 1.0, S->fa);
  cudaError_t e = ainv_full(S, S->fa, h, s);
  if (e == cudaSuccess) {
    csr_axpy_kernel<<<grid_of(S->n_h), kBlock, 0, s>>>(S->Gh, h, 0.0, nullptr, -1.0, S->fb);
    csr_axpy_kernel<<<grid_of(S->n_h), kBlock, 0, s>>>(S->B, u, 1.0, S->fb, S->alpha, S->fa);
    e = ainv_full(S, S->fa, p, s);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "schur_recover");
  return PP_OK;
}
