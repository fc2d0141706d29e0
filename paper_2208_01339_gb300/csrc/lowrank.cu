// Low-rank acceleration of the polynomial preconditioner (Section 3.1):
//   P_hat = p_k(A_hat) + V (V^T A_hat V)^{-1} V^T
// with V the Ritz vectors of the p smallest Ritz values of a Lanczos run on
// A_hat that keeps its basis (full reorthogonalisation), or caller vectors.
//
// Device pieces: a multi-column inner product (partials per block and
// column, summed in block order by a second kernel, so results are
// deterministic), the Gram-Schmidt update y -= Q h, the combination V = Q Y,
// and the per-application kernels: c = G^{-1} (V^T r) and z += V c fused
// with the inner products (r, z) and (q, z) that PCG needs.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "driver.cuh"

namespace pp {
namespace {

constexpr int kCols = 8;  // columns per block row of the multi-column dot

__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

// part[c * gridDim.x + blockIdx.x] = sum over this block's rows of Q_c . y,
// for the kCols columns c of block row blockIdx.y.
__global__ void __launch_bounds__(kBlock) mdot_partial_kernel(long long n, int ncol, const double* __restrict__ Q,
                                                              long long ldq, const double* __restrict__ y,
                                                              double* __restrict__ part, const Scalars* skip) {
  if (skip && load_done(skip)) return;
  const int c0 = blockIdx.y * kCols;
  double acc[kCols];
#pragma unroll
  for (int t = 0; t < kCols; ++t) acc[t] = 0.0;
  for (long long i = gtid(); i < n; i += gstride()) {
    const double yi = y[i];
#pragma unroll
    for (int t = 0; t < kCols; ++t)
      if (c0 + t < ncol) acc[t] += Q[(long long)(c0 + t) * ldq + i] * yi;
  }
  block_sum<kCols>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int t = 0; t < kCols; ++t)
      if (c0 + t < ncol) part[(long long)(c0 + t) * gridDim.x + blockIdx.x] = acc[t];
  }
}

// out[c] = sum_j part[c * gx + j], one block per column, fixed order.
__global__ void __launch_bounds__(kBlock) mdot_final_kernel(int gx, const double* __restrict__ part,
                                                            double* __restrict__ out) {
  const int c = blockIdx.x;
  double acc[1] = {0.0};
  for (int j = threadIdx.x; j < gx; j += blockDim.x) acc[0] += part[(long long)c * gx + j];
  block_sum<1>(acc);
  if (threadIdx.x == 0) out[c] = acc[0];
}

// y -= sum_c h[c] Q_c
__global__ void __launch_bounds__(kBlock) maxpy_kernel(long long n, int ncol, const double* __restrict__ Q,
                                                       long long ldq, const double* __restrict__ h,
                                                       double* __restrict__ y) {
  for (long long i = gtid(); i < n; i += gstride()) {
    double s = 0.0;
    for (int c = 0; c < ncol; ++c) s += h[c] * Q[(long long)c * ldq + i];
    y[i] -= s;
  }
}

// V_c = sum_j Y[j * p + c] Q_j, c < p, j < m (all n_pad rows).
__global__ void __launch_bounds__(kBlock) combine_kernel(long long n_pad, int m, const double* __restrict__ Q,
                                                         long long ldq, int p, const double* __restrict__ Y,
                                                         double* __restrict__ V) {
  for (long long i = gtid(); i < n_pad; i += gstride()) {
    for (int c = 0; c < p; ++c) {
      double s = 0.0;
      for (int j = 0; j < m; ++j) s += Y[j * p + c] * Q[(long long)j * ldq + i];
      V[(long long)c * ldq + i] = s;
    }
  }
}

// w = column sums of the partials (V^T r), then c = G^{-1} w.  One block.
__global__ void __launch_bounds__(kBlock) lr_coef_kernel(int p, int gx, const double* __restrict__ part,
                                                         const double* __restrict__ Ginv, double* __restrict__ cout,
                                                         const Scalars* skip) {
  if (skip && load_done(skip)) return;
  __shared__ double w[kMaxLowRank];
  for (int c = 0; c < p; ++c) {
    double acc[1] = {0.0};
    for (int j = threadIdx.x; j < gx; j += blockDim.x) acc[0] += part[(long long)c * gx + j];
    block_sum<1>(acc);
    if (threadIdx.x == 0) w[c] = acc[0];
  }
  __syncthreads();
  if (threadIdx.x < p) {
    double s = 0.0;
    for (int j = 0; j < p; ++j) s += Ginv[threadIdx.x * kMaxLowRank + j] * w[j];
    cout[threadIdx.x] = s;
  }
}

// z += V c, then (r, z) -> rz_out and, with NDOT = 2, (q, z) -> zq_out.
template <int NDOT>
__global__ void __launch_bounds__(kBlock) lr_update_kernel(long long n, int p, const double* __restrict__ V,
                                                           long long ldv, const double* __restrict__ cvec,
                                                           double* __restrict__ z, const double* __restrict__ r,
                                                           const double* __restrict__ q, double* rz_out,
                                                           double* zq_out, double* partials, unsigned int* counter,
                                                           const Scalars* skip) {
  if (skip && load_done(skip)) return;
  __shared__ double cs[kMaxLowRank];
  if (threadIdx.x < p) cs[threadIdx.x] = cvec[threadIdx.x];
  __syncthreads();
  double acc[NDOT > 0 ? NDOT : 1];
#pragma unroll
  for (int t = 0; t < (NDOT > 0 ? NDOT : 1); ++t) acc[t] = 0.0;
  for (long long i = gtid(); i < n; i += gstride()) {
    double zi = z[i];
    for (int c = 0; c < p; ++c) zi += cs[c] * V[(long long)c * ldv + i];
    z[i] = zi;
    if (NDOT > 0) acc[0] += r[i] * zi;
    if (NDOT > 1) acc[1] += q[i] * zi;
  }
  if constexpr (NDOT > 0) {
    if (grid_sum<NDOT>(acc, partials, counter) && threadIdx.x == 0) {
      *rz_out = acc[0];
      if (NDOT > 1) *zq_out = acc[1];
    }
  }
}

inline long long round8(long long v) { return (v + kCols - 1) / kCols * kCols; }
inline long long align256(long long b) { return (b + 255) / 256 * 256; }

// Multi-column inner products h[c] = Q_c . y, c < ncol (ncol <= max_cols).
cudaError_t mdot(pp_ctx* c, int ncol, const double* Q, const double* y, double* h, cudaStream_t s) {
  const int gx = c->grid_vec;
  dim3 grid(gx, (ncol + kCols - 1) / kCols);
  mdot_partial_kernel<<<grid, kBlock, 0, s>>>(c->n, ncol, Q, c->n_pad, y, c->lr_part, nullptr);
  mdot_final_kernel<<<ncol, kBlock, 0, s>>>(gx, c->lr_part, h);
  return cudaGetLastError();
}

// Symmetric tridiagonal eigen-decomposition by cyclic Jacobi rotations:
// eigenvalues ascending in w, eigenvectors as the columns of S (m x m,
// S[i * m + j] = component i of eigenvector j).
void tridiag_eig_jacobi(const std::vector<double>& a, const std::vector<double>& b, std::vector<double>& w,
                        std::vector<double>& S) {
  const int m = (int)a.size();
  std::vector<double> M((size_t)m * m, 0.0), E((size_t)m * m, 0.0);
  auto at = [&](int i, int j) -> double& { return M[(size_t)i * m + j]; };
  for (int i = 0; i < m; ++i) {
    at(i, i) = a[i];
    E[(size_t)i * m + i] = 1.0;
  }
  for (int i = 0; i + 1 < m; ++i) at(i, i + 1) = at(i + 1, i) = b[i];
  double fro = 0.0;
  for (double v : M) fro += v * v;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < m; ++i)
      for (int j = i + 1; j < m; ++j) off += 2.0 * at(i, j) * at(i, j);
    if (off <= 1e-32 * fro) break;
    for (int p = 0; p < m; ++p)
      for (int q = p + 1; q < m; ++q) {
        const double apq = at(p, q);
        if (std::fabs(apq) < 1e-300) continue;
        const double th = (at(q, q) - at(p, p)) / (2.0 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
        for (int k = 0; k < m; ++k) {
          const double akp = at(k, p), akq = at(k, q);
          at(k, p) = cs * akp - sn * akq;
          at(k, q) = sn * akp + cs * akq;
        }
        for (int k = 0; k < m; ++k) {
          const double apk = at(p, k), aqk = at(q, k);
          at(p, k) = cs * apk - sn * aqk;
          at(q, k) = sn * apk + cs * aqk;
        }
        for (int k = 0; k < m; ++k) {
          const double ekp = E[(size_t)k * m + p], ekq = E[(size_t)k * m + q];
          E[(size_t)k * m + p] = cs * ekp - sn * ekq;
          E[(size_t)k * m + q] = sn * ekp + cs * ekq;
        }
      }
  }
  std::vector<int> idx(m);
  for (int i = 0; i < m; ++i) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int x, int y) { return at(x, x) < at(y, y); });
  w.resize(m);
  S.assign((size_t)m * m, 0.0);
  for (int j = 0; j < m; ++j) {
    w[j] = at(idx[j], idx[j]);
    for (int i = 0; i < m; ++i) S[(size_t)i * m + j] = E[(size_t)i * m + idx[j]];
  }
}

}  // namespace

size_t lowrank_bytes(int cap, int m, long long n_pad, int grid_max) {
  if (cap <= 0) return 0;
  const long long cols = std::max(round8(cap), round8(m + 1));
  long long b = 0;
  b += align256(sizeof(LowRankState));
  b += align256((long long)cap * n_pad * 8);        // V
  b += align256((long long)(m + 1) * n_pad * 8);    // Q
  b += align256((long long)m * cap * 8);            // Y
  b += align256(cols * grid_max * 8);               // partials
  return (size_t)b;
}

void lowrank_carve(pp_ctx* c, void* base) {
  c->lr = nullptr;
  c->V = c->Q = c->lr_Y = c->lr_part = nullptr;
  if (c->lr_cap <= 0) return;
  char* p = (char*)base;
  auto take = [&](long long bytes) {
    char* q = p;
    p += align256(bytes);
    return q;
  };
  c->lr = (LowRankState*)take(sizeof(LowRankState));
  c->V = (double*)take((long long)c->lr_cap * c->n_pad * 8);
  c->Q = (double*)take((long long)(c->lr_m + 1) * c->n_pad * 8);
  c->lr_Y = (double*)take((long long)c->lr_m * c->lr_cap * 8);
  c->lr_part = (double*)take(std::max(round8(c->lr_cap), round8(c->lr_m + 1)) * kMaxGrid * 8);
}

// G = V^T A_hat V for the first p columns of V, inverted on the host
// (Cholesky, then the explicit inverse) and stored in lr->Ginv.  With
// unit_cols (Ritz vectors), theta_c = G_cc are Rayleigh quotients and the
// relative residuals ||A_hat v_c - theta_c v_c|| / theta_c are recorded.
int lowrank_build_G(pp_ctx* c, int p, bool unit_cols, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  VecLaunch L{c->grid_vec, c->partials, s};
  std::vector<double> G((size_t)p * p), av2(p);
  for (int j = 0; j < p && e == cudaSuccess; ++j) {
    StepParams sp;
    sp.mode = kSpmv;
    sp.x = c->V + (long long)j * c->n_pad;
    sp.y = c->t1;
    e = op_step(c, false, sp, nullptr, &c->sc->counters[kCntStep], s);
    if (e == cudaSuccess) e = mdot(c, p, c->V, c->t1, c->lr->h, s);
    if (e == cudaSuccess) e = vec_dot(L, c->n, c->t1, c->t1, &c->sc->vv, &c->sc->counters[kCntLan]);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&G[(size_t)j * p], c->lr->h, sizeof(double) * p,
                                              cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&av2[j], &c->sc->vv, sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "low-rank V^T A V");
  c->lr_theta.assign(p, 0.0);
  c->lr_ritz_resid = 0.0;
  for (int j = 0; j < p; ++j) {
    const double th = G[(size_t)j * p + j];
    c->lr_theta[j] = th;
    if (unit_cols && th > 0.0)
      c->lr_ritz_resid = std::max(c->lr_ritz_resid, std::sqrt(std::max(av2[j] - th * th, 0.0)) / th);
  }
  // G[j * p + i] = V_i . A V_j; use the lower triangle i >= j
  std::vector<double> Lc((size_t)p * p, 0.0);
  for (int j = 0; j < p; ++j) {
    double d = G[(size_t)j * p + j];
    for (int k = 0; k < j; ++k) d -= Lc[(size_t)j * p + k] * Lc[(size_t)j * p + k];
    // relative threshold: dependent columns leave d at rounding level
    if (!(d > 1e-13 * std::fabs(G[(size_t)j * p + j])) || !std::isfinite(d))
      return fail(c, PP_EBREAKDOWN, "V^T A V is not positive definite (dependent or zero correction vectors)");
    Lc[(size_t)j * p + j] = std::sqrt(d);
    for (int i = j + 1; i < p; ++i) {
      double t = G[(size_t)j * p + i];
      for (int k = 0; k < j; ++k) t -= Lc[(size_t)i * p + k] * Lc[(size_t)j * p + k];
      Lc[(size_t)i * p + j] = t / Lc[(size_t)j * p + j];
    }
  }
  // Ginv = L^{-T} L^{-1}, column by column
  std::vector<double> Ginv((size_t)kMaxLowRank * kMaxLowRank, 0.0), col(p);
  for (int j = 0; j < p; ++j) {
    for (int i = 0; i < p; ++i) col[i] = (i == j) ? 1.0 : 0.0;
    for (int i = 0; i < p; ++i) {
      double t = col[i];
      for (int k = 0; k < i; ++k) t -= Lc[(size_t)i * p + k] * col[k];
      col[i] = t / Lc[(size_t)i * p + i];
    }
    for (int i = p - 1; i >= 0; --i) {
      double t = col[i];
      for (int k = i + 1; k < p; ++k) t -= Lc[(size_t)k * p + i] * col[k];
      col[i] = t / Lc[(size_t)i * p + i];
    }
    for (int i = 0; i < p; ++i) Ginv[(size_t)i * kMaxLowRank + j] = col[i];
  }
  e = cudaMemcpyAsync(c->lr->Ginv, Ginv.data(), sizeof(double) * Ginv.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "low-rank G^{-1} upload");
  c->lr_p = p;
  return PP_OK;
}

// The vectors of the correction: Lanczos with a kept basis Q (columns of
// n_pad doubles) on the preconditioned operator B = p_k(A_hat) A_hat, which
// has the eigenvectors of A_hat, maps its smallest eigenvalues to the
// smallest of B (Theorem 2.3) and is far better conditioned, so its
// leftmost Ritz pairs converge in few steps.  Step j: w = B q_j -
// b_{j-1} q_{j-1}, a_j = (q_j, w), w -= a_j q_j, then classical Gram-Schmidt
// against q_0..q_j, twice, b_j = ||w||, q_{j+1} = w / b_j.  The Ritz
// vectors of the p smallest Ritz values give V = Q Y; G = V^T A_hat V
// follows.  Needs the coefficients of p_k.
int lowrank_lanczos(pp_ctx* c, cudaStream_t s) {
  const int m = c->lr_m;
  const long long ld = c->n_pad;
  Scalars* sc = c->sc;
  VecLaunch L{c->grid_vec, c->partials, s};
  double* Q = c->Q;
  cudaError_t e = cudaMemsetAsync(Q, 0, sizeof(double) * (size_t)(m + 1) * ld, s);
  if (e == cudaSuccess)
    e = lanczos_start(L, c->n, c->n_pad, splitmix_key(c->opt.seed, 3), c->perm, Q, &sc->vv, &sc->counters[kCntVec]);
  if (e == cudaSuccess) e = vec_scale_by_rsqrt(L, c->n, Q, &sc->vv);
  int steps = 0;
  std::vector<double> ha, hb;
  double h2[2] = {0.0, 0.0};
  for (int j = 0; j < m && e == cudaSuccess; ++j) {
    double* qj = Q + (long long)j * ld;
    double* w = Q + (long long)(j + 1) * ld;
    e = prec_op_apply(c, qj, w, s);
    if (e == cudaSuccess && j > 0) e = vec_axpby(L, c->n, -hb[j - 1], Q + (long long)(j - 1) * ld, 1.0, w);
    if (e == cudaSuccess) e = vec_dot(L, c->n, qj, w, &sc->lan_a[j], &sc->counters[kCntLan]);
    if (e == cudaSuccess)
      e = lanczos_orth(L, c->n, w, qj, &sc->lan_a[j], &sc->lan_b2[j], &sc->counters[kCntLan]);
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
      e = mdot(c, j + 1, Q, w, c->lr->h, s);
      if (e == cudaSuccess) {
        maxpy_kernel<<<c->grid_vec, kBlock, 0, s>>>(c->n, j + 1, Q, ld, c->lr->h, w);
        e = cudaGetLastError();
      }
    }
    if (e == cudaSuccess) e = vec_dot(L, c->n, w, w, &sc->lan_b2[j], &sc->counters[kCntLan]);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h2[0], &sc->lan_a[j], sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h2[1], &sc->lan_b2[j], sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) break;
    if (!std::isfinite(h2[0]) || !std::isfinite(h2[1])) return fail(c, PP_ENONFINITE, "non-finite Lanczos coefficient");
    ha.push_back(h2[0]);
    hb.push_back(std::sqrt(h2[1]));
    steps = j + 1;
    if (!(h2[1] > 1e-300)) break;  // invariant subspace
    if (j < m - 1) e = vec_scale_by_rsqrt(L, c->n, w, &sc->lan_b2[j]);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "Lanczos on the preconditioned operator");
  const int p = c->lr_cap;
  if (steps < p) return fail(c, PP_EBREAKDOWN, "Lanczos ended (invariant subspace) before lowrank Ritz pairs formed");
  std::vector<double> ta(ha.begin(), ha.begin() + steps), tb(hb.begin(), hb.begin() + steps - 1);
  std::vector<double> wv, S;
  tridiag_eig_jacobi(ta, tb, wv, S);
  std::vector<double> Y((size_t)steps * p);
  for (int cc = 0; cc < p; ++cc)
    for (int j = 0; j < steps; ++j) Y[(size_t)j * p + cc] = S[(size_t)j * steps + cc];
  e = cudaMemcpyAsync(c->lr_Y, Y.data(), sizeof(double) * Y.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    combine_kernel<<<c->grid_vec, kBlock, 0, s>>>(c->n_pad, steps, Q, ld, p, c->lr_Y, c->V);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "Ritz vectors");
  c->lr_steps_done = steps;
  return lowrank_build_G(c, p, true, s);
}

// Per application: c = G^{-1} V^T r (2 launches, before p_k) ...
cudaError_t lowrank_coefs(pp_ctx* c, const Scalars* skip, const double* r, cudaStream_t s) {
  const int p = c->lr_p;
  const int gx = c->grid_vec;
  dim3 grid(gx, (p + kCols - 1) / kCols);
  mdot_partial_kernel<<<grid, kBlock, 0, s>>>(c->n, p, c->V, c->n_pad, r, c->lr_part, skip);
  lr_coef_kernel<<<1, kBlock, 0, s>>>(p, gx, c->lr_part, c->lr->Ginv, c->lr->c, skip);
  return cudaGetLastError();
}

// ... and z += V c with (r, z) -> rz_out and, when q is given, (q, z) -> zq_out.
cudaError_t lowrank_update(pp_ctx* c, const Scalars* skip, double* z, const double* r, const double* q,
                           double* rz_out, double* zq_out, cudaStream_t s) {
  const int p = c->lr_p;
  unsigned int* cnt = &c->sc->counters[kCntLr];
  if (rz_out == nullptr)
    lr_update_kernel<0><<<c->grid_vec, kBlock, 0, s>>>(c->n, p, c->V, c->n_pad, c->lr->c, z, r, q, rz_out, zq_out,
                                                       c->partials, cnt, skip);
  else if (q == nullptr)
    lr_update_kernel<1><<<c->grid_vec, kBlock, 0, s>>>(c->n, p, c->V, c->n_pad, c->lr->c, z, r, q, rz_out, zq_out,
                                                       c->partials, cnt, skip);
  else
    lr_update_kernel<2><<<c->grid_vec, kBlock, 0, s>>>(c->n, p, c->V, c->n_pad, c->lr->c, z, r, q, rz_out, zq_out,
                                                       c->partials, cnt, skip);
  return cudaGetLastError();
}

}  // namespace pp

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" int pp_set_lowrank(pp_ctx* c, const double* U, int p, long long ldu, void* stream) {
  using namespace pp;
  if (!c) return fail(nullptr, PP_EINVAL, "ctx is NULL");
  if (c->kind == 2) return fail(c, PP_EUNSUPPORTED, "low-rank correction is not available for batch contexts");
  if (p < 0 || p > c->lr_cap)
    return fail(c, PP_EINVAL, "p must be in [0, opt.lowrank] (the capacity reserved at setup)");
  if (p == 0) {
    c->lr_p = 0;
    return PP_OK;
  }
  if (!U) return fail(c, PP_EINVAL, "U is NULL");
  if (ldu < c->n) return fail(c, PP_EINVAL, "ldu must be >= n");
  cudaStream_t s = (cudaStream_t)stream;
  VecLaunch L{c->grid_vec, c->partials, s};
  cudaError_t e = cudaSuccess;
  for (int j = 0; j < p && e == cudaSuccess; ++j)
    e = vec_unscale_in(L, c->n, c->n_pad, c->w, c->perm, U + (long long)j * ldu, c->V + (long long)j * c->n_pad);
  if (e != cudaSuccess) return cuda_fail(c, e, "pp_set_lowrank");
  const int rc = lowrank_build_G(c, p, false, s);
  if (rc) c->lr_p = 0;
  return rc;
}
