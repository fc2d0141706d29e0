// Vector kernels of the solver: seed scaling in/out, the PCG updates with
// their step lengths computed on the device from device-resident inner
// products, precision conversions and the Lanczos helpers.
//
// Internal vectors are padded (to a multiple of the SELL chunk) and their
// padding is kept at zero, so the pairwise (double2) loops below may run
// over ceil(n/2) pairs.  Caller-owned vectors are touched element-wise only.
#include <cmath>

#include "kernels.cuh"

namespace pp {
namespace {

__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

template <typename TO, bool DOT>
__global__ void __launch_bounds__(kBlock) scale_in_kernel(long long n, long long n_pad, const double* __restrict__ w,
                                                          const int* __restrict__ perm, const double* __restrict__ in,
                                                          TO* __restrict__ out, double* dot_out, double* partials,
                                                          unsigned int* counter) {
  double acc[1] = {0.0};
  for (long long i = gtid(); i < n_pad; i += gstride()) {
    double v = 0.0;
    if (i < n) v = w[i] * in[perm ? perm[i] : i];
    out[i] = (TO)v;
    if (DOT) acc[0] += v * v;
  }
  if (DOT) {
    if (grid_sum<1>(acc, partials, counter) && threadIdx.x == 0) *dot_out = acc[0];
  }
}

template <typename TI>
__global__ void __launch_bounds__(kBlock) scale_out_kernel(long long n, const double* __restrict__ w,
                                                           const int* __restrict__ perm, const TI* __restrict__ in,
                                                           double* __restrict__ out, int divide) {
  for (long long i = gtid(); i < n; i += gstride()) {
    const double v = (double)in[i];
    out[perm ? perm[i] : i] = divide ? v / w[i] : w[i] * v;
  }
}

__global__ void __launch_bounds__(kBlock) unscale_in_kernel(long long n, long long n_pad, const double* __restrict__ w,
                                                            const int* __restrict__ perm, const double* __restrict__ x,
                                                            double* __restrict__ xh) {
  for (long long i = gtid(); i < n_pad; i += gstride()) xh[i] = i < n ? x[perm ? perm[i] : i] / w[i] : 0.0;
}

// x += alpha p (UPD_X) and r -= alpha q with alpha = (r,z)/(p,q); ||r||^2
// and the stopping test (rtol, maxit) are evaluated by the last block.
// Without UPD_X the x update runs in the p update of the same iteration,
// which reads p anyway, and x_pending records a stop before it ran.
template <bool UPD_X>
__global__ void __launch_bounds__(kBlock) update_xr_kernel(long long n2, Scalars* sc, double2* __restrict__ x,
                                                           double2* __restrict__ r, const double2* __restrict__ p,
                                                           const double2* __restrict__ q, double* partials) {
  if (load_done(sc)) return;
  const double pq = sc->pq, rz = sc->rz;
  const bool bad = !(pq > 0.0) || !isfinite(pq);
  double acc[1] = {0.0};
  if (!bad) {
    const double alpha = rz / pq;
    for (long long i = gtid(); i < n2; i += gstride()) {
      double2 ri = r[i], qi = __ldcs(q + i);
      if constexpr (UPD_X) {
        double2 xi = x[i], pi = p[i];
        xi.x += alpha * pi.x;
        xi.y += alpha * pi.y;
        x[i] = xi;
      }
      ri.x -= alpha * qi.x;
      ri.y -= alpha * qi.y;
      r[i] = ri;
      acc[0] += ri.x * ri.x + ri.y * ri.y;
    }
  }
  if (grid_sum<1>(acc, partials, &sc->counters[kCntUpdXR]) && threadIdx.x == 0) {
    if (bad) {
      sc->done = 1;
      sc->status = isfinite(pq) ? -2 : -3;
    } else {
      const double rr = acc[0];
      sc->rr = rr;
      sc->iter += 1;
      if (!isfinite(rr)) {
        sc->done = 1;
        sc->status = -3;
      } else if (rr <= sc->rtol2) {
        sc->done = 1;
        sc->status = 0;
        if (!UPD_X) sc->x_pending = 1;
      } else if (sc->iter >= sc->maxit) {
        sc->done = 1;
        sc->status = 1;
        if (!UPD_X) sc->x_pending = 1;
      }
    }
  }
}

// The x update the stop left pending: x += alpha p with the last alpha.
__global__ void __launch_bounds__(kBlock) finish_x_kernel(long long n2, const Scalars* sc, double2* __restrict__ x,
                                                          const double2* __restrict__ p) {
  if (!*reinterpret_cast<const volatile int*>(&sc->x_pending)) return;
  const double alpha = sc->rz / sc->pq;
  for (long long i = gtid(); i < n2; i += gstride()) {
    double2 xi = x[i];
    const double2 pi = p[i];
    xi.x += alpha * pi.x;
    xi.y += alpha * pi.y;
    x[i] = xi;
  }
}

// p = z + beta p; beta = (r,z)_new/(r,z) (plain) or -(z_new,q)/(p,q)
// (flexible, FCG(1)); first = 1 gives p = z.
template <bool UPD_X>
__global__ void __launch_bounds__(kBlock) update_p_kernel(long long n2, Scalars* sc, const double2* __restrict__ z,
                                                          double2* __restrict__ p, double2* __restrict__ x, int first) {
  if (load_done(sc)) return;
  const double rzn = sc->rz_new;
  const bool bad = !(rzn > 0.0) || !isfinite(rzn);
  double beta = 0.0;
  if (!first) beta = sc->flexible ? -sc->zq / sc->pq : rzn / sc->rz;
  // with UPD_X, the x update of this iteration (alpha = (r,z)/(p,q) with the
  // direction p before it changes)
  const double alpha = UPD_X ? sc->rz / sc->pq : 0.0;
  if (!bad) {
    for (long long i = gtid(); i < n2; i += gstride()) {
      double2 zi = __ldcs(z + i), pi = p[i];
      if constexpr (UPD_X) {
        double2 xi = x[i];
        xi.x += alpha * pi.x;
        xi.y += alpha * pi.y;
        x[i] = xi;
      }
      pi.x = zi.x + beta * pi.x;
      pi.y = zi.y + beta * pi.y;
      p[i] = pi;
    }
  }
  if (grid_last(&sc->counters[kCntUpdP]) && threadIdx.x == 0) {
    if (bad) {
      sc->done = 1;
      sc->status = isfinite(rzn) ? -2 : -3;
      // the pending x update (UPD_X) is still valid: alpha came from (p,q) > 0
      if (UPD_X) sc->x_pending = 1;
    } else {
      sc->rz = rzn;
    }
  }
}

__global__ void pcg_init_kernel(Scalars* sc, double rtol, int maxit, int flexible) {
  sc->done = 0;
  sc->x_pending = 0;
  sc->status = 1;
  sc->iter = 0;
  sc->maxit = maxit;
  sc->flexible = flexible;
  const double bb = sc->bb;
  sc->rtol2 = rtol * rtol * bb;
  if (!isfinite(bb) || !isfinite(sc->rr)) {
    sc->done = 1;
    sc->status = -3;
  } else if (bb == 0.0 || sc->rr <= sc->rtol2) {
    sc->done = 1;
    sc->status = 0;
  } else if (maxit <= 0) {
    sc->done = 1;
    sc->status = 1;
  }
}

template <int NDOT>
__global__ void __launch_bounds__(kBlock) from32_dot_kernel(long long n, const Scalars* skip, const float* __restrict__ z32,
                                                            double* __restrict__ z, const double* __restrict__ r,
                                                            const double* __restrict__ q, double* rz_out,
                                                            double* zq_out, double* partials, unsigned int* counter) {
  if (skip && load_done(skip)) return;
  double acc[NDOT > 0 ? NDOT : 1];
  for (int i = 0; i < (NDOT > 0 ? NDOT : 1); ++i) acc[i] = 0.0;
  for (long long i = gtid(); i < n; i += gstride()) {
    const double zi = (double)z32[i];
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

template <typename T, int NDOT>
__global__ void __launch_bounds__(kBlock) scale_dot_kernel(long long n, const Scalars* skip, const T* __restrict__ r,
                                                           T* __restrict__ z, double inv_theta,
                                                           const double* __restrict__ rd, const double* __restrict__ q,
                                                           double* rz_out, double* zq_out, double* partials,
                                                           unsigned int* counter) {
  if (skip && load_done(skip)) return;
  double acc[NDOT > 0 ? NDOT : 1];
  for (int i = 0; i < (NDOT > 0 ? NDOT : 1); ++i) acc[i] = 0.0;
  const T it = (T)inv_theta;
  for (long long i = gtid(); i < n; i += gstride()) {
    const T zi = r[i] * it;
    z[i] = zi;
    if (NDOT > 0) acc[0] += rd[i] * (double)zi;
    if (NDOT > 1) acc[1] += q[i] * (double)zi;
  }
  if constexpr (NDOT > 0) {
    if (grid_sum<NDOT>(acc, partials, counter) && threadIdx.x == 0) {
      *rz_out = acc[0];
      if (NDOT > 1) *zq_out = acc[1];
    }
  }
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(kBlock) convert_kernel(long long n, const TI* __restrict__ in, TO* __restrict__ out,
                                                         const Scalars* skip) {
  if (skip && load_done(skip)) return;
  for (long long i = gtid(); i < n; i += gstride()) out[i] = (TO)in[i];
}

__global__ void __launch_bounds__(kBlock) lanczos_start_kernel(long long n, long long n_pad, uint64_t key,
                                                               const int* __restrict__ perm, double* __restrict__ v,
                                                               double* nrm2_out, double* partials,
                                                               unsigned int* counter) {
  double acc[1] = {0.0};
  for (long long i = gtid(); i < n_pad; i += gstride()) {
    double x = 0.0;
    if (i < n) {
      const long long orig = perm ? perm[i] : i;
      x = 2.0 * splitmix_uniform(key, (uint64_t)orig) - 1.0;
    }
    v[i] = x;
    acc[0] += x * x;
  }
  if (grid_sum<1>(acc, partials, counter) && threadIdx.x == 0) *nrm2_out = acc[0];
}

__global__ void __launch_bounds__(kBlock) scale_by_rsqrt_kernel(long long n, double* __restrict__ v,
                                                                const double* nrm2) {
  const double s = sqrt(*nrm2);
  for (long long i = gtid(); i < n; i += gstride()) v[i] = v[i] / s;
}

__global__ void __launch_bounds__(kBlock) lanczos_orth_kernel(long long n, double* __restrict__ w,
                                                              const double* __restrict__ v, const double* a,
                                                              double* b2_out, double* partials,
                                                              unsigned int* counter) {
  const double aj = *a;
  double acc[1] = {0.0};
  for (long long i = gtid(); i < n; i += gstride()) {
    const double wi = w[i] - aj * v[i];
    w[i] = wi;
    acc[0] += wi * wi;
  }
  if (grid_sum<1>(acc, partials, counter) && threadIdx.x == 0) *b2_out = acc[0];
}

__global__ void __launch_bounds__(kBlock) dot_kernel(long long n, const double* __restrict__ x,
                                                     const double* __restrict__ y, double* out, double* partials,
                                                     unsigned int* counter) {
  double acc[1] = {0.0};
  for (long long i = gtid(); i < n; i += gstride()) acc[0] += x[i] * y[i];
  if (grid_sum<1>(acc, partials, counter) && threadIdx.x == 0) *out = acc[0];
}

__global__ void __launch_bounds__(kBlock) axpby_kernel(long long n, double a, const double* __restrict__ x, double b,
                                                       double* __restrict__ y) {
  for (long long i = gtid(); i < n; i += gstride()) y[i] = a * x[i] + b * y[i];
}

__global__ void __launch_bounds__(kBlock) gather_weights_kernel(long long n, long long n_pad,
                                                                const double* __restrict__ w_orig,
                                                                const int* __restrict__ perm, double* __restrict__ w) {
  for (long long i = gtid(); i < n_pad; i += gstride())
    w[i] = (i < n && w_orig) ? w_orig[perm ? perm[i] : i] : 1.0;
}

}  // namespace

cudaError_t gather_weights(const VecLaunch& L, long long n, long long n_pad, const double* w_orig, const int* perm,
                           double* w_int) {
  gather_weights_kernel<<<L.grid, kBlock, 0, L.s>>>(n, n_pad, w_orig, perm, w_int);
  return cudaGetLastError();
}

cudaError_t vec_scale_in(const VecLaunch& L, long long n, long long n_pad, const double* w, const int* perm,
                         const double* in, void* out, int out_prec, double* dot_out, unsigned int* counter) {
  const bool dot = dot_out != nullptr;
  if (out_prec == kF64) {
    if (dot)
      scale_in_kernel<double, true><<<L.grid, kBlock, 0, L.s>>>(n, n_pad, w, perm, in, (double*)out, dot_out,
                                                               L.partials, counter);
    else
      scale_in_kernel<double, false><<<L.grid, kBlock, 0, L.s>>>(n, n_pad, w, perm, in, (double*)out, nullptr,
                                                                L.partials, counter);
  } else {
    if (dot)
      scale_in_kernel<float, true><<<L.grid, kBlock, 0, L.s>>>(n, n_pad, w, perm, in, (float*)out, dot_out,
                                                              L.partials, counter);
    else
      scale_in_kernel<float, false><<<L.grid, kBlock, 0, L.s>>>(n, n_pad, w, perm, in, (float*)out, nullptr,
                                                               L.partials, counter);
  }
  return cudaGetLastError();
}

cudaError_t vec_scale_out(const VecLaunch& L, long long n, const double* w, const int* perm, const void* in,
                          int in_prec, double* out, int divide) {
  if (in_prec == kF64)
    scale_out_kernel<double><<<L.grid, kBlock, 0, L.s>>>(n, w, perm, (const double*)in, out, divide);
  else
    scale_out_kernel<float><<<L.grid, kBlock, 0, L.s>>>(n, w, perm, (const float*)in, out, divide);
  return cudaGetLastError();
}

cudaError_t vec_unscale_in(const VecLaunch& L, long long n, long long n_pad, const double* w, const int* perm,
                           const double* x, double* xh) {
  unscale_in_kernel<<<L.grid, kBlock, 0, L.s>>>(n, n_pad, w, perm, x, xh);
  return cudaGetLastError();
}

cudaError_t vec_update_xr(const VecLaunch& L, long long n, Scalars* sc, double* x, double* r, const double* p,
                          const double* q) {
  if (x)
    update_xr_kernel<true><<<L.grid, kBlock, 0, L.s>>>((n + 1) / 2, sc, (double2*)x, (double2*)r, (const double2*)p,
                                                       (const double2*)q, L.partials);
  else
    update_xr_kernel<false><<<L.grid, kBlock, 0, L.s>>>((n + 1) / 2, sc, nullptr, (double2*)r, (const double2*)p,
                                                        (const double2*)q, L.partials);
  return cudaGetLastError();
}

cudaError_t vec_finish_x(const VecLaunch& L, long long n, const Scalars* sc, double* x, const double* p) {
  finish_x_kernel<<<L.grid, kBlock, 0, L.s>>>((n + 1) / 2, sc, (double2*)x, (const double2*)p);
  return cudaGetLastError();
}

cudaError_t vec_update_p(const VecLaunch& L, long long n, Scalars* sc, const double* z, double* p, int first,
                         double* x) {
  if (x)
    update_p_kernel<true><<<L.grid, kBlock, 0, L.s>>>((n + 1) / 2, sc, (const double2*)z, (double2*)p, (double2*)x,
                                                      first);
  else
    update_p_kernel<false><<<L.grid, kBlock, 0, L.s>>>((n + 1) / 2, sc, (const double2*)z, (double2*)p, nullptr,
                                                       first);
  return cudaGetLastError();
}

cudaError_t pcg_init(Scalars* sc, double rtol, int maxit, int flexible, cudaStream_t s) {
  pcg_init_kernel<<<1, 1, 0, s>>>(sc, rtol, maxit, flexible);
  return cudaGetLastError();
}

cudaError_t vec_from32_dot(const VecLaunch& L, long long n, const Scalars* skip, const float* z32, double* z,
                           const double* r, const double* q, double* rz_out, double* zq_out, unsigned int* counter) {
  if (rz_out == nullptr)
    from32_dot_kernel<0><<<L.grid, kBlock, 0, L.s>>>(n, skip, z32, z, r, q, rz_out, zq_out, L.partials, counter);
  else if (q == nullptr)
    from32_dot_kernel<1><<<L.grid, kBlock, 0, L.s>>>(n, skip, z32, z, r, q, rz_out, zq_out, L.partials, counter);
  else
    from32_dot_kernel<2><<<L.grid, kBlock, 0, L.s>>>(n, skip, z32, z, r, q, rz_out, zq_out, L.partials, counter);
  return cudaGetLastError();
}

cudaError_t vec_scale_dot(const VecLaunch& L, long long n, const Scalars* skip, const void* r, void* z, int prec,
                          double inv_theta, const double* rd, const double* q, double* rz_out, double* zq_out,
                          unsigned int* counter) {
  const int nd = rz_out == nullptr ? 0 : (q == nullptr ? 1 : 2);
  if (prec == kF64) {
    const double* rr = (const double*)r;
    double* zz = (double*)z;
    if (nd == 0) scale_dot_kernel<double, 0><<<L.grid, kBlock, 0, L.s>>>(n, skip, rr, zz, inv_theta, rd, q, rz_out, zq_out, L.partials, counter);
    if (nd == 1) scale_dot_kernel<double, 1><<<L.grid, kBlock, 0, L.s>>>(n, skip, rr, zz, inv_theta, rd, q, rz_out, zq_out, L.partials, counter);
    if (nd == 2) scale_dot_kernel<double, 2><<<L.grid, kBlock, 0, L.s>>>(n, skip, rr, zz, inv_theta, rd, q, rz_out, zq_out, L.partials, counter);
  } else {
    const float* rr = (const float*)r;
    float* zz = (float*)z;
    if (nd == 0) scale_dot_kernel<float, 0><<<L.grid, kBlock, 0, L.s>>>(n, skip, rr, zz, inv_theta, rd, q, rz_out, zq_out, L.partials, counter);
    if (nd == 1) scale_dot_kernel<float, 1><<<L.grid, kBlock, 0, L.s>>>(n, skip, rr, zz, inv_theta, rd, q, rz_out, zq_out, L.partials, counter);
    if (nd == 2) scale_dot_kernel<float, 2><<<L.grid, kBlock, 0, L.s>>>(n, skip, rr, zz, inv_theta, rd, q, rz_out, zq_out, L.partials, counter);
  }
  return cudaGetLastError();
}

cudaError_t vec_convert(const VecLaunch& L, long long n, const void* in, int in_prec, void* out, int out_prec,
                        const Scalars* skip) {
  if (in_prec == kF64 && out_prec == kF32)
    convert_kernel<double, float><<<L.grid, kBlock, 0, L.s>>>(n, (const double*)in, (float*)out, skip);
  else if (in_prec == kF32 && out_prec == kF64)
    convert_kernel<float, double><<<L.grid, kBlock, 0, L.s>>>(n, (const float*)in, (double*)out, skip);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t lanczos_start(const VecLaunch& L, long long n, long long n_pad, uint64_t key, const int* perm, double* v,
                          double* nrm2_out, unsigned int* counter) {
  lanczos_start_kernel<<<L.grid, kBlock, 0, L.s>>>(n, n_pad, key, perm, v, nrm2_out, L.partials, counter);
  return cudaGetLastError();
}

cudaError_t vec_scale_by_rsqrt(const VecLaunch& L, long long n, double* v, const double* nrm2) {
  scale_by_rsqrt_kernel<<<L.grid, kBlock, 0, L.s>>>(n, v, nrm2);
  return cudaGetLastError();
}

cudaError_t lanczos_orth(const VecLaunch& L, long long n, double* w, const double* v, const double* a, double* b2_out,
                         unsigned int* counter) {
  lanczos_orth_kernel<<<L.grid, kBlock, 0, L.s>>>(n, w, v, a, b2_out, L.partials, counter);
  return cudaGetLastError();
}

cudaError_t vec_dot(const VecLaunch& L, long long n, const double* x, const double* y, double* out,
                    unsigned int* counter) {
  dot_kernel<<<L.grid, kBlock, 0, L.s>>>(n, x, y, out, L.partials, counter);
  return cudaGetLastError();
}

cudaError_t vec_axpby(const VecLaunch& L, long long n, double a, const double* x, double b, double* y) {
  axpby_kernel<<<L.grid, kBlock, 0, L.s>>>(n, a, x, b, y);
  return cudaGetLastError();
}

}  // namespace pp
