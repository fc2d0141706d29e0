// Newton-form polynomial preconditioner (Algorithm 1): with zeta_0 =
// 1/theta_bar, zeta_1 from the shifted lower end alpha' = theta_bar - delta
// of the interval, and zeta_i = 2 / (1 + 2 zeta_{i-1} - zeta_{i-1}^2)
// (Eq. zetaNewt),
//   P_0 r = zeta_0 r,   P_{j+1} r = zeta_{j+1} (2 P_j r - P_j A P_j r),
// applied by recursion: degree 2^nlev - 1 with 2^nlev - 1 products by A.
// Level j keeps two vectors (Y_j = P_{j-1} r and W_j = A Y_j) in the
// workspace; the products run through the fused step kernels (plain
// product mode), the rest are two small streaming kernels.  FP64 only.
#include <cmath>

#include "driver.cuh"

namespace pp {
namespace {

__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

// out = zeta in (pairs of rows; the padding stays zero)
__global__ void __launch_bounds__(kBlock) newton_scale_kernel(long long n2, const Scalars* skip,
                                                              const double2* __restrict__ in,
                                                              double2* __restrict__ out, double zeta) {
  if (skip && load_done(skip)) return;
  for (long long i = gtid(); i < n2; i += gstride()) {
    const double2 v = in[i];
    out[i] = make_double2(zeta * v.x, zeta * v.y);
  }
}

// out = zeta (2 y - out)
__global__ void __launch_bounds__(kBlock) newton_combine_kernel(long long n2, const Scalars* skip,
                                                                const double2* __restrict__ y,
                                                                double2* __restrict__ out, double zeta) {
  if (skip && load_done(skip)) return;
  for (long long i = gtid(); i < n2; i += gstride()) {
    const double2 a = y[i], b = out[i];
    out[i] = make_double2(zeta * (2.0 * a.x - b.x), zeta * (2.0 * a.y - b.y));
  }
}

// (r, z) -> rz_out and, with NDOT = 2, (q, z) -> zq_out
template <int NDOT>
__global__ void __launch_bounds__(kBlock) newton_dots_kernel(long long n, const Scalars* skip,
                                                             const double* __restrict__ z,
                                                             const double* __restrict__ r,
                                                             const double* __restrict__ q, double* rz_out,
                                                             double* zq_out, double* partials, unsigned int* counter) {
  if (skip && load_done(skip)) return;
  double acc[NDOT];
#pragma unroll
  for (int t = 0; t < NDOT; ++t) acc[t] = 0.0;
  for (long long i = gtid(); i < n; i += gstride()) {
    const double zi = z[i];
    acc[0] += r[i] * zi;
    if (NDOT > 1) acc[1] += q[i] * zi;
  }
  if (grid_sum<NDOT>(acc, partials, counter) && threadIdx.x == 0) {
    *rz_out = acc[0];
    if (NDOT > 1) *zq_out = acc[1];
  }
}

cudaError_t rec(pp_ctx* c, const Scalars* skip, int j, const double* in, double* out, cudaStream_t s) {
  const long long n2 = c->n_pad / 2;
  if (j == 0) {
    newton_scale_kernel<<<c->grid_vec, kBlock, 0, s>>>(n2, skip, reinterpret_cast<const double2*>(in),
                                                       reinterpret_cast<double2*>(out), c->zeta[0]);
    return cudaGetLastError();
  }
  double* Y = c->newton_buf + (long long)(2 * (j - 1)) * c->n_pad;
  double* W = Y + c->n_pad;
  cudaError_t e = rec(c, skip, j - 1, in, Y, s);  // Y = P_{j-1} r
  if (e != cudaSuccess) return e;
  StepParams p;
  p.mode = kSpmv;
  p.x = Y;
  p.y = W;
  e = op_step(c, false, p, skip, &c->sc->counters[kCntStep], s);  // W = A Y
  if (e != cudaSuccess) return e;
  e = rec(c, skip, j - 1, W, out, s);  // out = P_{j-1} A P_{j-1} r
  if (e != cudaSuccess) return e;
  newton_combine_kernel<<<c->grid_vec, kBlock, 0, s>>>(n2, skip, reinterpret_cast<const double2*>(Y),
                                                       reinterpret_cast<double2*>(out), c->zeta[j]);
  return cudaGetLastError();
}

}  // namespace

int newton_levels(int k) {
  int nlev = 0;
  while ((1 << nlev) - 1 < k && nlev < 30) ++nlev;
  return ((1 << nlev) - 1 == k) ? nlev : -1;
}

void newton_coeffs(pp_ctx* c) {
  const int nlev = newton_levels(c->opt.k);
  c->zeta.assign((size_t)nlev + 1, 0.0);
  c->zeta[0] = 1.0 / c->theta_bar;
  if (nlev >= 1) {
    const double az = (c->theta_bar - c->delta) * c->zeta[0];
    c->zeta[1] = 2.0 / (1.0 + 2.0 * az - az * az);
  }
  for (int i = 2; i <= nlev; ++i) c->zeta[i] = 2.0 / (1.0 + 2.0 * c->zeta[i - 1] - c->zeta[i - 1] * c->zeta[i - 1]);
}

long long newton_launches(const pp_ctx* c) {
  const int nlev = newton_levels(c->opt.k);
  long long k = 1;  // K(0) = 1, K(j) = 2 K(j-1) + op_launches + 1
  for (int j = 1; j <= nlev; ++j) k = 2 * k + c->op_launches + 1;
  return k;
}

cudaError_t newton_apply(pp_ctx* c, const Scalars* skip, const double* r, double* z, cudaStream_t s) {
  return rec(c, skip, newton_levels(c->opt.k), r, z, s);
}

cudaError_t newton_dots(pp_ctx* c, const Scalars* skip, const double* z, const double* r, const double* q,
                        double* rz_out, double* zq_out, cudaStream_t s) {
  unsigned int* cnt = &c->sc->counters[kCntVec];
  if (q)
    newton_dots_kernel<2><<<c->grid_vec, kBlock, 0, s>>>(c->n, skip, z, r, q, rz_out, zq_out, c->partials, cnt);
  else
    newton_dots_kernel<1><<<c->grid_vec, kBlock, 0, s>>>(c->n, skip, z, r, q, rz_out, zq_out, c->partials, cnt);
  return cudaGetLastError();
}

}  // namespace pp
