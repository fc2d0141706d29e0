// Truncated flexible CG, FCG(m) (Notay 2000): with a preconditioner that is
// not a fixed SPD operator (p_k applied in FP32 or BF16), each new search
// direction is made A-orthogonal to the last m directions instead of the
// last one only:
//   p_{i+1} = z - sum_j (z, A p_j)/(p_j, A p_j) p_j,  alpha = (r, p)/(p, A p).
// The directions and their products live in rings of m slots; the slot of
// iteration i is i mod m, fixed at enqueue time (the host enqueues blocks of
// a multiple of m iterations), and the number of directions in the window
// is read from the device iteration counter.
#include "driver.cuh"

namespace pp {
namespace {

__device__ __forceinline__ long long gtid() { return (long long)blockIdx.x * blockDim.x + threadIdx.x; }
__device__ __forceinline__ long long gstride() { return (long long)gridDim.x * blockDim.x; }

// part[j * gridDim.x + blockIdx.x] = this block's share of (z, Q_j), j < M.
// Pairs of rows per thread (the vectors are padded to an even length with
// zeros).
template <int M>
__global__ void __launch_bounds__(kBlock) fcg_dots_partial_kernel(long long n2, const double* __restrict__ Q,
                                                                  long long ld, const double* __restrict__ z,
                                                                  double* __restrict__ part, const Scalars* sc) {
  if (load_done(sc)) return;
  double acc[M];
#pragma unroll
  for (int j = 0; j < M; ++j) acc[j] = 0.0;
  const double2* z2 = reinterpret_cast<const double2*>(z);
  for (long long i = gtid(); i < n2; i += gstride()) {
    const double2 zi = z2[i];
#pragma unroll
    for (int j = 0; j < M; ++j) {
      const double2 qj = __ldcs(reinterpret_cast<const double2*>(Q + (long long)j * ld) + i);
      acc[j] += qj.x * zi.x + qj.y * zi.y;
    }
  }
  block_sum<M>(acc);
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < M; ++j) part[(long long)j * gridDim.x + blockIdx.x] = acc[j];
}

// fcg_zq[j] = sum of the partials in block order; fcg_pq[s_cur] = pq.  One block.
__global__ void __launch_bounds__(kBlock) fcg_dots_final_kernel(int m, int gx, const double* __restrict__ part,
                                                                Scalars* sc, int s_cur) {
  if (load_done(sc)) return;
  for (int j = 0; j < m; ++j) {
    double acc[1] = {0.0};
    for (int t = threadIdx.x; t < gx; t += blockDim.x) acc[0] += part[(long long)j * gx + t];
    block_sum<1>(acc);
    if (threadIdx.x == 0) sc->fcg_zq[j] = acc[0];
  }
  if (threadIdx.x == 0) sc->fcg_pq[s_cur] = sc->pq;
}

// P[s_new] = z + sum over the window of beta_j P[j], beta_j = -zq_j / pq_j;
// (r, P[s_new]) -> sc->rz (the numerator of the next alpha).  first = 1:
// P[s_new] = z.  Each element of the slot being replaced is read before it
// is written by the same thread, so the oldest direction may share it.
template <int M>
__global__ void __launch_bounds__(kBlock) fcg_update_p_kernel(long long n2, double* __restrict__ P, long long ld,
                                                              int s_cur, int s_new, const double* __restrict__ z,
                                                              const double* __restrict__ r, Scalars* sc,
                                                              double* partials, int first) {
  if (load_done(sc)) return;
  __shared__ double beta_s[M];
  if (threadIdx.x == 0) {
    const int it = sc->iter;
    const int nv = first ? 0 : (it < M ? it : M);
    // beta by slot; slots outside the window get 0
    for (int j = 0; j < M; ++j) beta_s[j] = 0.0;
    for (int t = 0; t < nv; ++t) {
      const int j = (s_cur - t + M) % M;
      beta_s[j] = -sc->fcg_zq[j] / sc->fcg_pq[j];
    }
  }
  __syncthreads();
  double beta[M];
#pragma unroll
  for (int j = 0; j < M; ++j) beta[j] = beta_s[j];
  double acc[1] = {0.0};
  const double2* z2 = reinterpret_cast<const double2*>(z);
  const double2* r2 = reinterpret_cast<const double2*>(r);
  double2* pn = reinterpret_cast<double2*>(P + (long long)s_new * ld);
  for (long long i = gtid(); i < n2; i += gstride()) {
    double2 v = __ldcs(z2 + i);
    if (!first) {
#pragma unroll
      for (int j = 0; j < M; ++j) {
        const double2 pj = reinterpret_cast<const double2*>(P + (long long)j * ld)[i];
        v.x += beta[j] * pj.x;
        v.y += beta[j] * pj.y;
      }
    }
    pn[i] = v;
    const double2 ri = __ldcs(r2 + i);
    acc[0] += ri.x * v.x + ri.y * v.y;
  }
  if (grid_sum<1>(acc, partials, &sc->counters[kCntUpdP]) && threadIdx.x == 0) {
    const double rp = acc[0];
    if (!isfinite(rp)) {
      sc->done = 1;
      sc->status = -3;
    } else {
      sc->rz = rp;
    }
  }
}

template <int M>
cudaError_t fcg_launch(pp_ctx* c, int what, int s_cur, int s_new, int first, cudaStream_t s) {
  const long long n2 = (c->n + 1) / 2;
  if (what == 0)
    fcg_dots_partial_kernel<M><<<c->grid_vec, kBlock, 0, s>>>(n2, c->Qring, c->n_pad, c->z, c->fcg_part, c->sc);
  else
    fcg_update_p_kernel<M><<<c->grid_vec, kBlock, 0, s>>>(n2, c->Pring, c->n_pad, s_cur, s_new, c->z, c->r, c->sc,
                                                          c->partials, first);
  return cudaGetLastError();
}

cudaError_t fcg_dispatch(pp_ctx* c, int what, int s_cur, int s_new, int first, cudaStream_t s) {
  switch (c->fcg_m) {
    case 2: return fcg_launch<2>(c, what, s_cur, s_new, first, s);
    case 3: return fcg_launch<3>(c, what, s_cur, s_new, first, s);
    case 4: return fcg_launch<4>(c, what, s_cur, s_new, first, s);
    case 5: return fcg_launch<5>(c, what, s_cur, s_new, first, s);
    case 6: return fcg_launch<6>(c, what, s_cur, s_new, first, s);
    case 7: return fcg_launch<7>(c, what, s_cur, s_new, first, s);
    case 8: return fcg_launch<8>(c, what, s_cur, s_new, first, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t fcg_dots(pp_ctx* c, int s_cur, cudaStream_t s) {
  cudaError_t e = fcg_dispatch(c, 0, s_cur, 0, 0, s);
  if (e == cudaSuccess) {
    fcg_dots_final_kernel<<<1, kBlock, 0, s>>>(c->fcg_m, c->grid_vec, c->fcg_part, c->sc, s_cur);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t fcg_update_p(pp_ctx* c, int s_cur, int s_new, int first, cudaStream_t s) {
  return fcg_dispatch(c, 1, s_cur, s_new, first, s);
}

}  // namespace pp
