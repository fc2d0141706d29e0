// Setup kernels: the Jacobi seed W = diag(A)^{-1/2} (Section 3) and the
// construction of the seed-scaled matrix A_hat = W^T A W in SELL-C-sigma or
// CSR inside the caller's workspace, in FP64 / FP32 / BF16.
#include <cuda_bf16.h>

#include "kernels.cuh"

namespace pp {
namespace {

__global__ void jacobi_weights_kernel(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                      const double* __restrict__ val, double* __restrict__ w, int* bad_row) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p)
      if (col[p] == i) d += val[p];
    if (!(d > 0.0)) {
      atomicMin(bad_row, (int)i);
      w[i] = 1.0;
    } else {
      w[i] = 1.0 / sqrt(d);
    }
  }
}

template <typename TV>
__device__ __forceinline__ TV to_val(double v);
template <>
__device__ __forceinline__ double to_val<double>(double v) { return v; }
template <>
__device__ __forceinline__ float to_val<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_val<__nv_bfloat16>(double v) { return __double2bfloat16(v); }

// One thread per internal row (padding rows included).  Row s*C + e*32 + l
// puts entry j at slice_ptr[s] + j*C + l*VW + e (VW = C/32); padding entries
// point at the row itself (or column 0 for padding rows) with value 0.
template <typename TV>
__global__ void sell_fill_kernel(int n, long long n_pad, int C, const long long* __restrict__ sptr,
                                 const int* __restrict__ perm, const int* __restrict__ iperm,
                                 const int* __restrict__ rowptr, const int* __restrict__ col,
                                 const double* __restrict__ val, const double* __restrict__ w, int* __restrict__ out_col,
                                 TV* __restrict__ out_val) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n_pad;
       i += (long long)gridDim.x * blockDim.x) {
    const long long s = i / C;
    const int within = (int)(i - s * C);
    const int vw = C / 32;
    const int l = (within % 32) * vw + within / 32;  // position inside one entry column
    const long long base = sptr[s];
    const int wd = (int)((sptr[s + 1] - base) / C);
    int j = 0;
    if (i < n) {
      const int o = perm ? perm[i] : (int)i;
      const int beg = rowptr[o], len = rowptr[o + 1] - beg;
      const double wo = w ? w[o] : 1.0;
      for (; j < len; ++j) {
        const int c = col[beg + j];
        const double v = w ? (wo * val[beg + j]) * w[c] : val[beg + j];
        out_col[base + (long long)j * C + l] = iperm ? iperm[c] : c;
        out_val[base + (long long)j * C + l] = to_val<TV>(v);
      }
    }
    const int self = i < n ? (int)i : 0;
    for (; j < wd; ++j) {
      out_col[base + (long long)j * C + l] = self;
      out_val[base + (long long)j * C + l] = to_val<TV>(0.0);
    }
  }
}

template <typename TV>
__global__ void csr_fill_kernel(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ w, int* __restrict__ orp,
                                int* __restrict__ ocol, TV* __restrict__ oval) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += (long long)gridDim.x * blockDim.x) {
    orp[i] = rowptr[i];
    if (i == n) continue;
    const double wi = w ? w[i] : 1.0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const int c = col[p];
      ocol[p] = c;
      oval[p] = to_val<TV>(w ? (wi * val[p]) * w[c] : val[p]);
    }
  }
}

struct DiaFillArgs {
  int nd;
  int doff[kMaxDiag];
  long long dstride, dpad;
};

// One thread per row: entries with col >= row go to their diagonal.
__global__ void dia_fill_kernel(int n, const int* __restrict__ rowptr, const int* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ w, DiaFillArgs d,
                                double* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double wi = w ? w[i] : 1.0;
    for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
      const int c = col[p];
      const long long off = (long long)c - i;
      if (off < 0) continue;
      for (int t = 0; t < d.nd; ++t)
        if (d.doff[t] == off) {
          out[(long long)t * d.dstride + d.dpad + i] = w ? (wi * val[p]) * w[c] : val[p];
          break;
        }
    }
  }
}

template <typename TV>
__global__ void convert_values_kernel(long long m, const double* __restrict__ in, TV* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
    out[i] = to_val<TV>(in[i]);
}

int grid_for(long long m) {
  long long g = (m + kBlock - 1) / kBlock;
  if (g < 1) g = 1;
  if (g > 152 * 16) g = 152 * 16;
  return (int)g;
}

}  // namespace

cudaError_t csr_jacobi_weights(int n, const int* rowptr, const int* col, const double* val, double* w, int* bad_row,
                               cudaStream_t s) {
  jacobi_weights_kernel<<<grid_for(n), kBlock, 0, s>>>(n, rowptr, col, val, w, bad_row);
  return cudaGetLastError();
}

cudaError_t sell_fill(const MatDesc& d, const int* perm, const int* iperm, const int* rowptr, const int* col,
                      const double* val, const double* w, void* out_val, int out_prec, cudaStream_t s) {
  int* oc = const_cast<int*>(d.col);
  const int g = grid_for(d.n_pad);
  if (out_prec == kF64)
    sell_fill_kernel<double><<<g, kBlock, 0, s>>>(d.n, d.n_pad, d.C, d.slice_ptr, perm, iperm, rowptr, col, val, w, oc,
                                                  (double*)out_val);
  else if (out_prec == kF32)
    sell_fill_kernel<float><<<g, kBlock, 0, s>>>(d.n, d.n_pad, d.C, d.slice_ptr, perm, iperm, rowptr, col, val, w, oc,
                                                 (float*)out_val);
  else
    sell_fill_kernel<__nv_bfloat16><<<g, kBlock, 0, s>>>(d.n, d.n_pad, d.C, d.slice_ptr, perm, iperm, rowptr, col, val,
                                                         w, oc, (__nv_bfloat16*)out_val);
  return cudaGetLastError();
}

cudaError_t csr_fill(int n, const int* rowptr, const int* col, const double* val, const double* w, int* out_rowptr,
                     int* out_col, void* out_val, int out_prec, long long nnz, cudaStream_t s) {
  (void)nnz;
  const int g = grid_for((long long)n + 1);
  if (out_prec == kF64)
    csr_fill_kernel<double><<<g, kBlock, 0, s>>>(n, rowptr, col, val, w, out_rowptr, out_col, (double*)out_val);
  else if (out_prec == kF32)
    csr_fill_kernel<float><<<g, kBlock, 0, s>>>(n, rowptr, col, val, w, out_rowptr, out_col, (float*)out_val);
  else
    csr_fill_kernel<__nv_bfloat16><<<g, kBlock, 0, s>>>(n, rowptr, col, val, w, out_rowptr, out_col,
                                                        (__nv_bfloat16*)out_val);
  return cudaGetLastError();
}

cudaError_t dia_fill(const MatDesc& dst, const int* rowptr, const int* col, const double* val, const double* w,
                     cudaStream_t s) {
  DiaFillArgs d;
  d.nd = dst.ndiag;
  for (int t = 0; t < kMaxDiag; ++t) d.doff[t] = t < dst.ndiag ? dst.doff[t] : -1;
  d.dstride = dst.dstride;
  d.dpad = dst.dpad;
  dia_fill_kernel<<<grid_for(dst.n), kBlock, 0, s>>>(dst.n, rowptr, col, val, w, d, (double*)const_cast<void*>(dst.val));
  return cudaGetLastError();
}

cudaError_t sell_convert_values(long long m, const double* in, void* out, int out_prec, cudaStream_t s) {
  const int g = grid_for(m);
  if (out_prec == kF32)
    convert_values_kernel<float><<<g, kBlock, 0, s>>>(m, in, (float*)out);
  else if (out_prec == kBF16)
    convert_values_kernel<__nv_bfloat16><<<g, kBlock, 0, s>>>(m, in, (__nv_bfloat16*)out);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace pp
