// Setup kernels: the Jacobi seed W = diag(A)^{-1/2} (Section 3) and the
// construction of the seed-scaled matrix A_hat = W^T A W in SELL-C-sigma or
// CSR inside the caller's workspace, in FP64 / FP32 / BF16.
#include <cuda_bf16.h>

#include <mutex>

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

// DIA planning on the device (one thread per row): every column in range,
// no repeated entry, the diagonal present, a(j, i) == a(i, j) exactly for
// every off-diagonal entry, and the set of upper offsets j - i > 0 collected
// in an open-addressing table of kDiaSlots slots (offset + 1; 0 = empty).
// Of the errors found, the one of the smallest row (then the smallest code)
// is kept: err = row << 8 | code, reduced by atomicMin.
__device__ __forceinline__ void dia_plan_error(DiaPlanTable* t, int code, long long row) {
  atomicMin(&t->err, ((unsigned long long)row << 8) | (unsigned long long)code);
}

__global__ void dia_plan_kernel(int n, long long nnz, const int* __restrict__ rowptr, const int* __restrict__ col,
                                const double* __restrict__ val, DiaPlanTable* t) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int b = rowptr[i], e = rowptr[i + 1];
    if (e < b || (i == 0 && b != 0) || (i == n - 1 && (long long)e != nnz) || b < 0 || (long long)e > nnz) {
      dia_plan_error(t, kDiaBadRowptr, i);
      continue;
    }
    bool diag = false;
    for (int p = b; p < e; ++p) {
      const int j = col[p];
      if (j < 0 || j >= n) {
        dia_plan_error(t, kDiaBadCol, i);
        break;
      }
      for (int q = b; q < p; ++q)
        if (col[q] == j) dia_plan_error(t, kDiaRepeated, i);
      if (j == i) {
        diag = true;
        continue;
      }
      // the mirror entry a(j, i) must exist with the same value
      const int bj = rowptr[j], ej = rowptr[j + 1];
      bool mirror = false;
      if (bj >= 0 && ej >= bj && (long long)ej <= nnz)
        for (int q = bj; q < ej; ++q)
          if (col[q] == i) {
            mirror = val[q] == val[p];
            break;
          }
      if (!mirror) dia_plan_error(t, kDiaUnsymmetric, i);
      if (j < i) continue;
      const unsigned long long key = (unsigned long long)(j - i) + 1ull;
      unsigned int h = (unsigned int)((key * 0x9E3779B97F4A7C15ull) >> 58);  // 64 slots
      bool placed = false;
      for (int probe = 0; probe < kDiaSlots && !placed; ++probe, h = (h + 1) & (kDiaSlots - 1)) {
        const unsigned long long cur = *reinterpret_cast<volatile unsigned long long*>(&t->slot[h]);
        if (cur == key) {
          placed = true;
        } else if (cur == 0ull) {
          const unsigned long long old = atomicCAS(&t->slot[h], 0ull, key);
          if (old == 0ull) {
            atomicAdd(&t->count, 1);
            placed = true;
          } else if (old == key) {
            placed = true;
          }
        }
      }
      if (!placed) dia_plan_error(t, kDiaTooMany, i);
    }
    if (!diag) dia_plan_error(t, kDiaNoDiagonal, i);
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
  const long long cap = 16LL * num_sms();
  if (g > cap) g = cap;
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

namespace {
// The planning table: a few hundred bytes, so it lives in a file-scope device
// array rather than in a caller buffer (pp_workspace_size has none).  Its
// device address is looked up once per device; planning holds g_plan_mu from
// the clear to the read-back, so concurrent setups take turns.
__device__ DiaPlanTable g_dia_plan_table;
std::mutex g_plan_mu;
DiaPlanTable* g_plan_ptr[kMaxDevices] = {nullptr};
}  // namespace

cudaError_t dia_plan(int n, long long nnz, const int* rowptr, const int* col, const double* val, DiaPlanTable* out,
                     cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  const int dev = current_device();
  if (!g_plan_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_dia_plan_table);
    if (e != cudaSuccess) return e;
    g_plan_ptr[dev] = static_cast<DiaPlanTable*>(p);
  }
  DiaPlanTable* t = g_plan_ptr[dev];
  cudaError_t e = cudaMemsetAsync(t, 0, sizeof(DiaPlanTable), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(&t->err, 0xff, sizeof(t->err), s);
  if (e == cudaSuccess) {
    dia_plan_kernel<<<grid_for(n), kBlock, 0, s>>>(n, nnz, rowptr, col, val, t);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, t, sizeof(DiaPlanTable), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
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
