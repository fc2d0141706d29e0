// The learned part: a 3-layer MLP (8 -> 128 -> 128 -> 3, ReLU) that maps
// cheap per-instance statistics to the spectral interval multipliers and xi
// of the polynomial preconditioner.  BF16 weights and activations, FP32
// accumulation on the tensor cores (tcgen05.mma with the accumulator in
// tensor memory), FP32 master parameters updated by Adam -- forward,
// backward and the update all run in the kernels below.
//
// Computation (rounding points are part of the definition):
//   x0 = bf16(x);  h1 = relu(x0 W1^T + b1);  h2 = relu(bf16(h1) W2^T + b2)
//   y  = bf16(h2) W3^T + b3;                 L = sum (y - t)^2 / (2 B)
//   dY = (y - t)/B;  dW3 = bf16(dY)^T bf16(h2);  db3 = sum dY
//   dZ2 = (bf16(dY) W3) o [h2 > 0];  dW2 = bf16(dZ2)^T bf16(h1);  db2 = sum dZ2
//   dZ1 = (bf16(dZ2) W2) o [h1 > 0];  dW1 = bf16(dZ1)^T x0;       db1 = sum dZ1
// with W = bf16(master) in every product.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "driver.cuh"

namespace pp {
namespace {

constexpr int NIN = PP_MLP_NIN, NINP = 16, NH = PP_MLP_NHID, NOUT = PP_MLP_NOUT, NOUTP = 8;
// parameter layout (FP32 master)
constexpr int OW1 = 0, OB1 = OW1 + NH * NINP, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NOUTP * NH, NPARAM = OB3 + NOUTP;
static_assert(NPARAM == PP_MLP_NPARAM, "parameter count");

__device__ __forceinline__ unsigned short bf_bits(float f) {
  __nv_bfloat16 h = __float2bfloat16(f);
  return *reinterpret_cast<unsigned short*>(&h);
}
__device__ __forceinline__ float bf_float(unsigned short u) { return __uint_as_float(((unsigned int)u) << 16); }

// ---------------------------------------------------------------- tcgen05 --
// Strided BF16 GEMM on the 5th-generation tensor cores: C[m][n] = sum_k
// A(m,k) B(k,n) with A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn]
// (BF16, zero outside M x K / K x N), FP32 accumulation in tensor memory.
// Epilogue: + bias[n], ReLU, FP32 store (ldc), optional BF16 copy (ldcb).
//
// One CTA of 4 warps per 128 x NT tile of C (NT = N rounded up to 16, at
// most 128).  K runs in chunks of 32 through two shared-memory stages; all
// threads stage a chunk in the canonical K-major layout without swizzle
// (core matrices of 8 rows x 16 bytes: row group g, k group j at g*512 +
// j*128 bytes), then thread 0 issues two tcgen05.mma (K = 16 each) and
// commits them to the stage's mbarrier, which releases the stage two chunks
// later.  Warp 0 allocates the accumulator's TMEM columns; in the epilogue
// warp w reads rows 32w..32w+31 of the tile (TMEM lanes) with tcgen05.ld.
// Every mbarrier wait is bounded: on expiry the CTA sets *err, skips the
// rest of its work, frees its TMEM and returns.
constexpr int kTcM = 128, kTcNmax = 128, kTcKC = 32, kTcThreads = 128;
constexpr int kTcRowGroupBytes = (kTcKC / 8) * 128;  // SBO: next 8 rows
constexpr int kTcKGroupBytes = 128;                  // LBO: next 8 k
constexpr long long kTcSpin = 1LL << 22;

__device__ __forceinline__ uint32_t tc_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start, leading (K) and stride (M/N) byte
// offsets in 16-byte units, descriptor version 1 (bit 46), no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(kTcKGroupBytes >> 4) << 16) |
         ((uint64_t)(kTcRowGroupBytes >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at 24.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity) {
  for (long long it = 0; it < kTcSpin; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(tc_smem(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// bf16 element (row i, k j) of a staged chunk, in 16-bit units
__device__ __forceinline__ int tc_off(int i, int j) { return (i >> 3) * (kTcRowGroupBytes / 2) + (j >> 3) * 64 + (i & 7) * 8 + (j & 7); }

__global__ void __launch_bounds__(kTcThreads) tc_gemm_kernel(int M, int N, int K, const unsigned short* __restrict__ A,
                                                             long long sam, long long sak,
                                                             const unsigned short* __restrict__ B, long long sbk,
                                                             long long sbn, const float* __restrict__ bias, int relu,
                                                             float* __restrict__ C, int ldc,
                                                             unsigned short* __restrict__ Cb, int ldcb, int* err) {
  __shared__ __align__(1024) unsigned short sA[2][kTcM * kTcKC];
  __shared__ __align__(1024) unsigned short sB[2][kTcNmax * kTcKC];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ uint32_t s_tmem;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kTcM, n0 = blockIdx.y * kTcNmax;
  const int NT = min(kTcNmax, (N - n0 + 15) / 16 * 16);
  const uint32_t ncols = NT <= 32 ? 32u : (NT <= 64 ? 64u : 128u);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem(&s_tmem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&bar[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem(&bar[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = s_tmem;
  const uint32_t idesc = tc_idesc(kTcM, NT);
  const int nch = max(1, (K + kTcKC - 1) / kTcKC);
  bool bad = false;
  int issued = 0;  // chunks whose MMAs were committed
  for (int c = 0; c < nch && !bad; ++c) {
    const int st = c & 1, k0 = c * kTcKC;
    bool ok = true;
    if (c >= 2) ok = tc_wait(&bar[st], ((c - 2) >> 1) & 1);  // the MMAs of chunk c - 2 have read stage st
    if (__syncthreads_or(!ok)) {
      bad = true;
      break;
    }
    // stage A rows m0.., B rows (= output columns) n0.., k in [k0, k0 + 32)
    for (int e = tid; e < kTcM * kTcKC; e += kTcThreads) {
      const int i = sak == 1 ? e / kTcKC : e % kTcM, j = sak == 1 ? e % kTcKC : e / kTcM;
      const int m = m0 + i, k = k0 + j;
      sA[st][tc_off(i, j)] = (m < M && k < K) ? A[m * sam + k * sak] : (unsigned short)0;
    }
    for (int e = tid; e < NT * kTcKC; e += kTcThreads) {
      const int i = sbk == 1 ? e / kTcKC : e % NT, j = sbk == 1 ? e % kTcKC : e / NT;
      const int n = n0 + i, k = k0 + j;
      sB[st][tc_off(i, j)] = (n < N && k < K) ? B[k * sbk + n * sbn] : (unsigned short)0;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int kk = 0; kk < kTcKC / 16; ++kk) {
        const uint64_t ad = tc_desc(tc_smem(&sA[st][0]) + kk * 2 * kTcKGroupBytes);
        const uint64_t bd = tc_desc(tc_smem(&sB[st][0]) + kk * 2 * kTcKGroupBytes);
        const uint32_t acc = (c > 0 || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       tc_smem(&bar[st]))
                   : "memory");
    }
    issued = c + 1;
  }
  // the last commit covers every MMA issued before it
  if (!bad) {
    const bool ok = tc_wait(&bar[(nch - 1) & 1], ((nch - 1) >> 1) & 1);
    bad = __syncthreads_or(!ok);
  }
  if (!bad) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const int m = m0 + warp * 32 + lane;
    for (int c0 = 0; c0 < NT; c0 += 8) {
      uint32_t r[8];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
          : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (m < M) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int n = n0 + c0 + q;
          if (n >= N) continue;
          float v = __uint_as_float(r[q]);
          if (bias) v += bias[n];
          if (relu) v = v > 0.f ? v : 0.f;
          if (C) C[(long long)m * ldc + n] = v;
          if (Cb) Cb[(long long)m * ldcb + n] = bf_bits(v);
        }
      }
    }
  } else {
    if (tid == 0) atomicExch(err, 1);
    // let the MMAs still in flight finish (bounded) before their TMEM is freed
    if (issued > 0) tc_wait(&bar[(issued - 1) & 1], ((issued - 1) >> 1) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

__global__ void pack_input_kernel(int B, int Bp, const float* __restrict__ x, unsigned short* __restrict__ x0) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < Bp * NINP; e += gridDim.x * blockDim.x) {
    const int m = e / NINP, k = e % NINP;
    x0[e] = (m < B && k < NIN) ? bf_bits(x[m * NIN + k]) : 0;
  }
}

__global__ void weights_bf16_kernel(const float* __restrict__ p, unsigned short* __restrict__ w1,
                                    unsigned short* __restrict__ w2, unsigned short* __restrict__ w3) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < NH * NINP + NH * NH + NOUTP * NH;
       e += gridDim.x * blockDim.x) {
    if (e < NH * NINP)
      w1[e] = bf_bits(p[OW1 + e]);
    else if (e < NH * NINP + NH * NH)
      w2[e - NH * NINP] = bf_bits(p[OW2 + e - NH * NINP]);
    else
      w3[e - NH * NINP - NH * NH] = bf_bits(p[OW3 + e - NH * NINP - NH * NH]);
  }
}

// dY = (y - t)/B (FP32 and BF16 copies, padded), loss = sum (y-t)^2/(2B).
__global__ void loss_grad_kernel(int B, int Bp, const float* __restrict__ y, const float* __restrict__ t,
                                 float* __restrict__ dy, unsigned short* __restrict__ dyb, float* loss) {
  __shared__ float sh[256];
  float acc = 0.f;
  for (int e = threadIdx.x; e < Bp * NOUTP; e += blockDim.x) {
    const int m = e / NOUTP, n = e % NOUTP;
    float d = 0.f;
    if (m < B && n < NOUT) {
      const float r = y[m * NOUTP + n] - t[m * NOUT + n];
      acc += r * r;
      d = r / (float)B;
    }
    dy[e] = d;
    dyb[e] = bf_bits(d);
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = sh[0] / (2.0f * (float)B);
}

// dZ = dH o [H > 0] (FP32 and BF16)
__global__ void relu_back_kernel(int n, const float* __restrict__ dh, const float* __restrict__ h,
                                 float* __restrict__ dz, unsigned short* __restrict__ dzb) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const float v = h[e] > 0.f ? dh[e] : 0.f;
    dz[e] = v;
    dzb[e] = bf_bits(v);
  }
}

// db[n] = sum_m dz[m][n] over the first B rows (fixed order)
__global__ void bias_grad_kernel(int B, int N, int ld, const float* __restrict__ dz, float* __restrict__ db) {
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int m = 0; m < B; ++m) s += dz[(long long)m * ld + n];
    db[n] = s;
  }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < NPARAM; e += gridDim.x * blockDim.x) {
    const float gi = g[e];
    const float mi = b1 * m[e] + (1.f - b1) * gi;
    const float vi = b2 * v[e] + (1.f - b2) * gi * gi;
    m[e] = mi;
    v[e] = vi;
    p[e] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void copy_out_kernel(int B, const float* __restrict__ y, float* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * NOUT; e += gridDim.x * blockDim.x)
    out[e] = y[(e / NOUT) * NOUTP + e % NOUT];
}

}  // namespace
}  // namespace pp

struct pp_mlp {
  int max_batch = 0, bp = 0;
  long long step = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  unsigned short *w1 = nullptr, *w2 = nullptr, *w3 = nullptr;
  unsigned short *x0 = nullptr, *h1b = nullptr, *h2b = nullptr, *dyb = nullptr, *dz2b = nullptr, *dz1b = nullptr;
  float *h1 = nullptr, *h2 = nullptr, *y = nullptr, *dy = nullptr, *dh2 = nullptr, *dz2 = nullptr, *dh1 = nullptr,
        *dz1 = nullptr, *loss = nullptr;
  int* err = nullptr;  // set on the device when a tensor-core wait expires
};

namespace {

using namespace pp;

struct MBump {
  uintptr_t base, off = 0;
  explicit MBump(void* b) : base((uintptr_t)b) {}
  template <typename T>
  T* take(long long count) {
    off = (off + 255) & ~(uintptr_t)255;
    T* q = reinterpret_cast<T*>(base + off);
    off += (uintptr_t)(count > 0 ? count : 1) * sizeof(T);
    return q;
  }
};

size_t mlp_layout(pp_mlp* M, void* base, int max_batch) {
  MBump B(base);
  const int bp = (max_batch + 15) / 16 * 16;
  M->max_batch = max_batch;
  M->bp = bp;
  M->p = B.take<float>(NPARAM);
  M->g = B.take<float>(NPARAM);
  M->m = B.take<float>(NPARAM);
  M->v = B.take<float>(NPARAM);
  M->w1 = B.take<unsigned short>(NH * NINP);
  M->w2 = B.take<unsigned short>(NH * NH);
  M->w3 = B.take<unsigned short>(NOUTP * NH);
  M->x0 = B.take<unsigned short>((long long)bp * NINP);
  M->h1 = B.take<float>((long long)bp * NH);
  M->h1b = B.take<unsigned short>((long long)bp * NH);
  M->h2 = B.take<float>((long long)bp * NH);
  M->h2b = B.take<unsigned short>((long long)bp * NH);
  M->y = B.take<float>((long long)bp * NOUTP);
  M->dy = B.take<float>((long long)bp * NOUTP);
  M->dyb = B.take<unsigned short>((long long)bp * NOUTP);
  M->dh2 = B.take<float>((long long)bp * NH);
  M->dz2 = B.take<float>((long long)bp * NH);
  M->dz2b = B.take<unsigned short>((long long)bp * NH);
  M->dh1 = B.take<float>((long long)bp * NH);
  M->dz1 = B.take<float>((long long)bp * NH);
  M->dz1b = B.take<unsigned short>((long long)bp * NH);
  M->loss = B.take<float>(1);
  M->err = B.take<int>(1);
  return B.off + 256;
}

cudaError_t gemm(cudaStream_t s, int* err, int M, int N, int K, const unsigned short* A, long long sam,
                 long long sak, const unsigned short* B, long long sbk, long long sbn, const float* bias, int relu,
                 float* C, int ldc, unsigned short* Cb, int ldcb) {
  const dim3 grid((unsigned)((M + kTcM - 1) / kTcM), (unsigned)((N + kTcNmax - 1) / kTcNmax));
  tc_gemm_kernel<<<grid, kTcThreads, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, bias, relu, C, ldc, Cb, ldcb, err);
  return cudaGetLastError();
}

cudaError_t forward(pp_mlp* M, const float* x, int B, cudaStream_t s) {
  const int bp = (B + 15) / 16 * 16;
  weights_bf16_kernel<<<80, 256, 0, s>>>(M->p, M->w1, M->w2, M->w3);
  pack_input_kernel<<<(bp * NINP + 255) / 256, 256, 0, s>>>(B, bp, x, M->x0);
  // layer 1: [B x 16] W1^T (W1 stored [128 x 16]): B(k,n) = W1[n*16 + k]
  cudaError_t e = gemm(s, M->err, bp, NH, NINP, M->x0, NINP, 1, M->w1, 1, NINP, M->p + OB1, 1, M->h1, NH, M->h1b, NH);
  if (e == cudaSuccess) e = gemm(s, M->err, bp, NH, NH, M->h1b, NH, 1, M->w2, 1, NH, M->p + OB2, 1, M->h2, NH, M->h2b, NH);
  if (e == cudaSuccess) e = gemm(s, M->err, bp, NOUTP, NH, M->h2b, NH, 1, M->w3, 1, NH, M->p + OB3, 0, M->y, NOUTP, nullptr, 0);
  return e;
}

cudaError_t backward(pp_mlp* M, const float* t, int B, cudaStream_t s) {
  const int bp = (B + 15) / 16 * 16;
  loss_grad_kernel<<<1, 256, 0, s>>>(B, bp, M->y, t, M->dy, M->dyb, M->loss);
  // dW3 [8 x 128] = dY^T [8 x B] h2 [B x 128]: A(m=n_out, k=b) = dyb[b*8 + m], B(k=b, n) = h2b[b*128 + n]
  cudaError_t e = gemm(s, M->err, NOUTP, NH, B, M->dyb, 1, NOUTP, M->h2b, NH, 1, nullptr, 0, M->g + OW3, NH, nullptr, 0);
  bias_grad_kernel<<<1, 32, 0, s>>>(B, NOUTP, NOUTP, M->dy, M->g + OB3);
  // dH2 [B x 128] = dY [B x 8] W3 [8 x 128]: A(m, k) = dyb[m*8 + k], B(k, n) = w3[k*128 + n]
  if (e == cudaSuccess) e = gemm(s, M->err, bp, NH, NOUTP, M->dyb, NOUTP, 1, M->w3, NH, 1, nullptr, 0, M->dh2, NH, nullptr, 0);
  relu_back_kernel<<<(bp * NH + 255) / 256, 256, 0, s>>>(bp * NH, M->dh2, M->h2, M->dz2, M->dz2b);
  // dW2 [128 x 128] = dZ2^T h1
  if (e == cudaSuccess) e = gemm(s, M->err, NH, NH, B, M->dz2b, 1, NH, M->h1b, NH, 1, nullptr, 0, M->g + OW2, NH, nullptr, 0);
  bias_grad_kernel<<<4, 32, 0, s>>>(B, NH, NH, M->dz2, M->g + OB2);
  // dH1 = dZ2 W2 (W2 stored [out x in] = [n x k]): B(k=j, n=i) = w2[j*128 + i]
  if (e == cudaSuccess) e = gemm(s, M->err, bp, NH, NH, M->dz2b, NH, 1, M->w2, NH, 1, nullptr, 0, M->dh1, NH, nullptr, 0);
  relu_back_kernel<<<(bp * NH + 255) / 256, 256, 0, s>>>(bp * NH, M->dh1, M->h1, M->dz1, M->dz1b);
  // dW1 [128 x 16] = dZ1^T x0
  if (e == cudaSuccess) e = gemm(s, M->err, NH, NINP, B, M->dz1b, 1, NH, M->x0, NINP, 1, nullptr, 0, M->g + OW1, NINP, nullptr, 0);
  bias_grad_kernel<<<4, 32, 0, s>>>(B, NH, NH, M->dz1, M->g + OB1);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

// Reads the device flag of an expired tensor-core wait (synchronises the
// stream) and clears it: PP_ETIMEOUT if it was set.
int mlp_status(pp_mlp* M, cudaStream_t s, const char* where) {
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, M->err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && h) {
    e = cudaMemsetAsync(M->err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) return fail(nullptr, PP_ETIMEOUT, std::string(where) + ": a tensor-core wait expired");
  }
  if (e != cudaSuccess) return cuda_fail(nullptr, e, where);
  return PP_OK;
}

int check_batch(pp_mlp* M, int B) {
  if (!M) return fail(nullptr, PP_EINVAL, "mlp is NULL");
  if (B <= 0 || B > M->max_batch) return fail(nullptr, PP_EINVAL, "mlp batch out of range");
  return PP_OK;
}

}  // namespace

extern "C" int pp_mlp_workspace_size(int max_batch, size_t* bytes) {
  if (max_batch <= 0 || !bytes) return fail(nullptr, PP_EINVAL, "pp_mlp_workspace_size: bad argument");
  pp_mlp tmp;
  *bytes = mlp_layout(&tmp, nullptr, max_batch);
  return PP_OK;
}

extern "C" int pp_mlp_create(pp_mlp** out, int max_batch, unsigned long long seed, void* ws, size_t ws_bytes) {
  if (!out || max_batch <= 0 || !ws || ((uintptr_t)ws & 255)) return fail(nullptr, PP_EINVAL, "pp_mlp_create: bad argument");
  pp_mlp* M = new pp_mlp();
  const size_t need = mlp_layout(M, nullptr, max_batch);
  if (ws_bytes < need) {
    delete M;
    return fail(nullptr, PP_EINVAL, "pp_mlp_create: workspace too small, need " + std::to_string(need));
  }
  mlp_layout(M, ws, max_batch);
  // He-uniform weights from SplitMix64 (stream 7), zero biases and padding
  std::vector<float> p(NPARAM, 0.f);
  const uint64_t key = splitmix_key(seed, 7);
  uint64_t ctr = 0;
  auto fill = [&](int off, int rows, int cols, int used_rows, int used_cols, int fan_in) {
    const double a = std::sqrt(6.0 / fan_in);
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < cols; ++c) {
        const double u = splitmix_uniform(key, ctr++);
        if (r < used_rows && c < used_cols) p[off + r * cols + c] = (float)((2.0 * u - 1.0) * a);
      }
  };
  fill(OW1, NH, NINP, NH, NIN, NIN);
  fill(OW2, NH, NH, NH, NH, NH);
  fill(OW3, NOUTP, NH, NOUT, NH, NH);
  cudaError_t e = cudaMemcpy(M->p, p.data(), sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(M->m, 0, sizeof(float) * NPARAM);
  if (e == cudaSuccess) e = cudaMemset(M->v, 0, sizeof(float) * NPARAM);
  if (e == cudaSuccess) e = cudaMemset(M->g, 0, sizeof(float) * NPARAM);
  if (e == cudaSuccess) e = cudaMemset(M->err, 0, sizeof(int));
  if (e != cudaSuccess) {
    delete M;
    return cuda_fail(nullptr, e, "pp_mlp_create");
  }
  *out = M;
  return PP_OK;
}

extern "C" int pp_mlp_params(pp_mlp* M, float* get_host, const float* set_host) {
  if (!M) return fail(nullptr, PP_EINVAL, "mlp is NULL");
  cudaError_t e = cudaSuccess;
  if (get_host) e = cudaMemcpy(get_host, M->p, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && set_host) e = cudaMemcpy(M->p, set_host, sizeof(float) * NPARAM, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "pp_mlp_params");
  return PP_OK;
}

extern "C" int pp_mlp_forward(pp_mlp* M, const float* x, float* y, int batch, void* stream) {
  int rc = check_batch(M, batch);
  if (rc) return rc;
  if (!x || !y) return fail(nullptr, PP_EINVAL, "pp_mlp_forward: NULL vector");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = forward(M, x, batch, s);
  if (e == cudaSuccess) {
    copy_out_kernel<<<(batch * NOUT + 255) / 256, 256, 0, s>>>(batch, M->y, y);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "pp_mlp_forward");
  return mlp_status(M, s, "pp_mlp_forward");
}

extern "C" int pp_mlp_grad(pp_mlp* M, const float* x, const float* t, int batch, float* loss_host, float* grad_host,
                           void* stream) {
  int rc = check_batch(M, batch);
  if (rc) return rc;
  if (!x || !t) return fail(nullptr, PP_EINVAL, "pp_mlp_grad: NULL vector");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = forward(M, x, batch, s);
  if (e == cudaSuccess) e = backward(M, t, batch, s);
  if (e == cudaSuccess && loss_host) e = cudaMemcpyAsync(loss_host, M->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && grad_host)
    e = cudaMemcpyAsync(grad_host, M->g, sizeof(float) * NPARAM, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "pp_mlp_grad");
  return mlp_status(M, s, "pp_mlp_grad");
}

extern "C" int pp_mlp_train_step(pp_mlp* M, const float* x, const float* t, int batch, float lr, float* loss_host,
                                 void* stream) {
  int rc = check_batch(M, batch);
  if (rc) return rc;
  if (!x || !t || !(lr > 0.f)) return fail(nullptr, PP_EINVAL, "pp_mlp_train_step: bad argument");
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = forward(M, x, batch, s);
  if (e == cudaSuccess) e = backward(M, t, batch, s);
  if (e == cudaSuccess) {
    M->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)M->step), c2 = 1.f - std::pow(b2, (float)M->step);
    adam_kernel<<<80, 256, 0, s>>>(M->p, M->g, M->m, M->v, lr, b1, b2, 1e-8f, c1, c2);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && loss_host) e = cudaMemcpyAsync(loss_host, M->loss, sizeof(float), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && loss_host) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "pp_mlp_train_step");
  return loss_host ? mlp_status(M, s, "pp_mlp_train_step") : PP_OK;
}

extern "C" int pp_mlp_destroy(pp_mlp* M) {
  delete M;
  return PP_OK;
}
