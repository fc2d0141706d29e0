// polyprec_apply_csr_static: the Chebyshev apply z = p_k(A) r for callers
// that cannot allocate device memory (see include/polyprec.h).
//
// The two rotating vectors of the three-term recurrence live in the
// file-scope array below instead of a caller workspace.  Host code cannot
// use the array's name as a device address, so its address is looked up
// with cudaGetSymbolAddress once per device (on the first call made with
// that device current) and then passed to the kernels as a plain pointer.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "driver.cuh"

using namespace pp;

namespace {

constexpr long long kStaticMaxN = 262144;  // rows; 2 vectors x 2 MiB of FP64

// Shared by every call on a device and kept until the process exits.
static __device__ __align__(256) double g_static_scratch[2 * kStaticMaxN];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

int scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "polyprec_apply_csr_static: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(nullptr, PP_EUNSUPPORTED, "polyprec_apply_csr_static: device id too large");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr)
      return cuda_fail(nullptr, e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                       "polyprec_apply_csr_static: cudaGetSymbolAddress");
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return PP_OK;
}

}  // namespace

extern "C" int polyprec_apply_csr_static(int n, long long nnz, const int* rowptr, const int* col, const double* val,
                                         double alpha, double beta, double xi, int k, const double* r, double* z,
                                         void* stream) {
  if (n <= 0 || nnz < 0 || nnz > 2147483647LL || !rowptr || !col || !val || !r || !z || k < 0)
    return fail(nullptr, PP_EINVAL, "polyprec_apply_csr_static: invalid argument");
  // the recurrence reads r after step 1 has written z when k mod 3 == 1, so
  // the two must not share memory
  const uintptr_t rb = (uintptr_t)r, zb = (uintptr_t)z, bytes = (uintptr_t)n * sizeof(double);
  if (rb < zb + bytes && zb < rb + bytes)
    return fail(nullptr, PP_EINVAL, "polyprec_apply_csr_static: z must not overlap r");
  if ((long long)n > kStaticMaxN)
    return fail(nullptr, PP_EINVAL,
                "polyprec_apply_csr_static: n = " + std::to_string(n) + " exceeds the static limit of " +
                    std::to_string(kStaticMaxN) + " rows; use pcg_setup + polyprec_apply with a workspace");
  double theta_bar, delta, sigma_bar;
  std::vector<double> rho((size_t)k + 1);
  int rc = polyprec_coeffs(alpha, beta, xi, k, &theta_bar, &delta, &sigma_bar, rho.data());
  if (rc) return rc;
  double* scratch = nullptr;
  if ((rc = scratch_for_current_device(&scratch))) return rc;
  cudaStream_t s = (cudaStream_t)stream;

  MatDesc A{};
  A.format = PP_FMT_CSR;
  A.n = n;
  A.n_pad = n;
  A.rowptr = rowptr;
  A.col = col;
  A.val = val;
  A.prec = kF64;
  const double avg = (double)nnz / n;
  A.csr_group = avg < 3 ? 1 : (avg < 40 ? 8 : 32);
  const long long want = ((long long)n * A.csr_group + kBlock - 1) / kBlock;
  const int grid = (int)std::max(1LL, std::min<long long>(8LL * num_sms(), want));

  cudaError_t e = cudaSuccess;
  if (k == 0) {
    VecLaunch L{(int)std::max(1LL, std::min<long long>(8LL * num_sms(), ((long long)n + kBlock - 1) / kBlock)), nullptr, s};
    e = vec_scale_dot(L, n, nullptr, r, z, kF64, 1.0 / theta_bar, nullptr, nullptr, nullptr, nullptr, nullptr);
  } else {
    // Algorithm 2 with y_k landing in z; y_1 .. y_{k-1} rotate through the
    // two static vectors and z.
    void* buf[3] = {scratch, scratch + kStaticMaxN, z};
    const int off = ((2 - k) % 3 + 3) % 3;
    auto Y = [&](int j) { return buf[(j + off) % 3]; };
    for (int j = 1; j <= k && e == cudaSuccess; ++j) {
      StepParams p;
      p.r = r;
      p.y = Y(j);
      const StepCoeffs cf = cheb_step_coeffs(j, rho.data(), theta_bar, delta, sigma_bar);
      p.ca = cf.ca;
      p.cb = cf.cb;
      p.cc = cf.cc;
      if (j == 1) {
        p.mode = kCheb1;
        p.x = r;
      } else if (j == 2) {
        p.mode = kCheb2;
        p.x = Y(1);
      } else {
        p.mode = kChebK;
        p.x = Y(j - 1);
        p.xold = Y(j - 2);
      }
      e = launch_step(A, p, nullptr, nullptr, nullptr, grid, s);
    }
  }
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "polyprec_apply_csr_static");
  return PP_OK;
}
