// C-ABI entry points of libpolyprec (declared in include/polyprec.h): option
// defaults, the Chebyshev coefficients, workspace layout and SELL-C-sigma
// planning, and the setup of a sparse-matrix context.
//
// Method: Bergamaschi et al., arXiv 2208.01339 -- Section 2.2 and Eq.
// thetamod / Eq. rhocheb (coefficients), Section 3 (seed preconditioner).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "driver.cuh"

using namespace pp;

namespace {
thread_local std::string g_last_error;
}

// ---------------------------------------------------------------------------
// coefficients (Section 2.2, Eq. thetamod, Eq. rhocheb)
// ---------------------------------------------------------------------------
extern "C" int polyprec_coeffs(double alpha, double beta, double xi, int k, double* theta_bar, double* delta,
                               double* sigma_bar, double* rho) {
  if (!(alpha > 0.0) || !(beta > alpha) || !(xi >= 0.0) || k < 0 || !std::isfinite(beta) || !theta_bar || !delta ||
      !sigma_bar) {
    g_last_error = "polyprec_coeffs: need 0 < alpha < beta, xi >= 0, k >= 0";
    return PP_EINVAL;
  }
  const double half_sum = 0.5 * (beta + alpha);
  const double half_width = 0.5 * (beta - alpha);
  const double tb = half_sum * (1.0 + xi);  // Eq. thetamod; the half width is kept
  const double sb = tb / half_width;
  *theta_bar = tb;
  *delta = half_width;
  *sigma_bar = sb;
  if (rho) {
    rho[0] = 1.0 / sb;
    for (int j = 1; j <= k; ++j) rho[j] = 1.0 / (2.0 * sb - rho[j - 1]);
  }
  return PP_OK;
}

extern "C" void pp_options_default(pp_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->k = 20;
  o->xi = -1.0;
  o->interval = PP_INTERVAL_LANCZOS;
  o->lanczos_steps = 10;
  o->seed = 0;
  o->seed_scaling = PP_SEED_JACOBI;
  o->format = PP_FMT_AUTO;
  o->apply_prec = PP_PREC_F64;
  o->maxit = 10000;
  o->rtol = 1e-8;
  o->zero_guess = 1;
  o->check_every = 4;
  o->use_graphs = 0;
}

extern "C" const char* pp_last_error(const pp_ctx* ctx) {
  if (ctx) return ctx->err.c_str();
  return g_last_error.c_str();
}

// ---------------------------------------------------------------------------
// shared host helpers
// ---------------------------------------------------------------------------
namespace pp {

int fail(pp_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  g_last_error = msg;
  return code;
}

int cuda_fail(pp_ctx* c, cudaError_t e, const char* where) {
  return fail(c, PP_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

double auto_xi(double a, double b) {
  // xi = O(1/kappa) (Theorem 2.2): 10/kappa clipped to [1e-6, 1e-2].
  const double xi = 10.0 * a / b;
  return std::min(std::max(xi, 1e-6), 1e-2);
}

// Extreme eigenvalues of the symmetric tridiagonal T (diagonal a, off-
// diagonal b) by the cyclic Jacobi rotation method on the dense matrix.
void tridiag_extremes_jacobi(const std::vector<double>& a, const std::vector<double>& b, double* lmin, double* lmax) {
  const int m = (int)a.size();
  std::vector<double> M((size_t)m * m, 0.0);
  auto at = [&](int i, int j) -> double& { return M[(size_t)i * m + j]; };
  for (int i = 0; i < m; ++i) at(i, i) = a[i];
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
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; ++k) {
          const double akp = at(k, p), akq = at(k, q);
          at(k, p) = c * akp - s * akq;
          at(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {
          const double apk = at(p, k), aqk = at(q, k);
          at(p, k) = c * apk - s * aqk;
          at(q, k) = s * apk + c * aqk;
        }
      }
  }
  double lo = at(0, 0), hi = at(0, 0);
  for (int i = 1; i < m; ++i) {
    lo = std::min(lo, at(i, i));
    hi = std::max(hi, at(i, i));
  }
  *lmin = lo;
  *lmax = hi;
}

int validate_options(pp_ctx* c, const pp_options* o) {
  if (!o) return fail(c, PP_EINVAL, "options is NULL");
  if (o->k < 0 || o->k > 100000) return fail(c, PP_EINVAL, "k out of range [0, 100000]");
  if (o->interval != PP_INTERVAL_LANCZOS && o->interval != PP_INTERVAL_GIVEN)
    return fail(c, PP_EINVAL, "interval must be PP_INTERVAL_LANCZOS or PP_INTERVAL_GIVEN");
  if (o->interval == PP_INTERVAL_GIVEN && !(o->alpha > 0.0 && o->beta > o->alpha))
    return fail(c, PP_EINVAL, "given interval needs 0 < alpha < beta");
  if (o->interval == PP_INTERVAL_LANCZOS && (o->lanczos_steps < 1 || o->lanczos_steps > kMaxLanczos))
    return fail(c, PP_EINVAL, "lanczos_steps must be in [1, 512]");
  if (o->apply_prec < PP_PREC_F64 || o->apply_prec > PP_PREC_BF16)
    return fail(c, PP_EUNSUPPORTED, "apply_prec not supported");
  if (o->seed_scaling != PP_SEED_NONE && o->seed_scaling != PP_SEED_JACOBI)
    return fail(c, PP_EINVAL, "seed_scaling must be PP_SEED_NONE or PP_SEED_JACOBI");
  if (o->format < PP_FMT_AUTO || o->format > PP_FMT_DIA) return fail(c, PP_EUNSUPPORTED, "format not supported");
  if (!(o->rtol >= 0.0)) return fail(c, PP_EINVAL, "rtol must be >= 0");
  if (o->check_every < 0 || o->check_every > kMaxCheck) return fail(c, PP_EINVAL, "check_every must be in [0, 64]");
  if (o->sell_sigma < 0) return fail(c, PP_EINVAL, "sell_sigma must be >= 0");
  if (o->sell_variant < 0 || o->sell_variant > 3) return fail(c, PP_EINVAL, "sell_variant must be in [0, 3]");
  if (o->lowrank < 0 || o->lowrank > kMaxLowRank) return fail(c, PP_EINVAL, "lowrank must be in [0, 32]");
  if (o->flexible < 0 || o->flexible > kMaxFcg) return fail(c, PP_EINVAL, "flexible must be in [0, 8]");
  if (o->poly != PP_POLY_CHEB && o->poly != PP_POLY_NEWTON) return fail(c, PP_EINVAL, "poly must be CHEB or NEWTON");
  if (o->poly == PP_POLY_NEWTON && (newton_levels(o->k) < 0 || o->k > 16383))
    return fail(c, PP_EINVAL, "the Newton form needs k = 2^nlev - 1 <= 16383");
  if (o->poly == PP_POLY_NEWTON && o->apply_prec != PP_PREC_F64)
    return fail(c, PP_EUNSUPPORTED, "the Newton form is applied in FP64 only");
  if (o->lowrank > 0 && o->lowrank_steps != 0 && (o->lowrank_steps < o->lowrank || o->lowrank_steps > kMaxLanczos))
    return fail(c, PP_EINVAL, "lowrank > 0 needs lowrank <= lowrank_steps <= 512 (0: 30)");
  if (o->max_blocks < 0) return fail(c, PP_EINVAL, "max_blocks must be >= 0");
  if (o->lowrank > 30 && o->lowrank_steps == 0)
    return fail(c, PP_EINVAL, "lowrank > 30 needs lowrank_steps >= lowrank");
  return PP_OK;
}

int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) dev = 0;
  return dev < kMaxDevices ? dev : kMaxDevices - 1;
}

int num_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  // 152: the SM count of GB300, used only if the attribute query fails
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 152;
  return sms;
}

}  // namespace pp

// ---------------------------------------------------------------------------
// sparse-matrix context
// ---------------------------------------------------------------------------
namespace {

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

// Rows of each window of sigma consecutive rows are stably sorted by
// decreasing length; slices of C rows are padded to their longest row.
SellPlan plan_sell(const std::vector<int>& rowptr, int n, int C, int sigma) {
  SellPlan P;
  P.C = C;
  P.sigma = (sigma <= C) ? C : ((sigma + C - 1) / C) * C;
  P.nslices = ((long long)n + C - 1) / C;
  P.n_pad = P.nslices * C;
  std::vector<int> len(n);
  for (int i = 0; i < n; ++i) len[i] = rowptr[i + 1] - rowptr[i];
  P.has_perm = P.sigma > C;
  if (P.has_perm) {
    P.perm.resize(n);
    for (int i = 0; i < n; ++i) P.perm[i] = i;
    for (long long w0 = 0; w0 < n; w0 += P.sigma) {
      const long long w1 = std::min<long long>(n, w0 + P.sigma);
      std::stable_sort(P.perm.begin() + w0, P.perm.begin() + w1, [&](int x, int y) { return len[x] > len[y]; });
    }
  }
  P.sptr.assign(P.nslices + 1, 0);
  for (long long s = 0; s < P.nslices; ++s) {
    int wmax = 0;
    const long long e = std::min<long long>(n, (s + 1) * C);
    for (long long i = s * C; i < e; ++i) wmax = std::max(wmax, len[P.has_perm ? P.perm[i] : (int)i]);
    P.sptr[s + 1] = P.sptr[s] + (long long)wmax * C;
  }
  P.nnz_pad = P.sptr[P.nslices];
  return P;
}

int choose_format(const pp_options& o, int n) {
  if (o.format == PP_FMT_CSR || o.format == PP_FMT_SELL || o.format == PP_FMT_DIA) return o.format;
  return n < 262144 ? PP_FMT_CSR : PP_FMT_SELL;
}

int choose_C(const pp_options& o) {
  return (o.sell_C == 32 || o.sell_C == 64 || o.sell_C == 128) ? o.sell_C : 64;
}

struct DiaPlan {
  int nd = 0;
  int doff[kMaxDiag] = {0};
  long long dpad = 0;
};

// Symmetric diagonal storage applies when every row has its diagonal entry,
// no entry is repeated, the entries lie on at most kMaxDiag upper offsets
// (and their mirrors) and a(j, i) == a(i, j) exactly.  Checked on the device
// (dia_plan, which also validates rowptr); synchronous.
int plan_dia(const pp_csr* A, DiaPlan& P, cudaStream_t s, pp_ctx* c) {
  DiaPlanTable t;
  cudaError_t e = dia_plan(A->n, A->nnz, A->rowptr, A->col, A->val, &t, s);
  if (e != cudaSuccess) return cuda_fail(c, e, "DIA planning");
  if (t.err != ~0ull) {
    const long long row = (long long)(t.err >> 8);
    const std::string at = " (row " + std::to_string(row) + ")";
    switch ((int)(t.err & 0xff)) {
      case kDiaBadRowptr: return fail(c, PP_EINVAL, "rowptr is not monotone or does not span [0, nnz]" + at);
      case kDiaBadCol: return fail(c, PP_EINVAL, "column index out of range" + at);
      case kDiaRepeated: return fail(c, PP_EUNSUPPORTED, "DIA: repeated entry in a row" + at);
      case kDiaNoDiagonal: return fail(c, PP_EUNSUPPORTED, "DIA: a row has no diagonal entry" + at);
      case kDiaUnsymmetric: return fail(c, PP_EUNSUPPORTED, "DIA: the matrix is not symmetric" + at);
      default: return fail(c, PP_EUNSUPPORTED, "DIA: more than 16 upper diagonals");
    }
  }
  std::vector<long long> offs{0};
  for (int h = 0; h < kDiaSlots; ++h)
    if (t.slot[h]) offs.push_back((long long)t.slot[h] - 1);
  if (t.count != (int)offs.size() - 1) return fail(c, PP_ECUDA, "DIA planning: inconsistent offset table");
  if ((int)offs.size() > kMaxDiag) return fail(c, PP_EUNSUPPORTED, "DIA: more than 16 upper diagonals");
  std::sort(offs.begin(), offs.end());
  if (offs.back() > 0x7fffffffLL) return fail(c, PP_EUNSUPPORTED, "DIA: unsupported diagonal offsets");
  P.nd = (int)offs.size();
  for (int q = 0; q < P.nd; ++q) P.doff[q] = (int)offs[q];
  P.dpad = (offs.back() + 31) / 32 * 32;
  return PP_OK;
}

int read_rowptr(const pp_csr* A, std::vector<int>& h, cudaStream_t s, pp_ctx* c) {
  h.resize((size_t)A->n + 1);
  cudaError_t e = cudaMemcpyAsync(h.data(), A->rowptr, sizeof(int) * ((size_t)A->n + 1), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "reading rowptr");
  if (h[0] != 0 || (long long)h[A->n] != A->nnz) return fail(c, PP_EINVAL, "rowptr[0] != 0 or rowptr[n] != nnz");
  for (int i = 0; i < A->n; ++i)
    if (h[i + 1] < h[i]) return fail(c, PP_EINVAL, "rowptr is not monotone");
  return PP_OK;
}

int check_csr(const pp_csr* A, pp_ctx* c) {
  if (!A) return fail(c, PP_EINVAL, "matrix is NULL");
  if (A->n <= 0) return fail(c, PP_EINVAL, "n must be positive");
  if (A->nnz < 0 || A->nnz > 2147483647LL) return fail(c, PP_EUNSUPPORTED, "nnz must fit in int32");
  if (!A->rowptr || !A->col || !A->val) return fail(c, PP_EINVAL, "matrix arrays must not be NULL");
  return PP_OK;
}

void init_desc(pp_ctx* c, const pp_csr* A, const SellPlan& P, const DiaPlan& D) {
  c->A64 = MatDesc{};
  c->A64.format = choose_format(c->opt, A->n);
  c->A64.n = A->n;
  c->A64.prec = kF64;
  if (c->A64.format == PP_FMT_DIA) {
    c->n_pad = ((long long)A->n + 127) / 128 * 128;
    // with the Jacobi seed the scaled diagonal is 1 by construction: not stored
    const int unit = c->opt.seed_scaling == PP_SEED_JACOBI ? 1 : 0;
    c->A64.dia_unit = unit;
    c->A64.ndiag = D.nd - unit;
    for (int t = 0; t < kMaxDiag; ++t) c->A64.doff[t] = t < D.nd - unit ? D.doff[t + unit] : 0;
    c->A64.dpad = D.dpad;
    c->A64.dstride = D.dpad + c->n_pad;
    // FP32/BF16 steps on the 7-point stencil: direct loads (1), TMA-staged
    // tiles (2) or plane marching (3, and auto where the grid structure
    // allows it: measured fastest)
    c->A64.tma = c->opt.sell_variant == 0 ? 3 : c->opt.sell_variant;
    c->nnz_pad = (long long)std::max(1, D.nd - unit) * c->A64.dstride;
  } else if (c->A64.format == PP_FMT_SELL) {
    c->A64.C = P.C;
    c->A64.nslices = P.nslices;
    c->A64.tma = c->opt.sell_variant != 1;
    c->n_pad = P.n_pad;
    c->nnz_pad = P.nnz_pad;
  } else {
    const double avg = (double)A->nnz / A->n;
    c->A64.csr_group = avg < 3 ? 1 : (avg < 40 ? 8 : 32);
    c->n_pad = ((long long)A->n + 127) / 128 * 128;
    c->nnz_pad = A->nnz;
  }
  c->A64.n_pad = c->n_pad;
  c->n = A->n;
  c->nnz = A->nnz;
  c->mixed = c->opt.apply_prec != PP_PREC_F64;
}

// Carve the workspace; with a null base this only sizes it.
size_t layout(pp_ctx* c, void* base, const SellPlan& P) {
  Bump B(base);
  const long long n_pad = c->n_pad;
  c->sc = B.take<Scalars>(1);
  c->partials = B.take<double>(2LL * kMaxGrid);
  c->w = B.take<double>(n_pad);
  if (c->A64.format == PP_FMT_DIA) {
    c->A64.val = B.take<double>(c->nnz_pad);
    c->perm = c->iperm = nullptr;
  } else if (c->A64.format == PP_FMT_SELL) {
    c->A64.slice_ptr = B.take<long long>(P.nslices + 1);
    c->A64.col = B.take<int>(P.nnz_pad);
    c->A64.val = B.take<double>(P.nnz_pad);
    c->perm = P.has_perm ? B.take<int>(c->n) : nullptr;
    c->iperm = P.has_perm ? B.take<int>(c->n) : nullptr;
  } else {
    c->A64.rowptr = B.take<int>((long long)c->n + 1);
    c->A64.col = B.take<int>(c->nnz);
    c->A64.val = B.take<double>(c->nnz);
    c->perm = c->iperm = nullptr;
  }
  c->mixed_val = nullptr;
  if (c->mixed)
    c->mixed_val = c->opt.apply_prec == PP_PREC_F32 ? (void*)B.take<float>(c->nnz_pad)
                                                    : (void*)B.take<__nv_bfloat16>(c->nnz_pad);
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
  return B.off + 256;
}

}  // namespace

extern "C" int pp_workspace_size(const pp_csr* A, const pp_options* opt, size_t* bytes) {
  pp_ctx tmp;
  int rc = validate_options(&tmp, opt);
  if (rc) return rc;
  if ((rc = check_csr(A, &tmp))) return rc;
  if (!bytes) return fail(nullptr, PP_EINVAL, "bytes is NULL");
  tmp.opt = *opt;
  SellPlan P;
  DiaPlan D;
  const int fmt = choose_format(*opt, A->n);
  if (fmt == PP_FMT_SELL) {
    std::vector<int> h;
    if ((rc = read_rowptr(A, h, nullptr, &tmp))) return rc;
    P = plan_sell(h, A->n, choose_C(*opt), opt->sell_sigma);
  } else if (fmt == PP_FMT_DIA && (rc = plan_dia(A, D, nullptr, &tmp))) {
    return rc;
  }
  init_desc(&tmp, A, P, D);
  *bytes = layout(&tmp, nullptr, P);
  return PP_OK;
}

extern "C" int pcg_setup(pp_ctx** out, const pp_csr* A, const pp_options* opt, void* ws, size_t ws_bytes,
                         void* stream) {
  if (!out) return fail(nullptr, PP_EINVAL, "ctx pointer is NULL");
  *out = nullptr;
  pp_ctx* c = new pp_ctx();
  auto bail = [&](int code) {
    g_last_error = c->err;
    destroy_ctx_resources(c);
    delete c;
    return code;
  };
  int rc = validate_options(c, opt);
  if (rc) return bail(rc);
  if ((rc = check_csr(A, c))) return bail(rc);
  if (!ws || ((uintptr_t)ws & 255)) return bail(fail(c, PP_EINVAL, "workspace must be non-NULL and 256-byte aligned"));
  c->opt = *opt;
  if (c->opt.check_every <= 0) c->opt.check_every = 4;
  c->kind = 0;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);

  SellPlan P;
  DiaPlan D;
  if (choose_format(*opt, A->n) == PP_FMT_DIA) {
    if ((rc = plan_dia(A, D, s, c))) return bail(rc);  // validates rowptr on the device
  } else {
    std::vector<int> h;
    if ((rc = read_rowptr(A, h, s, c))) return bail(rc);
    if (choose_format(*opt, A->n) == PP_FMT_SELL) P = plan_sell(h, A->n, choose_C(*opt), opt->sell_sigma);
  }
  init_desc(c, A, P, D);
  const size_t need = layout(c, nullptr, P);
  if (ws_bytes < need) return bail(fail(c, PP_EINVAL, "workspace too small: need " + std::to_string(need) + " bytes"));
  layout(c, ws, P);
  c->ws = ws;
  c->ws_bytes = ws_bytes;
  c->num_sms = num_sms();

  cudaError_t e = cudaMemsetAsync(c->vec_begin, 0, (char*)c->vec_end - (char*)c->vec_begin, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->sc, 0, sizeof(Scalars), s);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "clearing workspace"));
  c->grid_vec = (int)std::max(1LL, std::min<long long>(std::min(kMaxGrid, c->num_sms * 8),
                                                       (c->n_pad / 2 + kBlock - 1) / kBlock));
  VecLaunch L{c->grid_vec, c->partials, s};

  // Seed W = diag(A)^{-1/2} (Section 3), in the caller's row order, kept in t1.
  double* w_orig = nullptr;
  if (opt->seed_scaling == PP_SEED_JACOBI) {
    w_orig = c->t1;
    int* d_bad = reinterpret_cast<int*>(c->t2);
    const int big = 0x7fffffff;
    int bad = big;
    e = cudaMemcpyAsync(d_bad, &big, sizeof(int), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = csr_jacobi_weights(A->n, A->rowptr, A->col, A->val, w_orig, d_bad, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "Jacobi weights"));
    if (bad != big)
      return bail(fail(c, PP_EINVAL, "non-positive diagonal at row " + std::to_string(bad) + " (Jacobi seed)"));
  }

  if (c->A64.format == PP_FMT_DIA) {
    e = cudaMemsetAsync(const_cast<void*>(c->A64.val), 0, sizeof(double) * (size_t)c->nnz_pad, s);
    if (e == cudaSuccess) e = dia_fill(c->A64, A->rowptr, A->col, A->val, w_orig, s);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "building the DIA matrix"));
  } else if (c->A64.format == PP_FMT_SELL) {
    e = cudaMemcpyAsync((void*)c->A64.slice_ptr, P.sptr.data(), sizeof(long long) * P.sptr.size(),
                        cudaMemcpyHostToDevice, s);
    std::vector<int> ip;
    if (e == cudaSuccess && P.has_perm) {
      ip.resize(A->n);
      for (int i = 0; i < A->n; ++i) ip[P.perm[i]] = i;
      e = cudaMemcpyAsync(c->perm, P.perm.data(), sizeof(int) * A->n, cudaMemcpyHostToDevice, s);
      if (e == cudaSuccess) e = cudaMemcpyAsync(c->iperm, ip.data(), sizeof(int) * A->n, cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess)
      e = sell_fill(c->A64, c->perm, c->iperm, A->rowptr, A->col, A->val, w_orig, (void*)c->A64.val, kF64, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // host plan arrays go out of scope
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "building the SELL matrix"));
  } else {
    e = csr_fill(A->n, A->rowptr, A->col, A->val, w_orig, const_cast<int*>(c->A64.rowptr),
                 const_cast<int*>(c->A64.col), const_cast<void*>(c->A64.val), kF64, A->nnz, s);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "building the CSR matrix"));
  }
  e = gather_weights(L, c->n, c->n_pad, w_orig, c->perm, c->w);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "seed weights"));
  c->Ap = c->A64;
  if (c->mixed) {
    c->Ap.prec = opt->apply_prec == PP_PREC_F32 ? kF32 : kBF16;
    c->Ap.val = c->mixed_val;
    e = sell_convert_values(c->nnz_pad, (const double*)c->A64.val, c->mixed_val, c->Ap.prec, s);
    if (e != cudaSuccess) return bail(cuda_fail(c, e, "converting matrix values"));
  }
  {
    const int mb = step_max_blocks_per_sm(c->A64, kChebK, 0);
    const long long work = c->A64.format == PP_FMT_SELL  ? c->A64.nslices * 32
                           : c->A64.format == PP_FMT_DIA ? (long long)A->n
                                                         : (long long)A->n * c->A64.csr_group;
    const long long want = (work + kBlock - 1) / kBlock;
    c->grid_step = (int)std::max(1LL, std::min<long long>(std::min(kMaxGrid, c->num_sms * mb), want));
    // DIA kernels size their grid per variant (one resident wave); this is the cap
    if (c->A64.format == PP_FMT_DIA) c->grid_step = (int)std::max(1LL, std::min<long long>(kMaxGrid, want));
    c->grid_step_lp = c->grid_step;
    if (opt->max_blocks > 0) {
      c->grid_step = std::min(c->grid_step, opt->max_blocks);
      c->grid_step_lp = std::min(c->grid_step_lp, opt->max_blocks);
      c->grid_vec = std::min(c->grid_vec, opt->max_blocks);
    }
  }
  rc = setup_interval_and_coeffs(c, s);
  if (rc) return bail(rc);
  cudaEventRecord(e1, s);
  e = cudaEventSynchronize(e1);
  if (e != cudaSuccess) return bail(cuda_fail(c, e, "setup"));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->t_setup_ms = ms;
  *out = c;
  return PP_OK;
}

extern "C" int pp_get_info(const pp_ctx* c, pp_info* info) {
  if (!c || !info) return fail(nullptr, PP_EINVAL, "NULL argument");
  std::memset(info, 0, sizeof(*info));
  info->n = c->n;
  info->format = c->kind == 1 ? 0 : c->A64.format;
  info->sell_C = c->A64.C;
  info->sell_sigma = c->opt.sell_sigma <= c->A64.C ? c->A64.C : c->opt.sell_sigma;
  info->nnz = c->nnz;
  info->nnz_padded = c->nnz_pad;
  info->alpha_hat = c->alpha_hat;
  info->beta_hat = c->beta_hat;
  info->xi = c->xi;
  info->theta_bar = c->theta_bar;
  info->delta = c->delta;
  info->sigma_bar = c->sigma_bar;
  info->k = c->opt.k;
  info->apply_prec = c->opt.apply_prec;
  info->lanczos_steps_done = c->lanczos_steps_done;
  info->t_setup_ms = c->t_setup_ms;
  info->grid_blocks = c->grid_step;
  info->ndiag = c->A64.format == PP_FMT_DIA ? c->A64.ndiag : 0;
  info->lowrank = c->lr_p;
  info->ritz_resid = c->lr_ritz_resid;
  info->lowrank_steps_done = c->lr_steps_done;
  info->theta_min = c->lr_theta.empty() ? 0.0 : *std::min_element(c->lr_theta.begin(), c->lr_theta.end());
  info->band_max = c->band_max;
  info->band_elems = c->band_elems;
  info->t_factor_ms = c->t_band_ms;
  info->t_trace_ms = c->t_trace_ms;
  return PP_OK;
}

extern "C" int pp_destroy(pp_ctx* c) {
  if (!c) return PP_OK;
  destroy_ctx_resources(c);
  delete c;
  return PP_OK;
}
