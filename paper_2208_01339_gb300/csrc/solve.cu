// Solve-time driver: the Lanczos interval estimate, the application of
// p_k by the three-term recurrence of Algorithm 2, and PCG (Section 1).
//
// The PCG scalars live on the device (Scalars); each iteration is a fixed
// sequence of kernels that read alpha/beta/the stopping state from device
// memory, so `check_every` iterations are enqueued (or replayed as one
// captured CUDA graph) between host reads of the convergence flag.  Work
// enqueued after convergence returns at once, so results do not depend on
// check_every.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "driver.cuh"

using namespace pp;

namespace pp {

cudaError_t op_step(pp_ctx* c, bool apply_matrix, const StepParams& p, const Scalars* skip, unsigned int* counter,
                    cudaStream_t s) {
  if (c->kind == 1) return schur_scaled_step(c, apply_matrix && c->mixed, p, skip, counter, s);
  StepParams q = p;
  q.err = &c->sc->dev_error;
  const bool lp = apply_matrix && c->mixed;
  return launch_step(lp ? c->Ap : c->A64, q, skip, c->partials, counter, lp ? c->grid_step_lp : c->grid_step, s);
}

namespace {

// Algorithm 2 in the apply precision: steps 2-8 with y_k written to zout.
// The three rotating buffers are chosen so that the last step lands in zout.
cudaError_t cheb_core(pp_ctx* c, const Scalars* skip, const void* rin, void* zout, int ndot, double* rz_out,
                      const double* q, double* zq_out, cudaStream_t s) {
  const int k = c->opt.k;
  void* buf[3];
  if (c->mixed) {
    buf[0] = c->u32;
    buf[1] = c->v32;
  } else {
    buf[0] = c->t1;
    buf[1] = c->t2;
  }
  buf[2] = zout;
  const int off = ((2 - k) % 3 + 3) % 3;
  auto Y = [&](int j) { return buf[(j + off) % 3]; };
  unsigned int* cnt = &c->sc->counters[kCntStep];
  const double* rho = c->rho.data();
  for (int j = 1; j <= k; ++j) {
    StepParams p;
    p.r = rin;
    p.y = Y(j);
    const StepCoeffs cf = cheb_step_coeffs(j, rho, c->theta_bar, c->delta, c->sigma_bar);
    p.ca = cf.ca;
    p.cb = cf.cb;
    p.cc = cf.cc;
    if (j == 1) {  // x = (2 rho_1/delta)(2 r - A r / theta)
      p.mode = kCheb1;
      p.x = rin;
    } else if (j == 2) {  // x_old = r / theta
      p.mode = kCheb2;
      p.x = Y(1);
    } else {
      p.mode = kChebK;
      p.x = Y(j - 1);
      p.xold = Y(j - 2);
    }
    if (j == k && ndot > 0) {
      p.ndot = ndot;
      p.dot_out0 = rz_out;
      p.aux = q;
      p.dot_out1 = zq_out;
    }
    cudaError_t e = op_step(c, true, p, skip, cnt, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// The PCG update x += alpha p runs in the p update of the same iteration
// (p = z + beta p reads p already) instead of in the r update, which saves
// one vector read per iteration; a solve that stops right after an r update
// applies the pending x update at its end.  FCG(m), m >= 2, keeps its own
// p update and the plain x update.
bool fuse_x_update(const pp_ctx* c) { return c->fcg_m == 0; }

// Records a timing event on s; while s is being captured into a graph the
// record becomes a node of the graph (an external event record), so every
// replay records it and the per-iteration step times stay measurable.
cudaError_t record_timing(cudaEvent_t ev, cudaStream_t s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &st);
  if (e != cudaSuccess) return e;
  return st == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
                                             : cudaEventRecord(ev, s);
}

// z = p_k(A_hat) r on the internal FP64 vectors r, z, with (r, z) -> rz_new
// and, for flexible CG, (q, z) -> zq.  With a low-rank correction in use
// (Section 3.1) c = G^{-1} V^T r is formed first and z += V c, fused with
// the inner products, follows the polynomial.  ev0/ev1 (may be null) are
// recorded around the k degree steps alone.
cudaError_t precond(pp_ctx* c, const Scalars* skip, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1) {
  Scalars* sc = c->sc;
  VecLaunch L{c->grid_vec, c->partials, s};
  // FCG(m), m >= 2, needs no inner product here: its own kernels form them
  const bool fcgm = c->fcg_m > 0;
  const double* q = (c->opt.flexible == 1) ? c->q : nullptr;
  const bool lr = c->lr_p > 0;
  const bool nodot = lr || fcgm;
  const int nd = nodot ? 0 : (q ? 2 : 1);
  double* rz = nodot ? nullptr : &sc->rz_new;
  const double* qd = nodot ? nullptr : q;
  cudaError_t e = lr ? lowrank_coefs(c, skip, c->r, s) : cudaSuccess;
  if (e != cudaSuccess) return e;
  if (c->opt.poly == PP_POLY_NEWTON) {
    if (ev0) e = record_timing(ev0, s);
    if (e == cudaSuccess) e = newton_apply(c, skip, c->r, c->z, s);
    if (e == cudaSuccess && ev1) e = record_timing(ev1, s);
    if (e == cudaSuccess && !nodot) e = newton_dots(c, skip, c->z, c->r, qd, rz, &sc->zq, s);
  } else if (c->opt.k == 0) {
    if (ev0) e = record_timing(ev0, s);
    if (e == cudaSuccess)
      e = vec_scale_dot(L, c->n, skip, c->r, c->z, kF64, 1.0 / c->theta_bar, c->r, qd, rz, &sc->zq,
                        &sc->counters[kCntVec]);
    if (e == cudaSuccess && ev1) e = record_timing(ev1, s);
  } else if (!c->mixed) {
    if (ev0) e = record_timing(ev0, s);
    if (e == cudaSuccess)
      e = cheb_core(c, skip, c->r, c->z, nd, rz, qd, &sc->zq, s);
    if (e == cudaSuccess && ev1) e = record_timing(ev1, s);
  } else {
    e = vec_convert(L, c->n, c->r, kF64, c->r32, kF32, skip);
    if (e == cudaSuccess && ev0) e = record_timing(ev0, s);
    if (e == cudaSuccess) e = cheb_core(c, skip, c->r32, c->z32, 0, nullptr, nullptr, nullptr, s);
    if (e == cudaSuccess && ev1) e = record_timing(ev1, s);
    if (e == cudaSuccess)
      e = vec_from32_dot(L, c->n, skip, c->z32, c->z, c->r, qd, rz, &sc->zq, &sc->counters[kCntVec]);
  }
  if (e == cudaSuccess && lr)
    e = lowrank_update(c, skip, c->z, c->r, fcgm ? nullptr : q, fcgm ? nullptr : &sc->rz_new, &sc->zq, s);
  return e;
}

}  // namespace

// y = p_k(A_hat) A_hat x (x, y FP64; q is scratch; the polynomial runs in the
// apply precision and writes through t1/t2 or the FP32 buffers).
cudaError_t prec_op_apply(pp_ctx* c, const double* x, double* y, cudaStream_t s) {
  VecLaunch L{c->grid_vec, c->partials, s};
  StepParams sp;
  sp.mode = kSpmv;
  sp.x = x;
  sp.y = c->q;
  cudaError_t e = op_step(c, false, sp, nullptr, &c->sc->counters[kCntStep], s);
  if (e != cudaSuccess) return e;
  if (c->opt.k == 0)
    return vec_scale_dot(L, c->n, nullptr, c->q, y, kF64, 1.0 / c->theta_bar, nullptr, nullptr, nullptr, nullptr,
                         nullptr);
  if (!c->mixed) return cheb_core(c, nullptr, c->q, y, 0, nullptr, nullptr, nullptr, s);
  e = vec_convert(L, c->n, c->q, kF64, c->r32, kF32, nullptr);
  if (e == cudaSuccess) e = cheb_core(c, nullptr, c->r32, c->z32, 0, nullptr, nullptr, nullptr, s);
  if (e == cudaSuccess) e = vec_from32_dot(L, c->n, nullptr, c->z32, y, nullptr, nullptr, nullptr, nullptr, nullptr);
  return e;
}

namespace {

// Kernel launches of one precond() call.
long long precond_launches(const pp_ctx* c) {
  const long long k = c->opt.k;
  long long n = k == 0 ? 1 : (c->mixed ? k * c->op_launches + 2 : k * c->op_launches);
  if (c->opt.poly == PP_POLY_NEWTON) n = newton_launches(c) + ((c->lr_p > 0 || c->fcg_m > 0) ? 0 : 1);
  if (c->lr_p > 0) n += 3;
  return n;
}

// One PCG iteration (q = A p; x, r update; z = P r; p update).  b is the
// iteration's index within its block: FCG(m) takes its ring slot b mod m.
cudaError_t pcg_iteration(pp_ctx* c, cudaStream_t s, cudaEvent_t ev0, cudaEvent_t ev1, int b) {
  Scalars* sc = c->sc;
  VecLaunch L{c->grid_vec, c->partials, s};
  const int m = c->fcg_m;
  const int s_cur = m ? b % m : 0;
  double* pv = m ? c->Pring + (long long)s_cur * c->n_pad : c->p;
  double* qv = m ? c->Qring + (long long)s_cur * c->n_pad : c->q;
  StepParams p;
  p.mode = kSpmv;
  p.ndot = 1;
  p.x = pv;
  p.y = qv;
  p.dot_out0 = &sc->pq;
  cudaError_t e = op_step(c, false, p, sc, &sc->counters[kCntStep], s);
  const bool fuse = fuse_x_update(c);
  if (e == cudaSuccess) e = vec_update_xr(L, c->n, sc, fuse ? nullptr : c->xh, c->r, pv, qv);
  if (e == cudaSuccess) e = precond(c, sc, s, ev0, ev1);
  if (m) {
    if (e == cudaSuccess) e = fcg_dots(c, s_cur, s);
    if (e == cudaSuccess) e = fcg_update_p(c, s_cur, (b + 1) % m, 0, s);
  } else if (e == cudaSuccess) {
    e = vec_update_p(L, c->n, sc, c->z, c->p, 0, fuse ? c->xh : nullptr);
  }
  return e;
}

int ensure_events(pp_ctx* c, size_t count) {
  while (c->events.size() < count) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaEventCreate");
    c->events.push_back(ev);
  }
  return PP_OK;
}

int build_graph(pp_ctx* c, int B) {
  if (c->graph_exec && c->graph_block == B) return PP_OK;
  if (c->graph_exec) {
    cudaGraphExecDestroy(c->graph_exec);
    c->graph_exec = nullptr;
  }
  cudaError_t e = cudaSuccess;
  if (!c->cap_stream) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamCreate");
  e = cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamBeginCapture");
  cudaError_t e2 = cudaSuccess;
  // the first iteration of the block records its step-time events (made
  // by ensure_events) through the graph's own nodes at every replay: one
  // sample per block keeps the event nodes off the other iterations
  for (int b = 0; b < B && e2 == cudaSuccess; ++b)
    e2 = pcg_iteration(c, c->cap_stream, b == 0 ? c->events[2] : nullptr, b == 0 ? c->events[3] : nullptr, b);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(c->cap_stream, &g);
  if (e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(c, e2, "capturing PCG iterations");
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&c->graph_exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
  c->graph_block = B;
  return PP_OK;
}

int check_vec_args(pp_ctx* c, const void* a, const void* b) {
  if (!c) return fail(nullptr, PP_EINVAL, "ctx is NULL");
  if (!a || !b) return fail(c, PP_EINVAL, "vector argument is NULL");
  return PP_OK;
}

}  // namespace

int setup_interval_and_coeffs(pp_ctx* c, cudaStream_t s) {
  double a = 0.0, b = 0.0;
  c->lr_p = 0;
  if (c->opt.interval == PP_INTERVAL_GIVEN) {
    a = c->opt.alpha;
    b = c->opt.beta;
    c->lanczos_steps_done = 0;
  } else {
    const int m = c->opt.lanczos_steps;
    Scalars* sc = c->sc;
    VecLaunch L{c->grid_vec, c->partials, s};
    double* buf[3] = {c->t1, c->t2, c->z};
    cudaError_t e = lanczos_start(L, c->n, c->n_pad, splitmix_key(c->opt.seed, 3), c->perm, buf[0], &sc->vv,
                                  &sc->counters[kCntVec]);
    if (e == cudaSuccess) e = vec_scale_by_rsqrt(L, c->n, buf[0], &sc->vv);
    int iv = 0, ivp = -1, iw = 1;
    for (int j = 0; j < m && e == cudaSuccess; ++j) {
      StepParams p;
      p.mode = kLanczos;
      p.ndot = 1;
      p.x = buf[iv];
      p.xold = ivp >= 0 ? buf[ivp] : nullptr;
      p.y = buf[iw];
      p.dev_coef = j > 0 ? &sc->lan_b2[j - 1] : nullptr;
      p.dot_out0 = &sc->lan_a[j];
      e = op_step(c, false, p, nullptr, &sc->counters[kCntStep], s);
      if (e == cudaSuccess) e = lanczos_orth(L, c->n, buf[iw], buf[iv], &sc->lan_a[j], &sc->lan_b2[j],
                                             &sc->counters[kCntLan]);
      if (e == cudaSuccess && j < m - 1) {
        e = vec_scale_by_rsqrt(L, c->n, buf[iw], &sc->lan_b2[j]);
        const int spare = ivp >= 0 ? ivp : 2;
        ivp = iv;
        iv = iw;
        iw = spare;
      }
    }
    std::vector<double> ha(m), hb2(m);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ha.data(), sc->lan_a, sizeof(double) * m, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb2.data(), sc->lan_b2, sizeof(double) * m, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "Lanczos");
    std::vector<double> ta, tb;
    for (int j = 0; j < m; ++j) {
      ta.push_back(ha[j]);
      if (j == m - 1) break;
      const double bj = std::sqrt(hb2[j]);
      if (!(bj > 1e-300)) break;  // invariant subspace
      tb.push_back(bj);
    }
    for (double v : ta)
      if (!std::isfinite(v)) return fail(c, PP_ENONFINITE, "non-finite Lanczos coefficient");
    c->lanczos_steps_done = (int)ta.size();
    tridiag_extremes_jacobi(ta, tb, &a, &b);
    if (!(a > 0.0)) return fail(c, PP_EBREAKDOWN, "Lanczos estimate of the smallest eigenvalue is not positive");
    if (!(b > a)) b = a * (1.0 + 1e-12) + 1e-300;
  }
  auto set_coeffs = [&](double lo, double hi) {
    c->alpha_hat = lo;
    c->beta_hat = hi;
    c->xi = c->opt.xi >= 0.0 ? c->opt.xi : auto_xi(lo, hi);
    c->rho.assign((size_t)c->opt.k + 2, 0.0);
    if (polyprec_coeffs(lo, hi, c->xi, c->opt.k, &c->theta_bar, &c->delta, &c->sigma_bar, c->rho.data()) != PP_OK)
      return fail(c, PP_EINVAL, "invalid spectral interval for the coefficients");
    if (c->opt.poly == PP_POLY_NEWTON) newton_coeffs(c);
    return PP_OK;
  };
  int rc = set_coeffs(a, b);
  if (rc || c->lr_cap <= 0) return rc;
  // Section 3.1: leftmost eigenvectors for the low-rank correction, found
  // with the polynomial just built.  The interval stays: the polynomial
  // keeps its lower end and the correction lifts the leftmost images.
  return lowrank_lanczos(c, s);
}

void destroy_ctx_resources(pp_ctx* c) {
  for (cudaEvent_t e : c->events) cudaEventDestroy(e);
  c->events.clear();
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  c->graph_exec = nullptr;
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  c->cap_stream = nullptr;
  if (c->schur) schur_free(c->schur);
  c->schur = nullptr;
  if (c->batch) batch_free(c->batch);
  c->batch = nullptr;
}

// Device time of one application of p_k on the internal vectors (r -> z,
// in the apply precision), averaged over `reps` after one warm-up.
int time_internal_apply(pp_ctx* c, int reps, cudaStream_t s, float* ms_per_apply) {
  VecLaunch L{c->grid_vec, c->partials, s};
  int rc = ensure_events(c, 2);
  if (rc) return rc;
  cudaError_t e = lanczos_start(L, c->n, c->n_pad, splitmix_key(c->opt.seed, 3), c->perm, c->r, &c->sc->vv,
                                &c->sc->counters[kCntVec]);
  if (e == cudaSuccess && c->mixed) e = vec_convert(L, c->n, c->r, kF64, c->r32, kF32, nullptr);
  void* rin = c->mixed ? (void*)c->r32 : (void*)c->r;
  void* zout = c->mixed ? (void*)c->z32 : (void*)c->z;
  if (e == cudaSuccess) e = cheb_core(c, nullptr, rin, zout, 0, nullptr, nullptr, nullptr, s);
  if (e == cudaSuccess) e = cudaEventRecord(c->events[0], s);
  for (int i = 0; i < reps && e == cudaSuccess; ++i) e = cheb_core(c, nullptr, rin, zout, 0, nullptr, nullptr, nullptr, s);
  if (e == cudaSuccess) e = cudaEventRecord(c->events[1], s);
  if (e == cudaSuccess) e = cudaEventSynchronize(c->events[1]);
  if (e != cudaSuccess) return cuda_fail(c, e, "timing p_k");
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->events[0], c->events[1]);
  *ms_per_apply = ms / (float)std::max(reps, 1);
  return PP_OK;
}

}  // namespace pp

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" int polyprec_apply(pp_ctx* c, const double* r, double* z, int nrhs, void* stream) {
  int rc = check_vec_args(c, r, z);
  if (rc) return rc;
  if (nrhs < 0) return fail(c, PP_EINVAL, "nrhs must be >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  VecLaunch L{c->grid_vec, c->partials, s};
  const int prec = c->mixed ? kF32 : kF64;
  void* rin = c->mixed ? (void*)c->r32 : (void*)c->r;
  void* zin = c->mixed ? (void*)c->z32 : (void*)c->z;
  for (int j = 0; j < nrhs; ++j) {
    const double* rj = r + (size_t)j * c->n;
    double* zj = z + (size_t)j * c->n;
    if (c->lr_p > 0) {  // FP64 r for V^T r, the polynomial in the apply precision, z += V c in FP64
      cudaError_t e = vec_scale_in(L, c->n, c->n_pad, c->w, c->perm, rj, c->r, kF64, nullptr, nullptr);
      if (e == cudaSuccess && c->mixed) e = vec_convert(L, c->n, c->r, kF64, c->r32, kF32, nullptr);
      if (e == cudaSuccess) e = lowrank_coefs(c, nullptr, c->r, s);
      if (e == cudaSuccess) {
        if (c->opt.poly == PP_POLY_NEWTON)
          e = newton_apply(c, nullptr, c->r, c->z, s);
        else if (c->opt.k == 0)
          e = vec_scale_dot(L, c->n, nullptr, rin, zin, prec, 1.0 / c->theta_bar, nullptr, nullptr, nullptr, nullptr,
                            nullptr);
        else
          e = cheb_core(c, nullptr, rin, zin, 0, nullptr, nullptr, nullptr, s);
      }
      if (e == cudaSuccess && c->mixed)
        e = vec_from32_dot(L, c->n, nullptr, c->z32, c->z, nullptr, nullptr, nullptr, nullptr, nullptr);
      if (e == cudaSuccess) e = lowrank_update(c, nullptr, c->z, c->r, nullptr, nullptr, nullptr, s);
      if (e == cudaSuccess) e = vec_scale_out(L, c->n, c->w, c->perm, c->z, kF64, zj, 0);
      if (e != cudaSuccess) return cuda_fail(c, e, "polyprec_apply");
      continue;
    }
    cudaError_t e = vec_scale_in(L, c->n, c->n_pad, c->w, c->perm, rj, rin, prec, nullptr, nullptr);
    if (e == cudaSuccess && c->opt.poly == PP_POLY_NEWTON) {
      e = newton_apply(c, nullptr, (const double*)rin, (double*)zin, s);
    } else if (e == cudaSuccess) {
      if (c->opt.k == 0)
        e = vec_scale_dot(L, c->n, nullptr, rin, zin, prec, 1.0 / c->theta_bar, nullptr, nullptr, nullptr, nullptr,
                          nullptr);
      else
        e = cheb_core(c, nullptr, rin, zin, 0, nullptr, nullptr, nullptr, s);
    }
    if (e == cudaSuccess) e = vec_scale_out(L, c->n, c->w, c->perm, zin, prec, zj, 0);
    if (e != cudaSuccess) return cuda_fail(c, e, "polyprec_apply");
  }
  return PP_OK;
}

extern "C" int pp_operator_apply(pp_ctx* c, const double* x, double* y, int nrhs, void* stream) {
  int rc = check_vec_args(c, x, y);
  if (rc) return rc;
  if (nrhs < 0) return fail(c, PP_EINVAL, "nrhs must be >= 0");
  if (c->kind == 1) {
    for (int j = 0; j < nrhs; ++j) {
      rc = schur_apply(c, x + (size_t)j * c->n, y + (size_t)j * c->n, stream);
      if (rc) return rc;
    }
    return PP_OK;
  }
  cudaStream_t s = (cudaStream_t)stream;
  VecLaunch L{c->grid_vec, c->partials, s};
  for (int j = 0; j < nrhs; ++j) {
    // A = W^{-1} A_hat W^{-1}
    cudaError_t e = vec_unscale_in(L, c->n, c->n_pad, c->w, c->perm, x + (size_t)j * c->n, c->t1);
    StepParams p;
    p.mode = kSpmv;
    p.x = c->t1;
    p.y = c->t2;
    if (e == cudaSuccess) e = op_step(c, false, p, nullptr, &c->sc->counters[kCntStep], s);
    if (e == cudaSuccess) e = vec_scale_out(L, c->n, c->w, c->perm, c->t2, kF64, y + (size_t)j * c->n, 1);
    if (e != cudaSuccess) return cuda_fail(c, e, "pp_operator_apply");
  }
  return PP_OK;
}

extern "C" int pcg_solve(pp_ctx* c, const double* b, double* x, pp_stats* st, void* stream) {
  int rc = check_vec_args(c, b, x);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  Scalars* sc = c->sc;
  VecLaunch L{c->grid_vec, c->partials, s};
  int B = std::max(1, std::min(c->opt.check_every, kMaxCheck));
  if (c->fcg_m) B = std::min(kMaxCheck / c->fcg_m * c->fcg_m, (B + c->fcg_m - 1) / c->fcg_m * c->fcg_m);
  const bool graphs = c->opt.use_graphs != 0;
  if ((rc = ensure_events(c, 2 + 2 * (size_t)(B + 1)))) return rc;
  cudaEvent_t ev_start = c->events[0], ev_end = c->events[1];
  auto ev_pair = [&](int i, int which) { return c->events[2 + 2 * i + which]; };
  if (graphs && (rc = build_graph(c, B))) return rc;

  cudaError_t e = cudaEventRecord(ev_start, s);
  if (c->opt.zero_guess) {
    if (e == cudaSuccess) e = vec_scale_in(L, c->n, c->n_pad, c->w, c->perm, b, c->r, kF64, &sc->bb, &sc->counters[kCntVec]);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->xh, 0, sizeof(double) * c->n_pad, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&sc->rr, &sc->bb, sizeof(double), cudaMemcpyDeviceToDevice, s);
  } else {
    if (e == cudaSuccess) e = vec_scale_in(L, c->n, c->n_pad, c->w, c->perm, b, c->bh, kF64, &sc->bb, &sc->counters[kCntVec]);
    if (e == cudaSuccess) e = vec_unscale_in(L, c->n, c->n_pad, c->w, c->perm, x, c->xh);
    StepParams p;
    p.mode = kResid;
    p.ndot = 1;
    p.x = c->xh;
    p.r = c->bh;
    p.y = c->r;
    p.dot_out0 = &sc->rr;
    if (e == cudaSuccess) e = op_step(c, false, p, nullptr, &sc->counters[kCntStep], s);
  }
  if (e == cudaSuccess) e = pcg_init(sc, c->opt.rtol, c->opt.maxit, c->opt.flexible, s);
  if (e == cudaSuccess) e = precond(c, sc, s, ev_pair(B, 0), ev_pair(B, 1));
  if (e == cudaSuccess)
    e = c->fcg_m ? fcg_update_p(c, 0, 0, 1, s) : vec_update_p(L, c->n, sc, c->z, c->p, 1);
  if (e != cudaSuccess) return cuda_fail(c, e, "pcg_solve start");

  const long long pre = precond_launches(c);
  long long launches = 1 + (c->opt.zero_guess ? 0 : 1 + c->op_launches) + 1 + pre + 1;
  int host[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // done, status, iter, maxit, flexible, lan_steps, dev_error, pad
  double t_apply = 0.0;
  long long applies = 0;
  bool first_block = true;
  int iter_before = 0;
  for (;;) {
    launches += (long long)B * (c->op_launches + 2 + pre + (c->fcg_m ? 2 : 0));
    if (graphs) {
      e = cudaGraphLaunch(c->graph_exec, s);
    } else {
      for (int bi = 0; bi < B && e == cudaSuccess; ++bi) e = pcg_iteration(c, s, ev_pair(bi, 0), ev_pair(bi, 1), bi);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(host, &sc->done, sizeof(host), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(c, e, "pcg_solve iteration");
    {  // step times of the iterations this block ran (a graph replay records its first one)
      float ms = 0.f;
      if (first_block && host[2] >= 1) {
        cudaEventElapsedTime(&ms, ev_pair(B, 0), ev_pair(B, 1));
        t_apply += ms;
        applies += 1;
      }
      int executed = host[2] - iter_before;
      int applied = executed - (host[0] ? 1 : 0);
      if (graphs) applied = applied > 0 ? 1 : 0;  // the block's sampled first iteration
      for (int bi = 0; bi < applied; ++bi) {
        cudaEventElapsedTime(&ms, ev_pair(bi, 0), ev_pair(bi, 1));
        t_apply += ms;
        applies += 1;
      }
    }
    first_block = false;
    iter_before = host[2];
    if (host[0]) break;
  }
  e = cudaSuccess;
  if (fuse_x_update(c)) {
    e = vec_finish_x(L, c->n, sc, c->xh, c->p);
    launches += 1;
  }
  if (e == cudaSuccess) e = vec_scale_out(L, c->n, c->w, c->perm, c->xh, kF64, x, 0);
  if (e == cudaSuccess) e = cudaEventRecord(ev_end, s);
  double rr = 0.0, bb = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&rr, &sc->rr, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&bb, &sc->bb, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(c, e, "pcg_solve finish");
  const int status = host[6] ? PP_ETIMEOUT : host[1];
  const int iters = host[2];
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->iterations = iters;
    st->mvp = (long long)iters * (c->opt.k + 1) + (c->opt.zero_guess ? 0 : 1);
    st->dots = (3LL + c->lr_p + c->fcg_m) * iters;
    st->rel_res = bb > 0.0 ? std::sqrt(rr / bb) : 0.0;
    st->alpha_hat = c->alpha_hat;
    st->beta_hat = c->beta_hat;
    st->xi = c->xi;
    st->theta_bar = c->theta_bar;
    st->delta = c->delta;
    st->sigma_bar = c->sigma_bar;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev_start, ev_end);
    st->t_solve_ms = ms;
    st->t_apply_ms = t_apply;
    st->apply_launches = applies * c->opt.k;
    st->kernel_launches = launches + 1;
    st->status = status;
  }
  if (status < 0) {
    const char* why = status == PP_EBREAKDOWN   ? "breakdown: (p,Ap) <= 0 or (r,z) <= 0"
                      : status == PP_ETIMEOUT ? "a bounded device wait expired (staged copy did not arrive)"
                                              : "non-finite value in PCG";
    fail(c, status, why);
  }
  return status;
}
