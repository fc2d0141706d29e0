// Autotuner of the storage of the fused degree step: it builds the matrix
// in every candidate layout that applies and fits in the caller's
// workspace (CSR; symmetric DIA for banded matrices, for FP32/BF16 applies
// with direct or TMA-staged loads; SELL-C-sigma with
// C = 32, 64, 128 rows per slice -- 1, 2 or 4 rows per lane -- and sort
// windows sigma = C or 1024, with direct loads or TMA-staged slices),
// times applications of p_k on it with CUDA events and reports the
// fastest.  Nothing of the method changes: every layout
// holds the same seed-scaled matrix, and the iterates agree to rounding.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "driver.cuh"

using namespace pp;

namespace {

struct Candidate {
  int format, C, sigma, variant;
};

std::vector<Candidate> candidates(int apply_prec) {
  // preference order for ties: fewest bytes per step first
  std::vector<Candidate> out;
  if (apply_prec == PP_PREC_F64) {
    out.push_back({PP_FMT_DIA, 0, 0, 0});
  } else {  // FP32/BF16 DIA steps: direct loads, TMA-staged tiles, plane marching
    out.push_back({PP_FMT_DIA, 0, 0, 1});
    out.push_back({PP_FMT_DIA, 0, 0, 2});
    out.push_back({PP_FMT_DIA, 0, 0, 3});
  }
  for (int C : {32, 64, 128})
    for (int sigma : {0, 1024})
      for (int variant : {1, 2}) out.push_back({PP_FMT_SELL, C, sigma, variant});
  out.push_back({PP_FMT_CSR, 0, 0, 0});
  return out;
}

pp_options candidate_options(const pp_options& base, const Candidate& cd) {
  pp_options o = base;
  o.format = cd.format;
  o.sell_C = cd.C;
  o.sell_sigma = cd.sigma;
  o.sell_variant = cd.variant;
  // the timing needs valid coefficients only: a fixed interval, no Lanczos
  o.interval = PP_INTERVAL_GIVEN;
  o.alpha = 1e-2;
  o.beta = 2.0;
  o.xi = 0.0;
  o.k = std::max(1, std::min(base.k, 8));
  o.lowrank = 0;
  o.lowrank_steps = 0;
  o.use_graphs = 0;
  return o;
}

}  // namespace

extern "C" int pp_autotune_workspace_size(const pp_csr* A, const pp_options* opt, size_t* bytes) {
  if (!opt || !bytes) return fail(nullptr, PP_EINVAL, "NULL argument");
  size_t most = 0;
  for (const Candidate& cd : candidates(opt->apply_prec)) {
    pp_options o = candidate_options(*opt, cd);
    size_t b = 0;
    const int rc = pp_workspace_size(A, &o, &b);
    if (rc == PP_EUNSUPPORTED) continue;  // layout not applicable to this matrix
    if (rc) return rc;
    most = std::max(most, b);
  }
  *bytes = most;
  return PP_OK;
}

extern "C" int pp_autotune(const pp_csr* A, pp_options* opt, void* ws, size_t ws_bytes, pp_tune_entry* entries,
                           int max_entries, int* count, void* stream) {
  if (!A || !opt) return fail(nullptr, PP_EINVAL, "NULL argument");
  if (!ws || ((uintptr_t)ws & 255)) return fail(nullptr, PP_EINVAL, "workspace must be non-NULL and 256-byte aligned");
  if (max_entries < 0) return fail(nullptr, PP_EINVAL, "max_entries must be >= 0");
  int rc = validate_options(nullptr, opt);
  if (rc) return rc;
  const std::vector<Candidate> cands = candidates(opt->apply_prec);
  int tried = 0, best = -1;
  double best_us = 0.0;
  std::vector<pp_tune_entry> res;
  for (const Candidate& cd : cands) {
    pp_options o = candidate_options(*opt, cd);
    pp_tune_entry e{};
    e.format = cd.format;
    e.sell_C = cd.C;
    e.sell_sigma = cd.sigma;
    e.sell_variant = cd.variant;
    e.us_per_step = 0.0;
    size_t need = 0;
    e.status = pp_workspace_size(A, &o, &need);
    if (e.status == PP_OK && need > ws_bytes) e.status = PP_EINVAL;  // does not fit: skipped
    if (e.status == PP_OK) {
      pp_ctx* c = nullptr;
      e.status = pcg_setup(&c, A, &o, ws, ws_bytes, stream);
      if (e.status == PP_OK) {
        float ms = 0.f;
        e.status = time_internal_apply(c, 5, (cudaStream_t)stream, &ms);
        if (e.status == PP_OK) {
          e.us_per_step = 1e3 * (double)ms / o.k;
          e.sell_C = c->A64.format == PP_FMT_SELL ? c->A64.C : 0;
        }
        pp_destroy(c);
      }
      if (e.status == PP_ECUDA) {
        res.push_back(e);
        if (entries)
          for (int i = 0; i < (int)res.size() && i < max_entries; ++i) entries[i] = res[i];
        if (count) *count = (int)res.size();
        return PP_ECUDA;  // the device is in an unknown state: stop
      }
    }
    if (e.status == PP_OK && (best < 0 || e.us_per_step < best_us)) {
      best = (int)res.size();
      best_us = e.us_per_step;
    }
    res.push_back(e);
    ++tried;
  }
  if (entries)
    for (int i = 0; i < (int)res.size() && i < max_entries; ++i) entries[i] = res[i];
  if (count) *count = tried;
  if (best < 0) return fail(nullptr, PP_EINVAL, "no candidate layout fits in the workspace");
  // timings within 3% of the fastest are a tie: take the first in preference
  // order, so that the choice does not flip on timing noise
  for (int i = 0; i < (int)res.size(); ++i)
    if (res[i].status == PP_OK && res[i].us_per_step <= 1.03 * best_us) {
      best = i;
      break;
    }
  opt->format = res[best].format;
  opt->sell_C = res[best].sell_C;
  opt->sell_sigma = res[best].sell_sigma;
  opt->sell_variant = res[best].sell_variant;
  return PP_OK;
}
