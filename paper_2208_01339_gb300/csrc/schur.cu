// Fracture-network Schur complement (Section 4.2): placeholder until the
// fracture solver lands.
#include "driver.cuh"

using namespace pp;

namespace pp {
struct SchurImpl {};
cudaError_t schur_scaled_step(pp_ctx*, const StepParams&, const Scalars*, unsigned int*, cudaStream_t) {
  return cudaErrorNotSupported;
}
void schur_free(SchurImpl* s) { delete s; }
}  // namespace pp

extern "C" int pp_schur_workspace_size(const pp_dfn*, const pp_options*, size_t*) {
  return fail(nullptr, PP_EUNSUPPORTED, "not built");
}
extern "C" int schur_setup(pp_ctx**, const pp_dfn*, const pp_options*, void*, size_t, void*) {
  return fail(nullptr, PP_EUNSUPPORTED, "not built");
}
extern "C" int schur_apply(pp_ctx* c, const double*, double*, void*) { return fail(c, PP_EUNSUPPORTED, "not built"); }
extern "C" int schur_diag(pp_ctx* c, double*, void*) { return fail(c, PP_EUNSUPPORTED, "not built"); }
extern "C" int schur_rhs(pp_ctx* c, const double*, double*, void*) { return fail(c, PP_EUNSUPPORTED, "not built"); }
extern "C" int schur_recover(pp_ctx* c, const double*, const double*, double*, double*, void*) {
  return fail(c, PP_EUNSUPPORTED, "not built");
}
extern "C" int schur_ainv(pp_ctx* c, const double*, double*, void*) { return fail(c, PP_EUNSUPPORTED, "not built"); }
