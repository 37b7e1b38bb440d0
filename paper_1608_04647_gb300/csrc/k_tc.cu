// Grouped persistent tensor-core (tcgen05) form of the two contractions.
#include "srm_internal.cuh"

namespace srm {

srm_status tc_setup(Ctx* c) {
  (void)c;
  set_error("the batched tensor-core form is not built yet");
  return SRM_ERR_UNSUPPORTED;
}
void tc_destroy(Ctx* c) { c->tc = nullptr; }
cudaError_t launch_p_tc(Ctx*) { return cudaErrorNotSupported; }
cudaError_t launch_a_tc(Ctx*) { return cudaErrorNotSupported; }

}  // namespace srm
