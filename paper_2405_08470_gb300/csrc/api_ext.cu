// api_ext.cu - CP-ALS, CP-loss and autotuning entry points (filled in below).
#include "engine.h"

using namespace spm;

extern "C" {

int cp_als_iter(spmttkrp_plan_t, void* const*, float*, double*) {
  return fail(SPM_ERR_UNSUPPORTED, "cp_als_iter: not built yet");
}
int cp_loss_fwd(spmttkrp_plan_t, const void* const*, float*) {
  return fail(SPM_ERR_UNSUPPORTED, "cp_loss_fwd: not built yet");
}
int cp_loss_bwd(spmttkrp_plan_t, const void* const*, const float*, float* const*) {
  return fail(SPM_ERR_UNSUPPORTED, "cp_loss_bwd: not built yet");
}
int spmttkrp_autotune(spmttkrp_plan_t, const void* const*, float* const*, int) {
  return fail(SPM_ERR_UNSUPPORTED, "spmttkrp_autotune: not built yet");
}

}  // extern "C"
