// K-e: observed-entry loss and its adjoint (placeholder until the kernels land).
#include "internal.cuh"

namespace tk {
tucker_status launch_loss_grad(Ctx *c, const float *const *, const float *, double *, float *const *, float *,
                               cudaStream_t) {
  c->last_error = "tucker_loss_grad is not available in this build";
  return TUCKER_ESTATE;
}
}  // namespace tk
