// Step kernel instantiations for __half population storage (float arithmetic).
#include "lbm_launch.cuh"

namespace lbm {
cudaError_t launch_step_f16(lbm_ctx* c) { return dispatch_model<float, __half, float>(c); }
}  // namespace lbm
