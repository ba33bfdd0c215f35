// Step kernel instantiations for float population storage (float arithmetic).
#include "lbm_launch.cuh"

namespace lbm {
cudaError_t launch_step_f32(lbm_ctx* c) { return dispatch_model<float, float, float>(c); }
}  // namespace lbm
