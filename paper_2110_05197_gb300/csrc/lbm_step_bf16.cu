// Step kernel instantiations for __nv_bfloat16 population storage (float arithmetic).
#include "lbm_launch.cuh"

namespace lbm {
cudaError_t launch_step_bf16(lbm_ctx* c) { return dispatch_model<float, __nv_bfloat16, float>(c); }
}  // namespace lbm
