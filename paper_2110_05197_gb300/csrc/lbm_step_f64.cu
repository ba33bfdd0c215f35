// Step kernel instantiations for double population storage (double arithmetic).
#include "lbm_launch.cuh"

namespace lbm {
cudaError_t launch_step_f64(lbm_ctx* c) { return dispatch_model<double, double, double>(c); }
}  // namespace lbm
