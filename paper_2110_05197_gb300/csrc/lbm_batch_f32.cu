// Batched step kernel instantiation for float population storage (float arithmetic).
#include <algorithm>

#include "lbm_batch.cuh"

namespace lbm {
const BatchOps* batch_ops_f32() { return make_batch_ops<float, float, float>(); }
}  // namespace lbm
