// Batched step kernel instantiation for __half population storage (float arithmetic).
#include <algorithm>

#include "lbm_batch.cuh"

namespace lbm {
const BatchOps* batch_ops_f16() { return make_batch_ops<float, __half, float>(); }
}  // namespace lbm
