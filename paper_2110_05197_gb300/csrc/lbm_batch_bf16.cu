// Batched step kernel instantiation for __nv_bfloat16 population storage (float arithmetic).
#include <algorithm>

#include "lbm_batch.cuh"

namespace lbm {
const BatchOps* batch_ops_bf16() { return make_batch_ops<float, __nv_bfloat16, float>(); }
}  // namespace lbm
