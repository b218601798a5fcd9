// Generic D3 step kernel, __nv_bfloat16 storage (see lbm_gen3.cuh).
#include "lbm_gen3.cuh"

namespace lbm {
LBM_GEN3_DEFINE(__nv_bfloat16)
}  // namespace lbm
