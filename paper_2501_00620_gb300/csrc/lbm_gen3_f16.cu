// Generic D3 step kernel, __half storage (see lbm_gen3.cuh).
#include "lbm_gen3.cuh"

namespace lbm {
LBM_GEN3_DEFINE(__half)
}  // namespace lbm
