// Generic D3 step kernel, double storage (see lbm_gen3.cuh).
#include "lbm_gen3.cuh"

namespace lbm {
LBM_GEN3_DEFINE(double)
}  // namespace lbm
