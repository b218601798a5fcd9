// Launchers of the occupancy-oriented step kernel, D2 lattice, fixed-state
// reservoirs in x (y, z periodic).
#include "lbm_fast_launch.cuh"

namespace lbm {

cudaError_t launch_step_fast_d2_fx(int dtype, int k, const TmaArgs& ta, cudaStream_t st) {
    return fast_by_dtype<2, true>(dtype, k, &ta, nullptr, st);
}

}  // namespace lbm
