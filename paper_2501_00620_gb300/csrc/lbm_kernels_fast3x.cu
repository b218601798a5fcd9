// Launchers of the occupancy-oriented step kernel, D3 lattice, fixed-state
// reservoirs in x (y, z periodic).
#include "lbm_fast_launch.cuh"

namespace lbm {

cudaError_t launch_step_fast_d3_fx(int dtype, int k, const TmaArgs& ta, cudaStream_t st) {
    return fast_by_dtype<3, true>(dtype, k, &ta, nullptr, st);
}

}  // namespace lbm
