// Launchers of the occupancy-oriented step kernel, D3 lattice, periodic in
// every axis (fixed-state launches are forwarded to lbm_kernels_fast3x.cu).
#include "lbm_fast_launch.cuh"

namespace lbm {

int n_fast_variants_d3() { return (int)(sizeof(kFast3) / sizeof(kFast3[0])); }
Variant fast_variant_d3(int k) { return Variant{kFast3[k].tx, kFast3[k].ty}; }
cudaError_t fast_box_d3(int dtype, int k, TmaBox* box) { return fast_by_dtype<3, false>(dtype, k, nullptr, box, nullptr); }
cudaError_t launch_step_fast_d3(int dtype, int k, const TmaArgs& ta, cudaStream_t st) {
    if (ta.s.fixed_x) return launch_step_fast_d3_fx(dtype, k, ta, st);
    return fast_by_dtype<3, false>(dtype, k, &ta, nullptr, st);
}

}  // namespace lbm
