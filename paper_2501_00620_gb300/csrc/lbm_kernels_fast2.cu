// Launchers of the occupancy-oriented step kernel, D2 lattice, periodic in
// every axis (fixed-state launches are forwarded to lbm_kernels_fast2x.cu).
#include "lbm_fast_launch.cuh"

namespace lbm {

int n_fast_variants_d2() { return (int)(sizeof(kFast2) / sizeof(kFast2[0])); }
Variant fast_variant_d2(int k) { return Variant{kFast2[k].tx, kFast2[k].ty}; }
cudaError_t fast_box_d2(int dtype, int k, TmaBox* box) { return fast_by_dtype<2, false>(dtype, k, nullptr, box, nullptr); }
cudaError_t launch_step_fast_d2(int dtype, int k, const TmaArgs& ta, cudaStream_t st) {
    if (ta.s.fixed_x) return launch_step_fast_d2_fx(dtype, k, ta, st);
    return fast_by_dtype<2, false>(dtype, k, &ta, nullptr, st);
}

}  // namespace lbm
