// Launchers of the pair kernel, D3 lattice, FP32 storage, periodic in every
// axis.
#include "lbm_pair_launch.cuh"

namespace lbm {

int n_pair_variants_d3() { return (int)(sizeof(kPair3) / sizeof(kPair3[0])); }
Variant pair_variant_d3(int k) { return Variant{kPair3[k].tx, kPair3[k].ty}; }
cudaError_t pair_box_d3(int dtype, int k, TmaBox* box) {
    if (dtype != DT_F32) return cudaErrorInvalidValue;
    return pair_by_variant<3, float>(k, nullptr, box, nullptr);
}
cudaError_t launch_step_pair_d3(int dtype, int k, const TmaArgs& ta, cudaStream_t st) {
    if (dtype != DT_F32 || ta.s.fixed_x) return cudaErrorNotSupported;
    return pair_by_variant<3, float>(k, &ta, nullptr, st);
}

}  // namespace lbm
