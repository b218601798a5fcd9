// Launchers of the pair kernel, D2 lattice, FP32 storage, periodic in every
// axis.
#include "lbm_pair_launch.cuh"

namespace lbm {

int n_pair_variants_d2() { return (int)(sizeof(kPair2) / sizeof(kPair2[0])); }
Variant pair_variant_d2(int k) { return Variant{kPair2[k].tx, kPair2[k].ty}; }
cudaError_t pair_box_d2(int dtype, int k, TmaBox* box) {
    if (dtype != DT_F32) return cudaErrorInvalidValue;
    return pair_by_variant<2, float>(k, nullptr, box, nullptr);
}
cudaError_t launch_step_pair_d2(int dtype, int k, const TmaArgs& ta, cudaStream_t st) {
    if (dtype != DT_F32 || ta.s.fixed_x) return cudaErrorNotSupported;
    return pair_by_variant<2, float>(k, &ta, nullptr, st);
}

}  // namespace lbm
