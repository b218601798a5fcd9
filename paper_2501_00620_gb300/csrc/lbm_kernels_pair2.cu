// Launchers of the pair kernel, D2 lattice, FP32 or 16-bit (shifted)
// population storage, periodic in every axis.
#include "lbm_pair_launch.cuh"

namespace lbm {

int n_pair_variants_d2() { return (int)(sizeof(kPair2) / sizeof(kPair2[0])); }
Variant pair_variant_d2(int k) { return Variant{kPair2[k].tx, kPair2[k].ty}; }
cudaError_t pair_box_d2(int dtype, int k, TmaBox* box) {
    switch (dtype) {
        case DT_F32: return pair_by_variant<2, float>(k, nullptr, box, nullptr);
        case DT_F16: return pair_by_variant<2, __half>(k, nullptr, box, nullptr);
        case DT_BF16: return pair_by_variant<2, __nv_bfloat16>(k, nullptr, box, nullptr);
        default: return cudaErrorInvalidValue;
    }
}
cudaError_t launch_step_pair_d2(int dtype, int k, const TmaArgs& ta, cudaStream_t st) {
    if (ta.s.fixed_x) return cudaErrorNotSupported;
    switch (dtype) {
        case DT_F32: return pair_by_variant<2, float>(k, &ta, nullptr, st);
        case DT_F16: return pair_by_variant<2, __half>(k, &ta, nullptr, st);
        case DT_BF16: return pair_by_variant<2, __nv_bfloat16>(k, &ta, nullptr, st);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace lbm
