// Launchers of the staged step kernel with the body-force and MRT terms in
// stage 2 (kFastExt2, kFastExt3): FP32 storage, periodic lattices.
#include "lbm_fast_launch.cuh"

namespace lbm {

cudaError_t fast_ext_box(int D, TmaBox* box) {
    if (D == 3) {
        fast_box<3, float, kFastExt3.tx, kFastExt3.ty, kFastExt3.pfb, kFastExt3.mb>(box);
        return cudaSuccess;
    }
    if (D == 2) {
        fast_box<2, float, kFastExt2.tx, kFastExt2.ty, kFastExt2.pfb, kFastExt2.mb>(box);
        return cudaSuccess;
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_step_fast_ext(int D, const TmaArgs& ta, cudaStream_t st) {
    if (ta.s.fixed_x) return cudaErrorInvalidValue;
    if (D == 3) return launch_fast<3, float, kFastExt3.tx, kFastExt3.ty, kFastExt3.pfb, kFastExt3.mb, false>(ta, st);
    if (D == 2) return launch_fast<2, float, kFastExt2.tx, kFastExt2.ty, kFastExt2.pfb, kFastExt2.mb, false>(ta, st);
    return cudaErrorInvalidValue;
}

}  // namespace lbm
