// Launchers of the in-place two-pass step (lbm_step_aa.cuh).
#include "lbm_internal.h"
#include "lbm_step_aa.cuh"

namespace lbm {

namespace {

template <int D, typename FS>
cudaError_t aa_launch(const StepArgs& a, int form, void* aux, cudaStream_t st) {
    using real = typename Store<FS>::real;
    const unsigned blocks = (unsigned)((a.N + 255) / 256);
    aa_aux_kernel<D, FS><<<blocks, 256, 0, st>>>(a, form, static_cast<real*>(aux));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    aa_collide_kernel<D, FS><<<blocks, 256, 0, st>>>(a, form, static_cast<const real*>(aux));
    return cudaGetLastError();
}

template <int D, typename FS>
cudaError_t aa_get(const StepArgs& a, double* fo, cudaStream_t st) {
    aa_get_state_kernel<D, FS><<<(unsigned)((a.N + 255) / 256), 256, 0, st>>>(a, fo);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step_aa(int D, int dtype, const StepArgs& a, int form, void* aux, cudaStream_t st) {
    if (dtype == DT_F64) {
        if (D == 1) return aa_launch<1, double>(a, form, aux, st);
        if (D == 2) return aa_launch<2, double>(a, form, aux, st);
        if (D == 3) return aa_launch<3, double>(a, form, aux, st);
    } else if (dtype == DT_F32) {
        if (D == 1) return aa_launch<1, float>(a, form, aux, st);
        if (D == 2) return aa_launch<2, float>(a, form, aux, st);
        if (D == 3) return aa_launch<3, float>(a, form, aux, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_aa_get_state(int D, int dtype, const StepArgs& a, double* fo, cudaStream_t st) {
    if (dtype == DT_F64) {
        if (D == 1) return aa_get<1, double>(a, fo, st);
        if (D == 2) return aa_get<2, double>(a, fo, st);
        if (D == 3) return aa_get<3, double>(a, fo, st);
    } else if (dtype == DT_F32) {
        if (D == 1) return aa_get<1, float>(a, fo, st);
        if (D == 2) return aa_get<2, float>(a, fo, st);
        if (D == 3) return aa_get<3, float>(a, fo, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbm
