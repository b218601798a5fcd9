// Launchers of the TMA-staged step kernel for the D3 lattice (tile shape and
// prefetch depth per variant).
#include "lbm_internal.h"
#include "lbm_fast_launch.cuh"
#include "lbm_step_tma.cuh"

namespace lbm {

namespace {
constexpr int kD = 3;
constexpr Variant kTmaVariants[] = {{32, 8}, {32, 4}, {64, 4}, {32, 4}};
constexpr int kNV = sizeof(kTmaVariants) / sizeof(kTmaVariants[0]);

template <typename FS, int TX, int TY, int PF>
cudaError_t launch_one(const TmaArgs& ta, cudaStream_t st) {
    using Sh = TmaShape<kD, FS, TX, TY, PF>;
    auto kern = step_tma_kernel<kD, FS, TX, TY, PF>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const StepArgs& a = ta.s;
    const int np = kD == 3 ? a.nz : a.ny;
    dim3 grid(a.nx / TX, kD == 3 ? a.ny / TY : 1, (np + a.chunk - 1) / a.chunk);
    kern<<<grid, Sh::NT, Sh::SMEM, st>>>(ta);
    return cudaGetLastError();
}

template <typename FS, int TX, int TY, int PF>
void box_of(TmaBox* b) {
    using Sh = TmaShape<kD, FS, TX, TY, PF>;
    b->sxf = Sh::SXF;
    b->sxb = Sh::SXB;
    b->sy = Sh::SY;
    b->pxf = Sh::PXF;
    b->smem = Sh::SMEM;
}

template <typename FS>
cudaError_t by_variant(int v, const TmaArgs* ta, TmaBox* box, cudaStream_t st) {
    switch (v) {
        case 0: if (box) { box_of<FS, 32, 8, 1>(box); return cudaSuccess; } return launch_one<FS, 32, 8, 1>(*ta, st);
        case 1: if (box) { box_of<FS, 32, 4, 1>(box); return cudaSuccess; } return launch_one<FS, 32, 4, 1>(*ta, st);
        case 2: if (box) { box_of<FS, 64, 4, 1>(box); return cudaSuccess; } return launch_one<FS, 64, 4, 1>(*ta, st);
        case 3: if (box) { box_of<FS, 32, 4, 2>(box); return cudaSuccess; } return launch_one<FS, 32, 4, 2>(*ta, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t by_dtype(int dtype, int v, const TmaArgs* ta, TmaBox* box, cudaStream_t st) {
    switch (dtype) {
        case DT_F32: return by_variant<float>(v, ta, box, st);
        case DT_F16: return by_variant<__half>(v, ta, box, st);
        case DT_BF16: return by_variant<__nv_bfloat16>(v, ta, box, st);
        default: return cudaErrorInvalidValue;
    }
}
}  // namespace

// Indices past this file's table select the occupancy-oriented kernel
// (lbm_kernels_fast3.cu).
int n_tma_variants_d3() { return kNV + n_fast_variants_d3(); }
Variant tma_variant_d3(int v) { return v < kNV ? kTmaVariants[v] : fast_variant_d3(v - kNV); }
cudaError_t tma_box_d3(int dtype, int v, TmaBox* box) {
    return v < kNV ? by_dtype(dtype, v, nullptr, box, nullptr) : fast_box_d3(dtype, v - kNV, box);
}
cudaError_t launch_step_tma_d3(int dtype, int v, const TmaArgs& ta, cudaStream_t st) {
    return v < kNV ? by_dtype(dtype, v, &ta, nullptr, st) : launch_step_fast_d3(dtype, v - kNV, ta, st);
}

}  // namespace lbm
