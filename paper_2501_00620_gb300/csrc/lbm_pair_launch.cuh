// Launch helpers of the pair kernel (lbm_step_pair.cuh): the tile table per
// lattice and one launcher per (storage, tile).
#pragma once

#include "lbm_internal.h"
#include "lbm_step_pair.cuh"

namespace lbm {

// Tile TX x TY (sites) and resident blocks per SM the launch bounds aim at.
// PF: one more variance plane in flight.
struct PairVariant {
    int tx, ty, mb, pf;
};

// D3Q19: 64 x 4 sites (32 pairs per row, one warp each) at two blocks per SM;
// 64 x 8 at one block per SM (more registers per thread, a smaller ring);
// 64 x 8 warp-specialized (mb = 0), one block per SM.
constexpr PairVariant kPair3[] = {{64, 4, 2, 0}, {64, 8, 1, 1}, {64, 8, 0, 1}};
// D2Q9: strips of 128 sites (64 pairs) at four, six and eight blocks per SM
// (the register budget per thread falls as the blocks per SM grow).
constexpr PairVariant kPair2[] = {{128, 1, 4, 1}, {128, 1, 6, 1}, {128, 1, 8, 1}};

// MB = 0 selects the warp-specialized form (one block per SM).
template <int D, typename FS, int TX, int TY, int MB, int PF>
cudaError_t launch_pair(const TmaArgs& ta, cudaStream_t st) {
    using Sh = PairShape<D, FS, TX, TY, MB == 0 ? 1 : MB, MB == 0 ? 1 : PF, MB == 0>;
    auto kern = [] {
        if constexpr (MB == 0)
            return step_pair_ws_kernel<D, FS, TX, TY>;
        else
            return step_pair_kernel<D, FS, TX, TY, MB, PF>;
    }();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const StepArgs& a = ta.s;
    const int np = march_extent(a, D);
    dim3 grid(a.nx / TX, D == 3 ? a.ny / TY : 1, (np + a.chunk - 1) / a.chunk);
    kern<<<grid, Sh::NT, Sh::SMEM, st>>>(ta);
    return cudaGetLastError();
}

template <int D, typename FS, int TX, int TY, int MB, int PF>
void pair_box(TmaBox* b) {
    using Sh = PairShape<D, FS, TX, TY, MB == 0 ? 1 : MB, MB == 0 ? 1 : PF, MB == 0>;
    b->pxf = 16 / (int)sizeof(FS);
    b->sxf = TX + 2 * b->pxf;  // population map: L2 prefetch box
    b->sxb = Sh::SXB;
    b->sy = Sh::SY;
    b->smem = Sh::SMEM;
}

#define LBM_PAIR_CASE(D, TAB, K)                                                    \
    case K:                                                                         \
        if (box) {                                                                  \
            pair_box<D, FS, TAB[K].tx, TAB[K].ty, TAB[K].mb, TAB[K].pf>(box);       \
            return cudaSuccess;                                                     \
        }                                                                           \
        return launch_pair<D, FS, TAB[K].tx, TAB[K].ty, TAB[K].mb, TAB[K].pf>(*ta, st);

template <int D, typename FS>
cudaError_t pair_by_variant(int k, const TmaArgs* ta, TmaBox* box, cudaStream_t st) {
    if constexpr (D == 3) {
        switch (k) {
            LBM_PAIR_CASE(3, kPair3, 0)
            LBM_PAIR_CASE(3, kPair3, 1)
            LBM_PAIR_CASE(3, kPair3, 2)
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (k) {
            LBM_PAIR_CASE(2, kPair2, 0)
            LBM_PAIR_CASE(2, kPair2, 1)
            LBM_PAIR_CASE(2, kPair2, 2)
            default: return cudaErrorInvalidValue;
        }
    }
}
#undef LBM_PAIR_CASE

// Defined in lbm_kernels_pair{2,3}.cu (periodic lattices; FP32 storage, 2D also FP16/BF16).
int n_pair_variants_d2();
int n_pair_variants_d3();
Variant pair_variant_d2(int k);
Variant pair_variant_d3(int k);
cudaError_t pair_box_d2(int dtype, int k, TmaBox* box);
cudaError_t pair_box_d3(int dtype, int k, TmaBox* box);
cudaError_t launch_step_pair_d2(int dtype, int k, const TmaArgs& ta, cudaStream_t st);
cudaError_t launch_step_pair_d3(int dtype, int k, const TmaArgs& ta, cudaStream_t st);

}  // namespace lbm
