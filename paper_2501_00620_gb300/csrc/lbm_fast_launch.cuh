// Launch helpers of the occupancy-oriented step kernel (lbm_step_fast.cuh):
// the tile table per lattice and one launcher per (storage, tile, boundary).
#pragma once

#include <algorithm>

#include "lbm_internal.h"
#include "lbm_step_fast.cuh"

namespace lbm {

// Tile TX x TY, PFB flags (bit 0: extra variance plane in flight, bit 1:
// populations to stage 2 through shared memory, bit 2: that hand-off in
// tensor memory), resident blocks per SM MB.
struct FastVariant {
    int tx, ty, pfb, mb;
};

// D3Q19: 32 x 8 at two blocks per SM; 32 x 4 at three; 32 x 4 with one more
// variance plane in flight and the populations handed to stage 2 through
// shared memory, at two blocks per SM; 32 x 4 with one more variance plane
// in flight at three; the third with the hand-off in tensor memory at three
// (the fastest on 256^3).
constexpr FastVariant kFast3[] = {{32, 8, 0, 2}, {32, 4, 0, 3}, {32, 4, 3, 2}, {32, 4, 1, 3},
                                  {32, 4, 7, 3}};
// Tiles for FP32 storage only, instantiated in their own translation unit
// (lbm_kernels_fastx.cu), variants kOwnBase + k, on the fastest D3Q19 and
// D2Q9 tile shapes:
//  k = 0: the body-force and MRT terms in stage 2 (PFB bit 3): the kernels of
//         forced or MRT periodic lattices;
//  k = 1: the same with half-way bounce-back walls normal to the march axis
//         (PFB bit 4): the kernels of walled lattices.
constexpr FastVariant kFastOwn3[] = {{32, 4, 15, 3}, {32, 4, 31, 3}};
constexpr FastVariant kFastOwn2[] = {{128, 1, 15, 6}, {128, 1, 31, 6}};
// D2Q9: strips of 128 sites; with the populations handed to stage 2 through
// shared memory; with that hand-off in tensor memory at six blocks per SM.
constexpr FastVariant kFast2[] = {{128, 1, 0, 5}, {128, 1, 1, 5}, {128, 1, 3, 5}, {128, 1, 7, 6}};


template <int D, typename FS, int TX, int TY, int PFB, int MB, bool FX>
cudaError_t launch_fast(const TmaArgs& ta, cudaStream_t st) {
    using Sh = FastShape<D, FS, TX, TY, PFB, MB>;
    auto kern = step_fast_kernel<D, FS, TX, TY, PFB, MB, FX>;
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

template <int D, typename FS, int TX, int TY, int PFB, int MB>
void fast_box(TmaBox* b) {
    using Sh = FastShape<D, FS, TX, TY, PFB, MB>;
    b->pxf = 16 / (int)sizeof(FS);
    b->sxf = TX + 2 * b->pxf;  // population map: L2 prefetch box
    b->sxb = Sh::SXB;
    b->sy = Sh::SY;
    b->smem = Sh::SMEM;
}

// Dispatch over the tile table of lattice D for storage FS and boundary FX;
// with box != nullptr only the geometry is returned.
#define LBM_FAST_CASE(D, TAB, K)                                                                        \
    case K:                                                                                             \
        if (box) {                                                                                      \
            fast_box<D, FS, TAB[K].tx, TAB[K].ty, TAB[K].pfb, TAB[K].mb>(box);                          \
            return cudaSuccess;                                                                         \
        }                                                                                               \
        return launch_fast<D, FS, TAB[K].tx, TAB[K].ty, TAB[K].pfb, TAB[K].mb, FX>(*ta, st);

template <int D, typename FS, bool FX>
cudaError_t fast_by_variant(int k, const TmaArgs* ta, TmaBox* box, cudaStream_t st) {
    if constexpr (D == 3) {
        switch (k) {
            LBM_FAST_CASE(3, kFast3, 0)
            LBM_FAST_CASE(3, kFast3, 1)
            LBM_FAST_CASE(3, kFast3, 2)
            LBM_FAST_CASE(3, kFast3, 3)
            LBM_FAST_CASE(3, kFast3, 4)
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (k) {
            LBM_FAST_CASE(2, kFast2, 0)
            LBM_FAST_CASE(2, kFast2, 1)
            LBM_FAST_CASE(2, kFast2, 2)
            LBM_FAST_CASE(2, kFast2, 3)
            default: return cudaErrorInvalidValue;
        }
    }
}
#undef LBM_FAST_CASE

template <int D, bool FX>
cudaError_t fast_by_dtype(int dtype, int k, const TmaArgs* ta, TmaBox* box, cudaStream_t st) {
    switch (dtype) {
        case DT_F32: return fast_by_variant<D, float, FX>(k, ta, box, st);
        case DT_F16: return fast_by_variant<D, __half, FX>(k, ta, box, st);
        case DT_BF16: return fast_by_variant<D, __nv_bfloat16, FX>(k, ta, box, st);
        default: return cudaErrorInvalidValue;
    }
}

// Defined in lbm_kernels_fast{2,3}.cu (periodic) and lbm_kernels_fast{2,3}x.cu
// (fixed-state in x).
int n_fast_variants_d2();
int n_fast_variants_d3();
Variant fast_variant_d2(int k);
Variant fast_variant_d3(int k);
cudaError_t fast_box_d2(int dtype, int k, TmaBox* box);
cudaError_t fast_box_d3(int dtype, int k, TmaBox* box);
cudaError_t launch_step_fast_d2(int dtype, int k, const TmaArgs& ta, cudaStream_t st);
cudaError_t launch_step_fast_d3(int dtype, int k, const TmaArgs& ta, cudaStream_t st);
cudaError_t launch_step_fast_d2_fx(int dtype, int k, const TmaArgs& ta, cudaStream_t st);
cudaError_t launch_step_fast_d3_fx(int dtype, int k, const TmaArgs& ta, cudaStream_t st);

}  // namespace lbm
