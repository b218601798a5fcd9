// Generic step kernel of the D3 lattice: tile table and per-storage-type
// launchers.  Each storage type is instantiated in its own translation unit
// (lbm_gen3_<type>.cu), because one D3Q19 instantiation takes about a minute
// to compile.
#pragma once

#include "lbm_internal.h"

namespace lbm {

// Tiles (TX x TY) of the generic D3 step kernel.
constexpr int kGen3Tiles = 2;
__host__ __device__ constexpr Variant gen3_tile(int v) { return v == 0 ? Variant{32, 8} : Variant{32, 4}; }

template <typename FS>
cudaError_t gen3_launch(int v, const StepArgs& a, cudaStream_t st);
template <typename FS>
size_t gen3_smem(int v);

template <typename FS, int TX, int TY>
cudaError_t gen3_launch_one(const StepArgs& a, cudaStream_t st) {
    using Sh = StepShape<3, FS, TX, TY>;
    auto kern = step_kernel<3, FS, TX, TY>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid = step_grid(3, -1, a.nx, a.ny, march_extent(a, 3), a.chunk);
    grid.x = (a.nx + TX - 1) / TX;
    grid.y = (a.ny + TY - 1) / TY;
    kern<<<grid, TX * TY, Sh::smem, st>>>(a);
    return cudaGetLastError();
}

// Defines gen3_launch<FS> and gen3_smem<FS> for one storage type.
#define LBM_GEN3_DEFINE(FS)                                                                   \
    template <>                                                                               \
    cudaError_t gen3_launch<FS>(int v, const StepArgs& a, cudaStream_t st) {                  \
        switch (v) {                                                                          \
            case 0: return gen3_launch_one<FS, gen3_tile(0).tx, gen3_tile(0).ty>(a, st);      \
            case 1: return gen3_launch_one<FS, gen3_tile(1).tx, gen3_tile(1).ty>(a, st);      \
            default: return cudaErrorInvalidValue;                                            \
        }                                                                                     \
    }                                                                                         \
    template <>                                                                               \
    size_t gen3_smem<FS>(int v) {                                                             \
        switch (v) {                                                                          \
            case 0: return StepShape<3, FS, gen3_tile(0).tx, gen3_tile(0).ty>::smem;          \
            case 1: return StepShape<3, FS, gen3_tile(1).tx, gen3_tile(1).ty>::smem;          \
            default: return 0;                                                                \
        }                                                                                     \
    }

// Explicit specializations defined in lbm_gen3_*.cu.
template <> cudaError_t gen3_launch<double>(int, const StepArgs&, cudaStream_t);
template <> cudaError_t gen3_launch<float>(int, const StepArgs&, cudaStream_t);
template <> cudaError_t gen3_launch<__half>(int, const StepArgs&, cudaStream_t);
template <> cudaError_t gen3_launch<__nv_bfloat16>(int, const StepArgs&, cudaStream_t);
template <> size_t gen3_smem<double>(int);
template <> size_t gen3_smem<float>(int);
template <> size_t gen3_smem<__half>(int);
template <> size_t gen3_smem<__nv_bfloat16>(int);

}  // namespace lbm
