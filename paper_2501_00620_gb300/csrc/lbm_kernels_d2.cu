// Launchers for the D2 lattice (tile variants x storage types).
#include "lbm_internal.h"
#include "lbm_step_strip.cuh"

namespace lbm {

namespace {
constexpr int kD = 2;
// 0-2: generic kernel strips; 3: strip kernel (lbm_step_strip.cuh), 254 sites
// per 256-thread block, FP32/16-bit storage.
constexpr Variant kVariants[] = {{256, 1}, {128, 1}, {512, 1}, {kStripNT - 2, 1}};
constexpr int kNV = sizeof(kVariants) / sizeof(kVariants[0]);

template <typename FS, int TX, int TY>
cudaError_t launch_one(const StepArgs& a, cudaStream_t st) {
    using Sh = StepShape<kD, FS, TX, TY>;
    auto kern = step_kernel<kD, FS, TX, TY>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid = step_grid(kD, -1, a.nx, march_extent(a, kD), a.nz, a.chunk);
    grid.x = (a.nx + TX - 1) / TX;
    if (kD == 3) grid.y = (a.ny + TY - 1) / TY;
    kern<<<grid, TX * TY, Sh::smem, st>>>(a);
    return cudaGetLastError();
}

template <typename FS, bool FX>
cudaError_t launch_strip_fx(const StepArgs& a, cudaStream_t st) {
    using Sh = StripShape<FS, kStripNT>;
    auto kern = step_strip_kernel<FS, kStripNT, FX>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((a.nx + Sh::TX - 1) / Sh::TX, 1, (march_extent(a, 2) + a.chunk - 1) / a.chunk);
    kern<<<grid, kStripNT, Sh::SMEM, st>>>(a);
    return cudaGetLastError();
}

template <typename FS>
cudaError_t launch_strip(const StepArgs& a, cudaStream_t st) {
    if constexpr (std::is_same<FS, double>::value) {
        return cudaErrorInvalidValue;  // FP32 arithmetic only
    } else {
        if (9 * a.N >= (1LL << 31)) return cudaErrorInvalidValue;  // 32-bit plane offsets i N + s
        return a.fixed_x ? launch_strip_fx<FS, true>(a, st) : launch_strip_fx<FS, false>(a, st);
    }
}

template <typename FS>
cudaError_t launch_dtype(int v, const StepArgs& a, cudaStream_t st) {
    switch (v) {
        case 0: return launch_one<FS, 256, 1>(a, st);
        case 1: return launch_one<FS, 128, 1>(a, st);
        case 2: return launch_one<FS, 512, 1>(a, st);
        case 3: return launch_strip<FS>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename FS>
size_t smem_of(int v) {
    switch (v) {
        case 0: return StepShape<kD, FS, 256, 1>::smem;
        case 1: return StepShape<kD, FS, 128, 1>::smem;
        case 2: return StepShape<kD, FS, 512, 1>::smem;
        case 3: return StripShape<FS, kStripNT>::SMEM;
        default: return 0;
    }
}

template <typename F>
cudaError_t by_dtype(int dtype, F&& f) {
    switch (dtype) {
        case DT_F64: return f(double{});
        case DT_F32: return f(float{});
        case DT_F16: return f(__half{});
        case DT_BF16: return f(__nv_bfloat16{});
        default: return cudaErrorInvalidValue;
    }
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }
}  // namespace

// K steps of a small D2 lattice in one cooperative launch: the generic
// kernel's strips of kMultiTX2 sites (a.chunk rows each) meet at a grid-wide
// barrier after every step.  cudaErrorCooperativeLaunchTooLarge if the grid
// cannot be resident at once.
template <typename FS>
cudaError_t launch_multi_d2_fs(const StepArgs& a0, const StepArgs& a1, int K, cudaStream_t st) {
    constexpr int TX = kMultiTX2;
    using Sh = StepShape<kD, FS, TX, 1>;
    auto kern = step_multi_kernel<kD, FS, TX, 1>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const dim3 grid((a0.nx + TX - 1) / TX, 1, (march_extent(a0, kD) + a0.chunk - 1) / a0.chunk);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX, Sh::smem);
    if (e != cudaSuccess) return e;
    if ((long long)per_sm * device_sms() < (long long)grid.x * grid.z) return cudaErrorCooperativeLaunchTooLarge;
    StepArgs p0 = a0, p1 = a1;
    void* args[] = {&p0, &p1, &K};
    return cudaLaunchCooperativeKernel((const void*)kern, grid, dim3(TX), args, Sh::smem, st);
}

cudaError_t launch_step_multi_d2(int dtype, const StepArgs& a0, const StepArgs& a1, int K, cudaStream_t st) {
    return by_dtype(dtype, [&](auto tag) { return launch_multi_d2_fs<decltype(tag)>(a0, a1, K, st); });
}

cudaError_t launch_step_d2(int dtype, int v, const StepArgs& a, cudaStream_t st) {
    return by_dtype(dtype, [&](auto tag) { return launch_dtype<decltype(tag)>(v, a, st); });
}

size_t step_smem_d2(int dtype, int v) {
    switch (dtype) {
        case DT_F64: return smem_of<double>(v);
        case DT_F32: return smem_of<float>(v);
        case DT_F16: return smem_of<__half>(v);
        case DT_BF16: return smem_of<__nv_bfloat16>(v);
    }
    return 0;
}

int n_variants_d2() { return kNV; }
Variant variant_d2(int v) { return kVariants[v]; }

cudaError_t launch_init_d2(int dtype, const double* rho, const double* u, const double* T, void* f, void* b,
                            long long N, cudaStream_t st) {
    return by_dtype(dtype, [&](auto tag) {
        using FS = decltype(tag);
        init_kernel<kD, FS><<<blocks_for(N, 256), 256, 0, st>>>(
            rho, u, T, static_cast<FS*>(f), static_cast<typename Store<FS>::breal*>(b), N);
        return cudaGetLastError();
    });
}

cudaError_t launch_reservoir_d2(int dtype, const double* rho, const double* u, const double* T, int nx,
                                 long long rows, long long N, void* gf, void* gb, void* gaux, cudaStream_t st) {
    return by_dtype(dtype, [&](auto tag) {
        using R = typename Store<decltype(tag)>::real;
        reservoir_kernel<kD, R><<<blocks_for(2 * rows, 256), 256, 0, st>>>(
            rho, u, T, nx, rows, N, static_cast<R*>(gf), static_cast<R*>(gb), static_cast<R*>(gaux));
        return cudaGetLastError();
    });
}

cudaError_t launch_get_state_d2(int dtype, const void* f, const void* b, double* fo, double* bo, long long N,
                                 cudaStream_t st) {
    return by_dtype(dtype, [&](auto tag) {
        using FS = decltype(tag);
        get_state_kernel<kD, FS><<<blocks_for(N, 256), 256, 0, st>>>(
            static_cast<const FS*>(f), static_cast<const typename Store<FS>::breal*>(b), fo, bo, N);
        return cudaGetLastError();
    });
}

cudaError_t launch_set_state_d2(int dtype, void* f, void* b, const double* fi, const double* bi, long long N,
                                 cudaStream_t st) {
    return by_dtype(dtype, [&](auto tag) {
        using FS = decltype(tag);
        set_state_kernel<kD, FS><<<blocks_for(N, 256), 256, 0, st>>>(
            static_cast<FS*>(f), static_cast<typename Store<FS>::breal*>(b), fi, bi, N);
        return cudaGetLastError();
    });
}

}  // namespace lbm
