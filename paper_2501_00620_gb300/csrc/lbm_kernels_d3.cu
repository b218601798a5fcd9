// Launchers for the D3 lattice: storage-type dispatch, init, reservoir and
// state kernels.  The generic step kernel is instantiated per storage type in
// lbm_gen3_*.cu (one translation unit each, so that they compile in parallel).
#include "lbm_gen3.cuh"

namespace lbm {

namespace {
constexpr int kD = 3;
constexpr int kNV = kGen3Tiles;

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

cudaError_t launch_step_d3(int dtype, int v, const StepArgs& a, cudaStream_t st) {
    return by_dtype(dtype, [&](auto tag) { return gen3_launch<decltype(tag)>(v, a, st); });
}

size_t step_smem_d3(int dtype, int v) {
    switch (dtype) {
        case DT_F64: return gen3_smem<double>(v);
        case DT_F32: return gen3_smem<float>(v);
        case DT_F16: return gen3_smem<__half>(v);
        case DT_BF16: return gen3_smem<__nv_bfloat16>(v);
    }
    return 0;
}

int n_variants_d3() { return kNV; }
Variant variant_d3(int v) { return gen3_tile(v); }

cudaError_t launch_init_d3(int dtype, const double* rho, const double* u, const double* T, void* f, void* b,
                            long long N, cudaStream_t st) {
    return by_dtype(dtype, [&](auto tag) {
        using FS = decltype(tag);
        init_kernel<kD, FS><<<blocks_for(N, 256), 256, 0, st>>>(
            rho, u, T, static_cast<FS*>(f), static_cast<typename Store<FS>::breal*>(b), N);
        return cudaGetLastError();
    });
}

cudaError_t launch_reservoir_d3(int dtype, const double* rho, const double* u, const double* T, int nx,
                                 long long rows, long long N, void* gf, void* gb, void* gaux, cudaStream_t st) {
    return by_dtype(dtype, [&](auto tag) {
        using R = typename Store<decltype(tag)>::real;
        reservoir_kernel<kD, R><<<blocks_for(2 * rows, 256), 256, 0, st>>>(
            rho, u, T, nx, rows, N, static_cast<R*>(gf), static_cast<R*>(gb), static_cast<R*>(gaux));
        return cudaGetLastError();
    });
}

cudaError_t launch_get_state_d3(int dtype, const void* f, const void* b, double* fo, double* bo, long long N,
                                 cudaStream_t st) {
    return by_dtype(dtype, [&](auto tag) {
        using FS = decltype(tag);
        get_state_kernel<kD, FS><<<blocks_for(N, 256), 256, 0, st>>>(
            static_cast<const FS*>(f), static_cast<const typename Store<FS>::breal*>(b), fo, bo, N);
        return cudaGetLastError();
    });
}

cudaError_t launch_set_state_d3(int dtype, void* f, void* b, const double* fi, const double* bi, long long N,
                                 cudaStream_t st) {
    return by_dtype(dtype, [&](auto tag) {
        using FS = decltype(tag);
        set_state_kernel<kD, FS><<<blocks_for(N, 256), 256, 0, st>>>(
            static_cast<FS*>(f), static_cast<typename Store<FS>::breal*>(b), fi, bi, N);
        return cudaGetLastError();
    });
}

}  // namespace lbm
