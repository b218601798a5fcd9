// Dimension dispatch for the kernel launchers.
#include <algorithm>

#include "lbm_internal.h"
#include "lbm_fast_launch.cuh"
#include "lbm_pair_launch.cuh"

namespace lbm {

#define LBM_DECLARE_D(DD)                                                                                       \
    cudaError_t launch_step_d##DD(int dtype, int v, const StepArgs& a, cudaStream_t st);                         \
    size_t step_smem_d##DD(int dtype, int v);                                                                    \
    int n_variants_d##DD();                                                                                      \
    Variant variant_d##DD(int v);                                                                                \
    cudaError_t launch_init_d##DD(int dtype, const double* rho, const double* u, const double* T, void* f,       \
                                 void* b, long long N, cudaStream_t st);                                        \
    cudaError_t launch_reservoir_d##DD(int dtype, const double* rho, const double* u, const double* T, int nx,   \
                                      long long rows, long long N, void* gf, void* gb, void* gaux,              \
                                      cudaStream_t st);                                                         \
    cudaError_t launch_get_state_d##DD(int dtype, const void* f, const void* b, double* fo, double* bo,          \
                                      long long N, cudaStream_t st);                                            \
    cudaError_t launch_set_state_d##DD(int dtype, void* f, void* b, const double* fi, const double* bi,          \
                                      long long N, cudaStream_t st);
LBM_DECLARE_D(1)
LBM_DECLARE_D(2)
LBM_DECLARE_D(3)
#undef LBM_DECLARE_D

#define LBM_BY_D(D, call1, call2, call3, bad) \
    ((D) == 1 ? (call1) : (D) == 2 ? (call2) : (D) == 3 ? (call3) : (bad))

int device_sms() {
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
    if (!cache[dev]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
        cache[dev] = n;
    }
    return cache[dev];
}

int n_variants(int D) { return LBM_BY_D(D, n_variants_d1(), n_variants_d2(), n_variants_d3(), 0); }

const char* kernel_name(int D, int v) {
    if (v == kStdVariant) return "std_step_kernel";
    if (v == kInplaceVariant) return "aa_collide_kernel";
    if (v >= kPairBase) return "step_pair_kernel";
    if (v >= kTmaBase) return "step_fast_kernel";
    return (D == 2 && v == 3) ? "step_strip_kernel" : "step_kernel";
}

int n_tma_variants(int D) { return D == 2 ? n_fast_variants_d2() : (D == 3 ? n_fast_variants_d3() : 0); }
int n_pair_variants(int D) { return D == 2 ? n_pair_variants_d2() : (D == 3 ? n_pair_variants_d3() : 0); }

Variant variant(int D, int v) {
    if (v >= kOwnBase && v < kOwnBase + n_own_variants(D)) return own_variant(D, v - kOwnBase);
    if (v >= kPairBase && v < kStdVariant) {
        const int k = v - kPairBase;
        return D == 2 ? pair_variant_d2(k) : (D == 3 ? pair_variant_d3(k) : Variant{0, 0});
    }
    if (v >= kTmaBase) {
        const int k = v - kTmaBase;
        return D == 2 ? fast_variant_d2(k) : (D == 3 ? fast_variant_d3(k) : Variant{0, 0});
    }
    return LBM_BY_D(D, variant_d1(v), variant_d2(v), variant_d3(v), (Variant{0, 0}));
}

cudaError_t tma_box(int D, int dtype, int v, TmaBox* box) {
    if (v >= kOwnBase && v < kPairBase)
        return dtype == DT_F32 && v < kOwnBase + n_own_variants(D) ? fast_own(D, v - kOwnBase, nullptr, box, nullptr)
                                                                    : cudaErrorInvalidValue;
    if (v >= kPairBase) {
        const int kk = v - kPairBase;
        return D == 2 ? pair_box_d2(dtype, kk, box) : (D == 3 ? pair_box_d3(dtype, kk, box) : cudaErrorInvalidValue);
    }
    const int k = v - kTmaBase;
    return D == 2 ? fast_box_d2(dtype, k, box) : (D == 3 ? fast_box_d3(dtype, k, box) : cudaErrorInvalidValue);
}

size_t step_smem(int D, int dtype, int v) {
    if (v >= kTmaBase) {
        TmaBox b{};
        return tma_box(D, dtype, v, &b) == cudaSuccess ? (size_t)b.smem : (size_t)0;
    }
    return LBM_BY_D(D, step_smem_d1(dtype, v), step_smem_d2(dtype, v), step_smem_d3(dtype, v), (size_t)0);
}

cudaError_t launch_step_tma(int D, int dtype, int v, const TmaArgs& ta, cudaStream_t st) {
    if (v >= kOwnBase && v < kPairBase)
        return dtype == DT_F32 && v < kOwnBase + n_own_variants(D) ? fast_own(D, v - kOwnBase, &ta, nullptr, st)
                                                                    : cudaErrorInvalidValue;
    if (v >= kPairBase) {
        const int kk = v - kPairBase;
        return D == 2 ? launch_step_pair_d2(dtype, kk, ta, st)
                      : (D == 3 ? launch_step_pair_d3(dtype, kk, ta, st) : cudaErrorInvalidValue);
    }
    const int k = v - kTmaBase;
    return D == 2 ? launch_step_fast_d2(dtype, k, ta, st)
                  : (D == 3 ? launch_step_fast_d3(dtype, k, ta, st) : cudaErrorInvalidValue);
}

dim3 step_grid(int D, int v, int nx, int ny, int nz, int chunk) {
    if (v == kStdVariant) return std_grid(D, nx, ny, nz, chunk);
    Variant t = v >= 0 ? variant(D, v) : Variant{1, 1};
    dim3 g(1, 1, 1);
    g.x = (nx + t.tx - 1) / t.tx;
    if (D == 3) {
        g.y = (ny + t.ty - 1) / t.ty;
        g.z = (nz + chunk - 1) / chunk;
    } else if (D == 2) {
        g.z = (ny + chunk - 1) / chunk;
    }
    return g;
}

cudaError_t launch_step(int D, int dtype, int v, const StepArgs& a, cudaStream_t st) {
    return LBM_BY_D(D, launch_step_d1(dtype, v, a, st), launch_step_d2(dtype, v, a, st),
                    launch_step_d3(dtype, v, a, st), cudaErrorInvalidValue);
}

// Grid-stride scan of the start fields on the device (a host loop over
// N values would cost more than the copy of them).  Writes only on failure.
__global__ void check_fields_kernel(const double* __restrict__ rho, const double* __restrict__ T, long long N,
                                    int* bad) {
    bool ok = true;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N;
         k += (long long)gridDim.x * blockDim.x)
        ok &= (rho[k] > 0.0) && (T[k] > 0.0);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) *bad = 1;
}

cudaError_t launch_check_fields(const double* rho, const double* T, long long N, int* bad, cudaStream_t st) {
    const long long want = (N + 255) / 256;
    const int blocks = (int)std::max(1LL, std::min<long long>(want, 8LL * device_sms()));
    check_fields_kernel<<<blocks, 256, 0, st>>>(rho, T, N, bad);
    return cudaGetLastError();
}

cudaError_t launch_init(int D, int dtype, const double* rho, const double* u, const double* T, void* f, void* b,
                        long long N, cudaStream_t st) {
    return LBM_BY_D(D, launch_init_d1(dtype, rho, u, T, f, b, N, st), launch_init_d2(dtype, rho, u, T, f, b, N, st),
                    launch_init_d3(dtype, rho, u, T, f, b, N, st), cudaErrorInvalidValue);
}

cudaError_t launch_reservoir(int D, int dtype, const double* rho, const double* u, const double* T, int nx,
                             long long rows, long long N, void* gf, void* gb, void* gaux, cudaStream_t st) {
    return LBM_BY_D(D, launch_reservoir_d1(dtype, rho, u, T, nx, rows, N, gf, gb, gaux, st),
                    launch_reservoir_d2(dtype, rho, u, T, nx, rows, N, gf, gb, gaux, st),
                    launch_reservoir_d3(dtype, rho, u, T, nx, rows, N, gf, gb, gaux, st), cudaErrorInvalidValue);
}

cudaError_t launch_get_state(int D, int dtype, const void* f, const void* b, double* fo, double* bo, long long N,
                             cudaStream_t st) {
    return LBM_BY_D(D, launch_get_state_d1(dtype, f, b, fo, bo, N, st),
                    launch_get_state_d2(dtype, f, b, fo, bo, N, st),
                    launch_get_state_d3(dtype, f, b, fo, bo, N, st), cudaErrorInvalidValue);
}

cudaError_t launch_set_state(int D, int dtype, void* f, void* b, const double* fi, const double* bi, long long N,
                             cudaStream_t st) {
    return LBM_BY_D(D, launch_set_state_d1(dtype, f, b, fi, bi, N, st),
                    launch_set_state_d2(dtype, f, b, fi, bi, N, st),
                    launch_set_state_d3(dtype, f, b, fi, bi, N, st), cudaErrorInvalidValue);
}

}  // namespace lbm
