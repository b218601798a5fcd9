// Launchers of the cluster-resident multi-step kernel (lbm_step_cluster.cuh):
// small periodic D2Q9 lattices, FP32 or FP64 storage.
#include "lbm_internal.h"
#include "lbm_step_cluster.cuh"

namespace lbm {

namespace {

// Blocks per cluster and threads per block of each variant.  Clusters of more
// than 8 blocks are a non-portable size, allowed per kernel.
struct ClusterVariant {
    int c, nt;
};
constexpr ClusterVariant kCluster[] = {{16, 256}, {16, 512}, {8, 512}};
constexpr int kNC = sizeof(kCluster) / sizeof(kCluster[0]);

// Largest dynamic shared memory of one block (bytes): the 227 KB a block may
// opt into, less room for the kernel's static shared memory.
constexpr size_t kMaxSmem = 227 * 1024 - 1024;

ClusterBands bands_of(int ny, int c) { return ClusterBands{ny / c, ny % c}; }

template <typename FS> size_t smem_for(int nx, int ny, int c, int* P) {
    const ClusterBands b = bands_of(ny, c);
    *P = b.rows(0) * nx;  // the first band is the largest
    return ClusterShape<FS>::smem(*P);
}

template <typename FS, int NT>
cudaError_t launch_fs(int c, const StepArgs& a0, const StepArgs& a1, int K, cudaStream_t st, bool probe) {
    auto kern = step_cluster_kernel<FS, NT>;
    int P = 0;
    const size_t smem = smem_for<FS>(a0.nx, a0.ny, c, &P);
    if (a0.ny < c || smem > kMaxSmem) return cudaErrorInvalidValue;
    static size_t attr_smem = 0;  // per instantiation
    if (smem > attr_smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_smem = smem;
    }
    static bool nonportable = false;  // per instantiation
    if (c > 8 && !nonportable) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        nonportable = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (probe) {
        // can one such cluster be resident at all on this device?
        int n = 0;
        cudaError_t e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
        if (e != cudaSuccess) return e;
        return n >= 1 ? cudaSuccess : cudaErrorNotSupported;
    }
    return cudaLaunchKernelEx(&cfg, kern, a0, a1, K, P, bands_of(a0.ny, c));
}

template <typename FS>
cudaError_t launch_dtype(int v, const StepArgs& a0, const StepArgs& a1, int K, cudaStream_t st, bool probe) {
    switch (v) {
        case 0: return launch_fs<FS, 256>(kCluster[0].c, a0, a1, K, st, probe);
        case 1: return launch_fs<FS, 512>(kCluster[1].c, a0, a1, K, st, probe);
        case 2: return launch_fs<FS, 512>(kCluster[2].c, a0, a1, K, st, probe);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int n_cluster_variants() { return kNC; }
int cluster_blocks(int v) { return (v >= 0 && v < kNC) ? kCluster[v].c : 0; }

bool cluster_fits_d2(int dtype, int v, int nx, int ny) {
    if (v < 0 || v >= kNC || ny < kCluster[v].c) return false;
    int P = 0;
    if (dtype == DT_F32) return smem_for<float>(nx, ny, kCluster[v].c, &P) <= kMaxSmem;
    if (dtype == DT_F64) return smem_for<double>(nx, ny, kCluster[v].c, &P) <= kMaxSmem;
    return false;
}

cudaError_t launch_step_cluster_d2(int dtype, int v, const StepArgs& a0, const StepArgs& a1, int K, cudaStream_t st,
                                   bool probe) {
    if (dtype == DT_F32) return launch_dtype<float>(v, a0, a1, K, st, probe);
    if (dtype == DT_F64) return launch_dtype<double>(v, a0, a1, K, st, probe);
    return cudaErrorNotSupported;
}

}  // namespace lbm
