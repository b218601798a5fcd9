// One fused time step on caller-owned device buffers that allocates no
// device memory (see lbm_step_noalloc in include/lbm.h).
//
// Who needs it: callers that must not allocate on the device while they run
// -- real-time loops that cannot afford the synchronisation an allocator may
// impose, and host frameworks or plugins that own all device memory and do
// not let a library take any.  Such a caller keeps the state in buffers it
// allocated up front and advances it with this call.
//
// The kernel is the generic fused step in FP64 storage with the periodic
// boundary.  Its scratch memory -- the per-block partial sums of the
// conservation diagnostics, the completion ticket of the last-block
// reduction, the step counter and the status flag -- lives in the
// file-scope device array g_noalloc_scratch below instead of in buffers
// the library allocates.  Every GPU that loads the library holds this array
// (kNoallocScratchBytes) until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/lbm.h"
#include "lbm_step.cuh"

namespace lbm {
void set_last_error(const std::string& m);  // lbm_capi.cu
}

namespace {

// Size of the shared scratch: a 256-byte header (ticket, step counter, flag)
// followed by the per-block partial sums (dim+2 doubles per block).
constexpr size_t kNoallocScratchBytes = 1u << 20;  // 1 MiB
constexpr size_t kHeaderBytes = 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Tile shapes of the generic FP64 kernel used here (one fixed variant per
// dimension, no autotuning: tuning would need scratch buffers of its own).
constexpr int kChunk = 64;

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};  // device address of g_noalloc_scratch per device

lbm_status fail(lbm_status s, const std::string& m) {
    lbm::set_last_error(m);  // reported by lbm_last_error()
    return s;
}

template <int D, int TX, int TY>
cudaError_t set_smem_attr() {
    using Sh = lbm::StepShape<D, double, TX, TY>;
    return cudaFuncSetAttribute(lbm::step_kernel<D, double, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Sh::smem);
}

// One-time set-up per device (with that device current): look up the device
// address of the scratch array -- in host code the array's name is only a
// host-side stand-in -- and allow the kernels' dynamic shared memory.
lbm_status setup_device(int dev, void** out) {
    std::lock_guard<std::mutex> g(g_mu);
    if (dev < 0 || dev >= kMaxDevices) return fail(LBM_EINVAL, "device ordinal out of range");
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return fail(LBM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        e = set_smem_attr<1, 256, 1>();
        if (e == cudaSuccess) e = set_smem_attr<2, 128, 1>();
        if (e == cudaSuccess) e = set_smem_attr<3, 32, 8>();
        if (e != cudaSuccess) return fail(LBM_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return LBM_OK;
}

template <int D, int TX, int TY>
cudaError_t launch(const lbm::StepArgs& a, cudaStream_t st) {
    using Sh = lbm::StepShape<D, double, TX, TY>;
    dim3 grid((a.nx + TX - 1) / TX, D == 3 ? (a.ny + TY - 1) / TY : 1,
              D == 3 ? (a.nz + a.chunk - 1) / a.chunk : (D == 2 ? (a.ny + a.chunk - 1) / a.chunk : 1));
    lbm::step_kernel<D, double, TX, TY><<<grid, TX * TY, Sh::smem, st>>>(a);
    return cudaGetLastError();
}

size_t blocks_needed(int dim, int nx, int ny, int nz) {
    if (dim == 1) return (size_t)((nx + 255) / 256);
    if (dim == 2) return (size_t)((nx + 127) / 128) * ((ny + kChunk - 1) / kChunk);
    return (size_t)((nx + 31) / 32) * ((ny + 7) / 8) * ((nz + kChunk - 1) / kChunk);
}

// Largest number of thread blocks whose diagnostics partials fit the array.
size_t max_blocks(int dim) { return (kNoallocScratchBytes - kHeaderBytes) / (sizeof(double) * (size_t)(dim + 2)); }

}  // namespace

extern "C" {

lbm_status lbm_step_noalloc(int dim, int nx, int ny, int nz, double tau, double T0, int thermal,
                            const double* f_in, const double* b_in, double* f_out, double* b_out,
                            double* diag_out, void* stream) {
    if (dim < 1 || dim > 3 || nx < 1 || ny < 1 || nz < 1 || (dim < 2 && ny != 1) || (dim < 3 && nz != 1))
        return fail(LBM_EINVAL, "invalid lattice extents");
    if (!(tau > 0) || !(T0 > 0)) return fail(LBM_EINVAL, "tau and T0 must be > 0");
    if (!f_in || !b_in || !f_out || !b_out) return fail(LBM_EINVAL, "NULL state buffer");
    if (f_in == f_out || b_in == b_out) return fail(LBM_EINVAL, "input and output buffers must differ");
    const size_t nblocks = blocks_needed(dim, nx, ny, nz);
    if (nblocks > max_blocks(dim))
        return fail(LBM_EINVAL, "lattice too large for the no-allocation step: needs " + std::to_string(nblocks) +
                                    " blocks of diagnostics scratch, the fixed array holds " +
                                    std::to_string(max_blocks(dim)));
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(LBM_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    void* scratch = nullptr;
    lbm_status st = setup_device(dev, &scratch);
    if (st != LBM_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned char* base = static_cast<unsigned char*>(scratch);
    // The ticket, step counter and flag must start at zero; the partial sums
    // are written before they are read.
    e = cudaMemsetAsync(base, 0, kHeaderBytes, s);
    if (e != cudaSuccess) return fail(LBM_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));

    lbm::StepArgs a{};
    a.fin = f_in;
    a.bin = b_in;
    a.fout = f_out;
    a.bout = b_out;
    a.nx = nx;
    a.ny = ny;
    a.nz = nz;
    a.chunk = kChunk;
    a.N = (long long)nx * ny * nz;
    a.omega = 1.0 / (tau + 0.5);
    a.tau = tau;
    a.T0 = T0;
    a.thermal = thermal ? 1 : 0;
    a.fixed_x = 0;
    a.rows = (long long)ny * nz;
    a.write_state = 1;
    a.want_diag = 1;
    a.ticket = reinterpret_cast<unsigned int*>(base);
    a.step_ctr = reinterpret_cast<long long*>(base + 64);
    a.flag = reinterpret_cast<int*>(base + 128);
    a.partial = reinterpret_cast<double*>(base + kHeaderBytes);
    a.diag_out = diag_out;
    a.hist = nullptr;
    a.hist_cap = 1;
    e = dim == 1 ? launch<1, 256, 1>(a, s) : (dim == 2 ? launch<2, 128, 1>(a, s) : launch<3, 32, 8>(a, s));
    if (e != cudaSuccess) return fail(LBM_ECUDA, std::string("step launch: ") + cudaGetErrorString(e));
    int flag = 0;
    e = cudaMemcpyAsync(&flag, a.flag, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(LBM_ECUDA, std::string("no-allocation step: ") + cudaGetErrorString(e));
    if (flag & 1) return fail(LBM_EUNSTABLE, "state became non-physical (rho <= 0 or not finite)");
    return LBM_OK;
}

}  // extern "C"
