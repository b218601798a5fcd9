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
#include <cuda.h>
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
// Per device: the context in which the kernels' shared-memory attribute was
// set.  A device reset (cudaDeviceReset) ends that context; the next call on
// the device runs in a new one, whose ID differs, and sets it again.
struct DeviceSetup {
    unsigned long long ctx_id = 0;  // 0: not set up
};
DeviceSetup g_setup[kMaxDevices];

lbm_status fail(lbm_status s, const std::string& m) {
    lbm::set_last_error(m);  // reported by lbm_last_error()
    return s;
}

// Unique ID of the current context (driver entry points through the runtime,
// so the library needs no link to libcuda).
cudaError_t current_context_id(unsigned long long* id) {
    using GetCurrent = CUresult (*)(CUcontext*);
    using GetId = CUresult (*)(CUcontext, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    if (!get_current || !get_id) {
        void* p1 = nullptr;
        void* p2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p1, 12000, cudaEnableDefault, &q1);
        if (e == cudaSuccess)
            e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &p2, 12000, cudaEnableDefault, &q2);
        if (e != cudaSuccess) return e;
        if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !p1 || !p2)
            return cudaErrorNotSupported;
        get_current = reinterpret_cast<GetCurrent>(p1);
        get_id = reinterpret_cast<GetId>(p2);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
    return get_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

template <int D, int TX, int TY>
cudaError_t set_smem_attr() {
    using Sh = lbm::StepShape<D, double, TX, TY>;
    return cudaFuncSetAttribute(lbm::step_kernel<D, double, TX, TY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Sh::smem);
}

// Set-up per call (with the device current): look up the device address of
// the scratch array -- in host code the array's name is only a host-side
// stand-in -- which also makes the device's primary context current; then,
// once per device and context, allow the kernels' dynamic shared memory.
// The address is looked up on every call, so it is never stale.
lbm_status setup_device(int dev, void** out) {
    std::lock_guard<std::mutex> g(g_mu);
    if (dev < 0 || dev >= kMaxDevices) return fail(LBM_EINVAL, "device ordinal out of range");
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return fail(LBM_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    unsigned long long id = 0;
    e = current_context_id(&id);
    if (e != cudaSuccess) return fail(LBM_ECUDA, std::string("current context: ") + cudaGetErrorString(e));
    DeviceSetup& d = g_setup[dev];
    if (d.ctx_id != id) {
        e = set_smem_attr<1, 256, 1>();
        if (e == cudaSuccess) e = set_smem_attr<2, 128, 1>();
        if (e == cudaSuccess) e = set_smem_attr<3, 32, 8>();
        if (e != cudaSuccess) return fail(LBM_ECUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e));
        d.ctx_id = id;
    }
    *out = p;
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
    const size_t nblocks = blocks_needed(dim, nx, ny, nz);
    if (nblocks > max_blocks(dim))
        return fail(LBM_EINVAL, "lattice too large for the no-allocation step: needs " + std::to_string(nblocks) +
                                    " blocks of diagnostics scratch, the fixed array holds " +
                                    std::to_string(max_blocks(dim)));
    {
        // The step reads f_in, b_in while it writes f_out, b_out: an output
        // that overlaps any of the four buffers (in part, or a b plane inside
        // an f buffer) would race.  The two inputs may alias each other.
        const int Q = dim == 1 ? 3 : (dim == 2 ? 9 : 19), NB = dim == 1 ? 1 : (dim == 2 ? 3 : 6);
        const size_t N = (size_t)nx * ny * nz;
        const uintptr_t lo[4] = {(uintptr_t)f_in, (uintptr_t)b_in, (uintptr_t)f_out, (uintptr_t)b_out};
        const size_t len[4] = {Q * N * sizeof(double), NB * N * sizeof(double), Q * N * sizeof(double),
                               NB * N * sizeof(double)};
        for (int o = 2; o < 4; ++o)
            for (int k = 0; k < 4; ++k)
                if (k != o && lo[o] < lo[k] + len[k] && lo[k] < lo[o] + len[o])
                    return fail(LBM_EINVAL, "output buffers must not overlap each other or the inputs");
    }
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
    lbm::set_step_params(a, tau, T0);
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
