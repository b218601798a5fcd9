// Internal interface between the C-ABI runtime and the kernel launchers.
// Not part of the public header.
#pragma once

#include <cuda_runtime.h>

#include "lbm_step.cuh"
#include "lbm_tma.cuh"

namespace lbm {

enum Dtype { DT_F64 = 0, DT_F32 = 1, DT_F16 = 2, DT_BF16 = 3 };

struct Variant {
    int tx, ty;
};

// Threads per block of the D2Q9 strip kernel (lbm_step_strip.cuh): NT - 2
// tile sites per strip.
constexpr int kStripNT = 256;

// Variant indices: 0..n_variants(D)-1 select the generic kernel's tiles;
// kTmaBase + k selects the k-th tile of the staged kernel (lbm_step_fast.cuh).
constexpr int kTmaBase = 100;

// kOwnBase + k selects the k-th FP32-only tile of the staged kernel
// (lbm_kernels_fastx.cu); own_kind: 1 for the tile with the body-force and
// MRT terms in stage 2 (periodic lattices with a body force or, D3Q19, the
// MRT collision), 2 for the tile that adds half-way bounce-back walls
// (walled lattices, with or without force and MRT).
constexpr int kOwnBase = 150;

// kPairBase + k selects the k-th tile of the pair kernel (lbm_step_pair.cuh):
// periodic lattices, FP32 storage (2D: also FP16/BF16).
constexpr int kPairBase = 200;

// Variant index of the in-place two-pass step (lbm_step_aa.cuh).
constexpr int kInplaceVariant = 900;

// Variant index of the standard-lattice comparator kernel (lbm_std.cu).
constexpr int kStdVariant = 1000;

// Slice geometry of a TMA variant (for the host-side tensor maps).
struct TmaBox {
    int sxf, sxb, sy, pxf, smem;
};

// Multiprocessor count of the current device (cached per device).
int device_sms();

int n_variants(int D);
// Name of the kernel template variant v launches (for reports).
const char* kernel_name(int D, int v);
int n_tma_variants(int D);
int n_pair_variants(int D);
Variant variant(int D, int v);
size_t step_smem(int D, int dtype, int v);
cudaError_t tma_box(int D, int dtype, int v, TmaBox* box);

// Grid of a step launch for extents and chunk.
dim3 step_grid(int D, int v, int nx, int ny, int nz, int chunk);

cudaError_t launch_step(int D, int dtype, int v, const StepArgs& a, cudaStream_t st);
// K steps of the D1 lattice in one cooperative launch (generic variant v):
// a0 reads buffer 0, a1 buffer 1; step k uses a0 if k is even.  Returns
// cudaErrorCooperativeLaunchTooLarge if the grid cannot be resident.
cudaError_t launch_step_multi_d1(int dtype, int v, const StepArgs& a0, const StepArgs& a1, int K,
                                 cudaStream_t st);
cudaError_t launch_step_tma(int D, int dtype, int v, const TmaArgs& ta, cudaStream_t st);
int n_own_variants(int D);
Variant own_variant(int D, int k);
int own_kind(int D, int k);
cudaError_t fast_own(int D, int k, const TmaArgs* ta, TmaBox* box, cudaStream_t st);
// K steps of a small D2 lattice in one cooperative launch (the generic
// kernel's strips of kMultiTX2 sites, a0.chunk rows per block).
constexpr int kMultiTX2 = 128;
constexpr int kMultiChunk2 = 8;
cudaError_t launch_step_multi_d2(int dtype, const StepArgs& a0, const StepArgs& a1, int K, cudaStream_t st);
// K steps of a small periodic D2 lattice held in the shared memory of one
// thread-block cluster (lbm_step_cluster.cuh), FP32 or FP64 storage, cluster
// variant v (kClusterBase + v in reports).  cluster_fits_d2: the lattice fits
// variant v (rows per block, shared memory).  probe = true only checks that
// such a cluster can be resident on the device (no launch).
constexpr int kClusterBase = 300;
int n_cluster_variants();
int cluster_blocks(int v);
bool cluster_fits_d2(int dtype, int v, int nx, int ny);
cudaError_t launch_step_cluster_d2(int dtype, int v, const StepArgs& a0, const StepArgs& a1, int K, cudaStream_t st,
                                   bool probe = false);
cudaError_t launch_init(int D, int dtype, const double* rho, const double* u, const double* T, void* f,
                        void* b, long long N, cudaStream_t st);
// Sets *bad (device) to 1 if some rho[k] or T[k] (k < N, device arrays) is
// not > 0 (NaN included); leaves it unchanged otherwise.
cudaError_t launch_check_fields(const double* rho, const double* T, long long N, int* bad, cudaStream_t st);
cudaError_t launch_reservoir(int D, int dtype, const double* rho, const double* u, const double* T, int nx,
                             long long rows, long long N, void* gf, void* gb, void* gaux, cudaStream_t st);
cudaError_t launch_get_state(int D, int dtype, const void* f, const void* b, double* fo, double* bo,
                             long long N, cudaStream_t st);
cudaError_t launch_set_state(int D, int dtype, void* f, void* b, const double* fi, const double* bi,
                             long long N, cudaStream_t st);

// In-place two-pass step (lbm_kernels_aa.cu): pass 1 (aux) then pass 2 on the
// population buffer in memory form `form` (0: emitted layout, 1: arrived
// populations in opposite planes); the emitted state of a form-1 buffer as
// FP64 population planes.
cudaError_t launch_step_aa(int D, int dtype, const StepArgs& a, int form, void* aux, cudaStream_t st);
cudaError_t launch_aa_get_state(int D, int dtype, const StepArgs& a, double* fo, cudaStream_t st);

// Standard-lattice comparator (lbm_std.cu): grid of a step launch, one step,
// and the start (equilibrium of Eq. 4 for the fields, populations only).
dim3 std_grid(int D, int nx, int ny, int nz, int chunk);
cudaError_t launch_std_step(int D, int dtype, const StepArgs& a, cudaStream_t st);
cudaError_t launch_std_init(int D, int dtype, const double* rho, const double* u, const double* T, void* f,
                            long long N, cudaStream_t st);

}  // namespace lbm
