// Many time steps of the bump-function lattice Boltzmann method (arXiv
// 2501.00620, Sec. II.C) per launch for small periodic D2Q9 lattices, with
// the whole state resident in the shared memory of ONE thread-block cluster.
//
// A lattice of at most a few tens of thousands of sites is too small to fill
// the GPU, and its step takes about as long as a launch and the march of a
// block through its planes: the time goes to latency, not to bandwidth.  Here
// the C blocks of one cluster (one block per SM, C <= 16) each hold a band of
// rows of the lattice -- both A-B population buffers, both variance buffers
// and the (u0, rho b) aux values -- and step it K times without touching
// global memory between the first load and the last store.  A site whose
// neighbour row lies in another block's band reads it through distributed
// shared memory (the neighbour block's shared memory mapped into the cluster
// window).
//
// One step is two passes separated by cluster barriers:
//   pass 1: pull (Eq. 49), mass-weighted variance transport (Eq. 66),
//           moments and rho b (Eqs. 56-57, 67-68) of every site of the band;
//           (u0, rho b) into the aux slots;
//   pass 2: the gradients F, G from the neighbours' aux values (Eqs. 59,
//           61), collision (Eq. 55, Appendix A) into the other buffers,
//           diagnostics of the state at t.  Where a block has a thread for
//           every site of its band, the site's pulled populations and
//           moments stay in registers from pass 1; otherwise pass 2 pulls,
//           transports and takes the moments again (reads of shared memory).
// The arithmetic is that of the other kernels (lbm_site.cuh).  Every thread
// of every block reaches every cluster barrier (no early exit), and a barrier
// follows the last read of another block's shared memory, so no block leaves
// while another may still read its memory.
#pragma once

#include <cooperative_groups.h>

#include "lbm_site.cuh"

namespace lbm {

// Rows of the lattice held by each block: the first `extra` blocks hold
// base + 1 rows, the others base (base >= 1).
struct ClusterBands {
    int base, extra;
    __host__ __device__ __forceinline__ int y0(int r) const { return r * base + (r < extra ? r : extra); }
    __host__ __device__ __forceinline__ int rows(int r) const { return base + (r < extra ? 1 : 0); }
    __device__ __forceinline__ int owner(int y) const {
        const int cut = extra * (base + 1);
        return y < cut ? y / (base + 1) : extra + (y - cut) / base;
    }
};

// Shared-memory layout of a block, in storage words of P sites per plane
// (P = the largest band's site count, the same in every block so that a
// remote band is addressed like the local one):
//   [0, Q P) populations, parity 0; [Q P, 2Q P) parity 1;
//   [2Q P, (2Q + NB) P) variance, parity 0; then parity 1;
//   then NA = D + NB aux planes (u0, rho b); then the FP64 reduction slots.
template <typename FS> struct ClusterShape {
    static constexpr int Q = 9, NB = 3, NA = 2 + NB;
    static constexpr int WORDS = 2 * Q + 2 * NB + NA;
    __host__ __device__ static constexpr size_t red_offset(int P) {
        return ((size_t)P * WORDS * sizeof(FS) + 15) / 16 * 16;
    }
    // reduction slots (doubles): [0, 64) per-warp sums; [64, 68) the band's
    // sums; [68, 132) block 0's copies of every band's sums
    static constexpr int RED_BAND = 64, RED_ALL = 68, RED_N = 132;
    __host__ __device__ static constexpr size_t smem(int P) { return red_offset(P) + RED_N * sizeof(double); }
};

// Pull, variance transport and moments of site (x, y) from the buffers of one
// parity: frow/brow[d] point at plane 0 of row y - 1 + d in the block that
// holds it.
template <typename FS>
__device__ __forceinline__ void cluster_site(const StepArgs& a, int P, int x, int nx, const FS* const* frow,
                                             const FS* const* brow, FS* df, FS* bt, FS& rho, FS* j, FS& E, FS* u0,
                                             FS* rb) {
    using L = Lattice<2>;
    constexpr int Q = L::Q, NB = L::NB;
    FS bsum[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) bsum[k] = FS(-0.0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int ex = L::e(i, 0), ey = L::e(i, 1);
        int xs = x - ex;  // the emitter of f_i(x) is x - e_i
        xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
        const FS v = frow[1 - ey][i * P + xs];
        df[i] = v;
        const FS fi = FS(L::w(i)) + v;
#pragma unroll
        for (int k = 0; k < NB; ++k) bsum[k] += fi * brow[1 - ey][k * P + xs];
    }
    FS omega, tau, T0;
    step_params(a, omega, tau, T0);
    (void)tau;
    site_moments<2, FS>(df, bsum, omega, T0, a.thermal, bt, rho, j, E, u0, rb);
}

// The diagnostics record of step number st, by the last warp of block 0 (the
// warp with the fewest sites) while the bands' sums are stable (between the
// barrier that ends a step and the one that ends the next step's first
// pass): lane r copies block r's four sums (distributed shared memory), then
// lane k adds value k over the blocks in rank order and writes it to the
// history record and diag_out.  The step counter lives in a register of this
// warp for the whole launch (no global read per step).
template <typename FS>
__device__ __forceinline__ void cluster_record(const StepArgs& a, cooperative_groups::cluster_group& cl, double* red,
                                               int nblocks, int lane, long long st) {
    using Sh = ClusterShape<FS>;
    if (lane < nblocks) {
        const double* v = cl.map_shared_rank(red, lane) + Sh::RED_BAND;
        const double v0 = v[0], v1 = v[1], v2 = v[2], v3 = v[3];
        double* o = red + Sh::RED_ALL + 4 * lane;
        o[0] = v0, o[1] = v1, o[2] = v2, o[3] = v3;
    }
    __syncwarp();
    if (lane < 4) {
        double tot = 0.0;
        for (int r = 0; r < nblocks; ++r) tot += red[Sh::RED_ALL + 4 * r + lane];
        if (a.diag_out) a.diag_out[lane] = tot;
        if (a.hist) {
            double* rec = a.hist + (st % a.hist_cap) * 5;
            if (lane == 0) rec[0] = double(st);
            rec[1 + lane] = tot;
        }
    }
    __syncwarp();
}

// Plane-0 address of row y (periodic) in the block of the cluster that holds
// it (distributed shared memory; the own block's memory through the same
// window).
template <typename FS>
__device__ __forceinline__ const FS* cluster_row(cooperative_groups::cluster_group& cl, FS* sm,
                                                 const ClusterBands& bands, int y, int ny, int nx) {
    y = y < 0 ? y + ny : (y >= ny ? y - ny : y);
    const int r = bands.owner(y);
    return cl.map_shared_rank(sm, r) + (size_t)(y - bands.y0(r)) * nx;
}

// a0 / a1: step arguments of the two parities (a0 reads the buffers that hold
// the state at the start).  K steps; the state after them is stored into the
// global buffers of parity K % 2.  Diagnostics: each block reduces its band
// (fixed order), block 0 sums the blocks' values in rank order through
// distributed shared memory and writes the step's history record.
template <typename FS, int NT>
__global__ void __launch_bounds__(NT, 1)
    step_cluster_kernel(const StepArgs a0, const StepArgs a1, int K, int P, ClusterBands bands) {
    namespace cg = cooperative_groups;
    using L = Lattice<2>;
    using Sh = ClusterShape<FS>;
    constexpr int Q = L::Q, NB = L::NB;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FS* sm = reinterpret_cast<FS*>(smem_raw);
    double* red = reinterpret_cast<double*>(smem_raw + Sh::red_offset(P));
    cg::cluster_group cl = cg::this_cluster();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int rank = (int)cl.block_rank();
    const int nx = a0.nx, ny = a0.ny;
    const long long N = a0.N;
    const int y0 = bands.y0(rank);
    const int S = bands.rows(rank) * nx;  // sites of this block's band
    const long long g0 = (long long)y0 * nx;
    const size_t OFF_B = (size_t)2 * Q * P, OFF_A = OFF_B + (size_t)2 * NB * P;
    // one site per thread (the band fits the block): its coordinates, row
    // addresses and stage-1 values are kept across the passes
    const bool one = S <= NT;
    const bool mine = tid < S;

    // the band's state at t (parity 0 buffers); each block reads only its own
    // rows of the global buffers
    {
        const FS* __restrict__ fin = static_cast<const FS*>(a0.fin);
        const FS* __restrict__ bin = static_cast<const FS*>(a0.bin);
        for (int i = 0; i < Q; ++i)
            for (int s = tid; s < S; s += NT) sm[(size_t)i * P + s] = fin[i * N + g0 + s];
        for (int k = 0; k < NB; ++k)
            for (int s = tid; s < S; s += NT) sm[OFF_B + (size_t)k * P + s] = bin[k * N + g0 + s];
    }
    // every block has started and loaded its band before any remote read
    cl.sync();
    // the history index of the first step (read once; block 0's last warp
    // keeps the count and writes it back after the last step)
    const long long st0 = (a0.want_diag && rank == 0 && warp == NT / 32 - 1) ? *a0.step_ctr : 0;

    int x1 = 0;
    const FS* row1[3] = {sm, sm, sm};
    if (one && mine) {
        x1 = tid % nx;
        const int y = y0 + tid / nx;
#pragma unroll
        for (int d = 0; d < 3; ++d) row1[d] = cluster_row(cl, sm, bands, y - 1 + d, ny, nx);
    }
    FS kdf[Q], kbt[NB], krho = FS(1), kj[2], kE = FS(0);
#pragma unroll
    for (int i = 0; i < Q; ++i) kdf[i] = FS(0);
#pragma unroll
    for (int k = 0; k < NB; ++k) kbt[k] = FS(0);
    kj[0] = kj[1] = FS(0);

    int bad = 0;
    for (int step = 0; step < K; ++step) {
        const int cur = step & 1;
        const StepArgs& a = cur ? a1 : a0;
        const size_t fc = (size_t)cur * Q * P, bc = OFF_B + (size_t)cur * NB * P;
        // the previous step's diagnostics: block 0 sums the bands' values
        if (step > 0 && a.want_diag && rank == 0 && warp == NT / 32 - 1)
            cluster_record<FS>(a, cl, red, (int)cl.num_blocks(), lane, st0 + step - 1);
        // pass 1: (u0, rho b) of every site of the band
        for (int s = tid; s < S; s += NT) {
            int x;
            const FS* row[3];
            if (one) {
                x = x1;
#pragma unroll
                for (int d = 0; d < 3; ++d) row[d] = row1[d];
            } else {
                x = s % nx;
                const int y = y0 + s / nx;
#pragma unroll
                for (int d = 0; d < 3; ++d) row[d] = cluster_row(cl, sm, bands, y - 1 + d, ny, nx);
            }
            const FS* frow[3] = {row[0] + fc, row[1] + fc, row[2] + fc};
            const FS* brow[3] = {row[0] + bc, row[1] + bc, row[2] + bc};
            FS u0[2], rb[NB];
            cluster_site<FS>(a, P, x, nx, frow, brow, kdf, kbt, krho, kj, kE, u0, rb);
#pragma unroll
            for (int c = 0; c < 2; ++c) sm[OFF_A + (size_t)c * P + s] = u0[c];
#pragma unroll
            for (int k = 0; k < NB; ++k) sm[OFF_A + (size_t)(2 + k) * P + s] = rb[k];
        }
        cl.sync();  // the aux values of every band are complete
        // pass 2: gradients, collision, store into the other parity
        StepArgs la = a;
        la.fout = sm + (size_t)(1 - cur) * Q * P;
        la.bout = sm + OFF_B + (size_t)(1 - cur) * NB * P;
        la.N = P;
        la.mout = nullptr;
        la.write_state = 1;
        DiagAcc<FS, 4> acc;
        for (int s = tid; s < S; s += NT) {
            int x;
            const FS* row[3];
            if (one) {
                x = x1;
#pragma unroll
                for (int d = 0; d < 3; ++d) row[d] = row1[d];
            } else {
                x = s % nx;
                const int y = y0 + s / nx;
#pragma unroll
                for (int d = 0; d < 3; ++d) row[d] = cluster_row(cl, sm, bands, y - 1 + d, ny, nx);
                // several sites per thread: pull, transport and moments again
                const FS* frow[3] = {row[0] + fc, row[1] + fc, row[2] + fc};
                const FS* brow[3] = {row[0] + bc, row[1] + bc, row[2] + bc};
                FS u0[2], rb[NB];
                cluster_site<FS>(a, P, x, nx, frow, brow, kdf, kbt, krho, kj, kE, u0, rb);
            }
            FS F[2], G[NB];
#pragma unroll
            for (int c = 0; c < 2; ++c) F[c] = FS(-0.0);
#pragma unroll
            for (int k = 0; k < NB; ++k) G[k] = FS(-0.0);
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const int ex = L::e(i, 0), ey = L::e(i, 1);
                int xn = x + ex;  // the neighbour x + e_i
                xn = xn < 0 ? xn + nx : (xn >= nx ? xn - nx : xn);
                const FS* ar = row[1 + ey] + OFF_A;
                FS rbn[NB], un[2];
#pragma unroll
                for (int k = 0; k < NB; ++k) rbn[k] = ar[(size_t)(2 + k) * P + xn];
#pragma unroll
                for (int c = 0; c < 2; ++c) un[c] = ar[(size_t)c * P + xn];
                fd_add<2, FS>(i, rbn, un, F, G);
            }
#pragma unroll
            for (int c = 0; c < 2; ++c) F[c] *= FS(-3);
#pragma unroll
            for (int k = 0; k < NB; ++k) G[k] *= FS(-3);
            site_collide<2, FS, FS, int, DiagAcc<FS, 4>>(la, s, kdf, kbt, krho, kj, kE, F, G, acc, bad);
        }
        if (a.want_diag) {
            // the band's sums in a fixed order: lanes (float-float pairs for
            // FP32 arithmetic), then warps
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if constexpr (DiagAcc<FS, 4>::kFF) {
                    float h, l;
                    acc.ff(k, h, l);
                    ff_warp_sum(h, l);
                    if (lane == 0) reinterpret_cast<float2*>(red)[warp * 4 + k] = make_float2(h, l);
                } else {
                    double v = acc.get(k);
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                    if (lane == 0) red[warp * 4 + k] = v;
                }
            }
            __syncthreads();
            if constexpr (DiagAcc<FS, 4>::kFF) {
                // the warps' pairs through the same tree in warp 0
                if (warp == 0) {
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const float2 p = lane < NT / 32 ? reinterpret_cast<const float2*>(red)[lane * 4 + k]
                                                        : make_float2(0.0f, 0.0f);
                        float h = p.x, l = p.y;
                        ff_warp_sum(h, l);
                        if (lane == 0) red[Sh::RED_BAND + k] = double(h) + double(l);
                    }
                }
            } else if (tid < 4) {
                double v = 0.0;
                for (int w = 0; w < NT / 32; ++w) v += red[w * 4 + tid];
                red[Sh::RED_BAND + tid] = v;
            }
        }
        // the new state and the band sums are complete, and every read of the
        // old state and of the aux values is done, before the next step
        cl.sync();
    }
    if (K > 0 && a0.want_diag && rank == 0 && warp == NT / 32 - 1) {
        cluster_record<FS>((K & 1) ? a0 : a1, cl, red, (int)cl.num_blocks(), lane, st0 + K - 1);
        if (lane == 0 && a0.write_state) *a0.step_ctr = st0 + K;
    }
    // block 0 has read every band's sums before any block leaves
    cl.sync();

    // the state after K steps: into the global buffers of parity K % 2
    {
        FS* __restrict__ fo = static_cast<FS*>((K & 1) ? a0.fout : const_cast<void*>(a0.fin));
        FS* __restrict__ bo = static_cast<FS*>((K & 1) ? a0.bout : const_cast<void*>(a0.bin));
        const size_t fr = (size_t)(K & 1) * Q * P, br = OFF_B + (size_t)(K & 1) * NB * P;
        for (int i = 0; i < Q; ++i)
            for (int s = tid; s < S; s += NT) fo[i * N + g0 + s] = sm[fr + (size_t)i * P + s];
        for (int k = 0; k < NB; ++k)
            for (int s = tid; s < S; s += NT) bo[k * N + g0 + s] = sm[br + (size_t)k * P + s];
    }
    if (bad) atomicOr(a0.flag, bad);
}

}  // namespace lbm
