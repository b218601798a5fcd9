// TMA-staged fused step of the bump-function lattice Boltzmann method
// (arXiv 2501.00620, Sec. II.C) for D2Q9 / D3Q19 with FP32 or 16-bit
// population storage on sm_103a.  Same arithmetic as the generic kernel
// (lbm_site.cuh); only the data movement differs.
//
// A block owns a TX x TY tile (2D: a TX-wide strip) and marches along the
// slowest axis.  For the stage-1 plane q (pull + moments of the tile plus a
// one-site ring), population i is read from input plane q - e_i,march, so
// each (population, plane) slice is needed exactly once: one tiled bulk
// tensor copy per population per plane lands it in shared memory (double
// buffered, issued one plane ahead), and the variance planes q-1, q, q+1
// are kept in a four-slot ring, one new plane per step.  Every gather is a
// shared-memory load at a compile-time offset.  Copies complete on mbarrier
// transaction counts; every wait is bounded (time limit) and a timeout sets
// flag bit 2 and ends the block after draining its copies.
//
// Threads: one per tile site (stage 1 for its site, then stage 2), plus one
// per ring site (stage 1 only), rounded up to whole warps, so that stage 1
// takes a single pass in every warp and one block barrier per plane
// suffices (aux planes live in four slots).
//
// Slice geometry: x from x0 - PX (PX = 16 bytes / element size, so the copy
// starts on a 16-byte boundary) over TX + 2 PX columns; y (3D) from y0 - 2
// over TY + 4 rows.  At the domain edges the copy reads out of bounds
// (zero fill); edge blocks then patch the halo columns/rows that the pull
// reads with the periodic image or the fixed-state reservoir.
#pragma once

#include "lbm_site.cuh"
#include "lbm_tma.cuh"

namespace lbm {

template <int D, typename FS, int TX, int TY, int PF> struct TmaShape {
    using L = Lattice<D>;
    static constexpr int Q = L::Q, NB = L::NB, NAUX = D + NB;
    static constexpr int ESF = sizeof(FS);
    static constexpr int PXF = 16 / ESF;
    static constexpr int PXB = 4;
    static constexpr int SXF = TX + 2 * PXF;
    static constexpr int SXB = TX + 2 * PXB;
    static constexpr int SY = (D == 3) ? TY + 4 : 1;
    static constexpr int RX = TX + 2;
    static constexpr int RY = (D == 3) ? TY + 2 : 1;
    static constexpr int RS = RX * RY;
    static constexpr int NAP = round_up(NAUX, 2);                   // aux floats per site (site-major)
    static constexpr int NINT = TX * ((D == 3) ? TY : 1);            // tile sites
    static constexpr int NRING = RS - NINT;                          // ring sites
    static constexpr int NT = round_up(NINT + NRING, 32);            // threads
    static constexpr int FSLICE = SY * SXF;                         // elements of one population slice
    static constexpr int FPITCH = round_up(FSLICE * ESF, 128);      // bytes between population slices
    static constexpr int BSLICE = SY * SXB;                         // floats of one variance component
    static constexpr int BPITCH = round_up(NB * BSLICE * 4, 128);   // bytes between variance slots
    // PF planes of prefetch: population slots hold planes q .. q+PF, variance
    // slots planes q-1 .. q+1+PF, aux slots q-2 .. q+1
    static constexpr int NPS = PF + 1, NBS = PF + 3, NAS = 4;
    static constexpr int OFF_B = NPS * Q * FPITCH;
    static constexpr int OFF_AUX = OFF_B + NBS * BPITCH;
    static constexpr int OFF_RED = OFF_AUX + round_up(NAS * NAP * RS * 4, 16);
    static constexpr int OFF_BAR = OFF_RED + 32 * (D + 2) * 8;
    static constexpr int SMEM = OFF_BAR + (NPS + NBS) * 8;
    // resident blocks per SM the register budget aims for: what shared memory
    // allows, but leaving at least 96 registers per thread
    static constexpr int MINB_SMEM = (227 * 1024) / SMEM;
    static constexpr int MINB_REG = 65536 / (NT * 96);
    static constexpr int MINB = (MINB_SMEM < MINB_REG ? MINB_SMEM : MINB_REG) > 0
                                    ? (MINB_SMEM < MINB_REG ? MINB_SMEM : MINB_REG)
                                    : 1;
    static constexpr uint32_t FBYTES = Q * FSLICE * ESF;            // transaction bytes per population slot
    static constexpr uint32_t BBYTES = NB * BSLICE * 4;             // per variance slot
    static_assert(SXF <= 256 && SXB <= 256, "TMA box width is limited to 256 elements");
    static_assert(SY <= 256, "TMA box height is limited to 256 elements");
    static_assert(NT <= 1024, "too many threads");
};

// Per-block state of the march; every method is force-inlined so that the
// carried site values stay in registers.
template <int D, typename FS, int TX, int TY, int PF> struct TmaBlock {
    using L = Lattice<D>;
    using Sh = TmaShape<D, FS, TX, TY, PF>;
    using real = float;
    using real2 = float2;
    static constexpr int Q = L::Q, NB = L::NB, NAUX = Sh::NAUX, NAP = Sh::NAP;
    static constexpr int RX = Sh::RX, RS = Sh::RS;
    static constexpr int SXF = Sh::SXF, SXB = Sh::SXB, PXF = Sh::PXF, PXB = Sh::PXB, SY = Sh::SY;

    const TmaArgs& ta;
    const StepArgs& a;
    unsigned char* smem;
    int tid, x0, y0, nx, ny, np, p0, p1;
    bool xlo, xhi, ylo, yhi, edge;
    uint32_t pphase = 0, bphase = 0, p_pending = 0, b_pending = 0;
    bool timed_out = false;  // a wait of this thread gave up

    __device__ __forceinline__ TmaBlock(const TmaArgs& t, unsigned char* sm) : ta(t), a(t.s), smem(sm) {
        tid = threadIdx.x;
        x0 = blockIdx.x * TX;
        y0 = (D == 3) ? blockIdx.y * TY : 0;
        nx = a.nx;
        ny = a.ny;
        np = (D == 3) ? a.nz : a.ny;
        p0 = blockIdx.z * a.chunk;
        p1 = min(p0 + a.chunk, np);
        xlo = (x0 == 0);
        xhi = (x0 + TX == nx);
        ylo = (D == 3) && (y0 == 0);
        yhi = (D == 3) && (y0 + TY == ny);
        edge = xlo || xhi || ylo || yhi;
    }

    __device__ __forceinline__ FS* pslice(int ps, int i) const {
        return reinterpret_cast<FS*>(smem + (ps * Q + i) * Sh::FPITCH);
    }
    __device__ __forceinline__ float* bslot(int bs) const {
        return reinterpret_cast<float*>(smem + Sh::OFF_B + bs * Sh::BPITCH);
    }
    // aux planes are site-major: NAP floats per region site, (u0, rho b, pad),
    // so a neighbour's values are NAP/2 aligned 64-bit loads
    __device__ __forceinline__ real* aux(int q) const {
        return reinterpret_cast<real*>(smem + Sh::OFF_AUX) + ((q - p0 + 1) & 3) * NAP * RS;
    }
    __device__ __forceinline__ uint64_t* pbar() const { return reinterpret_cast<uint64_t*>(smem + Sh::OFF_BAR); }
    __device__ __forceinline__ uint64_t* bbar() const { return pbar() + Sh::NPS; }
    __device__ __forceinline__ int ps_of(int q) const { return (q - (p0 - 1)) % Sh::NPS; }
    __device__ __forceinline__ int bs_of(int q) const { return (q - (p0 - 2)) % Sh::NBS; }
    // q ranges over [p0 - 3, p1 + 1 + PF] with PF < np: one conditional add or
    // subtract wraps it
    __device__ __forceinline__ int wrapq(int q) const { return q < 0 ? q + np : (q >= np ? q - np : q); }
    static __device__ __forceinline__ int march(int i) { return (D == 3) ? L::e(i, 2) : L::e(i, 1); }

    // ---- producer (thread 0) ---------------------------------------------------
    __device__ __forceinline__ void issue_pops(int q) {
        const int ps = ps_of(q);
        mbar_arrive_expect_tx(pbar() + ps, Sh::FBYTES);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int plane = wrapq(q - march(i));
            if (D == 3)
                tma_load_4d(pslice(ps, i), &ta.fmap, pbar() + ps, x0 - PXF, y0 - 2, plane, i);
            else
                tma_load_3d(pslice(ps, i), &ta.fmap, pbar() + ps, x0 - PXF, plane, i);
        }
    }
    __device__ __forceinline__ void issue_b(int q) {
        const int bs = bs_of(q);
        mbar_arrive_expect_tx(bbar() + bs, Sh::BBYTES);
        const int plane = wrapq(q);
        if (D == 3)
            tma_load_4d(bslot(bs), &ta.bmap, bbar() + bs, x0 - PXB, y0 - 2, plane, 0);
        else
            tma_load_3d(bslot(bs), &ta.bmap, bbar() + bs, x0 - PXB, plane, 0);
    }

    // A wait that gives up leaves its slot pending with the same parity, so
    // that the drain waits for exactly that copy.
    __device__ __forceinline__ void wait_p(int q) {
        const int ps = ps_of(q);
        if (mbar_wait_bounded(pbar() + ps, (pphase >> ps) & 1u, kWaitLimit)) {
            pphase ^= 1u << ps;
            p_pending &= ~(1u << ps);
        } else {
            timed_out = true;
        }
    }
    __device__ __forceinline__ void wait_b(int q) {
        const int bs = bs_of(q);
        if (mbar_wait_bounded(bbar() + bs, (bphase >> bs) & 1u, kWaitLimit)) {
            bphase ^= 1u << bs;
            b_pending &= ~(1u << bs);
        } else {
            timed_out = true;
        }
    }
    __device__ __forceinline__ void drain() {
        for (int k = 0; k < Sh::NPS; ++k)
            if (p_pending & (1u << k)) mbar_wait_bounded(pbar() + k, (pphase >> k) & 1u, kWaitLimit);
        for (int k = 0; k < Sh::NBS; ++k)
            if (b_pending & (1u << k)) mbar_wait_bounded(bbar() + k, (bphase >> k) & 1u, kWaitLimit);
    }

    // ---- halo patches of edge blocks (after the copy has landed) ----------------
    // Positions the pull reads outside the domain: x in {-2,-1} / {nx,nx+1}
    // (all slice rows) and, in 3D, y in {-2,-1} / {ny,ny+1} (x from x0-2 to
    // x0+TX+1).
    __device__ __forceinline__ int halo_count() const {
        const int cx = (xlo ? 2 : 0) + (xhi ? 2 : 0);
        const int cy = (ylo ? 2 : 0) + (yhi ? 2 : 0);
        return cx * SY + cy * (TX + 4);
    }
    __device__ __forceinline__ void halo_pos(int k, int& gx, int& gy) const {
        const int cx = (xlo ? 2 : 0) + (xhi ? 2 : 0);
        if (k < cx * SY) {
            const int col = k / SY, row = k % SY;
            gx = (xlo && col < 2) ? -2 + col : nx + (col - (xlo ? 2 : 0));
            gy = (D == 3) ? y0 - 2 + row : 0;
        } else {
            k -= cx * SY;
            const int rr = k / (TX + 4), col = k % (TX + 4);
            gx = x0 - 2 + col;
            gy = (ylo && rr < 2) ? -2 + rr : ny + (rr - (ylo ? 2 : 0));
        }
    }
    __device__ __forceinline__ long long site_of(int wx, int wy, int plane) const {
        return (D == 3) ? wx + (long long)nx * (wy + (long long)ny * plane) : wx + (long long)nx * plane;
    }
    // The population loop is unrolled (compile-time velocity), the halo
    // positions are spread over the threads.
    __device__ __forceinline__ void patch_pops(int q) {
        const FS* __restrict__ fin = static_cast<const FS*>(a.fin);
        const real* __restrict__ gf = static_cast<const real*>(a.gf);
        const int ps = ps_of(q);
        const int cnt = halo_count();
        for (int k = tid; k < cnt; k += Sh::NT) {
            int gx, gy;
            halo_pos(k, gx, gy);
            const int sx = gx - (x0 - PXF), sy = (D == 3) ? gy - (y0 - 2) : 0;
            const int wy = (D == 3) ? (gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy)) : 0;
            const bool res = a.fixed_x && (gx < 0 || gx >= nx);
            const int wx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int plane = wrapq(q - march(i));
                FS v;
                if (res) {
                    const long long row = (D == 3) ? wy + (long long)ny * plane : plane;
                    v = FS(gf[((long long)(gx < 0 ? 0 : 1) * Q + i) * a.rows + row]);
                } else {
                    v = fin[(long long)i * a.N + site_of(wx, (D == 3) ? wy : plane, plane)];
                }
                pslice(ps, i)[sy * SXF + sx] = v;
            }
        }
        fence_proxy_async_smem();  // the slot is refilled by a bulk copy later
    }
    __device__ __forceinline__ void patch_b(int q) {
        const float* __restrict__ bin = static_cast<const float*>(a.bin);
        const real* __restrict__ gb = static_cast<const real*>(a.gb);
        const int bs = bs_of(q);
        const int plane = wrapq(q);
        const int cnt = halo_count();
        for (int k = tid; k < cnt; k += Sh::NT) {
            int gx, gy;
            halo_pos(k, gx, gy);
            const int sx = gx - (x0 - PXB), sy = (D == 3) ? gy - (y0 - 2) : 0;
            const int wy = (D == 3) ? (gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy)) : plane;
            const bool res = a.fixed_x && (gx < 0 || gx >= nx);
            const int wx = gx < 0 ? gx + nx : (gx >= nx ? gx - nx : gx);
            const long long row = (D == 3) ? wy + (long long)ny * plane : plane;
            const long long s = site_of(wx, wy, plane);
#pragma unroll
            for (int k2 = 0; k2 < NB; ++k2)
                bslot(bs)[k2 * Sh::BSLICE + sy * SXB + sx] =
                    res ? gb[((long long)(gx < 0 ? 0 : 1) * NB + k2) * a.rows + row] : bin[(long long)k2 * a.N + s];
        }
        fence_proxy_async_smem();
    }

    // ---- stage 1: pull + moments of region site (rx, ry) at plane q --------------
    // Returns false for a fixed-state reservoir site (aux written from the
    // reservoir, no site values).
    __device__ __forceinline__ bool stage1(int rx, int ry, int q, real* df, real* bt, real& rho, real* j,
                                           real& E) {
        const int gx = x0 - 1 + rx;
        const int r = rx + RX * ry;
        real* ax = aux(q);
        if (a.fixed_x && (gx < 0 || gx >= nx)) {
            const real* __restrict__ gaux = static_cast<const real*>(a.gaux);
            const int qq = wrapq(q);
            int gy = (D == 3) ? y0 - 1 + ry : qq;
            if (D == 3) gy = gy < 0 ? gy + ny : (gy >= ny ? gy - ny : gy);
            const long long row = (D == 3) ? gy + (long long)ny * qq : qq;
#pragma unroll
            for (int k = 0; k < NAUX; ++k)
                ax[r * NAP + k] = gaux[((long long)(gx < 0 ? 0 : 1) * NAUX + k) * a.rows + row];
            return false;
        }
        const FS* pbase = pslice(ps_of(q), 0) + ((D == 3) ? (ry + 1) * SXF : 0) + (rx - 1 + PXF);
        const int bo = ((D == 3) ? (ry + 1) * SXB : 0) + (rx - 1 + PXB);
        const float* bm = bslot(bs_of(q - 1)) + bo;
        const float* b0 = bslot(bs_of(q)) + bo;
        const float* bp = bslot(bs_of(q + 1)) + bo;
        real bsum[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k) bsum[k] = real(-0.0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int off = (D == 3) ? -L::e(i, 1) * SXF - L::e(i, 0) : -L::e(i, 0);
            const real v =
                real(*(reinterpret_cast<const FS*>(reinterpret_cast<const unsigned char*>(pbase) + i * Sh::FPITCH) +
                       off));
            const int offb = (D == 3) ? -L::e(i, 1) * SXB - L::e(i, 0) : -L::e(i, 0);
            const int m = march(i);
            const float* bsrc = (m == 1) ? bm : ((m == -1) ? bp : b0);
            df[i] = v;
            const real fi = real(L::w(i)) + v;
#pragma unroll
            for (int k = 0; k < NB; ++k) bsum[k] += fi * bsrc[k * Sh::BSLICE + offb];
        }
        real u0[D], rb[NB];
        site_moments<D, real>(df, bsum, real(a.omega), real(a.T0), a.thermal, bt, rho, j, E, u0, rb);
        real2* dst = reinterpret_cast<real2*>(ax + r * NAP);
        real vals[NAP];
#pragma unroll
        for (int c = 0; c < D; ++c) vals[c] = u0[c];
#pragma unroll
        for (int k = 0; k < NB; ++k) vals[D + k] = rb[k];
        if (NAP > NAUX) vals[NAP - 1] = real(0);
#pragma unroll
        for (int k = 0; k < NAP / 2; ++k) dst[k] = make_float2(vals[2 * k], vals[2 * k + 1]);
        return true;
    }

    // ---- stage 2: gradients, collision and store for tile site (tx, ty) at p ----
    __device__ __forceinline__ void stage2(int tx, int ty, int p, const real* c_df, const real* c_bt, real c_rho,
                                           const real* c_j, real c_E, DiagAcc<real, D + 2>& acc, int& bad) {
        const long long s = (D == 3) ? (x0 + tx) + (long long)nx * ((y0 + ty) + (long long)ny * p)
                                     : (x0 + tx) + (long long)nx * p;
        const int rc = ((tx + 1) + RX * ((D == 3) ? ty + 1 : 0)) * NAP;
        const real* am = aux(p - 1) + rc;
        const real* a0 = aux(p) + rc;
        const real* ap = aux(p + 1) + rc;
        real F[D], G[NB];
#pragma unroll
        for (int c = 0; c < D; ++c) F[c] = real(-0.0);
#pragma unroll
        for (int k = 0; k < NB; ++k) G[k] = real(-0.0);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int m = march(i);
            const real* as = (m == 1) ? ap : ((m == -1) ? am : a0);
            const int r = L::e(i, 0) + ((D == 3) ? RX * L::e(i, 1) : 0);
            const real2* src = reinterpret_cast<const real2*>(as + r * NAP);
            real vals[NAP];
#pragma unroll
            for (int k = 0; k < NAP / 2; ++k) {
                const real2 v2 = src[k];
                vals[2 * k] = v2.x;
                vals[2 * k + 1] = v2.y;
            }
            fd_add<D, real>(i, vals + D, vals, F, G);
        }
#pragma unroll
        for (int c = 0; c < D; ++c) F[c] *= real(-3);
#pragma unroll
        for (int k = 0; k < NB; ++k) G[k] *= real(-3);
        site_collide<D, FS, real>(a, s, c_df, c_bt, c_rho, c_j, c_E, F, G, acc, bad);
    }
};

template <int D, typename FS, int TX, int TY, int PF>
__global__ void __launch_bounds__(TmaShape<D, FS, TX, TY, PF>::NT, TmaShape<D, FS, TX, TY, PF>::MINB)
    step_tma_kernel(const __grid_constant__ TmaArgs ta) {
    using L = Lattice<D>;
    using Sh = TmaShape<D, FS, TX, TY, PF>;
    using real = float;
    constexpr int Q = L::Q, NB = L::NB;
    constexpr int NINT = Sh::NINT, NRING = Sh::NRING, NT = Sh::NT, RX = Sh::RX;

    extern __shared__ __align__(128) unsigned char smem[];
    TmaBlock<D, FS, TX, TY, PF> blk(ta, smem);
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int k = 0; k < Sh::NPS + Sh::NBS; ++k) mbar_init(blk.pbar() + k, 1);
        fence_barrier_init();
    }
    __syncthreads();

    // role of this thread: tile site (stage 1 + stage 2), ring site (stage 1)
    // or idle padding of the last warp
    const bool interior = tid < NINT;
    const bool ring = !interior && tid < NINT + NRING;
    int rx = 0, ry = 0, tx = 0, ty = 0;
    if (interior) {
        tx = tid % TX;
        ty = tid / TX;
        rx = tx + 1;
        ry = (D == 3) ? ty + 1 : 0;
    } else if (ring) {
        const int k = tid - NINT;
        if (D < 3) {
            rx = (k == 0) ? 0 : RX - 1;
        } else if (k < RX) {
            rx = k;
        } else if (k < 2 * RX) {
            rx = k - RX;
            ry = Sh::RY - 1;
        } else if (k < 2 * RX + TY) {
            ry = k - 2 * RX + 1;
        } else {
            rx = RX - 1;
            ry = k - 2 * RX - TY + 1;
        }
    }

    real c_df[Q], c_bt[NB], c_rho = real(1), c_j[D], c_E = real(0);
    real n_df[Q], n_bt[NB], n_rho = real(1), n_j[D], n_E = real(0);
    DiagAcc<real, D + 2> acc;
    int bad = 0;

    const int p0 = blk.p0, p1 = blk.p1;
    // prologue: variance planes p0-2 .. p0+PF-1, population planes p0-1 .. p0+PF-2
    for (int q = p0 - 2; q <= min(p0 + PF - 1, p1 + 1); ++q) {
        if (tid == 0) blk.issue_b(q);
        blk.b_pending |= 1u << blk.bs_of(q);
    }
    for (int q = p0 - 1; q <= min(p0 + PF - 2, p1); ++q) {
        if (tid == 0) blk.issue_pops(q);
        blk.p_pending |= 1u << blk.ps_of(q);
    }
    blk.wait_b(p0 - 2);
    blk.wait_b(p0 - 1);
    if (blk.edge) {
        blk.patch_b(p0 - 2);
        blk.patch_b(p0 - 1);
    }
    bool aborted = false;
    for (int q = p0 - 1; q <= p1; ++q) {
        if (tid == 0) {
            fence_proxy_async_smem();
            if (q + PF <= p1) blk.issue_pops(q + PF);
            if (q + 1 + PF <= p1 + 1) blk.issue_b(q + 1 + PF);
        }
        if (q + PF <= p1) blk.p_pending |= 1u << blk.ps_of(q + PF);
        if (q + 1 + PF <= p1 + 1) blk.b_pending |= 1u << blk.bs_of(q + 1 + PF);
        // each thread waits for the copies itself; the data is then visible
        // to it without a block barrier
        blk.wait_p(q);
        blk.wait_b(q + 1);
        if (blk.edge) {
            blk.patch_pops(q);
            blk.patch_b(q + 1);
            __syncthreads();
        }
        if (interior) {
            blk.stage1(rx, ry, q, n_df, n_bt, n_rho, n_j, n_E);
        } else if (ring) {
            real d_df[Q], d_bt[NB], d_rho, d_j[D], d_E;
            blk.stage1(rx, ry, q, d_df, d_bt, d_rho, d_j, d_E);
        }
        // The one barrier per plane: the aux of plane q is complete, and all
        // reads of the population slot of q and the variance slot of q-1 are
        // done, so thread 0 may refill them in the next iteration.  It also
        // tells every thread at once whether any wait gave up.
        if (__syncthreads_or(blk.timed_out)) {
            aborted = true;
            break;
        }
        if (interior && q - 1 >= p0) blk.stage2(tx, ty, q - 1, c_df, c_bt, c_rho, c_j, c_E, acc, bad);
#pragma unroll
        for (int i = 0; i < Q; ++i) c_df[i] = n_df[i];
#pragma unroll
        for (int k = 0; k < NB; ++k) c_bt[k] = n_bt[k];
        c_rho = n_rho;
#pragma unroll
        for (int c = 0; c < D; ++c) c_j[c] = n_j[c];
        c_E = n_E;
    }
    if (aborted) {
        // drain this block's copies still in flight, then leave
        if (tid == 0) {
            atomicOr(ta.s.flag, 4);
            blk.drain();
        }
        return;
    }
    if (bad) atomicOr(ta.s.flag, bad);
    if (ta.s.want_diag)
        block_diagnostics<D, NT>(ta.s, acc, reinterpret_cast<double*>(smem + Sh::OFF_RED));
}

}  // namespace lbm
