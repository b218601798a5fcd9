// Fused step of the bump-function lattice Boltzmann method (arXiv 2501.00620,
// Sec. II.C) for D2Q9 / D3Q19 with FP32 or 16-bit population storage, laid
// out for occupancy on sm_103a.  The per-site arithmetic is the one of the
// other step kernels (lbm_site.cuh); only the data movement differs.
//
// * Populations are pulled straight from global memory (read-only path).
//   The pull is a permutation -- every emitted value is read by exactly one
//   site -- so staging them in shared memory buys no reuse; leaving them out
//   frees shared memory for more resident blocks.
// * The variance planes, which the mass-weighted transport (Eq. 66) reads at
//   all Q neighbours, are staged by tiled bulk tensor copies (TMA) in a ring
//   of 3 + PFB plane slots.  The copy of plane q+2+PFB is issued right after
//   the block barrier that frees its slot, so it lands while stage 2 runs.
// * (u0, rho b) of the tile plus a one-site ring live in four shared plane
//   slots (stage 1 writes plane q; stage 2 of plane q-1 reads q-2 .. q), so
//   one block barrier per plane suffices.
// * A tile site hands (bbar, rho, j0, Ebar) from stage 1 to stage 2 through
//   its own column of two shared slots (plane parity) and pulls its
//   populations a second time in stage 2 (cache hits); nothing is carried in
//   registers across the barrier, which keeps MB blocks per SM resident.
//
// A block owns a TX x TY tile (2D: a TX-wide strip) and marches along the
// slowest axis (z in 3D, y in 2D) over `chunk` planes.  Threads: one per tile
// site (stage 1, then stage 2 one plane later) plus one per ring site (stage 1
// only), rounded up to whole warps.  FX selects the fixed-state boundary in x
// (frozen equilibrium reservoirs); otherwise every axis is periodic.
#pragma once

#include "lbm_site.cuh"
#include "lbm_tma.cuh"

namespace lbm {

template <int D, typename FS, int TX, int TY, int PFB, int MB> struct FastShape {
    using L = Lattice<D>;
    static constexpr int Q = L::Q, NB = L::NB, NAUX = D + NB;
    static constexpr int PXB = 4;                                   // 16-byte aligned x start of a b copy
    static constexpr int SXB = TX + 2 * PXB;
    static constexpr int SY = (D == 3) ? TY + 4 : 1;
    static constexpr int RX = TX + 2;
    static constexpr int RY = (D == 3) ? TY + 2 : 1;
    static constexpr int RS = RX * RY;
    static constexpr int NAP = round_up(NAUX, 2);                   // aux floats per site (site-major)
    static constexpr int NINT = TX * ((D == 3) ? TY : 1);
    static constexpr int NRING = RS - NINT;
    static constexpr int NT = round_up(NINT + NRING, 32);
    static constexpr int BSLICE = SY * SXB;                         // floats of one variance component
    static constexpr int BPITCH = round_up(NB * BSLICE * 4, 128);   // bytes between variance slots
    static constexpr int NBS = 3 + PFB, NAS = 4;
    static constexpr int NSV = NB + D + 2;                          // carried site values: bbar, rho, j0, Ebar
    static constexpr int OFF_AUX = NBS * BPITCH;
    static constexpr int OFF_SV = OFF_AUX + round_up(NAS * NAP * RS * 4, 16);
    static constexpr int OFF_RED = OFF_SV + 2 * NSV * NINT * 4;
    static constexpr int OFF_BAR = OFF_RED + 32 * (D + 2) * 8;
    static constexpr int SMEM = OFF_BAR + NBS * 8;
    static constexpr uint32_t BBYTES = NB * BSLICE * 4;             // transaction bytes per variance slot
    static_assert(SXB <= 256 && SY <= 256, "TMA box edges are limited to 256 elements");
    static_assert(NT <= 1024, "too many threads");
    static_assert(MB * (SMEM + 1024) <= 228 * 1024, "MB blocks do not fit in shared memory");
};

template <int D, typename FS, int TX, int TY, int PFB, int MB, bool FX> struct FastBlock {
    using L = Lattice<D>;
    using Sh = FastShape<D, FS, TX, TY, PFB, MB>;
    using real = float;
    using real2 = float2;
    static constexpr int Q = L::Q, NB = L::NB, NAUX = Sh::NAUX, NAP = Sh::NAP;
    static constexpr int RX = Sh::RX, RS = Sh::RS, SXB = Sh::SXB, PXB = Sh::PXB, SY = Sh::SY;

    const TmaArgs& ta;
    const StepArgs& a;
    unsigned char* smem;
    int tid, x0, y0, nx, ny, np, p0, p1, pstride;
    bool xlo, xhi, ylo, yhi, edge;
    uint32_t bphase = 0, b_pending = 0;
    bool timed_out = false;  // a wait of this thread gave up
    // this thread's region site: wrapped coordinates and source offsets
    int rx = 0, ry = 0, gxw = 0, gyw = 0;
    int xs[3], ys[3];    // x and y*nx of the sources x - e, y - e for e = -1, 0, 1
    int xo = 0;          // FX: bit e+1 set if source column x - e lies outside [0, nx)
    bool reservoir = false;

    __device__ __forceinline__ FastBlock(const TmaArgs& t, unsigned char* sm) : ta(t), a(t.s), smem(sm) {
        tid = threadIdx.x;
        x0 = blockIdx.x * TX;
        y0 = (D == 3) ? blockIdx.y * TY : 0;
        nx = a.nx;
        ny = a.ny;
        np = (D == 3) ? a.nz : a.ny;
        pstride = (D == 3) ? nx * ny : nx;
        p0 = blockIdx.z * a.chunk;
        p1 = min(p0 + a.chunk, np);
        xlo = (x0 == 0);
        xhi = (x0 + TX == nx);
        ylo = (D == 3) && (y0 == 0);
        yhi = (D == 3) && (y0 + TY == ny);
        edge = xlo || xhi || ylo || yhi;
    }

    static __device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
    // q ranges over [p0 - 3, p1 + 2 + PFB] with PFB + 3 <= np: one conditional add or subtract wraps it
    __device__ __forceinline__ int wrapq(int q) const { return wrap(q, np); }
    static __device__ __forceinline__ int march(int i) { return (D == 3) ? L::e(i, 2) : L::e(i, 1); }

    __device__ __forceinline__ float* bslot(int bs) const {
        return reinterpret_cast<float*>(smem + bs * Sh::BPITCH);
    }
    __device__ __forceinline__ real* aux(int q) const {
        return reinterpret_cast<real*>(smem + Sh::OFF_AUX) + ((q - p0 + 1) & 3) * NAP * RS;
    }
    __device__ __forceinline__ uint64_t* bbar() const { return reinterpret_cast<uint64_t*>(smem + Sh::OFF_BAR); }
    // site values of plane q for tile site t: component k at [k * NINT + t]
    __device__ __forceinline__ real* sv(int q) const {
        return reinterpret_cast<real*>(smem + Sh::OFF_SV) + (q & 1) * Sh::NSV * Sh::NINT + tid;
    }
    __device__ __forceinline__ int bs_of(int q) const { return (q - (p0 - 2)) % Sh::NBS; }

    // Region site (rx, ry) of this thread: x from x0 - 1, y from y0 - 1.
    __device__ __forceinline__ void set_site(int rx_, int ry_) {
        rx = rx_;
        ry = ry_;
        const int gx = x0 - 1 + rx;
        reservoir = FX && (gx < 0 || gx >= nx);
        gxw = wrap(gx, nx);
#pragma unroll
        for (int e = -1; e <= 1; ++e) {
            const int sx = gxw - e;
            xs[e + 1] = wrap(sx, nx);
            if (FX && (sx < 0 || sx >= nx)) xo |= 1 << (e + 1);
        }
        gyw = (D == 3) ? wrap(y0 - 1 + ry, ny) : 0;
#pragma unroll
        for (int e = -1; e <= 1; ++e) ys[e + 1] = (D == 3) ? wrap(gyw - e, ny) * nx : 0;
    }
    // Offsets of the source planes q - e (e = -1, 0, 1) along the march axis.
    __device__ __forceinline__ void planes(int q, int* zs) const {
#pragma unroll
        for (int e = -1; e <= 1; ++e) zs[e + 1] = wrapq(q - e) * pstride;
    }

    // Pull: df_i = stored deviation of fbar*_i at (x - e_i) (Eq. 49).
    __device__ __forceinline__ void pull(int q, const int* zs, real* df) const {
        const FS* __restrict__ fin = static_cast<const FS*>(a.fin);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int ex = L::e(i, 0), ey = L::e(i, 1), ez = L::e(i, 2);
            const int m = march(i);
            const int sidx = xs[ex + 1] + ((D == 3) ? ys[ey + 1] : 0) + zs[m + 1];
            if (FX && ex != 0 && (xo & (1 << (ex + 1)))) {
                const real* __restrict__ gf = static_cast<const real*>(a.gf);
                const long long row = (D == 3) ? (long long)wrap(gyw - ey, ny) + (long long)ny * wrapq(q - ez)
                                               : (long long)wrapq(q - ey);
                df[i] = gf[((long long)(ex > 0 ? 0 : 1) * Q + i) * a.rows + row];
            } else {
                df[i] = Store<FS>::ld(fin, (long long)i * a.N + sidx);
            }
        }
    }

    // ---- variance copies (thread 0 issues; every thread waits itself) --------
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
        for (int k = 0; k < Sh::NBS; ++k)
            if (b_pending & (1u << k)) mbar_wait_bounded(bbar() + k, (bphase >> k) & 1u, kWaitLimit);
    }

    // ---- halo patch of the variance slot in edge blocks ------------------------
    // The copy reads out of bounds (zero fill) at the domain edges; the
    // transport reads x in {-2,-1} / {nx,nx+1} (all slice rows) and, in 3D,
    // y in {-2,-1} / {ny,ny+1} (x from x0-2 to x0+TX+1): those positions get
    // the periodic image or the fixed-state reservoir.
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
    __device__ __forceinline__ void patch_b(int q) {
        const float* __restrict__ bin = static_cast<const float*>(a.bin);
        const real* __restrict__ gb = static_cast<const real*>(a.gb);
        float* slot = bslot(bs_of(q));
        const int plane = wrapq(q);
        const int cnt = halo_count();
        for (int k = tid; k < cnt; k += Sh::NT) {
            int gx, gy;
            halo_pos(k, gx, gy);
            const int sx = gx - (x0 - PXB), sy = (D == 3) ? gy - (y0 - 2) : 0;
            const int wy = (D == 3) ? wrap(gy, ny) : plane;
            const int wx = wrap(gx, nx);
            const long long row = (D == 3) ? wy + (long long)ny * plane : plane;
            const long long s = (D == 3) ? wx + (long long)nx * row : wx + (long long)nx * plane;
            const bool res = FX && (gx < 0 || gx >= nx);
#pragma unroll
            for (int k2 = 0; k2 < NB; ++k2)
                slot[k2 * Sh::BSLICE + sy * SXB + sx] =
                    res ? gb[((long long)(gx < 0 ? 0 : 1) * NB + k2) * a.rows + row] : bin[(long long)k2 * a.N + s];
        }
        fence_proxy_async_smem();  // the slot is refilled by a bulk copy later
    }

    // ---- stage 1: pull + moments of this thread's region site at plane q -------
    // Writes (u0, rho b) to the aux plane q; returns the site values for a tile
    // site.  A fixed-state reservoir site writes the reservoir's aux instead.
    __device__ __forceinline__ void stage1(int q, const int* zs, bool tile) {
        real* ax = aux(q) + (rx + RX * ry) * NAP;
        if (FX && reservoir) {
            const real* __restrict__ gaux = static_cast<const real*>(a.gaux);
            const int qq = wrapq(q);
            const long long row = (D == 3) ? gyw + (long long)ny * qq : qq;
            const int side = (x0 - 1 + rx) < 0 ? 0 : 1;
#pragma unroll
            for (int k = 0; k < NAUX; ++k) ax[k] = gaux[((long long)side * NAUX + k) * a.rows + row];
            return;
        }
        real df[Q];
        pull(q, zs, df);
        const int bo = ((D == 3) ? (ry + 1) * SXB : 0) + (rx - 1 + PXB);
        const float* bm = bslot(bs_of(q - 1)) + bo;
        const float* b0 = bslot(bs_of(q)) + bo;
        const float* bp = bslot(bs_of(q + 1)) + bo;
        real bsum[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k) bsum[k] = real(-0.0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int offb = (D == 3) ? -L::e(i, 1) * SXB - L::e(i, 0) : -L::e(i, 0);
            const int m = march(i);
            const float* bsrc = (m == 1) ? bm : ((m == -1) ? bp : b0);
            const real fi = real(L::w(i)) + df[i];
#pragma unroll
            for (int k = 0; k < NB; ++k) bsum[k] += fi * bsrc[k * Sh::BSLICE + offb];
        }
        real u0[D], rb[NB], bt[NB], rho, j[D], E;
        real omega, tau, T0;
        step_params(a, omega, tau, T0);
        site_moments<D, real>(df, bsum, omega, T0, a.thermal, bt, rho, j, E, u0, rb);
        if (tile) {
            real* v = sv(q);
            constexpr int NI = Sh::NINT;
#pragma unroll
            for (int k = 0; k < NB; ++k) v[k * NI] = bt[k];
            v[NB * NI] = rho;
#pragma unroll
            for (int c = 0; c < D; ++c) v[(NB + 1 + c) * NI] = j[c];
            v[(NB + 1 + D) * NI] = E;
        }
        real vals[NAP];
#pragma unroll
        for (int c = 0; c < D; ++c) vals[c] = u0[c];
#pragma unroll
        for (int k = 0; k < NB; ++k) vals[D + k] = rb[k];
        if (NAP > NAUX) vals[NAP - 1] = real(0);
        real2* dst = reinterpret_cast<real2*>(ax);
#pragma unroll
        for (int k = 0; k < NAP / 2; ++k) dst[k] = make_float2(vals[2 * k], vals[2 * k + 1]);
    }

    // ---- stage 2: gradients, collision and store of this tile site at plane p ----
    __device__ __forceinline__ void stage2(int p, const int* zsp, DiagAcc<real, D + 2>& acc, int& bad) {
        const long long s = (long long)xs[1] + ((D == 3) ? ys[1] : 0) + zsp[1];
        const int rc = (rx + RX * ry) * NAP;
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
        const real* v = sv(p);
        constexpr int NI = Sh::NINT;
        real c_bt[NB], c_j[D];
#pragma unroll
        for (int k = 0; k < NB; ++k) c_bt[k] = v[k * NI];
        const real c_rho = v[NB * NI];
#pragma unroll
        for (int c = 0; c < D; ++c) c_j[c] = v[(NB + 1 + c) * NI];
        const real c_E = v[(NB + 1 + D) * NI];
        real df[Q];
        pull(p, zsp, df);  // second pull of the same values: cache hits
        site_collide<D, FS, real>(a, s, df, c_bt, c_rho, c_j, c_E, F, G, acc, bad);
    }
};

template <int D, typename FS, int TX, int TY, int PFB, int MB, bool FX>
__global__ void __launch_bounds__(FastShape<D, FS, TX, TY, PFB, MB>::NT, MB)
    step_fast_kernel(const __grid_constant__ TmaArgs ta) {
    using Sh = FastShape<D, FS, TX, TY, PFB, MB>;
    constexpr int NINT = Sh::NINT, NRING = Sh::NRING, NT = Sh::NT, RX = Sh::RX;

    extern __shared__ __align__(128) unsigned char smem[];
    FastBlock<D, FS, TX, TY, PFB, MB, FX> blk(ta, smem);
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int k = 0; k < Sh::NBS; ++k) mbar_init(blk.bbar() + k, 1);
        fence_barrier_init();
    }
    __syncthreads();

    // role of this thread: tile site (stage 1 + stage 2), ring site (stage 1)
    // or idle padding of the last warp
    const bool interior = tid < NINT;
    const bool ring = !interior && tid < NINT + NRING;
    int rx = 0, ry = 0;
    if (interior) {
        rx = tid % TX + 1;
        ry = (D == 3) ? tid / TX + 1 : 0;
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
    blk.set_site(rx, ry);

    DiagAcc<float, D + 2> acc;
    int bad = 0;

    const int p0 = blk.p0, p1 = blk.p1;
    // prologue: variance planes p0-2 .. p0+PFB (the slots' first fill)
    for (int q = p0 - 2; q <= min(p0 + PFB, p1 + 1); ++q) {
        if (tid == 0) blk.issue_b(q);
        blk.b_pending |= 1u << blk.bs_of(q);
    }
    blk.wait_b(p0 - 2);
    blk.wait_b(p0 - 1);
    if (blk.edge) {
        blk.patch_b(p0 - 2);
        blk.patch_b(p0 - 1);
    }
    int zs[3], zsp[3] = {0, 0, 0};
    bool aborted = false;
    for (int q = p0 - 1; q <= p1; ++q) {
        blk.wait_b(q + 1);
        if (blk.edge) {
            blk.patch_b(q + 1);
            __syncthreads();
        }
        blk.planes(q, zs);
        if (interior || ring) blk.stage1(q, zs, interior);
        // The one barrier per plane: aux of plane q is complete and every read
        // of the variance slot of plane q-1 is done.  It also tells every
        // thread at once whether any wait gave up, so all leave together.
        if (__syncthreads_or(blk.timed_out)) {
            aborted = true;
            break;
        }
        const int qn = q + 2 + PFB;
        if (qn <= p1 + 1) {
            if (tid == 0) {
                fence_proxy_async_smem();
                blk.issue_b(qn);
            }
            blk.b_pending |= 1u << blk.bs_of(qn);
        }
        if (interior && q - 1 >= p0) blk.stage2(q - 1, zsp, acc, bad);
#pragma unroll
        for (int e = 0; e < 3; ++e) zsp[e] = zs[e];
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
