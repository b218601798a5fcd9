// Fused step of the bump-function lattice Boltzmann method (arXiv 2501.00620,
// Sec. II.C) for D2Q9 / D3Q19 with FP32 or 16-bit population storage, written
// for instruction economy on sm_103a.  The arithmetic is the one of the
// generic kernel (lbm_step.cuh, lbm_site.cuh) up to FP32 rounding order; only
// the data movement and the instruction selection differ.
//
// * Populations are pulled straight from global memory (read-only path) with
//   32-bit offsets from per-plane base pointers, after one bulk tensor
//   prefetch per block and plane has brought them into L2.  The pull is a
//   permutation -- every emitted value is read by exactly one site -- so
//   staging them in shared memory would buy no reuse.
// * The variance planes, which the mass-weighted transport (Eq. 66) reads at
//   all Q neighbours, are staged by tiled bulk tensor copies (TMA) in a ring
//   of 3 + PF plane slots (PF = PFB & 1).  In 3D they are stored as component
//   pairs, so the transport reads one 8-byte pair per neighbour and
//   accumulates it with the packed FP32x2 multiply-add of sm_100+ (two FP32
//   FMAs per instruction).
// * (u0, rho b) of the tile plus a one-site ring live in four shared plane
//   slots, site-major as float2 pairs grouped by the rows of rho b that a
//   neighbour direction needs; the gradient (Eqs. 59, 61) loads only those
//   pairs, folds the sign of e_i into the adds, and applies the lattice
//   weights once at the end (axis terms first, scaled by w_axis / w_edge).
// * A tile site hands (bbar, rho, j0, Ebar) from stage 1 to stage 2 and,
//   depending on PFB, either pulls its populations a second time or hands
//   them over too: through two shared slots (plane parity), or through its
//   own lane of tensor memory (tcgen05.st / tcgen05.ld), which the path
//   leaves otherwise unused and which does not count against the shared
//   memory that limits the blocks per SM.
// * Halo items of edge blocks (periodic images or reservoirs) are assigned
//   one per thread with their geometry computed once per block.
// * The conservation diagnostics are summed per thread in FP32 as deviations
//   from the rest state (rho - 1, E - D T0), which keeps the per-thread sums
//   small and exact to far below the storage rounding; blocks reduce in FP64.
//
// A block owns a TX x TY tile (2D: a TX-wide strip) and marches along the
// slowest axis (z in 3D, y in 2D) over `chunk` planes.  Threads: one per tile
// site (stage 1, then stage 2 one plane later) plus one per ring site (stage 1
// only), rounded up to whole warps.  FX selects the fixed-state boundary in x
// (frozen equilibrium reservoirs); otherwise every axis is periodic.
#pragma once

#include <utility>

#include "lbm_lean.cuh"
#include "lbm_mrt.cuh"
#include "lbm_tma.cuh"

namespace lbm {

// PFB: bit 0 -- one more variance plane in flight; bit 1 -- a tile site hands
// its pulled populations to stage 2 through shared memory instead of pulling
// them a second time; bit 2 (with bit 1) -- those populations and the site
// values live in tensor memory (TMEM) instead of shared memory, so that more
// blocks fit per SM; bit 3 -- stage 2 also applies a uniform body force
// (StepArgs::forced) and, on D3Q19, the MRT collision (StepArgs::mrt), as
// the generic kernel does.  MB: resident blocks per SM the launch bounds aim
// at.
template <int D, typename FS, int TX, int TY, int PFB, int MB> struct FastShape {
    using L = Lattice<D>;
    static constexpr int PF = PFB & 1;
    static constexpr bool DFS = (PFB & 2) != 0;
    static constexpr bool TM = (PFB & 4) != 0;
    static constexpr bool EXT = (PFB & 8) != 0;
    // bit 4: half-way bounce-back walls normal to the march axis (StepArgs::
    // walls, at rest or moving): at the first and last plane the populations
    // whose source lies beyond a wall are the site's own opposite emissions
    // (plus the momentum of a moving wall) and carry the site's own
    // variance; the gradient sees beyond a wall the image of the plane facing
    // it (same rho b, velocity 2 u_w - u0), as in the generic kernel
    static constexpr bool WL = (PFB & 16) != 0;
    static constexpr int Q = L::Q, NB = L::NB;
    static constexpr int PXB = 4;                                   // 16-byte aligned x start of a b copy
    static constexpr int SXB = TX + 2 * PXB;                        // sites per staged row
    static constexpr int SY = (D == 3) ? TY + 4 : 1;
    static constexpr int RX = TX + 2;
    static constexpr int RY = (D == 3) ? TY + 2 : 1;
    static constexpr int RS = RX * RY;
    static constexpr int NA2 = (D == 3) ? 5 : 3;                    // float2 of (u0, rho b) per site
    static constexpr int NINT = TX * ((D == 3) ? TY : 1);
    static constexpr int NRING = RS - NINT;
    static constexpr int NT = round_up(NINT + NRING, 32);
    static constexpr int BSLICE = SY * SXB;                         // sites of one staged slice
    static constexpr int BPITCH = round_up(NB * BSLICE * 4, 128);   // bytes between variance slots
    static constexpr int NBS = 3 + PF, NAS = 4;
    static constexpr int NSV = NB + D + 2;                          // carried site values: bbar, rho, j0, Ebar
    static constexpr int OFF_AUX = NBS * BPITCH;
    static constexpr int OFF_SV = OFF_AUX + round_up(NAS * NA2 * 8 * RS, 16);
    static constexpr int OFF_DF = OFF_SV + (TM ? 0 : 2 * NSV * NINT * 4);  // DFS: [2][Q][NINT] populations
    static constexpr int OFF_RED = OFF_DF + (DFS && !TM ? 2 * Q * NINT * 4 : 0);
    static constexpr int OFF_BAR = OFF_RED + (NT / 32) * (D + 2) * 8;  // per-warp diagnostics partials
    static constexpr int OFF_TADDR = OFF_BAR + NBS * 8;               // TM: TMEM base address
    static constexpr int SMEM = OFF_TADDR + 16;
    // TM: per tile thread 2 planes x 32 columns (19 populations, NB + D + 2
    // site values, padding) in its warp's TMEM lane quadrant (warp % 4);
    // tile warps sharing a quadrant take consecutive 64-column groups
    static constexpr int TGROUPS = (NINT / 32 + 3) / 4;
    static constexpr uint32_t TCOLS = TGROUPS <= 1 ? 64u : (TGROUPS <= 2 ? 128u : 256u);
    static_assert(!TM || (DFS && NINT % 32 == 0 && TGROUPS <= 4), "TMEM hand-off: whole tile warps, <= 16");
    static_assert(!TM || Q + NSV <= 32, "site values fit one 32-column group");
    static constexpr uint32_t BBYTES = NB * BSLICE * 4;             // transaction bytes per variance slot
    static_assert((D == 3 ? 2 * SXB : SXB) <= 256 && SY <= 256, "TMA box edges are limited to 256 elements");
    static_assert(NT <= 1024, "too many threads");
    static_assert(4 * SY + ((D == 3) ? 4 * (TX + 4) : 0) <= NT, "one halo item per thread at most");
    static_assert(MB * (SMEM + 1024) <= 228 * 1024, "MB blocks do not fit in shared memory");
};

template <int D, typename FS, int TX, int TY, int PFB, int MB, bool FX> struct FastBlock {
    using L = Lattice<D>;
    using Sh = FastShape<D, FS, TX, TY, PFB, MB>;
    static constexpr int Q = L::Q, NB = L::NB, NA2 = Sh::NA2;
    static constexpr int RX = Sh::RX, RS = Sh::RS, SXB = Sh::SXB, PXB = Sh::PXB, SY = Sh::SY;
    static constexpr int BSLICE = Sh::BSLICE;

    const TmaArgs& ta;
    const StepArgs& a;
    unsigned char* smem;
    int tid, x0, y0, nx, ny, np, p0, p1, pstride, Ni;
    bool xlo, xhi, ylo, yhi, edge;
    uint32_t bphase = 0, b_pending = 0;
    bool timed_out = false;  // a wait of this thread gave up
    // this thread's region site: wrapped coordinates and source offsets
    int rx = 0, ry = 0, gxw = 0, gyw = 0;
    // byte offsets (population storage) of the sources x - e and rows y - e,
    // e = -1, 0, 1: x * sizeof(FS) and y * nx * sizeof(FS)
    int xs[3], ys[3];
    int xo = 0;          // FX: bit e+1 set if source column x - e lies outside [0, nx)
    bool reservoir = false;
    uint32_t tbase = 0;  // TM: TMEM base address of the block

    // Tile (bx, by) over march planes [pp0, pp1); bph carries the phase bits
    // of the variance-slot barriers from the block's previous segment.
    __device__ __forceinline__ FastBlock(const TmaArgs& t, unsigned char* sm, int bx, int by, int pp0, int pp1,
                                         uint32_t bph)
        : ta(t), a(t.s), smem(sm), bphase(bph) {
        tid = threadIdx.x;
        x0 = bx * TX;
        y0 = (D == 3) ? by * TY : 0;
        nx = a.nx;
        ny = a.ny;
        np = (D == 3) ? a.nz : a.ny;
        pstride = (D == 3) ? nx * ny : nx;
        Ni = (int)a.N;
        p0 = pp0;
        p1 = pp1;
        xlo = (x0 == 0);
        xhi = (x0 + TX == nx);
        ylo = (D == 3) && (y0 == 0);
        yhi = (D == 3) && (y0 + TY == ny);
        edge = xlo || xhi || ylo || yhi;
    }

    static __device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
    // q ranges over [p0 - 3, p1 + 2 + PF] with PF + 3 <= np: one conditional add or subtract wraps it
    __device__ __forceinline__ int wrapq(int q) const { return wrap(q, np); }
    static __device__ __forceinline__ int march(int i) { return (D == 3) ? L::e(i, 2) : L::e(i, 1); }

    __device__ __forceinline__ float* bslot(int bs) const {
        return reinterpret_cast<float*>(smem + bs * Sh::BPITCH);
    }
    __device__ __forceinline__ float2* aux(int q) const {
        return reinterpret_cast<float2*>(smem + Sh::OFF_AUX) + ((q - p0 + 1) & 3) * NA2 * RS;
    }
    __device__ __forceinline__ uint64_t* bbar() const { return reinterpret_cast<uint64_t*>(smem + Sh::OFF_BAR); }
    // site values of plane q for tile site t: component k at [k * NINT + t]
    __device__ __forceinline__ float* sv(int q) const {
        return reinterpret_cast<float*>(smem + Sh::OFF_SV) + (q & 1) * Sh::NSV * Sh::NINT + tid;
    }
    __device__ __forceinline__ int bs_of(int q) const { return (q - (p0 - 2)) % Sh::NBS; }
    // TM: TMEM address of plane q's group in this thread's lane (lane
    // quadrant of the warp in bits 16+, column offset in the low bits)
    __device__ __forceinline__ uint32_t taddr(int q) const {
        return tbase + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16) + (uint32_t)((tid >> 7) * 64 + (q & 1) * 32);
    }
    // DFS: populations of plane q for tile site t: population i at [i * NINT + t]
    __device__ __forceinline__ float* dfs(int q) const {
        return reinterpret_cast<float*>(smem + Sh::OFF_DF) + (q & 1) * Q * Sh::NINT + tid;
    }

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
            xs[e + 1] = wrap(sx, nx) * (int)sizeof(FS);
            if (FX && (sx < 0 || sx >= nx)) xo |= 1 << (e + 1);
        }
        gyw = (D == 3) ? wrap(y0 - 1 + ry, ny) : 0;
#pragma unroll
        for (int e = -1; e <= 1; ++e) ys[e + 1] = (D == 3) ? wrap(gyw - e, ny) * nx * (int)sizeof(FS) : 0;
    }
    // Byte offsets of the source planes q - e (e = -1, 0, 1) along the march
    // axis.
    __device__ __forceinline__ void planes(int q, int* zs) const {
#pragma unroll
        for (int e = -1; e <= 1; ++e) zs[e + 1] = wrapq(q - e) * pstride * (int)sizeof(FS);
    }

    // Pull: df_i = stored deviation of fbar*_i at (x - e_i) (Eq. 49).  The
    // address is the block-uniform base of plane i plus a 32-bit byte offset
    // (one add of three per-thread offsets), not a 64-bit index computation
    // per population.
    // WL: wall = 1 at the first plane (sources at q - 1 lie below the lower
    // wall), 2 at the last (sources at q + 1 above the upper wall), else 0.
    __device__ __forceinline__ static bool bounced(int wall, int m) {
        return (wall & 1 && m == 1) || (wall & 2 && m == -1);
    }
    __device__ __forceinline__ void pull(int q, const int* zs, float* df, int wall = 0) const {
        const char* __restrict__ fin = static_cast<const char*>(a.fin);
        // moving walls: density of this site at t, the sum of its emissions
        float rho_self = 1.0f;
        if (Sh::WL && wall && a.walls_moving) {
            const unsigned own = (unsigned)(xs[1] + ((D == 3) ? ys[1] : 0) + zs[1]);
#pragma unroll
            for (int k = 0; k < Q; ++k)
                rho_self += Store<FS>::ld(
                    reinterpret_cast<const FS*>(fin + (size_t)k * (size_t)Ni * sizeof(FS) + own), 0);
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int ex = L::e(i, 0), ey = L::e(i, 1), ez = L::e(i, 2);
            const int m = march(i);
            const unsigned off = (unsigned)(xs[ex + 1] + ((D == 3) ? ys[ey + 1] : 0) + zs[m + 1]);
            if (Sh::WL && bounced(wall, m)) {
                // half-way bounce-back: the site's own opposite emission
                const unsigned own = (unsigned)(xs[1] + ((D == 3) ? ys[1] : 0) + zs[1]);
                const char* plane = fin + (size_t)opposite<D>(i) * (size_t)Ni * sizeof(FS);
                float v = Store<FS>::ld(reinterpret_cast<const FS*>(plane + own), 0);
                if (a.walls_moving) {
                    const int side = (wall & 1 && m == 1) ? 0 : 1;
                    float eu = 0.0f;
#pragma unroll
                    for (int c = 0; c < D; ++c)
                        if (L::e(i, c) != 0) eu += float(L::e(i, c)) * uw_param(a, side, c, 0.0f);
                    v += 6.0f * float(L::w(i)) * rho_self * eu;
                }
                df[i] = v;
            } else if (FX && ex != 0 && (xo & (1 << (ex + 1)))) {
                const float* __restrict__ gf = static_cast<const float*>(a.gf);
                const int row = (D == 3) ? wrap(gyw - ey, ny) + ny * wrapq(q - ez) : wrapq(q - ey);
                df[i] = gf[((ex > 0 ? 0 : 1) * Q + i) * (int)a.rows + row];
            } else {
                const char* plane = fin + (size_t)i * (size_t)Ni * sizeof(FS);
                df[i] = Store<FS>::ld(reinterpret_cast<const FS*>(plane + off), 0);
            }
        }
    }

    // L2 prefetch of the stored populations of march plane P (all Q planes,
    // the x and y range the tile and its ring pull from).  The first pull
    // from plane P is made by stage 1 of plane P - 1.
    __device__ __forceinline__ void prefetch_f(int P) const {
        constexpr int PXF = 16 / (int)sizeof(FS);
        if (D == 3)
            tma_prefetch_l2_4d(&ta.fmap, x0 - PXF, y0 - 2, wrapq(P), 0);
        else
            tma_prefetch_l2_3d(&ta.fmap, x0 - PXF, wrapq(P), 0);
    }

    // ---- variance copies (thread 0 issues; every thread waits itself) --------
    __device__ __forceinline__ void issue_b(int q) {
        const int bs = bs_of(q);
        mbar_arrive_expect_tx(bbar() + bs, Sh::BBYTES);
        if (a.debug_missing_copy && q == p0 - 2 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)
            return;  // armed, never filled: every wait on this slot runs into its time limit
        const int plane = wrapq(q);
        if (D == 3)  // pair planes: x in floats of the (2 nx)-wide pair rows
            tma_load_4d(bslot(bs), &ta.bmap, bbar() + bs, 2 * (x0 - PXB), y0 - 2, plane, 0);
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
    // halo items of this block per plane: at most 4 SY + 4 (TX + 4) <= NT
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
    // This thread's halo item (at most one: halo_count() <= NT), fixed for
    // the segment: its slot position and source column/row, computed once.
    int h_off = -1;   // float offset (2D) or float2 offset (3D) in a slot; -1: no item
    int h_src = 0;    // in-plane source index wx + nx wy (3D) or wx (2D)
    int h_wy = 0;     // source row y (3D)
    int h_res = -1;   // fixed-state reservoir side (0, 1) or -1
    __device__ __forceinline__ void setup_halo() {
        if (!edge || tid >= halo_count()) return;
        int gx, gy;
        halo_pos(tid, gx, gy);
        const int sx = gx - (x0 - PXB), sy = (D == 3) ? gy - (y0 - 2) : 0;
        h_off = sy * SXB + sx;
        h_wy = (D == 3) ? wrap(gy, ny) : 0;
        h_src = wrap(gx, nx) + ((D == 3) ? nx * h_wy : 0);
        if (FX && (gx < 0 || gx >= nx)) h_res = gx < 0 ? 0 : 1;
    }
    __device__ __forceinline__ void patch_b(int q) {
        if (h_off >= 0) {
            const float* __restrict__ bin = static_cast<const float*>(a.bin);
            const float* __restrict__ gb = static_cast<const float*>(a.gb);
            float* slot = bslot(bs_of(q));
            const int plane = wrapq(q);
            const int s = h_src + pstride * plane;
            const int row = (D == 3) ? h_wy + ny * plane : plane;
            float v[NB];
#pragma unroll
            for (int k2 = 0; k2 < NB; ++k2)
                v[k2] = (FX && h_res >= 0) ? gb[(h_res * NB + k2) * (int)a.rows + row]
                                           : bin[(int)BLayout<D, FS>::at(k2, s, Ni)];
            if (D == 3) {
                float2* s2 = reinterpret_cast<float2*>(slot) + h_off;
#pragma unroll
                for (int p = 0; p < NB / 2; ++p) s2[p * BSLICE] = make_float2(v[2 * p], v[2 * p + 1]);
            } else {
#pragma unroll
                for (int k2 = 0; k2 < NB; ++k2) slot[k2 * BSLICE + h_off] = v[k2];
            }
            fence_proxy_async_smem();  // the slot is refilled by a bulk copy later
        }
    }

    // ---- stage 1: pull + moments of this thread's region site at plane q -------
    // Writes (u0, rho b) to the aux plane q; keeps the site values for a tile
    // site.  A fixed-state reservoir site writes the reservoir's aux instead.
    __device__ __forceinline__ void stage1(int q, const int* zs, bool tile, int wall = 0) {
        float2* ax = aux(q) + (rx + RX * ry) * NA2;
        if (FX && reservoir) {
            const float* __restrict__ gaux = static_cast<const float*>(a.gaux);
            const int qq = wrapq(q);
            const int row = (D == 3) ? gyw + ny * qq : qq;
            const int side = (x0 - 1 + rx) < 0 ? 0 : 1;
            constexpr int NAUX = D + NB;
            float u0[D], rb[NB];
#pragma unroll
            for (int c = 0; c < D; ++c) u0[c] = gaux[(side * NAUX + c) * (int)a.rows + row];
#pragma unroll
            for (int k = 0; k < NB; ++k) rb[k] = gaux[(side * NAUX + D + k) * (int)a.rows + row];
            put_aux<D>(ax, u0, rb);
            return;
        }
        float df[Q];
        pull(q, zs, df, wall);
        const int bo = ((D == 3) ? (ry + 1) * SXB : 0) + (rx - 1 + PXB);
        float bsum[NB];
        if constexpr (D == 3) {
            // pairs (xx, yy), (zz, xy), (xz, yz), packed multiply-adds
            const int s0 = bs_of(q);
            const int sm = s0 == 0 ? Sh::NBS - 1 : s0 - 1, sp = s0 == Sh::NBS - 1 ? 0 : s0 + 1;
            const float2* bm = reinterpret_cast<const float2*>(bslot(sm)) + bo;
            const float2* b0 = reinterpret_cast<const float2*>(bslot(s0)) + bo;
            const float2* bp = reinterpret_cast<const float2*>(bslot(sp)) + bo;
            // two independent accumulator sets (in-plane sources, off-plane
            // sources) halve the dependency chains of the multiply-adds
            float2 acc[2][3];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int offb = -L::e(i, 1) * SXB - L::e(i, 0);
                const int m = march(i);
                const int h = (m == 0) ? 0 : 1;
                const bool first = (i == 0) || (i == 5);  // first in-plane / off-plane source
                // a bounced population carries the site's own variance
                const float2* src = (Sh::WL && bounced(wall, m)) ? b0
                                                                 : ((m == 1) ? bm : ((m == -1) ? bp : b0)) + offb;
                const float fi = float(L::w(i)) + df[i];
                const float2 f2 = make_float2(fi, fi);
#pragma unroll
                for (int p = 0; p < 3; ++p)
                    acc[h][p] = first ? __fmul2_rn(f2, src[p * BSLICE]) : __ffma2_rn(f2, src[p * BSLICE], acc[h][p]);
            }
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                const float2 t = __fadd2_rn(acc[0][p], acc[1][p]);
                bsum[2 * p] = t.x;
                bsum[2 * p + 1] = t.y;
            }
        } else {
            const float* bm = bslot(bs_of(q - 1)) + bo;
            const float* b0 = bslot(bs_of(q)) + bo;
            const float* bp = bslot(bs_of(q + 1)) + bo;
            float2 acc2;
            float accxy;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int offb = -L::e(i, 0);
                const int m = march(i);
                const float* src = (Sh::WL && bounced(wall, m)) ? b0
                                                                : ((m == 1) ? bm : ((m == -1) ? bp : b0)) + offb;
                const float fi = float(L::w(i)) + df[i];
                const float2 f2 = make_float2(fi, fi);
                const float2 bxy = make_float2(src[0], src[BSLICE]);
                if (i == 0) {
                    acc2 = __fmul2_rn(f2, bxy);
                    accxy = fi * src[2 * BSLICE];
                } else {
                    acc2 = __ffma2_rn(f2, bxy, acc2);
                    accxy = fmaf(fi, src[2 * BSLICE], accxy);
                }
            }
            bsum[0] = acc2.x;
            bsum[1] = acc2.y;
            bsum[2] = accxy;
        }
        float u0[D], rb[NB], bt[NB], rho, j[D], E;
        float omega, tau, T0;
        step_params(a, omega, tau, T0);
        site_moments<D, float>(df, bsum, omega, T0, a.thermal, bt, rho, j, E, u0, rb);
        if (Sh::TM && tile) {
            // populations and site values of plane q to this thread's TMEM lane
            float w[32];
#pragma unroll
            for (int i = 0; i < Q; ++i) w[i] = df[i];
#pragma unroll
            for (int k = 0; k < NB; ++k) w[Q + k] = bt[k];
            w[Q + NB] = rho;
#pragma unroll
            for (int c = 0; c < D; ++c) w[Q + NB + 1 + c] = j[c];
            w[Q + NB + 1 + D] = E;
#pragma unroll
            for (int k = Q + Sh::NSV; k < 32; ++k) w[k] = 0.0f;
            tmem_st32(taddr(q), w);
        } else if (tile) {
            if constexpr (Sh::DFS) {
                float* dv = dfs(q);
#pragma unroll
                for (int i = 0; i < Q; ++i) dv[i * Sh::NINT] = df[i];
            }
            float* v = sv(q);
            constexpr int NI = Sh::NINT;
#pragma unroll
            for (int k = 0; k < NB; ++k) v[k * NI] = bt[k];
            v[NB * NI] = rho;
#pragma unroll
            for (int c = 0; c < D; ++c) v[(NB + 1 + c) * NI] = j[c];
            v[(NB + 1 + D) * NI] = E;
        }
        put_aux<D>(ax, u0, rb);
    }

    // WL: aux of plane dst, beyond a wall, as the image of this thread's own
    // site in plane src (same rho b, velocity 2 u_w - u0 of wall `side`).
    __device__ __forceinline__ void write_image(int src, int dst, int side) const {
        const float2* as = aux(src) + (rx + RX * ry) * NA2;
        float2* ad = aux(dst) + (rx + RX * ry) * NA2;
        float2 g0 = as[0];
        g0.x = 2.0f * uw_param(a, side, 0, 0.0f) - g0.x;
        g0.y = 2.0f * uw_param(a, side, 1, 0.0f) - g0.y;
        ad[0] = g0;
#pragma unroll
        for (int k = 1; k < NA2; ++k) ad[k] = as[k];
        if constexpr (D == 3) {
            float2 g4 = as[4];
            g4.x = 2.0f * uw_param(a, side, 2, 0.0f) - g4.x;  // (u_z, rb_zz)
            ad[4] = g4;
        }
    }

    // ---- stage 2: gradients, collision and store of this tile site at plane p ----
    __device__ __forceinline__ void stage2(int p, const int* zsp, DiagDev<D + 2>& acc, int& bad) {
        const unsigned sb = (unsigned)(xs[1] + ((D == 3) ? ys[1] : 0) + zsp[1]);  // byte offset of the site
        const int s = (int)(sb / sizeof(FS));
        const int rc = rx + RX * ry;
        const float2* am = aux(p - 1);
        const float2* a0 = aux(p);
        const float2* ap = aux(p + 1);
        float F[D], G[NB];
        gradients<D>(
            [&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int m = (D == 3) ? L::e(i, 2) : L::e(i, 1);
                const float2* as = (m == 1) ? ap : ((m == -1) ? am : a0);
                return as + (rc + L::e(i, 0) + ((D == 3) ? RX * L::e(i, 1) : 0)) * NA2;
            },
            F, G);
        float c_bt[NB], c_j[D], c_rho, c_E;
        float df[Q];
        if constexpr (Sh::TM) {
            tmem_wait_st();  // this thread's store of plane p, an iteration ago
            float w[32];
            tmem_ld32(taddr(p), w);
#pragma unroll
            for (int i = 0; i < Q; ++i) df[i] = w[i];
#pragma unroll
            for (int k = 0; k < NB; ++k) c_bt[k] = w[Q + k];
            c_rho = w[Q + NB];
#pragma unroll
            for (int c = 0; c < D; ++c) c_j[c] = w[Q + NB + 1 + c];
            c_E = w[Q + NB + 1 + D];
        } else {
            const float* v = sv(p);
            constexpr int NI = Sh::NINT;
#pragma unroll
            for (int k = 0; k < NB; ++k) c_bt[k] = v[k * NI];
            c_rho = v[NB * NI];
#pragma unroll
            for (int c = 0; c < D; ++c) c_j[c] = v[(NB + 1 + c) * NI];
            c_E = v[(NB + 1 + D) * NI];
        }
        if constexpr (!Sh::TM) {
            if constexpr (Sh::DFS) {
                const float* dv = dfs(p);
#pragma unroll
                for (int i = 0; i < Q; ++i) df[i] = dv[i * Sh::NINT];
            } else {
                pull(p, zsp, df);  // second pull of the same values
            }
        }
        if constexpr (Sh::EXT) {
            if (a.forced) {
                // body force: F + rho a, G + (rho u a + a rho u) with the
                // corrected momentum rho u = j0 + F/2 (Eq. 57)
                float ga[D], ru[D];
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    ga[c] = acc_param(a, c, 0.0f);
                    F[c] += c_rho * ga[c];
                }
#pragma unroll
                for (int c = 0; c < D; ++c) ru[c] = c_j[c] + 0.5f * F[c];
#pragma unroll
                for (int c = 0; c < D; ++c)
#pragma unroll
                    for (int d2 = c; d2 < D; ++d2) G[sym<D>(c, d2)] += ru[c] * ga[d2] + ru[d2] * ga[c];
            }
        }
        site_collide<D, FS, float, int, DiagDev<D + 2>, PlaneDstBytes>(
            a, s, df, c_bt, c_rho, c_j, c_E, F, G, acc, bad, -1.0,
            PlaneDstBytes{sb, (unsigned)Ni * (unsigned)sizeof(FS)});
        if constexpr (Sh::EXT && D == 3) {
            if (a.mrt && a.write_state) mrt_correct<FS, float>(a, s, df, c_rho, c_j, F);
        }
    }
};

// One segment of the march: tile (bx, by), planes [p0, p1).  Returns false
// if a wait for a variance copy gave up (the block's copies in flight are
// drained and the error flag raised; the caller leaves the kernel).
template <int D, typename FS, int TX, int TY, int PFB, int MB, bool FX>
__device__ __forceinline__ bool fast_segment(const TmaArgs& ta, unsigned char* smem, int bx, int by, int p0,
                                             int p1, DiagDev<D + 2>& acc, int& bad, uint32_t& bphase,
                                             uint32_t tbase) {
    using Sh = FastShape<D, FS, TX, TY, PFB, MB>;
    constexpr int NINT = Sh::NINT, NRING = Sh::NRING, RX = Sh::RX;
    FastBlock<D, FS, TX, TY, PFB, MB, FX> blk(ta, smem, bx, by, p0, p1, bphase);
    blk.tbase = tbase;
    const int tid = threadIdx.x;

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
    blk.setup_halo();

    // prologue: variance planes p0-2 .. p0+PF (the slots' first fill)
    if (tid == 0) fence_proxy_async_smem();  // slots may hold generic-proxy halo writes of a previous segment
    for (int q = p0 - 2; q <= min(p0 + Sh::PF, p1 + 1); ++q) {
        if (tid == 0) blk.issue_b(q);
        blk.b_pending |= 1u << blk.bs_of(q);
    }
    // populations of the first planes the pulls read (p0-2 .. p0+2) into L2
    if (tid == 0)
        for (int P = p0 - 2; P <= min(p0 + 2, p1 + 1); ++P) blk.prefetch_f(P);
    blk.wait_b(p0 - 2);
    blk.wait_b(p0 - 1);
    if (blk.edge) {
        blk.patch_b(p0 - 2);
        blk.patch_b(p0 - 1);
    }
    int zs[3], zsp[3] = {0, 0, 0};
    for (int q = p0 - 1; q <= p1; ++q) {
        blk.wait_b(q + 1);
        if (blk.edge) {
            blk.patch_b(q + 1);
            __syncthreads();
        }
        blk.planes(q, zs);
        if constexpr (Sh::WL) {
            // walls: nothing lies beyond the lattice along the march axis;
            // the planes -1 and np hold the images of planes 0 and np - 1
            const int np = blk.np;
            if (interior || ring) {
                if (q >= 0 && q < np) {
                    const int wall = (q == 0 ? 1 : 0) | (q == np - 1 ? 2 : 0);
                    blk.stage1(q, zs, interior, wall);
                    if (q == 0 && p0 == 0) blk.write_image(0, -1, 0);
                } else if (q == np) {
                    blk.write_image(np - 1, np, 1);
                }
            }
        } else {
            if (interior || ring) blk.stage1(q, zs, interior);
        }
        // The one barrier per plane: aux of plane q is complete and every read
        // of the variance slot of plane q-1 is done.  It also tells every
        // thread at once whether any wait gave up, so all leave together.
        if (__syncthreads_or(blk.timed_out)) {
            // drain this block's copies still in flight, then leave
            if (tid == 0) {
                atomicOr(ta.s.flag, 4);
                blk.drain();
            }
            return false;
        }
        const int qn = q + 2 + Sh::PF;
        if (qn <= p1 + 1) {
            if (tid == 0) {
                fence_proxy_async_smem();
                blk.issue_b(qn);
            }
            blk.b_pending |= 1u << blk.bs_of(qn);
        }
        // populations two planes ahead of the next stage 1
        if (tid == 0 && q + 3 <= p1 + 1) blk.prefetch_f(q + 3);
        if (interior && q - 1 >= p0) blk.stage2(q - 1, zsp, acc, bad);
#pragma unroll
        for (int e = 0; e < 3; ++e) zsp[e] = zs[e];
    }
    bphase = blk.bphase;
    // the next segment rewrites the aux and site-value slots
    __syncthreads();
    return true;
}

// Grid: (nx/TX, ny/TY, chunks), one segment of the march per block.
template <int D, typename FS, int TX, int TY, int PFB, int MB, bool FX>
__global__ void __launch_bounds__(FastShape<D, FS, TX, TY, PFB, MB>::NT, MB)
    step_fast_kernel(const __grid_constant__ TmaArgs ta) {
    using Sh = FastShape<D, FS, TX, TY, PFB, MB>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Sh::OFF_BAR);
    if (tid == 0) {
        for (int k = 0; k < Sh::NBS; ++k) mbar_init(bars + k, 1);
        fence_barrier_init();
    }
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + Sh::OFF_TADDR);
    if constexpr (Sh::TM) {
        if (tid < 32) tmem_alloc(tslot, Sh::TCOLS);  // warp 0
        tmem_fence_before_sync();
    }
    __syncthreads();
    uint32_t tbase = 0;
    if constexpr (Sh::TM) {
        tmem_fence_after_sync();
        tbase = *tslot;
    }

    DiagDev<D + 2> acc(float(D) * ta.s.T0_f);
    int bad = 0;
    uint32_t bphase = 0;
    const int np = (D == 3) ? ta.s.nz : ta.s.ny;
    const int p0 = ta.s.halo + blockIdx.z * ta.s.chunk;
    const bool ok = fast_segment<D, FS, TX, TY, PFB, MB, FX>(ta, smem, blockIdx.x, blockIdx.y, p0,
                                                             min(p0 + ta.s.chunk, np - ta.s.halo), acc, bad, bphase,
                                                             tbase);
    if constexpr (Sh::TM) {
        // every thread's TMEM stores complete, then warp 0 frees the columns
        // (on the abort path too: the segment left with every thread)
        tmem_wait_st();
        tmem_fence_before_sync();
        __syncthreads();
        if (tid < 32) {
            tmem_fence_after_sync();
            tmem_dealloc(tbase, Sh::TCOLS);
        }
    }
    if (!ok) return;
    if (bad) atomicOr(ta.s.flag, bad);
    if (ta.s.want_diag)
        block_diagnostics<D, Sh::NT>(ta.s, acc, reinterpret_cast<double*>(smem + Sh::OFF_RED));
}

}  // namespace lbm
