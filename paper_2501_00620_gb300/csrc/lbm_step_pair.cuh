// Fused step of the bump-function lattice Boltzmann method (arXiv 2501.00620,
// Sec. II.C) for D2Q9 / D3Q19 with FP32 or 16-bit population storage and
// periodic boundaries, one thread per PAIR of x-adjacent sites.
//
// The arithmetic is that of the other kernels (lbm_site.cuh) up to FP32
// rounding order; this kernel differs in how it spends instructions:
// * Every per-site operation runs on both sites of the pair at once in packed
//   FP32x2 (add/sub/mul/fma.rn.f32x2), which halves the arithmetic
//   instructions of the moments, the gradients (Eqs. 59, 61) and the
//   collision (Eq. 55, Appendix A).
// * A pair starts at an even x, so the populations a pair pulls along a
//   direction with e_x = 0, and every population and variance value it
//   stores, move as one 8-byte (16-byte for variance pairs) access.
// * As in the staged kernel, the variance planes (read at all Q neighbours by
//   the mass-weighted transport, Eq. 66) are staged by tiled bulk tensor
//   copies (TMA) into a ring of three plane slots on mbarrier transaction
//   barriers, and the populations of the planes ahead are prefetched into L2
//   by bulk tensor prefetches.
// * (u0, rho b) of the tile and its one-site ring live in four shared plane
//   slots, component-major with x contiguous, so a neighbour pair with
//   e_x = 0 reads each component with one 8-byte load.
// * A tile pair hands its pulled populations and site values from stage 1 to
//   stage 2 through its own lane of tensor memory (tcgen05.st / tcgen05.ld),
//   which the path otherwise leaves unused.
//
// A block owns a TX x TY tile (2D: a TX-wide strip) and marches along the
// slowest axis (z in 3D, y in 2D) over `chunk` planes.  Region = tile plus a
// one-site ring, covered by pairs of columns x0 - 2 + 2k (the first and last
// pair of a row each hold one site the gradient never reads).  Threads: one
// per tile pair (stage 1, then stage 2 one plane later), then one per ring
// pair (stage 1 only).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_f2.cuh"
#include "lbm_lean.cuh"
#include "lbm_tma.cuh"

namespace lbm {

// Storage of a pair of adjacent populations (site x even, x + 1).
template <typename FS> struct PairIO;
template <> struct PairIO<float> {
    __device__ __forceinline__ static px::P ld2(const float* p, uint32_t k) {
        return px::P(__ldg(reinterpret_cast<const float2*>(p + k)));
    }
    __device__ __forceinline__ static float ld1(const float* p, uint32_t k) { return __ldg(p + k); }
    __device__ __forceinline__ static void st2(float* p, uint32_t k, px::P v) {
        *reinterpret_cast<float2*>(p + k) = v.v;
    }
};
template <> struct PairIO<__half> {
    __device__ __forceinline__ static px::P ld2(const __half* p, uint32_t k) {
        return px::P(__half22float2(__ldg(reinterpret_cast<const __half2*>(p + k))));
    }
    __device__ __forceinline__ static float ld1(const __half* p, uint32_t k) { return __half2float(__ldg(p + k)); }
    __device__ __forceinline__ static void st2(__half* p, uint32_t k, px::P v) {
        *reinterpret_cast<__half2*>(p + k) = __float22half2_rn(v.v);
    }
};
template <> struct PairIO<__nv_bfloat16> {
    __device__ __forceinline__ static px::P ld2(const __nv_bfloat16* p, uint32_t k) {
        return px::P(__bfloat1622float2(__ldg(reinterpret_cast<const __nv_bfloat162*>(p + k))));
    }
    __device__ __forceinline__ static float ld1(const __nv_bfloat16* p, uint32_t k) {
        return __bfloat162float(__ldg(p + k));
    }
    __device__ __forceinline__ static void st2(__nv_bfloat16* p, uint32_t k, px::P v) {
        *reinterpret_cast<__nv_bfloat162*>(p + k) = __float22bfloat162_rn(v.v);
    }
};

// WS: warp-specialized form -- NTILE threads run stage 1 for every region
// pair (tile pairs, then ring pairs), another NTILE threads run stage 2 of the
// tile pairs, handing over through mbarrier pipelines (more aux slots and
// hand-off buffers in flight); otherwise every thread runs stage 1 of its
// pair and a tile thread stage 2 too, one block barrier per plane.
template <int D, typename FS, int TX, int TY, int MB, int PF, bool WS = false> struct PairShape {
    using L = Lattice<D>;
    static constexpr int Q = L::Q, NB = L::NB;
    static constexpr int TXP = TX / 2;                    // pairs per tile row
    static constexpr int RXP = TXP + 2;                   // pairs per region row
    static constexpr int RY = (D == 3) ? TY + 2 : 1;      // region rows
    static constexpr int NTILE = TXP * ((D == 3) ? TY : 1);
    static constexpr int NREG = RXP * RY;
    static constexpr int NRING = NREG - NTILE;
    static constexpr int NT = WS ? 2 * NTILE : round_up(NREG, 32);
    static constexpr int NS1 = WS ? NTILE : NT;           // stage-1 threads
    static constexpr int PXB = 4;                         // staged sites left of x0 (16-byte aligned copy start)
    static constexpr int SXB = TX + 2 * PXB;              // staged sites per row
    static constexpr int SY = (D == 3) ? TY + 4 : 1;      // staged rows
    static constexpr int BSLICE = SY * SXB;               // sites of one staged slice
    static constexpr int BPITCH = round_up(NB * BSLICE * 4, 128);
    static constexpr int NBS = 3 + PF;                    // variance slots: planes q-1..q+1 (+ PF ahead)
    static constexpr int RXA = 2 * RXP;                   // aux columns (x from x0 - 2)
    static constexpr int NAUX = D + NB;                   // u0 (D), rho b (NB)
    static constexpr int APLANE = NAUX * RY * RXA;        // floats per aux slot
    static constexpr int NAS = WS ? 5 : 4;                // aux plane slots
    static constexpr int NTB = WS ? 4 : 2;                // hand-off buffers (planes) per thread
    static constexpr int KB = 8;                          // pipeline barriers per direction (WS)
    static constexpr int NSV = NB + D + 2;                // carried site values: bbar, rho, j0, Ebar
    static constexpr int TW = round_up(2 * (Q + NSV), 32);  // TMEM words per thread and plane
    static constexpr int OFF_AUX = NBS * BPITCH;
    static constexpr int OFF_RED = OFF_AUX + round_up(NAS * APLANE * 4, 16);
    static constexpr int OFF_BAR = OFF_RED + (NT / 32) * (D + 2) * 8;
    static constexpr int OFF_PIPE = OFF_BAR + NBS * 8;           // WS: full[KB], empty[KB]
    static constexpr int OFF_TADDR = OFF_PIPE + (WS ? 2 * KB * 8 : 0);
    static constexpr int SMEM = OFF_TADDR + 16;
    // tile warps sharing a TMEM lane quadrant (warp % 4) take consecutive
    // groups of 2 TW columns
    static constexpr int TGROUPS = (NTILE / 32 + 3) / 4;
    static constexpr int TCOLS0 = NTB * TW * TGROUPS;
    static constexpr uint32_t TCOLS = TCOLS0 <= 64 ? 64u : (TCOLS0 <= 128 ? 128u : (TCOLS0 <= 256 ? 256u : 512u));
    static constexpr uint32_t BBYTES = NB * BSLICE * 4;
    // halo items (positions of a staged slice outside the lattice): at most
    // 6 columns x SY rows and 4 rows x (TX + 6) columns, two per thread
    static constexpr int MAXHALO = 6 * SY + ((D == 3) ? 4 * (TX + 6) : 0);
    static_assert(TX % 64 == 0 || D == 2, "3D tiles: whole warps of pairs per row");
    static_assert(TX % 4 == 0, "pairs and 16-byte copy starts");
    static_assert(NTILE % 32 == 0 && TCOLS0 * MB <= 512, "tile pairs: whole warps, TMEM columns of every block");
    static_assert(!WS || (NTILE % 128 == 0 && NREG <= 2 * NTILE), "WS: whole warpgroups, two stage-1 rounds");
    static_assert((D == 3 ? 2 * SXB : SXB) <= 256 && SY <= 256, "TMA box edges are limited to 256 elements");
    static_assert(NT <= 1024, "too many threads");
    static_assert(NSV <= 16 && (TW == 32 || TW == 64), "site values in the first 32 hand-off words");
    static_assert(MAXHALO <= 2 * NS1, "two halo items per stage-1 thread at most");
    static_assert(MB * (SMEM + 1024) <= 228 * 1024, "MB blocks do not fit in shared memory");
};

template <int D, typename FS, int TX, int TY, int MB, int PF, bool WS = false> struct PairBlock {
    using L = Lattice<D>;
    using Sh = PairShape<D, FS, TX, TY, MB, PF, WS>;
    using P = px::P;
    static constexpr int Q = L::Q, NB = L::NB, NAUX = Sh::NAUX;
    static constexpr int SXB = Sh::SXB, PXB = Sh::PXB, SY = Sh::SY, BSLICE = Sh::BSLICE;
    static constexpr int RXA = Sh::RXA, RY = Sh::RY;

    const TmaArgs& ta;
    const StepArgs& a;
    unsigned char* smem;
    int tid, x0, y0, nx, ny, np, p0, p1, pstride;
    uint32_t Nu;
    bool xlo, xhi, ylo, yhi, edge;
    uint32_t bphase = 0, b_pending = 0;
    bool timed_out = false;
    int kp = 0, ry = 0;            // this thread's pair column and region row
    int xa = 0, yrow = 0;          // first site of the pair (unwrapped), row y (unwrapped)
    uint32_t xsa[3], xsb[3];       // wrapped source columns x - e of both sites, e = -1, 0, 1
    uint32_t ys[3];                // wrapped source rows (y - e) nx (3D)
    uint32_t tbase = 0;
    int tw = 0;                    // tile warp (TMEM lane quadrant tw % 4, column group tw / 4)
    int h_off[2] = {-1, -1};       // halo items: site offset in a slice, -1: none
    uint32_t h_src[2] = {0, 0};    // in-plane source index of the periodic image

    __device__ __forceinline__ PairBlock(const TmaArgs& t, unsigned char* sm, int bx, int by, int pp0, int pp1)
        : ta(t), a(t.s), smem(sm) {
        tid = threadIdx.x;
        x0 = bx * TX;
        y0 = (D == 3) ? by * TY : 0;
        nx = a.nx;
        ny = a.ny;
        np = (D == 3) ? a.nz : a.ny;
        pstride = (D == 3) ? nx * ny : nx;
        Nu = (uint32_t)a.N;
        p0 = pp0;
        p1 = pp1;
        xlo = (x0 == 0);
        xhi = (x0 + TX == nx);
        ylo = (D == 3) && (y0 == 0);
        yhi = (D == 3) && (y0 + TY == ny);
        edge = xlo || xhi || ylo || yhi;
    }

    static __device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
    __device__ __forceinline__ int wrapq(int q) const { return wrap(q, np); }
    static __device__ __forceinline__ constexpr int march(int i) { return (D == 3) ? L::e(i, 2) : L::e(i, 1); }

    __device__ __forceinline__ float* bslot(int bs) const { return reinterpret_cast<float*>(smem + bs * Sh::BPITCH); }
    __device__ __forceinline__ int bs_of(int q) const { return (q - (p0 - 2)) % Sh::NBS; }
    __device__ __forceinline__ float* aux(int q) const {
        return reinterpret_cast<float*>(smem + Sh::OFF_AUX) + ((q - p0 + 1) % Sh::NAS) * Sh::APLANE;
    }
    __device__ __forceinline__ uint64_t* bbar() const { return reinterpret_cast<uint64_t*>(smem + Sh::OFF_BAR); }
    // TMEM address of plane q's words in this thread's lane
    __device__ __forceinline__ uint32_t taddr(int q) const {
        return tbase + ((uint32_t)(32 * (tw & 3)) << 16) + (uint32_t)((tw >> 2) * Sh::NTB * Sh::TW) +
               (uint32_t)(((q - p0 + 1) % Sh::NTB) * Sh::TW);
    }

    // The pair-dependent state: saved and restored when one thread serves
    // two pairs (a tile pair and a ring pair) in the warp-specialized form.
    struct Site {
        int kp, ry, xa, yrow;
        uint32_t xsa[3], xsb[3], ys[3];
    };
    __device__ __forceinline__ Site site() const {
        Site t;
        t.kp = kp;
        t.ry = ry;
        t.xa = xa;
        t.yrow = yrow;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            t.xsa[e] = xsa[e];
            t.xsb[e] = xsb[e];
            t.ys[e] = ys[e];
        }
        return t;
    }
    __device__ __forceinline__ void use(const Site& t) {
        kp = t.kp;
        ry = t.ry;
        xa = t.xa;
        yrow = t.yrow;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            xsa[e] = t.xsa[e];
            xsb[e] = t.xsb[e];
            ys[e] = t.ys[e];
        }
    }

    __device__ __forceinline__ void set_pair(int kp_, int ry_) {
        kp = kp_;
        ry = ry_;
        xa = x0 - 2 + 2 * kp;
        yrow = (D == 3) ? y0 - 1 + ry : 0;
#pragma unroll
        for (int e = -1; e <= 1; ++e) {
            xsa[e + 1] = (uint32_t)wrap(xa - e, nx);
            xsb[e + 1] = (uint32_t)wrap(xa + 1 - e, nx);
            ys[e + 1] = (D == 3) ? (uint32_t)wrap(yrow - e, ny) * (uint32_t)nx : 0u;
        }
    }
    __device__ __forceinline__ void planes(int q, uint32_t* zs) const {
#pragma unroll
        for (int e = -1; e <= 1; ++e) zs[e + 1] = (uint32_t)wrapq(q - e) * (uint32_t)pstride;
    }

    // Pull of both sites: df_i = stored deviation of fbar*_i at (x - e_i) (Eq. 49).
    __device__ __forceinline__ void pull(const uint32_t* zs, P* df) const {
        const FS* __restrict__ fin = static_cast<const FS*>(a.fin);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int ex = L::e(i, 0), ey = L::e(i, 1);
            const int m = march(i);
            const uint32_t base = (uint32_t)i * Nu + ((D == 3) ? ys[ey + 1] : 0u) + zs[m + 1];
            if (ex == 0)
                df[i] = PairIO<FS>::ld2(fin, base + xsa[1]);
            else
                df[i] = P(PairIO<FS>::ld1(fin, base + xsa[ex + 1]), PairIO<FS>::ld1(fin, base + xsb[ex + 1]));
        }
    }

    __device__ __forceinline__ void prefetch_f(int Pl) const {
        constexpr int PXF = 16 / (int)sizeof(FS);
        if (D == 3)
            tma_prefetch_l2_4d(&ta.fmap, x0 - PXF, y0 - 2, wrapq(Pl), 0);
        else
            tma_prefetch_l2_3d(&ta.fmap, x0 - PXF, wrapq(Pl), 0);
    }

    __device__ __forceinline__ void issue_b(int q) {
        const int bs = bs_of(q);
        mbar_arrive_expect_tx(bbar() + bs, Sh::BBYTES);
        if (a.debug_missing_copy && q == p0 - 2 && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0)
            return;  // armed, never filled: every wait on this slot runs into its time limit
        const int plane = wrapq(q);
        if (D == 3)
            tma_load_4d(bslot(bs), &ta.bmap, bbar() + bs, 2 * (x0 - PXB), y0 - 2, plane, 0);
        else
            tma_load_3d(bslot(bs), &ta.bmap, bbar() + bs, x0 - PXB, plane, 0);
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
        for (int k = 0; k < Sh::NBS; ++k)
            if (b_pending & (1u << k)) mbar_wait_bounded(bbar() + k, (bphase >> k) & 1u, kWaitLimit);
    }

    // ---- halo of the staged variance slice in edge blocks -----------------
    // The copy zero-fills positions outside the lattice; the transport reads
    // x in [x0 - 3, x0 + TX + 2] and (3D) rows [y0 - 2, y0 + TY + 1]: those
    // outside get their periodic image.
    __device__ __forceinline__ int halo_count() const {
        const int cx = (xlo ? 3 : 0) + (xhi ? 3 : 0);
        const int cy = (ylo ? 2 : 0) + (yhi ? 2 : 0);
        return cx * SY + cy * (TX + 6);
    }
    __device__ __forceinline__ void halo_pos(int k, int& gx, int& gy) const {
        const int cx = (xlo ? 3 : 0) + (xhi ? 3 : 0);
        if (k < cx * SY) {
            const int col = k / SY, row = k % SY;
            gx = (xlo && col < 3) ? -3 + col : nx + (col - (xlo ? 3 : 0));
            gy = (D == 3) ? y0 - 2 + row : 0;
        } else {
            k -= cx * SY;
            const int rr = k / (TX + 6), col = k % (TX + 6);
            gx = x0 - 3 + col;
            gy = (ylo && rr < 2) ? -2 + rr : ny + (rr - (ylo ? 2 : 0));
        }
    }
    __device__ __forceinline__ void setup_halo() {
        if (!edge) return;
        const int n = halo_count();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = tid + h * Sh::NS1;
            if (tid >= Sh::NS1 || k >= n) continue;
            int gx, gy;
            halo_pos(k, gx, gy);
            h_off[h] = ((D == 3) ? (gy - (y0 - 2)) * SXB : 0) + gx - (x0 - PXB);
            h_src[h] = (uint32_t)wrap(gx, nx) + ((D == 3) ? (uint32_t)nx * (uint32_t)wrap(gy, ny) : 0u);
        }
    }
    __device__ __forceinline__ void patch_b(int q) {
        const float* __restrict__ bin = static_cast<const float*>(a.bin);
        float* slot = bslot(bs_of(q));
        const uint32_t plane = (uint32_t)wrapq(q) * (uint32_t)pstride;
        bool any = false;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (h_off[h] < 0) continue;
            any = true;
            const uint32_t s = h_src[h] + plane;
            if (D == 3) {
                const float2* __restrict__ b2 = reinterpret_cast<const float2*>(bin);
                float2* s2 = reinterpret_cast<float2*>(slot) + h_off[h];
#pragma unroll
                for (int p = 0; p < NB / 2; ++p) s2[p * BSLICE] = __ldg(b2 + p * Nu + s);
            } else {
#pragma unroll
                for (int k2 = 0; k2 < NB; ++k2) slot[k2 * BSLICE + h_off[h]] = __ldg(bin + k2 * Nu + s);
            }
        }
        if (any) fence_proxy_async_smem();  // the slot is refilled by a bulk copy later
    }

    // ---- stage 1: pull, transport and moments of this thread's pair at plane q
    __device__ __forceinline__ void stage1(int q, const P* df, bool tile) {
        P bsum[NB];
        const int ca = 2 * kp + 2;  // slice column of site a (x - (x0 - PXB)) before the shift by -e_x
        if constexpr (D == 3) {
            // component pairs (xx, yy), (zz, xy), (xz, yz) of each site,
            // accumulated per site with packed multiply-adds; two accumulator
            // sets (in-plane, off-plane sources) shorten the chains
            const int s0 = bs_of(q);
            const int sm = s0 == 0 ? Sh::NBS - 1 : s0 - 1, sp = s0 == Sh::NBS - 1 ? 0 : s0 + 1;  // planes q -+ 1
            const float2* bm = reinterpret_cast<const float2*>(bslot(sm));
            const float2* b0 = reinterpret_cast<const float2*>(bslot(s0));
            const float2* bp = reinterpret_cast<const float2*>(bslot(sp));
            float2 acca[2][3], accb[2][3];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int ex = L::e(i, 0), ey = L::e(i, 1), m = march(i);
                const int h = (m == 0) ? 0 : 1;
                const bool first = (i == 0) || (i == 5);
                const float2* src = ((m == 1) ? bm : ((m == -1) ? bp : b0)) + (ry + 1 - ey) * SXB + ca - ex;
                const P fi = P(float(L::w(i))) + df[i];
                const float2 fa = make_float2(fi.a(), fi.a()), fb = make_float2(fi.b(), fi.b());
#pragma unroll
                for (int p = 0; p < 3; ++p) {
                    float2 va, vb;
                    if (ex == 0) {
                        const float4 v4 = *reinterpret_cast<const float4*>(src + p * BSLICE);
                        va = make_float2(v4.x, v4.y);
                        vb = make_float2(v4.z, v4.w);
                    } else {
                        va = src[p * BSLICE];
                        vb = src[p * BSLICE + 1];
                    }
                    acca[h][p] = first ? __fmul2_rn(fa, va) : __ffma2_rn(fa, va, acca[h][p]);
                    accb[h][p] = first ? __fmul2_rn(fb, vb) : __ffma2_rn(fb, vb, accb[h][p]);
                }
            }
#pragma unroll
            for (int p = 0; p < 3; ++p) {
                const float2 ta2 = __fadd2_rn(acca[0][p], acca[1][p]);
                const float2 tb2 = __fadd2_rn(accb[0][p], accb[1][p]);
                bsum[2 * p] = P(ta2.x, tb2.x);
                bsum[2 * p + 1] = P(ta2.y, tb2.y);
            }
        } else {
            const float* bm = bslot(bs_of(q - 1));
            const float* b0 = bslot(bs_of(q));
            const float* bp = bslot(bs_of(q + 1));
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const int ex = L::e(i, 0), m = march(i);
                const float* src = ((m == 1) ? bm : ((m == -1) ? bp : b0)) + ca - ex;
                const P fi = P(float(L::w(i))) + df[i];
#pragma unroll
                for (int k = 0; k < NB; ++k) {
                    const P v = (ex == 0) ? P(*reinterpret_cast<const float2*>(src + k * BSLICE))
                                          : P(src[k * BSLICE], src[k * BSLICE + 1]);
                    bsum[k] = (i == 0) ? fi * v : px::fma(fi, v, bsum[k]);
                }
            }
        }
        float omega, tau, T0;
        step_params(a, omega, tau, T0);
        P bt[NB], rho, j[D], E, u0[D], rb[NB];
        moments(df, bsum, omega, T0, a.thermal, bt, rho, j, E, u0, rb);
        float* ax = aux(q) + ry * RXA + 2 * kp;
#pragma unroll
        for (int c = 0; c < D; ++c) *reinterpret_cast<float2*>(ax + c * RY * RXA) = u0[c].v;
#pragma unroll
        for (int k = 0; k < NB; ++k) *reinterpret_cast<float2*>(ax + (D + k) * RY * RXA) = rb[k].v;
        if (tile) {
            // hand-off words (pairs a, b): rho, j0, Ebar, bbar, then the
            // populations, so that stage 2 loads the site values and the
            // first populations (group 0) before the rest (group 1)
            float w[Sh::TW];
            auto put = [&](int k, P v) {
                w[2 * k] = v.a();
                w[2 * k + 1] = v.b();
            };
            put(0, rho);
#pragma unroll
            for (int c = 0; c < D; ++c) put(1 + c, j[c]);
            put(D + 1, E);
#pragma unroll
            for (int k = 0; k < NB; ++k) put(D + 2 + k, bt[k]);
#pragma unroll
            for (int i = 0; i < Q; ++i) put(Sh::NSV + i, df[i]);
#pragma unroll
            for (int k = 2 * (Q + Sh::NSV); k < Sh::TW; ++k) w[k] = 0.0f;
#pragma unroll
            for (int g = 0; g < Sh::TW / 32; ++g) tmem_st32(taddr(q) + 32 * g, w + 32 * g);
        }
    }

    // Moments of both sites (Eqs. 56-57, 66-68): rho, j0, bbar = bsum / rho,
    // Ebar, u0 = j0 / rho, T_unc (thermal) or T0, and
    // rho b = rho (bbar - (omega/2)(bbar - b^eq(u0, T_unc))) as a deviation
    // of the shifted variance (diagonal minus rho/3).
    static __device__ __forceinline__ void moments(const P* df, const P* bsum, float omega, float T0, int thermal,
                                                   P* bt, P& rho, P* j, P& E, P* u0, P* rb) {
        P ps[Q], pd[Q];
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if (i > opposite<D>(i)) continue;
            ps[i] = df[i] + df[opposite<D>(i)];
            pd[i] = df[i] - df[opposite<D>(i)];
        }
        P r = df[0];
#pragma unroll
        for (int i = 1; i < Q; ++i)
            if (i < opposite<D>(i)) r += ps[i];
        rho = r + P(1.0f);
        const P irho = px::recip(rho);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            bool first = true;
            P acc;
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                if (!(i < opposite<D>(i) && L::e(i, c) != 0)) continue;
                if (first)
                    acc = pd[i];  // the first member of each pair has e_c = +1 here
                else
                    acc = L::e(i, c) > 0 ? acc + pd[i] : acc - pd[i];
                first = false;
            }
            j[c] = acc;
        }
#pragma unroll
        for (int k = 0; k < NB; ++k) bt[k] = bsum[k] * irho;
        P trb = bt[0];
#pragma unroll
        for (int c = 1; c < D; ++c) trb += bt[c];
        P e = px::fma(rho, trb, P(float(-D * (1.0 / 3.0))) * df[0]);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if (i > opposite<D>(i)) continue;
            const double coef = norm2<D>(i) - D * (1.0 / 3.0);
            if (coef == 1.0)
                e += ps[i];
            else if (coef != 0.0)
                e = px::fma(P(float(coef)), ps[i], e);
        }
        E = e;
#pragma unroll
        for (int c = 0; c < D; ++c) u0[c] = j[c] * irho;
        P Tu = P(T0);
        if (thermal) {
            P uu = u0[0] * u0[0];
#pragma unroll
            for (int c = 1; c < D; ++c) uu = px::fma(u0[c], u0[c], uu);
            Tu = ((e - rho * uu) * irho) * P(float(1.0 / D));
        }
        const P hw = P(0.5f * omega);
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
            for (int d2 = c; d2 < D; ++d2) {
                const int k = sym<D>(c, d2);
                const P uc3 = u0[c] * P(float(1.0 / 3.0));
                const P beq = (c == d2) ? px::fma(uc3, u0[d2], Tu) : uc3 * u0[d2];
                P t = px::fma(hw, beq - bt[k], bt[k]);
                if (c == d2) t = t - P(float(1.0 / 3.0));
                rb[k] = rho * t;
            }
    }

    // ---- stage 2: gradients, collision and store of this tile pair at plane p --
    // One neighbour's term of F = -div(rho b) and G = -div(rho u0 b + rho u0 b)
    // (Eqs. 59, 61) for both sites (unscaled: v = e_i . rho b, F += v,
    // G_bc += u_c v_b + u_b v_c, the diagonal counted once).
    template <int I>
    __device__ __forceinline__ void grad_nb(const float* am, const float* a0, const float* ap, P* F, P* G) const {
        constexpr int ex = L::e(I, 0), ey = L::e(I, 1), ez = L::e(I, 2);
        constexpr int m = (D == 3) ? ez : ey;
        const float* as = (m == 1) ? ap : ((m == -1) ? am : a0);
        const float* nb = as + ((D == 3) ? (ry + ey) * RXA : 0) + 2 * kp + ex;
        constexpr int CS = RY * RXA;  // component stride
        auto ld = [&](int comp) -> P {
            const float* p = nb + comp * CS;
            if constexpr (ex == 0)
                return P(*reinterpret_cast<const float2*>(p));
            else
                return P(p[0], p[1]);
        };
        if constexpr (D == 3) {
            // rho b components: xx 3, yy 4, zz 5, xy 6, xz 7, yz 8
            constexpr int rowc[3][3] = {{3, 6, 7}, {6, 4, 8}, {7, 8, 5}};
            P v[3];
            constexpr int e3[3] = {ex, ey, ez};
            // rows of the positive components first, then the negative ones
            // subtracted (a direction with no positive component starts from 0)
            bool first = true;
#pragma unroll
            for (int pass = 0; pass < 2; ++pass)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    if (e3[c] == 0 || (pass == 0) != (e3[c] > 0)) continue;
#pragma unroll
                    for (int b2 = 0; b2 < 3; ++b2) {
                        const P r = ld(rowc[c][b2]);
                        if (first)
                            v[b2] = (e3[c] > 0) ? r : P(0.0f) - r;
                        else
                            v[b2] = (e3[c] > 0) ? v[b2] + r : v[b2] - r;
                    }
                    first = false;
                }
            const P ux = ld(0), uy = ld(1), uz = ld(2);
#pragma unroll
            for (int b2 = 0; b2 < 3; ++b2) F[b2] += v[b2];
            G[0] = px::fma(ux, v[0], G[0]);
            G[1] = px::fma(uy, v[1], G[1]);
            G[2] = px::fma(uz, v[2], G[2]);
            G[3] = px::fma(uy, v[0], px::fma(ux, v[1], G[3]));
            G[4] = px::fma(uz, v[0], px::fma(ux, v[2], G[4]));
            G[5] = px::fma(uz, v[1], px::fma(uy, v[2], G[5]));
        } else {
            // rho b components: xx 2, yy 3, xy 4
            constexpr int rowc[2][2] = {{2, 4}, {4, 3}};
            constexpr int e2[2] = {ex, ey};
            P v[2];
            bool first = true;
#pragma unroll
            for (int pass = 0; pass < 2; ++pass)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    if (e2[c] == 0 || (pass == 0) != (e2[c] > 0)) continue;
#pragma unroll
                    for (int b2 = 0; b2 < 2; ++b2) {
                        const P r = ld(rowc[c][b2]);
                        if (first)
                            v[b2] = (e2[c] > 0) ? r : P(0.0f) - r;
                        else
                            v[b2] = (e2[c] > 0) ? v[b2] + r : v[b2] - r;
                    }
                    first = false;
                }
            const P ux = ld(0), uy = ld(1);
            F[0] += v[0];
            F[1] += v[1];
            G[0] = px::fma(ux, v[0], G[0]);
            G[1] = px::fma(uy, v[1], G[1]);
            G[2] = px::fma(uy, v[0], px::fma(ux, v[1], G[2]));
        }
    }

    template <int... Is>
    __device__ __forceinline__ void gradients(const float* am, const float* a0, const float* ap, P* F, P* G,
                                              std::integer_sequence<int, Is...>) const {
#pragma unroll
        for (int c = 0; c < D; ++c) F[c] = P(0.0f);
#pragma unroll
        for (int k = 0; k < NB; ++k) G[k] = P(0.0f);
        ((norm2<D>(Is + 1) == 1 ? grad_nb<Is + 1>(am, a0, ap, F, G) : void()), ...);
        const P ratio = P(float(L::w(1) / L::w(Q - 1)));
#pragma unroll
        for (int c = 0; c < D; ++c) F[c] = F[c] * ratio;
#pragma unroll
        for (int k = 0; k < NB; ++k) G[k] = G[k] * ratio;
        ((norm2<D>(Is + 1) == 2 ? grad_nb<Is + 1>(am, a0, ap, F, G) : void()), ...);
        const float sc = float(-3.0 * L::w(Q - 1));
#pragma unroll
        for (int c = 0; c < D; ++c) F[c] = F[c] * P(sc);
#pragma unroll
        for (int k = 0; k < NB; ++k) G[k] = G[k] * P(k < D ? 2.0f * sc : sc);
    }

    template <typename Acc>
    __device__ __forceinline__ void stage2(int p, const uint32_t* zsp, Acc& acc, int& bad) {
        P F[D], G[NB];
        gradients(aux(p - 1), aux(p), aux(p + 1), F, G, std::make_integer_sequence<int, Q - 1>{});
        tmem_wait_st();  // this thread's store of plane p, an iteration ago
        float w[32];
        tmem_ld32(taddr(p), w);
        P bt[NB], rho, j[D], E;
        rho = P(w[0], w[1]);
#pragma unroll
        for (int c = 0; c < D; ++c) j[c] = P(w[2 * (1 + c)], w[2 * (1 + c) + 1]);
        E = P(w[2 * (D + 1)], w[2 * (D + 1) + 1]);
#pragma unroll
        for (int k = 0; k < NB; ++k) bt[k] = P(w[2 * (D + 2 + k)], w[2 * (D + 2 + k) + 1]);
        // populations in group 0: the rest go to collide as a TMEM address
        P df[Q];
        constexpr int NLO = 16 - Sh::NSV;  // populations in group 0
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (i < NLO) df[i] = P(w[2 * (Sh::NSV + i)], w[2 * (Sh::NSV + i) + 1]);
        const uint32_t s = (uint32_t)xa + ((D == 3) ? (uint32_t)yrow * (uint32_t)nx : 0u) + zsp[1];
        collide(s, df, taddr(p) + 32, bt, rho, j, E, F, G, acc, bad);
    }

    // Corrected u = (j0 + F/2)/rho (Eq. 57), temperature, diagnostics, SRT
    // update fbar* = fbar + omega (f^eq + tau Phi - fbar) (Eq. 55, Appendix A,
    // Eqs. 58-61) and bbar* = bbar + omega (b^eq - bbar) (Eqs. 63, 65) of
    // both sites, stored at s, s + 1.
    template <typename Acc>
    __device__ __forceinline__ void collide(uint32_t s, P* df, uint32_t thi, const P* bt, P rho, const P* j, P E,
                                            const P* F, const P* G, Acc& acc, int& bad) const {
        float omegaf, tauf, T0f;
        step_params(a, omegaf, tauf, T0f);
        const P omega = P(omegaf), tau = P(tauf);
        P trG = G[0];
#pragma unroll
        for (int c = 1; c < D; ++c) trG += G[c];
        const P irho = px::recip(rho);
        P u[D];
#pragma unroll
        for (int c = 0; c < D; ++c) u[c] = px::fma(P(0.5f), F[c], j[c]) * irho;
        P uu = u[0] * u[0];
#pragma unroll
        for (int c = 1; c < D; ++c) uu = px::fma(u[c], u[c], uu);
        const P Ecorr = px::fma(P(0.5f), trG, E);
        const P Tm = ((Ecorr - rho * uu) * irho) * P(float(1.0 / D));
        const P T = a.thermal ? Tm : P(T0f);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float r = h ? rho.b() : rho.a();
            const float ec = h ? Ecorr.b() : Ecorr.a();
            const float q2 = h ? uu.b() : uu.a();
            const float tm = h ? Tm.b() : Tm.a();
            if (!(r > 0.0f) || !isfinite(ec) || !isfinite(q2)) bad |= 1;
            if (a.thermal && !(tm > 0.0f)) bad |= 2;
        }
        if (a.want_diag) acc.add(rho, j, F, Ecorr);
        if (a.mout) {
            const long long N = a.N;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long sh = (long long)s + h;
                a.mout[sh] = double(h ? rho.b() : rho.a());
#pragma unroll
                for (int c = 0; c < D; ++c) a.mout[(1 + c) * N + sh] = double(h ? u[c].b() : u[c].a());
                a.mout[(1 + D) * N + sh] = double(h ? Tm.b() : Tm.a());
            }
        }
        if (!a.write_state) return;
        FS* __restrict__ fo = static_cast<FS*>(a.fout);
        const P dr = rho - P(1.0f);
        const P om1 = P(1.0f - omegaf);
        P mom[D];
#pragma unroll
        for (int c = 0; c < D; ++c) mom[c] = px::fma(tau, F[c], rho * u[c]);
        const P F0 = P(-1.5f * tauf) * trG;
        const P t45 = P(4.5f * tauf);
        P g45[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k) g45[k] = t45 * G[k];
        const P C0 = dr + F0;
        P ev[Q];
        if constexpr (D == 3) {
            P X[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) X[c] = u[c] * u[c];
            const P S = X[0] + X[1] + X[2];
            const P m2S = P(-2.0f) * S;
            const P q3 = px::fma(X[0], X[1], px::fma(X[0], X[2], X[1] * X[2]));
            ev[0] = P(float(1.0 / 3.0)) * px::fma(rho, px::fma(P(float(-2.0 / 3.0)), S, P(-2.0f) * q3), C0);
#pragma unroll
            for (int aa = 0; aa < 3; ++aa) {
                // axis pair along aa: e_aa = +1 is its first member
                const P t = px::fma(P(6.0f), S - X[aa], P(4.0f));
                const P inner = px::fma(X[aa], t, m2S);
                ev[aa == 0 ? 1 : (aa == 1 ? 2 : 5)] = P(float(1.0 / 18.0)) * (px::fma(rho, inner, C0) + g45[aa]);
            }
#pragma unroll
            for (int i = 7; i < Q; ++i) {
                if (i > opposite<3>(i)) continue;
                const int aa = L::e(i, 0) != 0 ? 0 : 1;
                const int bb = L::e(i, 2) != 0 ? 2 : 1;
                const int sab = L::e(i, aa) * L::e(i, bb);
                const P eu = sab > 0 ? u[aa] + u[bb] : u[aa] - u[bb];
                const P Xab = px::fma(P(6.0f) * X[aa], X[bb], X[aa] + X[bb]);
                const P gs = sab > 0 ? px::fma(P(2.0f), g45[sym<3>(aa, bb)], g45[aa] + g45[bb])
                                     : (g45[aa] + g45[bb]) - P(2.0f) * g45[sym<3>(aa, bb)];
                const P inner = px::fma(P(3.0f), eu * eu, P(0.0f) - Xab);
                ev[i] = P(float(1.0 / 36.0)) * (px::fma(rho, inner, C0) + gs);
            }
        } else {
            const P X = u[0] * u[0], Y = u[1] * u[1];
            const P m20 = px::fma(P(2.0f) * rho, X, dr) * P(float(1.0 / 3.0));
            const P m02 = px::fma(P(2.0f) * rho, Y, dr) * P(float(1.0 / 3.0));
            const P m11 = (P(float(2.0 / 3.0)) * rho) * (u[0] * u[1]);
            const P m22 = px::fma(rho, px::fma(P(2.0f), X + Y, P(-6.0f) * (X * Y)), dr) * P(float(1.0 / 9.0));
            ev[0] = px::fma(P(float(4.0 / 9.0)), F0, (dr - m20) - (m02 - m22));
            ev[1] = px::fma(P(0.5f), m20 - m22, P(float(1.0 / 9.0)) * (F0 + g45[0]));
            ev[2] = px::fma(P(0.5f), m02 - m22, P(float(1.0 / 9.0)) * (F0 + g45[1]));
            const P g01 = F0 + g45[0] + g45[1];
            ev[5] = px::fma(P(0.25f), m22 + m11, P(float(1.0 / 36.0)) * px::fma(P(2.0f), g45[2], g01));
            ev[6] = px::fma(P(0.25f), m22 - m11, P(float(1.0 / 36.0)) * (g01 - P(2.0f) * g45[2]));
        }
        if constexpr (Sh::TW > 32) {
            // the populations of group 1, loaded only now
            float w[32];
            tmem_ld32(thi, w);
            constexpr int NLO = 16 - Sh::NSV;
#pragma unroll
            for (int i = NLO; i < Q; ++i) df[i] = P(w[2 * (i - NLO)], w[2 * (i - NLO) + 1]);
        }
        PairIO<FS>::st2(fo, s, px::fma(om1, df[0], omega * ev[0]));
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int ib = opposite<D>(i);
            if (i > ib) continue;
            P eM;
            bool first = true;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                if (L::e(i, c) == 0) continue;
                eM = first ? mom[c] : (L::e(i, c) > 0 ? eM + mom[c] : eM - mom[c]);
                first = false;
            }
            const P A = omega * ev[i];
            const P B = P(float(3.0 * L::w(i)) * omegaf) * eM;
            PairIO<FS>::st2(fo, (uint32_t)i * Nu + s, px::fma(om1, df[i], A + B));
            PairIO<FS>::st2(fo, (uint32_t)ib * Nu + s, px::fma(om1, df[ib], A - B));
        }
        P bnew[NB];
#pragma unroll
        for (int c = 0; c < D; ++c)
#pragma unroll
            for (int d2 = c; d2 < D; ++d2) {
                const int k = sym<D>(c, d2);
                const P uc3 = u[c] * P(float(1.0 / 3.0));
                const P beq = (c == d2) ? px::fma(uc3, u[d2], T) : uc3 * u[d2];
                bnew[k] = px::fma(omega, beq - bt[k], bt[k]);
            }
        float* __restrict__ bo = static_cast<float*>(a.bout);
        if constexpr (D == 3) {
            // pair planes: (xx, yy), (zz, xy), (xz, yz) of site s, then of s + 1
#pragma unroll
            for (int pp = 0; pp < 3; ++pp)
                *reinterpret_cast<float4*>(bo + (size_t)pp * 2 * Nu + 2 * (size_t)s) =
                    make_float4(bnew[2 * pp].a(), bnew[2 * pp + 1].a(), bnew[2 * pp].b(), bnew[2 * pp + 1].b());
        } else {
#pragma unroll
            for (int k = 0; k < NB; ++k) *reinterpret_cast<float2*>(bo + (uint32_t)k * Nu + s) = bnew[k].v;
        }
    }
};

// Conservation diagnostics of both sites of a pair, summed per thread in
// packed FP32 as deviations from the rest state (mass as rho - 1, energy as
// E - D T0), then in FP64 per block.
template <int D> struct PairDiag {
    static constexpr bool kFF = true;  // reduced as float-float pairs (block_diagnostics)
    using P = px::P;
    P m, e, j[D];
    float eref;
    int n;
    __device__ __forceinline__ explicit PairDiag(float er) : m(0.0f), e(0.0f), eref(er), n(0) {
#pragma unroll
        for (int c = 0; c < D; ++c) j[c] = P(0.0f);
    }
    __device__ __forceinline__ void add(P rho, const P* jj, const P* F, P Ecorr) {
        m += rho - P(1.0f);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            j[c] += jj[c];
            j[c] = px::fma(P(0.5f), F[c], j[c]);  // exact halving, one rounding as an add
        }
        e += Ecorr - P(eref);
        n += 2;
    }
    __device__ __forceinline__ double get(int k) const {
        if (k == 0) return double(m.a()) + double(m.b()) + double(n);
        if (k == D + 1) return double(e.a()) + double(e.b()) + double(n) * double(eref);
        return double(j[k - 1].a()) + double(j[k - 1].b());
    }
    // value k = (h + l) + cnt() * cref(k): the two sites' sums as an exact
    // float-float pair
    __device__ __forceinline__ void ff(int k, float& h, float& l) const {
        const P v = k == 0 ? m : (k == D + 1 ? e : j[k - 1]);
        h = v.a();
        l = 0.0f;
        ff_add(h, l, v.b(), 0.0f);
    }
    __device__ __forceinline__ int cnt() const { return n; }
    __device__ __forceinline__ float cref(int k) const { return k == 0 ? 1.0f : (k == D + 1 ? eref : 0.0f); }
};

template <int D, typename FS, int TX, int TY, int MB, int PF>
__device__ __forceinline__ bool pair_segment(const TmaArgs& ta, unsigned char* smem, int bx, int by, int p0, int p1,
                                             PairDiag<D>& acc, int& bad, uint32_t tbase) {
    using Sh = PairShape<D, FS, TX, TY, MB, PF>;
    constexpr int NTILE = Sh::NTILE, NRING = Sh::NRING, RXP = Sh::RXP, TXP = Sh::TXP;
    PairBlock<D, FS, TX, TY, MB, PF> blk(ta, smem, bx, by, p0, p1);
    blk.tbase = tbase;
    const int tid = threadIdx.x;
    const bool tile = tid < NTILE;
    const bool ring = !tile && tid < NTILE + NRING;
    int kp = 0, ry = 0;
    if (tile) {
        kp = tid % TXP + 1;
        ry = (D == 3) ? tid / TXP + 1 : 0;
    } else if (ring) {
        const int k = tid - NTILE;
        if (D < 3) {
            kp = (k == 0) ? 0 : RXP - 1;
        } else if (k < RXP) {
            kp = k;
        } else if (k < 2 * RXP) {
            kp = k - RXP;
            ry = Sh::RY - 1;
        } else if (k < 2 * RXP + TY) {
            ry = k - 2 * RXP + 1;
        } else {
            kp = RXP - 1;
            ry = k - 2 * RXP - TY + 1;
        }
    }
    blk.set_pair(kp, ry);
    blk.tw = tid >> 5;
    blk.setup_halo();

    if (tid == 0) fence_proxy_async_smem();
    for (int q = p0 - 2; q <= min(p0 + PF, p1 + 1); ++q) {
        if (tid == 0) blk.issue_b(q);
        blk.b_pending |= 1u << blk.bs_of(q);
    }
    if (tid == 0)
        for (int Pl = p0 - 2; Pl <= min(p0 + 2, p1 + 1); ++Pl) blk.prefetch_f(Pl);
    blk.wait_b(p0 - 2);
    blk.wait_b(p0 - 1);
    if (blk.edge) {
        blk.patch_b(p0 - 2);
        blk.patch_b(p0 - 1);
    }
    // The pulls of a plane are issued one stage ahead: a tile pair loads plane
    // q + 1 before its stage 2 of plane q - 1, a ring pair before it waits for
    // the variance copy of the next plane, so that the L2 latency of the
    // loads overlaps that work.
    uint32_t zs[3], zsp[3] = {0u, 0u, 0u};
    px::P dfn[Sh::Q];
    blk.planes(p0 - 1, zs);
    if (tile || ring) blk.pull(zs, dfn);
    for (int q = p0 - 1; q <= p1; ++q) {
        blk.wait_b(q + 1);
        if (blk.edge) {
            blk.patch_b(q + 1);
            __syncthreads();
        }
        if (tile || ring) blk.stage1(q, dfn, tile);
        // one barrier per plane: aux of plane q complete, every read of the
        // variance slot of plane q - 1 done; it also tells every thread
        // whether a wait gave up
        if (__syncthreads_or(blk.timed_out)) {
            if (tid == 0) {
                atomicOr(ta.s.flag, 4);
                blk.drain();
            }
            return false;
        }
        const int qn = q + 2 + PF;
        if (qn <= p1 + 1) {
            if (tid == 0) {
                fence_proxy_async_smem();
                blk.issue_b(qn);
            }
            blk.b_pending |= 1u << blk.bs_of(qn);
        }
        if (tid == 0 && q + 3 <= p1 + 1) blk.prefetch_f(q + 3);
#pragma unroll
        for (int e = 0; e < 3; ++e) zsp[e] = zs[e];
        if (q + 1 <= p1) {
            blk.planes(q + 1, zs);
            if (tile || ring) blk.pull(zs, dfn);
        }
        if (tile && q - 1 >= p0) {
            uint32_t zs2[3];
            blk.planes(q - 1, zs2);
            blk.stage2(q - 1, zs2, acc, bad);
        }
    }
    __syncthreads();
    return true;
}

// Grid: (nx/TX, ny/TY, chunks), one segment of the march per block.
// Registers per thread: the MB blocks of an SM spread their warps over its
// four sub-partitions, each with 16 K registers (allocated per warp in steps
// of 8 per thread).
template <int D, typename FS, int TX, int TY, int MB, int PF> struct PairRegs {
    static constexpr int WARPS = PairShape<D, FS, TX, TY, MB, PF>::NT / 32 * MB;
    static constexpr int PER_SMSP = (WARPS + 3) / 4;
    static constexpr int R0 = 16384 / (32 * PER_SMSP) / 8 * 8;
    static constexpr int R = R0 > 255 ? 255 : R0;
};

template <int D, typename FS, int TX, int TY, int MB, int PF>
__global__ void __launch_bounds__(PairShape<D, FS, TX, TY, MB, PF>::NT) __maxnreg__((PairRegs<D, FS, TX, TY, MB, PF>::R))
    step_pair_kernel(const __grid_constant__ TmaArgs ta) {
    using Sh = PairShape<D, FS, TX, TY, MB, PF>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Sh::OFF_BAR);
    if (tid == 0) {
        for (int k = 0; k < Sh::NBS; ++k) mbar_init(bars + k, 1);
        fence_barrier_init();
    }
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + Sh::OFF_TADDR);
    if (tid < 32) tmem_alloc(tslot, Sh::TCOLS);  // warp 0
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const uint32_t tbase = *tslot;

    PairDiag<D> acc(float(D) * ta.s.T0_f);
    int bad = 0;
    const int np = (D == 3) ? ta.s.nz : ta.s.ny;
    const int p0 = ta.s.halo + blockIdx.z * ta.s.chunk;
    const bool ok = pair_segment<D, FS, TX, TY, MB, PF>(ta, smem, blockIdx.x, blockIdx.y, p0,
                                                    min(p0 + ta.s.chunk, np - ta.s.halo), acc, bad, tbase);
    // every thread's TMEM stores complete, then warp 0 frees the columns (on
    // the abort path too: the segment left with every thread)
    tmem_wait_st();
    tmem_fence_before_sync();
    __syncthreads();
    if (tid < 32) {
        tmem_fence_after_sync();
        tmem_dealloc(tbase, Sh::TCOLS);
    }
    if (!ok) return;
    if (bad) atomicOr(ta.s.flag, bad);
    if (ta.s.want_diag)
        block_diagnostics<D, Sh::NT>(ta.s, acc, reinterpret_cast<double*>(smem + Sh::OFF_RED));
}

// Ring pair k (0 .. NRING - 1) of a region: top row, bottom row, then the
// left and right columns of the tile rows.
template <int D, int TY, int RXP, int RY>
__device__ __forceinline__ void ring_pair(int k, int& kp, int& ry) {
    kp = 0;
    ry = 0;
    if (D < 3) {
        kp = (k == 0) ? 0 : RXP - 1;
    } else if (k < RXP) {
        kp = k;
    } else if (k < 2 * RXP) {
        kp = k - RXP;
        ry = RY - 1;
    } else if (k < 2 * RXP + TY) {
        ry = k - 2 * RXP + 1;
    } else {
        kp = RXP - 1;
        ry = k - 2 * RXP - TY + 1;
    }
}

// Warp-specialized segment: threads [0, NTILE) run stage 1 (their tile pair,
// then ring pair tid if tid < NRING), threads [NTILE, 2 NTILE) stage 2 of
// tile pair tid - NTILE -- the same TMEM lane and column group as its stage-1
// thread.  full[q]: every stage-1 thread has finished plane q (its aux values
// and hand-off words are written); empty[p]: every stage-2 thread has
// finished plane p (its reads of the aux planes p - 1 .. p + 1 and of its
// hand-off buffer are done).  Stage 1 of plane q reuses the aux slot and the
// hand-off buffer of plane q - 5 / q - 4, so it waits for empty[q - 4].  All
// waits are bounded; a wait that gives up raises flag bit 4, and the
// stage-1 threads agree on leaving at their per-plane barrier.
template <int D, typename FS, int TX, int TY>
__device__ __forceinline__ bool pair_segment_ws(const TmaArgs& ta, unsigned char* smem, int bx, int by, int p0,
                                                int p1, PairDiag<D>& acc, int& bad, uint32_t tbase) {
    using Sh = PairShape<D, FS, TX, TY, 1, 1, true>;
    using Blk = PairBlock<D, FS, TX, TY, 1, 1, true>;
    using P = px::P;
    constexpr int NTILE = Sh::NTILE, NRING = Sh::NRING, RXP = Sh::RXP, TXP = Sh::TXP, KB = Sh::KB;
    Blk blk(ta, smem, bx, by, p0, p1);
    blk.tbase = tbase;
    const int tid = threadIdx.x;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + Sh::OFF_PIPE);
    uint64_t* empty = full + KB;
    // Barrier k of a direction serves planes k, k + KB, ... counted from the
    // first plane that arrives on it: q0 for full (stage 1 starts at the
    // ring plane p0 - 1), p0 for empty (stage 2 starts at p0).  The use
    // count gives the phase whose completion a wait asks for.
    const int q0 = p0 - 1;
    auto fidx = [&](int q) { return (q - q0) % KB; };
    auto fpar = [&](int q) { return (uint32_t)(((q - q0) / KB) & 1); };
    auto eidx = [&](int p) { return (p - p0) % KB; };
    auto epar = [&](int p) { return (uint32_t)(((p - p0) / KB) & 1); };
    bool gave_up = false;
    // launched at 128 registers per thread: stage 2 (no pulls, no transport)
    // gives 16 per thread to stage 1, which keeps two planes of pulls in flight
    static_assert(Sh::NT == 512 && NTILE == 256, "register split sized for 2 x 256 threads at 128 registers");
    if (tid < NTILE) {
        regs_raise<144>();
        blk.tw = tid >> 5;
        int rkp, rry;
        ring_pair<D, TY, RXP, Sh::RY>(tid, rkp, rry);
        const bool has_ring = tid < NRING;
        blk.set_pair(rkp, rry);
        const typename Blk::Site sr = blk.site();
        blk.set_pair(tid % TXP + 1, (D == 3) ? tid / TXP + 1 : 0);
        const typename Blk::Site st = blk.site();
        blk.setup_halo();
        if (tid == 0) fence_proxy_async_smem();
        for (int q = p0 - 2; q <= min(p0 + 1, p1 + 1); ++q) {
            if (tid == 0) blk.issue_b(q);
            blk.b_pending |= 1u << blk.bs_of(q);
        }
        if (tid == 0)
            for (int Pl = p0 - 2; Pl <= min(p0 + 2, p1 + 1); ++Pl) blk.prefetch_f(Pl);
        // pulls run one plane ahead: each pair's next plane is loaded right
        // after its current plane has been consumed
        P dft[Sh::Q], dfr[Sh::Q];
        {
            uint32_t zs[3];
            blk.planes(q0, zs);
            blk.pull(zs, dft);
            if (has_ring) {
                blk.use(sr);
                blk.pull(zs, dfr);
                blk.use(st);
            }
        }
        blk.wait_b(p0 - 2);
        blk.wait_b(p0 - 1);
        if (blk.edge) {
            blk.patch_b(p0 - 2);
            blk.patch_b(p0 - 1);
        }
        for (int q = q0; q <= p1; ++q) {
            const int pe = q - 4;  // plane whose aux slot / hand-off buffer this plane reuses
            if (pe >= p0 && !mbar_wait_bounded(empty + eidx(pe), epar(pe), kWaitLimit)) gave_up = true;
            blk.wait_b(q + 1);
            if (blk.edge) blk.patch_b(q + 1);
            // patched slot visible to every stage-1 thread, every stage-1 read
            // of the slot of plane q - 2 done; and all agree on giving up
            if (named_sync_or(1, NTILE, gave_up || blk.timed_out)) {
                if (tid == 0) {
                    atomicOr(ta.s.flag, 4);
                    blk.drain();
                }
                gave_up = true;
                break;
            }
            if (q >= p0 && q + 2 <= p1 + 1) {
                if (tid == 0) {
                    fence_proxy_async_smem();
                    blk.issue_b(q + 2);
                }
                blk.b_pending |= 1u << blk.bs_of(q + 2);
            }
            if (tid == 0 && q + 3 <= p1 + 1) blk.prefetch_f(q + 3);
            uint32_t zn[3];
            blk.planes(q < p1 ? q + 1 : q, zn);
            blk.stage1(q, dft, true);
            if (q < p1) blk.pull(zn, dft);
            if (has_ring) {
                blk.use(sr);
                blk.stage1(q, dfr, false);
                if (q < p1) blk.pull(zn, dfr);
                blk.use(st);
            }
            // this thread's hand-off stores complete before the arrival
            tmem_wait_st();
            tmem_fence_before_sync();
            mbar_arrive(full + fidx(q));
        }
    } else {
        regs_lower<112>();
        const int t = tid - NTILE;
        blk.tw = t >> 5;
        blk.set_pair(t % TXP + 1, (D == 3) ? t / TXP + 1 : 0);
        for (int p = p0; p < p1; ++p) {
            if (!mbar_wait_bounded(full + fidx(p + 1), fpar(p + 1), kWaitLimit)) {
                atomicOr(ta.s.flag, 4);
                gave_up = true;
                break;
            }
            tmem_fence_after_sync();
            uint32_t zs[3];
            blk.planes(p, zs);
            blk.stage2(p, zs, acc, bad);
            tmem_fence_before_sync();
            mbar_arrive(empty + eidx(p));
        }
    }
    return !gave_up;
}

template <int D, typename FS, int TX, int TY>
__global__ void __launch_bounds__(PairShape<D, FS, TX, TY, 1, 1, true>::NT, 1)
    step_pair_ws_kernel(const __grid_constant__ TmaArgs ta) {
    using Sh = PairShape<D, FS, TX, TY, 1, 1, true>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int tid = threadIdx.x;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + Sh::OFF_BAR);
    uint64_t* pipe = reinterpret_cast<uint64_t*>(smem + Sh::OFF_PIPE);
    if (tid == 0) {
        for (int k = 0; k < Sh::NBS; ++k) mbar_init(bars + k, 1);
        for (int k = 0; k < 2 * Sh::KB; ++k) mbar_init(pipe + k, Sh::NTILE);
        fence_barrier_init();
    }
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + Sh::OFF_TADDR);
    if (tid < 32) tmem_alloc(tslot, Sh::TCOLS);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const uint32_t tbase = *tslot;

    PairDiag<D> acc(float(D) * ta.s.T0_f);
    int bad = 0;
    const int np = (D == 3) ? ta.s.nz : ta.s.ny;
    const int p0 = ta.s.halo + blockIdx.z * ta.s.chunk;
    const bool ok = pair_segment_ws<D, FS, TX, TY>(ta, smem, blockIdx.x, blockIdx.y, p0,
                                                   min(p0 + ta.s.chunk, np - ta.s.halo), acc, bad, tbase);
    tmem_wait_st();
    tmem_fence_before_sync();
    const bool any_fail = __syncthreads_or(!ok);
    if (tid < 32) {
        tmem_fence_after_sync();
        tmem_dealloc(tbase, Sh::TCOLS);
    }
    if (any_fail) return;
    if (bad) atomicOr(ta.s.flag, bad);
    if (ta.s.want_diag)
        block_diagnostics<D, Sh::NT>(ta.s, acc, reinterpret_cast<double*>(smem + Sh::OFF_RED));
}

}  // namespace lbm
