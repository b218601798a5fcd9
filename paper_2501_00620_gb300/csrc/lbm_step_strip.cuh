// Fused step of the bump-function lattice Boltzmann method (arXiv 2501.00620,
// Sec. II.C) for D2Q9 with FP32 or 16-bit storage on lattices of any extent.
// The arithmetic is the staged kernel's (lbm_step_fast.cuh): the packed
// variance transport (Eq. 66), the lean gradient (Eqs. 59, 61) and the FP32
// deviation-sum diagnostics; the data movement needs no tensor map, so it
// serves rows of any length:
//
// * A block of NT threads owns a strip of NT - 2 sites in x (the last strip
//   of a row may be shorter) and marches along y over `chunk` rows.  Thread t
//   is region site x0 - 1 + t: the one-site ring of the strip is the first
//   and last active lane, so no warp is set aside for the ring.
// * Variance rows are staged in a ring of four shared rows with plain
//   coalesced loads, issued into registers before stage 1 of a row and
//   stored after it, so their latency overlaps stage 1.
// * (u0, rho b) of the strip and ring live in four shared row slots; tile
//   sites hand their site values to stage 2 through two shared slots and
//   either pull their populations again or (HANDOFF) hand those over too.
// * FX selects the fixed-state boundary in x (frozen reservoirs).
#pragma once

#include "lbm_lean.cuh"

namespace lbm {

// HANDOFF: tile sites hand their pulled populations to stage 2 through
// shared memory (18 KB more) instead of pulling them again -- a gain where
// registers, not shared memory, bound the blocks per SM (the serving kernel).
template <typename FS, int NT, bool HANDOFF = false> struct StripShape {
    static constexpr int Q = 9, NB = 3, NA2 = 3;
    static constexpr int TX = NT - 2;    // tile sites of a full strip
    static constexpr int BW = NT + 2;    // staged variance row: x from x0 - 2
    static constexpr int NBS = 4, NAS = 4;
    static constexpr int NSV = NB + 2 + 2;  // bbar, rho, j0 (2), Ebar
    static constexpr int OFF_AUX = round_up(NBS * NB * BW * 4, 16);
    static constexpr int OFF_SV = OFF_AUX + NAS * NT * NA2 * 8;
    static constexpr int OFF_DF = OFF_SV + 2 * NSV * NT * 4;  // [2][Q][NT] populations of tile sites
    static constexpr int OFF_RED = OFF_DF + (HANDOFF ? 2 * Q * NT * 4 : 0);
    static constexpr int SMEM = OFF_RED + 32 * 4 * 8;
    static_assert(NT % 32 == 0 && NT <= 1024, "whole warps");
};

// One strip (bx) over march rows [bz*chunk, bz*chunk + chunk) of the lattice
// in `a`.  Every thread of the block calls it; it contains block barriers.
template <typename FS, int NT, bool FX, bool HANDOFF = false>
__device__ __forceinline__ void strip_block(const StepArgs& a, int bx, int bz, unsigned char* smem,
                                            DiagDev<4>& acc, int& bad) {
    using L = Lattice<2>;
    using Sh = StripShape<FS, NT, HANDOFF>;
    constexpr int Q = Sh::Q, NB = Sh::NB, NA2 = Sh::NA2, BW = Sh::BW;
    const int tid = threadIdx.x;
    const int nx = a.nx, np = a.ny, Ni = (int)a.N, rows = (int)a.rows;
    const int x0 = bx * Sh::TX;
    const int txe = min(Sh::TX, nx - x0);  // tile sites of this strip
    const int p0 = a.halo + bz * a.chunk, p1 = min(p0 + a.chunk, np - a.halo);
    const bool interior = tid >= 1 && tid <= txe;
    const bool active = tid <= txe + 1;
    const int gx = x0 - 1 + tid;
    const bool reservoir = FX && (gx < 0 || gx >= nx);
    float omega, tau, T0;
    step_params(a, omega, tau, T0);
    (void)tau;

    auto modx = [nx](int v) {
        const int r = v % nx;
        return r < 0 ? r + nx : r;
    };
    // rows q in [p0 - 2, p1 + 1]: one conditional add or subtract when
    // np >= 3; the loops cover lattices of one or two rows
    auto wrapq = [np](int q) {
        while (q < 0) q += np;
        while (q >= np) q -= np;
        return q;
    };
    const int gxw = modx(gx);
    int xs[3];
    int xo = 0;  // FX: bit e+1 set if source column x - e lies outside [0, nx)
#pragma unroll
    for (int e = -1; e <= 1; ++e) {
        const int sx = gx - e;
        xs[e + 1] = modx(sx);
        if (FX && (sx < 0 || sx >= nx)) xo |= 1 << (e + 1);
    }

    float* bslots = reinterpret_cast<float*>(smem);
    float2* auxs = reinterpret_cast<float2*>(smem + Sh::OFF_AUX);
    float* svs = reinterpret_cast<float*>(smem + Sh::OFF_SV);
    auto bslot = [&](int r) { return bslots + ((r - (p0 - 2)) & 3) * (NB * BW); };
    auto aux = [&](int q) { return auxs + ((q - p0 + 1) & 3) * (NT * NA2); };
    auto sv = [&](int q) { return svs + (q & 1) * (Sh::NSV * NT) + tid; };
    float* dfbase = reinterpret_cast<float*>(smem + Sh::OFF_DF);
    auto dfs = [&](int q) { return dfbase + (q & 1) * (Q * NT) + tid; };

    // variance of row r at staged positions c = tid, tid + NT (x = x0 - 2 + c)
    const float* __restrict__ bin = static_cast<const float*>(a.bin);
    const float* __restrict__ gb = static_cast<const float*>(a.gb);
    const int ncol = txe + 4;
    auto load_row = [&](int r, float (*v)[NB]) {
        const int rr = wrapq(r);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = tid + h * NT;
            if (c >= ncol) continue;
            const int x = x0 - 2 + c;
            if (FX && (x < 0 || x >= nx)) {
#pragma unroll
                for (int k = 0; k < NB; ++k) v[h][k] = gb[((x < 0 ? 0 : 1) * NB + k) * rows + rr];
            } else {
                const int s = modx(x) + nx * rr;
#pragma unroll
                for (int k = 0; k < NB; ++k) v[h][k] = bin[k * Ni + s];
            }
        }
    };
    auto store_row = [&](int r, float (*v)[NB]) {
        float* sl = bslot(r);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = tid + h * NT;
            if (c >= ncol) continue;
#pragma unroll
            for (int k = 0; k < NB; ++k) sl[k * BW + c] = v[h][k];
        }
    };

    // Pull: df_i = stored deviation of fbar*_i at (x - e_i) (Eq. 49).
    const FS* __restrict__ fin = static_cast<const FS*>(a.fin);
    auto pull = [&](int q, float* df) {
        int ys[3];
#pragma unroll
        for (int e = -1; e <= 1; ++e) ys[e + 1] = wrapq(q - e);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int ex = L::e(i, 0), ey = L::e(i, 1);
            if (FX && ex != 0 && (xo & (1 << (ex + 1)))) {
                const float* __restrict__ gf = static_cast<const float*>(a.gf);
                df[i] = gf[((ex > 0 ? 0 : 1) * Q + i) * rows + ys[ey + 1]];
            } else {
                df[i] = Store<FS>::ld(fin + i * Ni, xs[ex + 1] + nx * ys[ey + 1]);
            }
        }
    };

    // Stage 1 at row q: pull, variance transport, moments; (u0, rho b) to
    // the aux row, site values of a tile site to its own column.
    auto stage1 = [&](int q) {
        float2* ax = aux(q) + tid * NA2;
        if (FX && reservoir) {
            const float* __restrict__ gaux = static_cast<const float*>(a.gaux);
            const int row = wrapq(q);
            const int side = gx < 0 ? 0 : 1;
            constexpr int NAUX = 2 + NB;
            float u0[2], rb[NB];
#pragma unroll
            for (int c = 0; c < 2; ++c) u0[c] = gaux[(side * NAUX + c) * rows + row];
#pragma unroll
            for (int k = 0; k < NB; ++k) rb[k] = gaux[(side * NAUX + 2 + k) * rows + row];
            put_aux<2>(ax, u0, rb);
            return;
        }
        float df[Q];
        pull(q, df);
        const float* bm = bslot(q - 1) + tid + 1;  // source row q-1 (e_y = +1), column x
        const float* b0 = bslot(q) + tid + 1;
        const float* bp = bslot(q + 1) + tid + 1;
        float2 acc2;
        float accxy;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int ey = L::e(i, 1);
            const float* src = ((ey == 1) ? bm : ((ey == -1) ? bp : b0)) - L::e(i, 0);
            const float fi = float(L::w(i)) + df[i];
            const float2 f2 = make_float2(fi, fi);
            const float2 bxy = make_float2(src[0], src[BW]);
            if (i == 0) {
                acc2 = __fmul2_rn(f2, bxy);
                accxy = fi * src[2 * BW];
            } else {
                acc2 = __ffma2_rn(f2, bxy, acc2);
                accxy = fmaf(fi, src[2 * BW], accxy);
            }
        }
        const float bsum[NB] = {acc2.x, acc2.y, accxy};
        float u0[2], rb[NB], bt[NB], rho, j[2], E;
        site_moments<2, float>(df, bsum, omega, T0, a.thermal, bt, rho, j, E, u0, rb);
        if (interior) {
            if constexpr (HANDOFF) {
                float* dv = dfs(q);
#pragma unroll
                for (int i = 0; i < Q; ++i) dv[i * NT] = df[i];
            }
            float* v = sv(q);
#pragma unroll
            for (int k = 0; k < NB; ++k) v[k * NT] = bt[k];
            v[NB * NT] = rho;
            v[(NB + 1) * NT] = j[0];
            v[(NB + 2) * NT] = j[1];
            v[(NB + 3) * NT] = E;
        }
        put_aux<2>(ax, u0, rb);
    };

    // Stage 2 at row p: gradients from the aux rows p-1..p+1, collision,
    // store (site_collide).
    auto stage2 = [&](int p) {
        const float2* am = aux(p - 1) + tid * NA2;
        const float2* a0 = aux(p) + tid * NA2;
        const float2* ap = aux(p + 1) + tid * NA2;
        float F[2], G[NB];
        gradients<2>(
            [&](auto I) {
                constexpr int i = decltype(I)::value;
                constexpr int ey = L::e(i, 1);
                const float2* as = (ey == 1) ? ap : ((ey == -1) ? am : a0);
                return as + L::e(i, 0) * NA2;
            },
            F, G);
        const float* v = sv(p);
        float c_bt[NB], c_j[2];
#pragma unroll
        for (int k = 0; k < NB; ++k) c_bt[k] = v[k * NT];
        const float c_rho = v[NB * NT];
        c_j[0] = v[(NB + 1) * NT];
        c_j[1] = v[(NB + 2) * NT];
        const float c_E = v[(NB + 3) * NT];
        float df[Q];
        if constexpr (HANDOFF) {
            const float* dv = dfs(p);  // the populations stage 1 pulled
#pragma unroll
            for (int i = 0; i < Q; ++i) df[i] = dv[i * NT];
        } else {
            pull(p, df);  // second pull of the same values
        }
        const int s = gxw + nx * wrapq(p);
        site_collide<2, FS, float, int, DiagDev<4>>(a, s, df, c_bt, c_rho, c_j, c_E, F, G, acc, bad);
    };

    // prologue: variance rows p0-2 .. p0
    {
        float v[2][NB];
        for (int r = p0 - 2; r <= p0; ++r) {
            load_row(r, v);
            store_row(r, v);
        }
    }
    __syncthreads();
    // L2 prefetch of this site's populations in row P (all Q planes): the
    // first pull from row P is made by stage 1 of row P - 1
    auto prefetch_row = [&](int P) {
        if (!active || reservoir) return;
        const int s = gxw + nx * wrapq(P);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const FS* pp = fin + i * Ni + s;
            asm volatile("prefetch.global.L2 [%0];" ::"l"(pp));
        }
    };
    for (int r = p0 - 2; r <= min(p0 + 1, p1 + 1); ++r) prefetch_row(r);
    for (int q = p0 - 1; q <= p1; ++q) {
        if (q + 3 <= p1 + 1) prefetch_row(q + 3);
        // variance row q+2 (read by stage 1 of row q+1) into registers now,
        // into its slot -- that of row q-2, last read before the previous
        // barrier -- after stage 1
        const bool more = q + 2 <= p1 + 1;
        float v[2][NB];
        if (more) load_row(q + 2, v);
        if (active) stage1(q);
        if (more) store_row(q + 2, v);
        // aux of row q complete; variance row q+2 staged
        __syncthreads();
        if (interior && q - 1 >= p0) stage2(q - 1);
    }
}

template <typename FS, int NT, bool FX>
__global__ void __launch_bounds__(NT) step_strip_kernel(const StepArgs a) {
    using Sh = StripShape<FS, NT>;
    extern __shared__ __align__(16) unsigned char smem[];
    DiagDev<4> acc(2.0f * a.T0_f);
    int bad = 0;
    strip_block<FS, NT, FX>(a, blockIdx.x, blockIdx.z, smem, acc, bad);
    if (bad) atomicOr(a.flag, bad);
    if (a.want_diag) block_diagnostics<2, NT>(a, acc, reinterpret_cast<double*>(smem + Sh::OFF_RED));
}

}  // namespace lbm
