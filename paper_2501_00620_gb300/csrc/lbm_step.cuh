// Fused single-pass update of the bump-function lattice Boltzmann method
// (arXiv 2501.00620, Sec. II.C), pull scheme with A-B buffers -- the generic
// kernel (any extents, FP64 included; loads through the L1/L2 caches).
//
// Stored state: the EMITTED (post-collision, about-to-stream) populations
// S_i(x) = fbar*_i(x) and variance bt*(x) of the last step.  One launch maps
// S(t) -> S(t+1):
//   stage 1 (every site of the tile plus a one-site ring):
//     pull fbar_i(x) = S_i(x - e_i) (Eq. 49) and the mass-weighted variance
//     bbar(x) = sum_i fbar_i bt*(x - e_i) / rho (Eq. 66); moments; rho*b for
//     the gradient (Eq. 68); u0 and rho*b go to shared memory.
//   stage 2 (tile sites): gradient corrections, equilibrium + forcing, SRT
//     update, store S(t+1) (site_collide).
// Walls (a.walls, D = 2, 3): half-way bounce-back walls normal to the march
// axis, half a site outside the lattice (Sec. III.A).  A population whose
// source lies beyond a wall is the site's own emission in the opposite
// direction, carrying the site's bt*; the gradient stencil sees, one plane
// beyond a wall, the image of the plane facing it (same rho*b, reversed u0).
// A moving wall (a.walls_moving, velocity u_w along the wall) adds its
// momentum to a bounced population, 6 w_i rho(x, t) e_i.u_w with rho(x, t)
// the sum of the site's own emissions, and the image velocity is reflected
// about the wall's, 2 u_w - u0 (Sec. III.D).
// Body force (a.forced): F + rho a and G + rho (u a + a u) with the corrected
// u = (j + F/2)/rho of Eq. 57.
// MRT (a.mrt, D = 3): the SRT result is stored, then the difference of the
// MRT step in the third- and fourth-order moments of Table M is added
// (lbm_mrt.cuh).
// The gradient needs rho*b on the neighbours, which exist only after the
// neighbours have pulled; the ring is recomputed per tile and the kernel
// marches along the slowest axis keeping three planes of (u0, rho b) in a
// rolling shared-memory window, so each stored value is read from HBM about
// once per step.
#pragma once

#include <cooperative_groups.h>
#include <cstdint>
#include <type_traits>

#include "lbm_mrt.cuh"
#include "lbm_site.cuh"

namespace lbm {

__device__ __forceinline__ int wrap1(int c, int n) { return c < 0 ? c + n : (c >= n ? c - n : c); }
__device__ __forceinline__ int modp(int c, int n) {
    int r = c % n;
    return r < 0 ? r + n : r;
}

// Shared-memory footprint of the aux window: 3 planes x (D + NB) x region.
template <int D, typename FS, int TX, int TY> struct StepShape {
    using L = Lattice<D>;
    using real = typename Store<FS>::real;
    static constexpr int RX = TX + 2;
    static constexpr int RY = (D == 3) ? TY + 2 : 1;
    static constexpr int RS = RX * RY;
    static constexpr int NAUX = D + L::NB;
    static constexpr int NSLOT = (D == 1) ? 1 : 3;
    static constexpr size_t aux_bytes = (sizeof(real) * NSLOT * NAUX * RS + 15) / 16 * 16;
    static constexpr size_t smem = aux_bytes + sizeof(double) * 32 * (D + 2);
};

// One tile (bx, by) x chunk bz of the fused step; the body of step_kernel,
// also run per work item by the batched serving kernel.
template <int D, typename FS, int TX, int TY>
__device__ __forceinline__ void step_block(const StepArgs& a, int bx, int by, int bz, unsigned char* smem_raw) {
    using L = Lattice<D>;
    using Sh = StepShape<D, FS, TX, TY>;
    using real = typename Store<FS>::real;
    using breal = typename Store<FS>::breal;
    constexpr int Q = L::Q, NB = L::NB, NAUX = Sh::NAUX;
    constexpr int RX = Sh::RX, RS = Sh::RS;
    constexpr int NT = TX * TY;
    constexpr int NRING = RS - TX * TY;

    real* aux = reinterpret_cast<real*>(smem_raw);  // [NSLOT][NAUX][RS]
    double* red = reinterpret_cast<double*>(smem_raw + Sh::aux_bytes);

    const FS* __restrict__ fin = static_cast<const FS*>(a.fin);
    const breal* __restrict__ bin = static_cast<const breal*>(a.bin);
    const real* __restrict__ gf = static_cast<const real*>(a.gf);
    const real* __restrict__ gb = static_cast<const real*>(a.gb);
    const real* __restrict__ gaux = static_cast<const real*>(a.gaux);

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int x0 = bx * TX;
    const int y0 = (D == 3) ? by * TY : 0;
    const int np = (D == 3) ? a.nz : (D == 2 ? a.ny : 1);
    const int p0 = (D == 1) ? 0 : a.halo + bz * a.chunk;
    const int p1 = (D == 1) ? 1 : min(p0 + a.chunk, np - a.halo);
    const long long N = a.N;
    real omega, tau, T0;
    step_params(a, omega, tau, T0);
    (void)tau;
    const int nx = a.nx, ny = a.ny, nz = a.nz;

    // interior site of this thread in region coordinates
    const int rxi = tx + 1, ryi = (D == 3) ? ty + 1 : 0;
    // ring site of this thread (if tid < NRING)
    int rxr = 0, ryr = 0;
    if (tid < NRING) {
        if (D < 3) {
            rxr = (tid == 0) ? 0 : RX - 1;
        } else if (tid < RX) {
            rxr = tid;
            ryr = 0;
        } else if (tid < 2 * RX) {
            rxr = tid - RX;
            ryr = Sh::RY - 1;
        } else if (tid < 2 * RX + TY) {
            rxr = 0;
            ryr = tid - 2 * RX + 1;
        } else {
            rxr = RX - 1;
            ryr = tid - 2 * RX - TY + 1;
        }
    }

    // interior values carried from stage 1 of plane p to stage 2 of plane p
    real c_df[Q], c_bt[NB], c_rho, c_j[D], c_E;
    real n_df[Q], n_bt[NB], n_rho, n_j[D], n_E;
    double c_E64 = -1.0, n_E64 = -1.0;  // FP64 Ebar of a small-T site (32/16-bit storage), else -1

    DiagAcc<real, D + 2> acc;
    int bad = 0;

    auto slot_of = [&](int p) { return (D == 1) ? 0 : (p - p0 + 1) % 3; };

    // Stage 1 for one region site at march plane q (wrapped).  Writes u0 and
    // rho*b into aux[slot]; returns the site's values if `keep`.
    auto stage1_site = [&](int rx, int ry, int q, int slot, int img, bool keep, real* o_df, real* o_bt,
                           real& o_rho, real* o_j, real& o_E) {
        int gx = x0 - 1 + rx;
        int gy = (D == 3) ? modp(y0 - 1 + ry, ny) : (D == 2 ? q : 0);
        int gz = (D == 3) ? q : 0;
        const int r = rx + RX * ry;
        const bool outside = a.fixed_x && (gx < 0 || gx >= nx);
        if (outside) {
            const int side = gx < 0 ? 0 : 1;
            const long long row = gy + (long long)ny * gz;
#pragma unroll
            for (int k = 0; k < NAUX; ++k)
                aux[(slot * NAUX + k) * RS + r] = gaux[((long long)side * NAUX + k) * a.rows + row];
            return;
        }
        if (!a.fixed_x) gx = modp(gx, nx);
        const long long self = gx + (long long)nx * (gy + (long long)ny * gz);
        // density of this site at t (sum of its emissions) for the momentum a
        // moving wall gives to the populations bounced there
        real rho_self = real(1);
        if (D > 1 && a.walls_moving) {
            const int gw = (D == 3) ? gz : gy;
            if (gw == 0 || gw == np - 1) {
#pragma unroll
                for (int k = 0; k < Q; ++k) rho_self += Store<FS>::ld(fin, (long long)k * N + self);
            }
        }
        // source of population i: its stored value and the variance it carries
        auto fetch = [&](int i, real& v, real* bv) {
            int sx = gx - L::e(i, 0);
            int sy = (D >= 2) ? wrap1(gy - L::e(i, 1), ny) : 0;
            int sz = (D == 3) ? wrap1(gz - L::e(i, 2), nz) : 0;
            const int sm = (D == 3) ? gz - L::e(i, 2) : gy - L::e(i, 1);
            if (D > 1 && a.walls && (sm < 0 || sm >= np)) {
                // half-way bounce-back: the site's own opposite emission,
                // plus the momentum of a moving wall
                v = Store<FS>::ld(fin, (long long)opposite<D>(i) * N + self);
                if (a.walls_moving) {
                    const int side = sm < 0 ? 0 : 1;
                    real eu = real(0);
#pragma unroll
                    for (int c = 0; c < D; ++c)
                        if (L::e(i, c) != 0) eu += real(L::e(i, c)) * uw_param(a, side, c, real(0));
                    v += real(6) * real(L::w(i)) * rho_self * eu;
                }
#pragma unroll
                for (int k = 0; k < NB; ++k) bv[k] = real(__ldg(bin + BLayout<D, FS>::at(k, self, N)));
            } else if (a.fixed_x && (sx < 0 || sx >= nx)) {
                const int side = sx < 0 ? 0 : 1;
                const long long row = sy + (long long)ny * sz;
                v = gf[((long long)side * Q + i) * a.rows + row];
#pragma unroll
                for (int k = 0; k < NB; ++k) bv[k] = gb[((long long)side * NB + k) * a.rows + row];
            } else {
                sx = wrap1(sx, nx);
                const long long s = sx + (long long)nx * (sy + (long long)ny * sz);
                v = Store<FS>::ld(fin, (long long)i * N + s);
#pragma unroll
                for (int k = 0; k < NB; ++k) bv[k] = real(__ldg(bin + BLayout<D, FS>::at(k, s, N)));
            }
        };
        real df[Q], bsum[NB];
#pragma unroll
        for (int k = 0; k < NB; ++k) bsum[k] = real(-0.0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            real v, bv[NB];
            fetch(i, v, bv);
            df[i] = v;
            const real fi = real(L::w(i)) + v;
#pragma unroll
            for (int k = 0; k < NB; ++k) bsum[k] += fi * bv[k];
        }
        real bt[NB], rho, j[D], E, u0[D], rb[NB];
        site_moments<D, real>(df, bsum, omega, T0, a.thermal, bt, rho, j, E, u0, rb);
        double E64 = -1.0;
        if constexpr (std::is_same<real, float>::value) {
            if (a.thermal && a.small_t_f > 0.0f) {
                real uu = real(0);
#pragma unroll
                for (int c = 0; c < D; ++c) uu += u0[c] * u0[c];
                const real Tu = (E - rho * uu) / (real(D) * rho);
                if (Tu < a.small_t_f * uu) {
                    // T << |u|^2: the transport (Eq. 66), the moments and
                    // rho b (Eq. 68) again in FP64 from the same sources
                    double bs[NB], r = 1.0, jj[D], e = 0.0;
#pragma unroll
                    for (int k = 0; k < NB; ++k) bs[k] = 0.0;
#pragma unroll
                    for (int c = 0; c < D; ++c) jj[c] = 0.0;
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        real v, bv[NB];
                        fetch(i, v, bv);
                        const double d = v, fi = L::w(i) + d;
#pragma unroll
                        for (int k = 0; k < NB; ++k) bs[k] += fi * (double)bv[k];
                        r += d;
#pragma unroll
                        for (int c = 0; c < D; ++c)
                            if (L::e(i, c) != 0) jj[c] += L::e(i, c) * d;
                        e += (norm2<D>(i) - D * (1.0 / 3.0)) * d;
                    }
                    double b64[NB], tr = 0.0;
#pragma unroll
                    for (int k = 0; k < NB; ++k) b64[k] = bs[k] / r;
#pragma unroll
                    for (int c = 0; c < D; ++c) tr += b64[c];
                    e += r * tr;
                    double u64[D], q = 0.0;
#pragma unroll
                    for (int c = 0; c < D; ++c) {
                        u64[c] = jj[c] / r;
                        q += u64[c] * u64[c];
                    }
                    const double Tu64 = (e - r * q) / (D * r);
                    const double hw = 0.5 * a.omega;
#pragma unroll
                    for (int c = 0; c < D; ++c)
#pragma unroll
                        for (int d2 = c; d2 < D; ++d2) {
                            const int k = sym<D>(c, d2);
                            const double beq = u64[c] * u64[d2] / 3.0 + (c == d2 ? Tu64 : 0.0);
                            double v = r * (b64[k] - hw * (b64[k] - beq));
                            if (c == d2) v -= r / 3.0;
                            rb[k] = real(v);
                        }
#pragma unroll
                    for (int k = 0; k < NB; ++k) bt[k] = real(b64[k]);
#pragma unroll
                    for (int c = 0; c < D; ++c) u0[c] = real(u64[c]);
                    E = real(e);
                    E64 = e;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NB; ++k) aux[(slot * NAUX + D + k) * RS + r] = rb[k];
#pragma unroll
        for (int c = 0; c < D; ++c)
            aux[(slot * NAUX + c) * RS + r] =
                img < 0 ? u0[c] : real(2) * uw_param(a, img, c, real(0)) - u0[c];
        if (keep) {
            n_E64 = E64;
#pragma unroll
            for (int i = 0; i < Q; ++i) o_df[i] = df[i];
#pragma unroll
            for (int k = 0; k < NB; ++k) o_bt[k] = bt[k];
            o_rho = rho;
#pragma unroll
            for (int c = 0; c < D; ++c) o_j[c] = j[c];
            o_E = E;
        }
    };

    auto stage1 = [&](int q, bool keep_next) {
        // beyond a wall: the image of the plane facing it (-1 -> 0, np -> np - 1);
        // img = the wall crossed (0 lower, 1 upper), -1 for a fluid plane
        const int img = (D > 1 && a.walls && (q < 0 || q >= np)) ? (q < 0 ? 0 : 1) : -1;
        const int qq = (D == 1) ? 0 : (img >= 0 ? (q < 0 ? -1 - q : 2 * np - 1 - q) : modp(q, np));
        const int slot = slot_of(q);
        stage1_site(rxi, ryi, qq, slot, img, keep_next, n_df, n_bt, n_rho, n_j, n_E);
        if (tid < NRING) {
            real d_df[Q], d_bt[NB], d_rho, d_j[D], d_E;
            stage1_site(rxr, ryr, qq, slot, img, false, d_df, d_bt, d_rho, d_j, d_E);
        }
    };

    // Stage 2 for the interior site of this thread at plane p.
    auto stage2 = [&](int p) {
        const int gx = x0 + tx;
        const int gy = (D == 3) ? y0 + ty : (D == 2 ? p : 0);
        const int gz = (D == 3) ? p : 0;
        if (gx >= nx || (D == 3 && gy >= ny)) return;
        const long long s = gx + (long long)nx * (gy + (long long)ny * gz);
        real F[D], G[NB];
#pragma unroll
        for (int c = 0; c < D; ++c) F[c] = real(-0.0);
#pragma unroll
        for (int k = 0; k < NB; ++k) G[k] = real(-0.0);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const int em = (D == 3) ? L::e(i, 2) : (D == 2 ? L::e(i, 1) : 0);
            const int slot = (D == 1) ? 0 : slot_of(p + em);
            const int r = (rxi + L::e(i, 0)) + RX * ((D == 3) ? ryi + L::e(i, 1) : 0);
            real rbn[NB], un[D];
#pragma unroll
            for (int k = 0; k < NB; ++k) rbn[k] = aux[(slot * NAUX + D + k) * RS + r];
#pragma unroll
            for (int c = 0; c < D; ++c) un[c] = aux[(slot * NAUX + c) * RS + r];
            fd_add<D, real>(i, rbn, un, F, G);
        }
#pragma unroll
        for (int c = 0; c < D; ++c) F[c] *= real(-3);
#pragma unroll
        for (int k = 0; k < NB; ++k) G[k] *= real(-3);
        if (a.forced) {
            real ga[D], ru[D];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                ga[c] = acc_param(a, c, real(0));
                F[c] += c_rho * ga[c];
            }
#pragma unroll
            for (int c = 0; c < D; ++c) ru[c] = c_j[c] + real(0.5) * F[c];
#pragma unroll
            for (int c = 0; c < D; ++c)
#pragma unroll
                for (int d2 = c; d2 < D; ++d2) G[sym<D>(c, d2)] += ru[c] * ga[d2] + ru[d2] * ga[c];
        }
        site_collide<D, FS, real>(a, s, c_df, c_bt, c_rho, c_j, c_E, F, G, acc, bad, c_E64);
        if constexpr (D == 3) {
            if (a.mrt && a.write_state) mrt_correct<FS, real>(a, s, c_df, c_rho, c_j, F);
        }
    };

    auto carry = [&]() {
#pragma unroll
        for (int i = 0; i < Q; ++i) c_df[i] = n_df[i];
#pragma unroll
        for (int k = 0; k < NB; ++k) c_bt[k] = n_bt[k];
        c_rho = n_rho;
#pragma unroll
        for (int c = 0; c < D; ++c) c_j[c] = n_j[c];
        c_E = n_E;
        c_E64 = n_E64;
    };

    if (D == 1) {
        stage1(0, true);
        carry();
        __syncthreads();
        stage2(0);
    } else {
        stage1(p0 - 1, false);
        stage1(p0, true);
        carry();
        for (int p = p0; p < p1; ++p) {
            stage1(p + 1, true);
            __syncthreads();
            stage2(p);
            __syncthreads();
            carry();
        }
    }

    if (bad) atomicOr(a.flag, bad);
    if (a.want_diag) block_diagnostics<D, NT>(a, acc, red);
}

template <int D, typename FS, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) step_kernel(const StepArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    step_block<D, FS, TX, TY>(a, blockIdx.x, blockIdx.y, blockIdx.z, smem_raw);
}

// K steps in one cooperative launch (small lattices, where a launch costs
// more than the step): the blocks run the tile body on the arguments of the
// current parity (a[0] reads buffer 0, a[1] buffer 1) and meet at a
// grid-wide barrier after every step.  Every block must be resident; the
// launcher checks that before it launches.
template <int D, typename FS, int TX, int TY>
__global__ void __launch_bounds__(TX* TY) step_multi_kernel(const StepArgs a0, const StepArgs a1, int K) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cooperative_groups::grid_group grid = cooperative_groups::this_grid();
    for (int k = 0; k < K; ++k) {
        step_block<D, FS, TX, TY>((k & 1) ? a1 : a0, blockIdx.x, blockIdx.y, blockIdx.z, smem_raw);
        __syncthreads();  // the next step reuses shared memory
        grid.sync();
    }
}

// ---------------------------------------------------------------------------
// Start: every site emits its local equilibrium, df = f^eq(rho, u) - w,
// bt = b^eq(u, T) + I/3 = T I + u u / 3 (Eq. 36, Appendix A).
template <int D, typename FS>
__device__ __forceinline__ void init_site(const double* __restrict__ rho, const double* __restrict__ u,
                                          const double* __restrict__ T, FS* __restrict__ f,
                                          typename Store<FS>::breal* __restrict__ b, long long N, long long s) {
    using L = Lattice<D>;
    using real = typename Store<FS>::real;
    real uu[D];
#pragma unroll
    for (int c = 0; c < D; ++c) uu[c] = real(u[c * N + s]);
    real df[L::Q];
    Equilibrium<D, real>::dev(real(rho[s]), uu, df);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) Store<FS>::st(f, i * N + s, df[i]);
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
        for (int d2 = c; d2 < D; ++d2)
            b[BLayout<D, FS>::at(sym<D>(c, d2), s, N)] = uu[c] * uu[d2] * real(1.0 / 3.0) + (c == d2 ? real(T[s]) : real(0));
}

template <int D, typename FS>
__global__ void init_kernel(const double* __restrict__ rho, const double* __restrict__ u,
                            const double* __restrict__ T, FS* __restrict__ f,
                            typename Store<FS>::breal* __restrict__ b, long long N) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s < N) init_site<D, FS>(rho, u, T, f, b, N, s);
}

// Reservoirs of the fixed-state boundary: for each row, the equilibrium of the
// edge site's initial state (side 0: x = 0, side 1: x = nx - 1).
template <int D, typename R>
__device__ __forceinline__ void reservoir_item(const double* __restrict__ rho, const double* __restrict__ u,
                                               const double* __restrict__ T, int nx, long long rows, long long N,
                                               R* __restrict__ gf, R* __restrict__ gb, R* __restrict__ gaux,
                                               long long t) {
    using L = Lattice<D>;
    constexpr int NB = L::NB, NAUX = D + NB;
    const int side = (int)(t / rows);
    const long long row = t % rows;
    const long long s = (side ? nx - 1 : 0) + (long long)nx * row;
    R uu[D];
#pragma unroll
    for (int c = 0; c < D; ++c) uu[c] = R(u[c * N + s]);
    const R r = R(rho[s]), TT = R(T[s]);
    R df[L::Q];
    Equilibrium<D, R>::dev(r, uu, df);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) gf[((long long)side * L::Q + i) * rows + row] = df[i];
#pragma unroll
    for (int c = 0; c < D; ++c) gaux[((long long)side * NAUX + c) * rows + row] = uu[c];
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
        for (int d2 = c; d2 < D; ++d2) {
            const int k = sym<D>(c, d2);
            const R bt = uu[c] * uu[d2] * R(1.0 / 3.0) + (c == d2 ? TT : R(0));
            gb[((long long)side * NB + k) * rows + row] = bt;
            // rho*b of a site at equilibrium: rho (b^eq) = rho (bt - I/3)
            gaux[((long long)side * NAUX + D + k) * rows + row] = r * (bt - (c == d2 ? R(1.0 / 3.0) : R(0)));
        }
}

template <int D, typename R>
__global__ void reservoir_kernel(const double* __restrict__ rho, const double* __restrict__ u,
                                 const double* __restrict__ T, int nx, long long rows, long long N,
                                 R* __restrict__ gf, R* __restrict__ gb, R* __restrict__ gaux) {
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < 2 * rows) reservoir_item<D, R>(rho, u, T, nx, rows, N, gf, gb, gaux, t);
}

// Emitted state <-> FP64 planes of fbar*_i and bbar* (unshifted).
template <int D, typename FS>
__global__ void get_state_kernel(const FS* __restrict__ f, const typename Store<FS>::breal* __restrict__ b,
                                 double* __restrict__ fo, double* __restrict__ bo, long long N) {
    using L = Lattice<D>;
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= N) return;
    if (fo)
#pragma unroll
        for (int i = 0; i < L::Q; ++i) fo[i * N + s] = L::w(i) + double(Store<FS>::ld(f, i * N + s));
    if (bo)
#pragma unroll
        for (int k = 0; k < L::NB; ++k) bo[k * N + s] = double(b[BLayout<D, FS>::at(k, s, N)]) - (k < D ? 1.0 / 3.0 : 0.0);
}

template <int D, typename FS>
__global__ void set_state_kernel(FS* __restrict__ f, typename Store<FS>::breal* __restrict__ b,
                                 const double* __restrict__ fi, const double* __restrict__ bi, long long N) {
    using L = Lattice<D>;
    using breal = typename Store<FS>::breal;
    using real = typename Store<FS>::real;
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= N) return;
    if (fi)
#pragma unroll
        for (int i = 0; i < L::Q; ++i) Store<FS>::st(f, i * N + s, real(fi[i * N + s] - L::w(i)));
    if (bi)
#pragma unroll
        for (int k = 0; k < L::NB; ++k) b[BLayout<D, FS>::at(k, s, N)] = breal(bi[k * N + s] + (k < D ? 1.0 / 3.0 : 0.0));
}

}  // namespace lbm
