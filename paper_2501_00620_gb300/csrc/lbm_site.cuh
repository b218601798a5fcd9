// Per-site arithmetic of one time step (arXiv 2501.00620, Sec. II.C), shared by
// the step kernels; the kernels differ only in how they move data.
//
// Variables: df_i = fbar_i - w_i (pulled populations as deviations from the
// rest weights); bt = bbar + I/3 (bump variance plus the lattice's own
// second moment per axis).
#pragma once

#include <type_traits>

#include "lbm_args.cuh"
#include "lbm_lattice.cuh"

namespace lbm {

// Per-thread accumulator of the conservation diagnostics (mass, momentum,
// energy; K = D + 2 values).  In FP64 arithmetic it is a plain sum.  In FP32
// arithmetic each value is a float-float pair (hi, lo) updated by the
// error-free TwoSum transformation (Knuth, TAOCP vol. 2, 4.2.2): the pair
// carries the exact sum of its inputs to about 2^-48 relative, as an FP64 sum
// would, while costing only FP32 instructions (GB300's FP64 rate is a small
// fraction of its FP32 rate).
template <typename R, int K> struct DiagAcc;

template <int K> struct DiagAcc<double, K> {
    static constexpr bool kFF = false;  // reduced in FP64 (block_diagnostics)
    double v[K];
    __device__ __forceinline__ DiagAcc() {
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] = 0.0;
    }
    __device__ __forceinline__ void add(int k, double x) { v[k] += x; }
    __device__ __forceinline__ double get(int k) const { return v[k]; }
};

template <int K> struct DiagAcc<float, K> {
    static constexpr bool kFF = true;  // reduced as float-float pairs (block_diagnostics)
    float hi[K], lo[K];
    __device__ __forceinline__ DiagAcc() {
#pragma unroll
        for (int k = 0; k < K; ++k) hi[k] = lo[k] = 0.0f;
    }
    __device__ __forceinline__ void add(int k, float x) {
        const float s = __fadd_rn(hi[k], x);
        const float bp = __fsub_rn(s, hi[k]);
        const float err = __fadd_rn(__fsub_rn(hi[k], __fsub_rn(s, bp)), __fsub_rn(x, bp));
        hi[k] = s;
        lo[k] = __fadd_rn(lo[k], err);
    }
    __device__ __forceinline__ double get(int k) const { return double(hi[k]) + double(lo[k]); }
    // value k = (h + l) + cnt() * cref(k)
    __device__ __forceinline__ void ff(int k, float& h, float& l) const {
        h = hi[k];
        l = lo[k];
    }
    __device__ __forceinline__ int cnt() const { return 0; }
    __device__ __forceinline__ float cref(int) const { return 0.0f; }
};

// Float-float sum h + l += h2 + l2: TwoSum of the high parts (Knuth, TAOCP
// vol. 2, 4.2.2), the low parts and the rounding error added.
__device__ __forceinline__ void ff_add(float& h, float& l, float h2, float l2) {
    const float s = __fadd_rn(h, h2);
    const float bp = __fsub_rn(s, h);
    const float err = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(h2, bp));
    h = s;
    l = __fadd_rn(__fadd_rn(l, l2), err);
}

// Warp sum of float-float pairs in a fixed tree order; lane 0 holds it.
__device__ __forceinline__ void ff_warp_sum(float& h, float& l) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, h, o);
        const float l2 = __shfl_down_sync(0xffffffffu, l, o);
        ff_add(h, l, h2, l2);
    }
}

// 1/x, correctly rounded (the same value as 1/x by IEEE division, in fewer
// instructions than the division sequence).
__device__ __forceinline__ float recip(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double recip(double x) { return __drcp_rn(x); }

// Stage 1 at one site, after the pull: from df_i and the mass-weighted
// variance sum bsum = sum_i fbar_i bt*(x - e_i) (Eq. 66 numerator) compute
//   rho = sum fbar (Eq. 56), j0 = sum fbar e, bt = bsum / rho,
//   Ebar = sum fbar |e|^2 + rho tr bbar = sum df (|e|^2 - D/3) + rho tr bt,
//   u0 = j0 / rho, T_unc (thermal) or T0, and for the gradient
//   rho*b = rho (bbar - (omega/2)(bbar - b^eq(u0, T_unc)))  (Eq. 68).
template <int D, typename R>
__device__ __forceinline__ void site_moments(const R* df, const R* bsum, R omega, R T0, int thermal, R* bt,
                                             R& rho, R* j, R& E, R* u0, R* rb) {
    using L = Lattice<D>;
    constexpr int Q = L::Q, NB = L::NB;
    // velocity pairs (e_i, -e_i): sums for the even moments, differences for
    // the odd ones
    R ps[Q], pd[Q];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (i > opposite<D>(i)) continue;
        ps[i] = df[i] + df[opposite<D>(i)];
        pd[i] = df[i] - df[opposite<D>(i)];
    }
    R r = df[0];
#pragma unroll
    for (int i = 1; i < Q; ++i)
        if (i < opposite<D>(i)) r += ps[i];
    rho = r + R(1);
    const R irho = recip(rho);
#pragma unroll
    for (int c = 0; c < D; ++c) {
        R acc = R(-0.0);
#pragma unroll
        for (int i = 1; i < Q; ++i)
            if (i < opposite<D>(i) && L::e(i, c) != 0) acc += R(L::e(i, c)) * pd[i];
        j[c] = acc;
    }
    R trb = R(-0.0);
#pragma unroll
    for (int k = 0; k < NB; ++k) bt[k] = bsum[k] * irho;
#pragma unroll
    for (int c = 0; c < D; ++c) trb += bt[c];
    // sum_i df_i (|e_i|^2 - D/3): coefficient 0 (D3Q19 axis pairs) skipped
    R e = rho * trb + R(-D * (1.0 / 3.0)) * df[0];
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        if (i > opposite<D>(i)) continue;
        constexpr double third = 1.0 / 3.0;
        const double coef = norm2<D>(i) - D * third;
        if (coef == 1.0)
            e += ps[i];
        else if (coef != 0.0)
            e += R(coef) * ps[i];
    }
    E = e;
    R uu = R(-0.0);
#pragma unroll
    for (int c = 0; c < D; ++c) {
        u0[c] = j[c] * irho;
        uu += u0[c] * u0[c];
    }
    const R Tu = thermal ? (e - rho * uu) * irho * R(1.0 / D) : T0;
    const R hw = R(0.5) * omega;
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
        for (int d2 = c; d2 < D; ++d2) {
            const int k = sym<D>(c, d2);
            const R beq = u0[c] * u0[d2] * R(1.0 / 3.0) + (c == d2 ? Tu : R(0));
            R v = rho * (bt[k] - hw * (bt[k] - beq));
            if (c == d2) v -= rho * R(1.0 / 3.0);
            rb[k] = v;
        }
}

// Gradient contribution of neighbour x + e_i with rho*b = rbn and u0 = un:
// v = e_i . (rho b); F += w_i v; G_bc += w_i (u0_c v_b + u0_b v_c).  The
// caller scales by -3 (= -1/cs2) at the end: F = -div(rho b) (Eq. 59),
// G = -div(rho u0 b + rho u0 b) (Eq. 61) with the lattice-weight central
// difference d_a phi = 3 sum_i w_i e_ia phi(x + e_i).
template <int D, typename R>
__device__ __forceinline__ void fd_add(int i, const R* rbn, const R* un, R* F, R* G) {
    using L = Lattice<D>;
    R v[D];
#pragma unroll
    for (int b2 = 0; b2 < D; ++b2) {
        v[b2] = R(-0.0);
#pragma unroll
        for (int c = 0; c < D; ++c)
            if (L::e(i, c) != 0) v[b2] += R(L::e(i, c)) * rbn[sym<D>(c, b2)];
    }
    const R wi = R(L::w(i));
    R wv[D];
#pragma unroll
    for (int b2 = 0; b2 < D; ++b2) {
        wv[b2] = wi * v[b2];
        F[b2] += wv[b2];
    }
#pragma unroll
    for (int b2 = 0; b2 < D; ++b2)
#pragma unroll
        for (int c = b2; c < D; ++c) {
            R& g = G[sym<D>(b2, c)];
            g = fma(un[c], wv[b2], g);
            g = fma(un[b2], wv[c], g);
        }
}

// BGK update and store of the populations, pair by pair.  For a velocity pair
// (e_i, -e_i) the target f^eq_i + tau Phi_i (Appendix A, Eqs. 55, 58-61)
// splits into a part even in e_i, shared by the pair, and the odd part
// 3 w_i e_i.(rho u + tau F) -- the first moments of the equilibrium and of
// the forcing -- so that
//   df*_(+/-) = (1 - omega) df_(+/-) + omega (even +/- odd).
// Even parts (deviations from w_i, with dr = rho - 1, X_a = u_a^2):
//   D3Q19 (Appendix A):  rest  (1/3)[dr + rho(-(2/3)S - 2(XY+XZ+YZ))]
//                        axis  (1/18)[dr + rho(X_a(4 + 6(S - X_a)) - 2S)]
//                        edge  (1/36)[dr + rho(3 eu^2 - X_a - X_b - 6 X_a X_b)]
//   D2Q9, D1Q3: the even halves of the tensor-product moment inversion.
// The forcing Phi_i = w_i [3 e_i.F + 9/2 e_i.G.e_i - 3/2 tr G] -- the
// second-order Hermite projection whose zeroth, first and second moments are
// 0, F and G (Eqs. 58-61) -- adds w_i tau (9/2 e_i.G.e_i - 3/2 tr G) to the
// even part and 3 w_i tau e_i.F to the odd part.
// Where the emitted population i of the site goes: plane i at the site
// (pull scheme, A-B buffers); the in-place scheme supplies its own map.
template <typename I> struct PlaneDst {
    static constexpr bool kBytes = false;
    I s;
    __device__ __forceinline__ I operator()(int i, I N) const { return (I)i * N + s; }
};
// The same destination as a 32-bit byte offset from the buffer (plane i at
// i * pb + sb), for kernels whose population buffers span less than 4 GiB:
// the per-plane part is block-uniform, the per-site part one register.
struct PlaneDstBytes {
    static constexpr bool kBytes = true;
    unsigned sb, pb;
    template <typename I> __device__ __forceinline__ unsigned operator()(int i, I) const { return (unsigned)i * pb + sb; }
};
template <typename T, typename = void> struct dst_bytes : std::false_type {};
template <typename T> struct dst_bytes<T, std::void_t<decltype(T::kBytes)>> : std::bool_constant<T::kBytes> {};
template <typename FS, typename R, typename Dst, typename I>
__device__ __forceinline__ void store_pop(FS* fo, const Dst& dst, int i, I N, R v) {
    if constexpr (dst_bytes<Dst>::value)
        Store<FS>::stb(fo, dst(i, N), v);
    else
        Store<FS>::st(fo, dst(i, N), v);
}

template <int D, typename FS, typename R, typename I = long long, typename Dst = PlaneDst<I>>
__device__ __forceinline__ void collide_store(FS* __restrict__ fo, I N, const R* df, R rho, const R* u,
                                              const R* F, const R* G, R trG, R omega, R tau, Dst dst) {
    using L = Lattice<D>;
    constexpr int Q = L::Q, NB = L::NB;
    const R dr = rho - R(1);
    const R om1 = R(1) - omega;
    R mom[D];
#pragma unroll
    for (int c = 0; c < D; ++c) mom[c] = fma(tau, F[c], rho * u[c]);
    const R F0 = R(-1.5) * tau * trG;
    const R t45 = R(4.5) * tau;
    R g45[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) g45[k] = t45 * G[k];
    R ev[Q];  // even part of the target, at the rest population and the first member of each pair
    if constexpr (D == 3) {
        const R X0 = u[0] * u[0], X1 = u[1] * u[1], X2 = u[2] * u[2];
        const R X[3] = {X0, X1, X2};
        const R S = X0 + X1 + X2;
        const R C0 = dr + F0;
        ev[0] = R(1.0 / 3.0) * (C0 + rho * (R(-2.0 / 3.0) * S - R(2) * (X0 * X1 + X0 * X2 + X1 * X2)));
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if (i > opposite<3>(i)) continue;
            if (norm2<3>(i) == 1) {
                const int a = L::e(i, 0) != 0 ? 0 : (L::e(i, 1) != 0 ? 1 : 2);
                ev[i] = R(1.0 / 18.0) * (C0 + rho * (X[a] * (R(4) + R(6) * (S - X[a])) - R(2) * S) + g45[a]);
            } else {
                const int a = L::e(i, 0) != 0 ? 0 : 1;
                const int b = L::e(i, 2) != 0 ? 2 : 1;
                const int sab = L::e(i, a) * L::e(i, b);
                const R eu = sab > 0 ? u[a] + u[b] : u[a] - u[b];
                const R gab = sab > 0 ? g45[sym<3>(a, b)] : -g45[sym<3>(a, b)];
                ev[i] = R(1.0 / 36.0) *
                        (C0 + rho * (R(3) * eu * eu - X[a] - X[b] - R(6) * X[a] * X[b]) + (g45[a] + g45[b] + R(2) * gab));
            }
        }
    } else if constexpr (D == 2) {
        const R X = u[0] * u[0], Y = u[1] * u[1];
        const R m20 = (dr + R(2) * rho * X) * R(1.0 / 3.0);
        const R m02 = (dr + R(2) * rho * Y) * R(1.0 / 3.0);
        const R m11 = R(2.0 / 3.0) * rho * u[0] * u[1];
        const R m22 = (dr + rho * (R(2) * (X + Y) - R(6) * X * Y)) * R(1.0 / 9.0);
        ev[0] = (dr - m20) - (m02 - m22) + R(4.0 / 9.0) * F0;
        ev[1] = R(0.5) * (m20 - m22) + R(1.0 / 9.0) * (F0 + g45[0]);
        ev[2] = R(0.5) * (m02 - m22) + R(1.0 / 9.0) * (F0 + g45[1]);
        ev[5] = R(0.25) * (m22 + m11) + R(1.0 / 36.0) * (F0 + g45[0] + g45[1] + R(2) * g45[2]);
        ev[6] = R(0.25) * (m22 - m11) + R(1.0 / 36.0) * (F0 + g45[0] + g45[1] - R(2) * g45[2]);
    } else {
        const R dm2 = (dr + R(2) * rho * u[0] * u[0]) * R(1.0 / 3.0);
        ev[0] = dr - dm2 + R(2.0 / 3.0) * F0;
        ev[1] = R(0.5) * dm2 + R(1.0 / 6.0) * (F0 + g45[0]);
    }
    store_pop<FS, R>(fo, dst, 0, N, fma(om1, df[0], omega * ev[0]));
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int ib = opposite<D>(i);
        if (i > ib) continue;
        R eM = R(-0.0);
#pragma unroll
        for (int c = 0; c < D; ++c)
            if (L::e(i, c) != 0) eM += R(L::e(i, c)) * mom[c];
        const R A = omega * ev[i];
        const R B = (R(3.0 * L::w(i)) * omega) * eM;
        store_pop<FS, R>(fo, dst, i, N, fma(om1, df[i], A + B));
        store_pop<FS, R>(fo, dst, ib, N, fma(om1, df[ib], A - B));
    }
}

// Stage 2 at one site, given F and G (already scaled): corrected velocity
// u = (j0 + F/2)/rho (Eq. 57), temperature, diagnostics, the SRT update
// fbar* = fbar + omega (f^eq + tau Phi - fbar) (Eq. 55, Appendix A, Eqs. 58-61)
// and bbar* = bbar + omega (b^eq - bbar) (Eqs. 63, 65), stored at site s.
// bad |= 1: rho <= 0 or non-finite; bad |= 2: T <= 0 in thermal mode.
// I is the index type of the site (int where the lattice has fewer than 2^31
// sites); Acc the diagnostics accumulator (DiagAcc or a kernel's own).
// FP64 temperature of the corrected moments (Eq. 57, thermal mode) from the
// site's pulled populations df, its energy Ebar (E64, summed in FP64 with
// an FP64 variance transport) and the FP32 gradients F, tr G:
// T = (Ebar + tr G / 2 - rho |u|^2) / (D rho), u = (j0 + F/2) / rho.  Used
// where T << |u|^2, where the FP32 difference cancels.
template <int D>
__device__ __forceinline__ double temperature64(const float* df, double E64, const float* F, float trG) {
    using L = Lattice<D>;
    double r = 1.0, j[D];
#pragma unroll
    for (int c = 0; c < D; ++c) j[c] = 0.0;
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        const double d = df[i];
        r += d;
#pragma unroll
        for (int c = 0; c < D; ++c)
            if (L::e(i, c) != 0) j[c] += L::e(i, c) * d;
    }
    double uu = 0.0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        const double u = (j[c] + 0.5 * (double)F[c]) / r;
        uu += u * u;
    }
    return (E64 + 0.5 * (double)trG - r * uu) / (D * r);
}

// E64: the site's Ebar summed in FP64 where stage 1 found T small (then T is
// recovered in FP64 here too); E64 < 0 marks "no FP64 value".
template <int D, typename FS, typename R, typename I = long long, typename Acc = DiagAcc<R, D + 2>,
          typename Dst = PlaneDst<I>>
__device__ __forceinline__ void site_collide(const StepArgs& a, I s, const R* c_df, const R* c_bt, R rho,
                                             const R* c_j, R c_E, const R* F, const R* G, Acc& acc, int& bad,
                                             double E64 = -1.0, Dst dst = Dst{}) {
    using L = Lattice<D>;
    using breal = typename Store<FS>::breal;
    const I N = (I)a.N;
    R omega, tau, T0;
    step_params(a, omega, tau, T0);
    R trG = R(-0.0);
#pragma unroll
    for (int c = 0; c < D; ++c) trG += G[c];
    const R irho = recip(rho);
    R u[D], uu = R(-0.0);
#pragma unroll
    for (int c = 0; c < D; ++c) {
        u[c] = (c_j[c] + R(0.5) * F[c]) * irho;
        uu += u[c] * u[c];
    }
    const R Ecorr = c_E + R(0.5) * trG;
    R Tm = (Ecorr - rho * uu) * irho * R(1.0 / D);
    double Tm64 = double(Tm);
    if constexpr (std::is_same<R, float>::value) {
        // small T: recover T in FP64 (the FP32 difference above cancels)
        if (E64 >= 0.0 && a.thermal) {
            Tm64 = temperature64<D>(c_df, E64, F, trG);
            Tm = float(Tm64);
        }
    }
    const R T = a.thermal ? Tm : T0;
    // fatal: the method divides by rho; non-finite values propagate
    if (!(rho > R(0)) || !isfinite(Ecorr) || !isfinite(uu)) bad |= 1;
    // not fatal: a negative moment temperature only makes b^eq more
    // negative (thermal mode); it occurs transiently at sharp fronts
    if (a.thermal && !(Tm > R(0))) bad |= 2;
    if (a.want_diag) {
        acc.add(0, rho);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            acc.add(1 + c, c_j[c]);
            acc.add(1 + c, R(0.5) * F[c]);  // exact halving
        }
        acc.add(D + 1, Ecorr);
    }
    if (a.mout) {
        a.mout[s] = double(rho);
#pragma unroll
        for (int c = 0; c < D; ++c) a.mout[(1 + c) * N + s] = double(u[c]);
        a.mout[(1 + D) * N + s] = Tm64;
    }
    if (!a.write_state) return;
    if constexpr (std::is_same<Dst, PlaneDst<I>>::value)
        collide_store<D, FS, R, I>(static_cast<FS*>(a.fout), N, c_df, rho, u, F, G, trG, omega, tau, PlaneDst<I>{s});
    else
        collide_store<D, FS, R, I>(static_cast<FS*>(a.fout), N, c_df, rho, u, F, G, trG, omega, tau, dst);
    breal* __restrict__ bo = static_cast<breal*>(a.bout);
    R bnew[L::NB];
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
        for (int d2 = c; d2 < D; ++d2) {
            const int k = sym<D>(c, d2);
            const R beq = u[c] * u[d2] * R(1.0 / 3.0) + (c == d2 ? T : R(0));
            bnew[k] = c_bt[k] + omega * (beq - c_bt[k]);
        }
    if constexpr (BLayout<D, FS>::paired) {
        float2* __restrict__ bo2 = reinterpret_cast<float2*>(bo);
#pragma unroll
        for (int p = 0; p < L::NB / 2; ++p) bo2[p * N + s] = make_float2(float(bnew[2 * p]), float(bnew[2 * p + 1]));
    } else {
#pragma unroll
        for (int k = 0; k < L::NB; ++k) bo[k * N + s] = breal(bnew[k]);
    }
}

// Block reduction of the per-thread diagnostics (fixed order: warp shuffle,
// then warps in order), per-block partials, and the last block's fixed-order
// sum of all partials into the history record / diag_out.  `red` holds
// 32 * (D + 2) doubles of shared memory.
template <int D, int NT, typename Acc>
__device__ __forceinline__ void block_diagnostics(const StepArgs& a, const Acc& acc, double* red) {
    constexpr int K = D + 2;
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    if constexpr (Acc::kFF) {
        // FP32 accumulators: float-float pairs and an exact site count through
        // the warp tree (GB300's FP64 rate is a small fraction of its FP32
        // rate); FP64 only for each warp's result
        int n = acc.cnt();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) n += __shfl_down_sync(0xffffffffu, n, o);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float h, l;
            acc.ff(k, h, l);
            ff_warp_sum(h, l);
            if (lane == 0) red[warp * K + k] = (double(h) + double(l)) + double(n) * double(acc.cref(k));
        }
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double v = acc.get(k);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (lane == 0) red[warp * K + k] = v;
        }
    }
    __syncthreads();
    const unsigned int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const unsigned int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    __shared__ int last;
    if (tid < K) {  // the warps in order, one value per thread
        double v = 0.0;
        for (int w = 0; w < NT / 32; ++w) v += red[w * K + tid];
        a.partial[(long long)bid * K + tid] = v;
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) last = (atomicAdd(a.ticket, 1u) == nblocks - 1);
    __syncthreads();
    if (!last) return;
    // The last block sums the per-block partials: thread t takes blocks
    // t, t + NT, ... in order, then the same fixed tree -- the result does not
    // depend on block scheduling.
    __threadfence();
    double v[K];
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = 0.0;
    // the partials of G blocks are loaded before they are added (in the same
    // order): G x K loads in flight per thread instead of K, which shortens
    // this serial tail of the step several times over
    constexpr int G = 8;
    unsigned int b2 = tid;
    for (; b2 + (G - 1) * NT < nblocks; b2 += G * NT) {
        double w[G][K];
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int k = 0; k < K; ++k) w[g][k] = __ldcg(a.partial + (long long)(b2 + g * NT) * K + k);
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int k = 0; k < K; ++k) v[k] += w[g][k];
    }
    for (; b2 < nblocks; b2 += NT)
#pragma unroll
        for (int k = 0; k < K; ++k) v[k] += __ldcg(a.partial + (long long)b2 * K + k);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < K; ++k) {
        if constexpr (Acc::kFF) {
            // the FP64 partial as a float-float pair (about 48 bits)
            float h = __double2float_rn(v[k]);
            float l = __double2float_rn(v[k] - double(h));
            ff_warp_sum(h, l);
            if (lane == 0) red[warp * K + k] = double(h) + double(l);
        } else {
            double x = v[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
            if (lane == 0) red[warp * K + k] = x;
        }
    }
    __syncthreads();
    double tot = 0.0;
    if (tid < K)
        for (int w = 0; w < NT / 32; ++w) tot += red[w * K + tid];
    __syncthreads();
    if (tid < K) red[tid] = tot;
    __syncthreads();
    if (tid == 0) {
        const long long st = *a.step_ctr;
        if (a.diag_out)
            for (int k = 0; k < K; ++k) a.diag_out[k] = red[k];
        if (a.hist) {
            double* rec = a.hist + (st % a.hist_cap) * (D + 3);
            rec[0] = double(st);
            for (int k = 0; k < K; ++k) rec[1 + k] = red[k];
        }
        if (a.write_state) *a.step_ctr = st + 1;
        *a.ticket = 0u;
    }
}

}  // namespace lbm
