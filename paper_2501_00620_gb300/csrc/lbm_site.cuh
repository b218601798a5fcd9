// Per-site arithmetic of one time step (arXiv 2501.00620, Sec. II.C), shared by
// the step kernels; the kernels differ only in how they move data.
//
// Variables: df_i = fbar_i - w_i (pulled populations as deviations from the
// rest weights); bt = bbar + I/3 (bump variance plus the lattice's own
// second moment per axis).
#pragma once

#include "lbm_args.cuh"
#include "lbm_lattice.cuh"

namespace lbm {

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
    R r = R(-0.0);
#pragma unroll
    for (int i = 0; i < Q; ++i) r += df[i];
    rho = r + R(1);
    const R irho = recip(rho);
#pragma unroll
    for (int c = 0; c < D; ++c) {
        R acc = R(-0.0);
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (L::e(i, c) != 0) acc += R(L::e(i, c)) * df[i];
        j[c] = acc;
    }
    R trb = R(-0.0);
#pragma unroll
    for (int k = 0; k < NB; ++k) bt[k] = bsum[k] * irho;
#pragma unroll
    for (int c = 0; c < D; ++c) trb += bt[c];
    R e = rho * trb;
#pragma unroll
    for (int i = 0; i < Q; ++i) e += R(norm2<D>(i) - D * (1.0 / 3.0)) * df[i];
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

// Stage 2 at one site, given F and G (already scaled): corrected velocity
// u = (j0 + F/2)/rho (Eq. 57), temperature, diagnostics, the SRT update
// fbar* = fbar + omega (f^eq + tau Phi - fbar) (Eq. 55, Appendix A, Eqs. 58-61)
// and bbar* = bbar + omega (b^eq - bbar) (Eqs. 63, 65), stored at site s.
// bad |= 1: rho <= 0 or non-finite; bad |= 2: T <= 0 in thermal mode.
template <int D, typename FS, typename R>
__device__ __forceinline__ void site_collide(const StepArgs& a, long long s, const R* c_df, const R* c_bt, R rho,
                                             const R* c_j, R c_E, const R* F, const R* G, double* acc,
                                             int& bad) {
    using L = Lattice<D>;
    using breal = typename Store<FS>::breal;
    constexpr int Q = L::Q;
    const long long N = a.N;
    const R omega = R(a.omega), tau = R(a.tau), T0 = R(a.T0);
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
    const R Tm = (Ecorr - rho * uu) * irho * R(1.0 / D);
    const R T = a.thermal ? Tm : T0;
    // fatal: the method divides by rho; non-finite values propagate
    if (!(rho > R(0)) || !isfinite(Ecorr) || !isfinite(uu)) bad |= 1;
    // not fatal: a negative moment temperature only makes b^eq more
    // negative (thermal mode); it occurs transiently at sharp fronts
    if (a.thermal && !(Tm > R(0))) bad |= 2;
    if (a.want_diag) {
        acc[0] += double(rho);
#pragma unroll
        for (int c = 0; c < D; ++c) acc[1 + c] += double(c_j[c]) + 0.5 * double(F[c]);
        acc[D + 1] += double(Ecorr);
    }
    if (a.mout) {
        a.mout[s] = double(rho);
#pragma unroll
        for (int c = 0; c < D; ++c) a.mout[(1 + c) * N + s] = double(u[c]);
        a.mout[(1 + D) * N + s] = double(Tm);
    }
    if (!a.write_state) return;
    R feq[Q];
    Equilibrium<D, R>::dev(rho, u, feq);
    // plane-strided stores from one running pointer per array
    FS* __restrict__ fo = static_cast<FS*>(a.fout) + s;
    breal* __restrict__ bo = static_cast<breal*>(a.bout) + s;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const R tgt = feq[i] + tau * forcing_term<D, R>(i, F, G, trG);
        Store<FS>::st(fo, 0, c_df[i] + omega * (tgt - c_df[i]));
        fo += N;
    }
    R bnew[L::NB];
#pragma unroll
    for (int c = 0; c < D; ++c)
#pragma unroll
        for (int d2 = c; d2 < D; ++d2) {
            const int k = sym<D>(c, d2);
            const R beq = u[c] * u[d2] * R(1.0 / 3.0) + (c == d2 ? T : R(0));
            bnew[k] = c_bt[k] + omega * (beq - c_bt[k]);
        }
#pragma unroll
    for (int k = 0; k < L::NB; ++k) {
        bo[0] = breal(bnew[k]);
        bo += N;
    }
}

// Block reduction of the per-thread diagnostics (fixed order: warp shuffle,
// then warps in order), per-block partials, and the last block's fixed-order
// sum of all partials into the history record / diag_out.  `red` holds
// 32 * (D + 2) doubles of shared memory.
template <int D, int NT>
__device__ __forceinline__ void block_diagnostics(const StepArgs& a, double* acc, double* red) {
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
    for (int k = 0; k < D + 2; ++k) {
        double v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[warp * (D + 2) + k] = v;
    }
    __syncthreads();
    const unsigned int nblocks = gridDim.x * gridDim.y * gridDim.z;
    const unsigned int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    __shared__ int last;
    if (tid == 0) {
        for (int k = 0; k < D + 2; ++k) {
            double v = 0.0;
            for (int w = 0; w < NT / 32; ++w) v += red[w * (D + 2) + k];
            a.partial[(long long)bid * (D + 2) + k] = v;
        }
        __threadfence();
        last = (atomicAdd(a.ticket, 1u) == nblocks - 1);
    }
    __syncthreads();
    if (!last) return;
    // The last block sums the per-block partials: thread t takes blocks
    // t, t + NT, ... in order, then the same fixed tree -- the result does not
    // depend on block scheduling.
    __threadfence();
    double v[D + 2];
#pragma unroll
    for (int k = 0; k < D + 2; ++k) v[k] = 0.0;
    for (unsigned int b2 = tid; b2 < nblocks; b2 += NT)
#pragma unroll
        for (int k = 0; k < D + 2; ++k) v[k] += __ldcg(a.partial + (long long)b2 * (D + 2) + k);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < D + 2; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
        if (lane == 0) red[warp * (D + 2) + k] = x;
    }
    __syncthreads();
    double tot = 0.0;
    if (tid < D + 2)
        for (int w = 0; w < NT / 32; ++w) tot += red[w * (D + 2) + tid];
    __syncthreads();
    if (tid < D + 2) red[tid] = tot;
    __syncthreads();
    if (tid == 0) {
        const long long st = *a.step_ctr;
        if (a.diag_out)
            for (int k = 0; k < D + 2; ++k) a.diag_out[k] = red[k];
        if (a.hist) {
            double* rec = a.hist + (st % a.hist_cap) * (D + 3);
            rec[0] = double(st);
            for (int k = 0; k < D + 2; ++k) rec[1 + k] = red[k];
        }
        if (a.write_state) *a.step_ctr = st + 1;
        *a.ticket = 0u;
    }
}

}  // namespace lbm
