// MRT collision of the bump scheme on D3Q19, in the moment basis of Table M
// (arXiv 2501.00620, Appendix B).  With M^a = sum_i m^a_i f_i, each moment
// relaxes at its own rate, M*^a = M^a + s_a (M^a_eq - M^a) + (1 - s_a/2) Phi^a,
// and f_i = w_i sum_a m^a_i N^a M^a with N^a = 1 / sum_i w_i (m^a_i)^2 (the
// rows of Table M are orthogonal under that weighted sum).  The conserved and
// second-order rows 0-9 relax at omega, as in the SRT step; the third-order
// rows 10-15 at s3 and the fourth-order rows 16-18 at s4.
//
// The generic kernel stores the SRT result and adds the difference of the
// two steps, which lives in rows 10-18 only:
//   f*_i(MRT) - f*_i(SRT) = w_i sum_{a >= 10} m^a_i N^a (s_a - omega) sum_k m^a_k (f^eq_k - f_k).
// The forcing term drops out of it: Phi_i = w_i p(e_i) with p a polynomial of
// degree two, i.e. a combination of rows 0-9, orthogonal to rows 10-18.
#pragma once

#include "lbm_site.cuh"

namespace lbm {

// Rows 10-18 of Table M with c = 1, as integers over kMrtDen[k].
__host__ __device__ constexpr int mrt_hi(int k, int i) {
    constexpr signed char t[9][19] = {
        {0, -2, 0, 2, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 0, 0, 0, 0},
        {0, 0, -2, 0, 2, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1},
        {0, 0, 0, 0, 0, -2, 2, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1},
        {0, 0, 0, 0, 0, 0, 0, 1, 1, -1, -1, -1, -1, 1, 1, 0, 0, 0, 0},
        {0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, -1, -1, 1, 1},
        {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, -1, 1, -1, -1, 1, -1, 1},
        {0, 1, 1, 1, 1, -2, -2, -2, -2, -2, -2, 1, 1, 1, 1, 1, 1, 1, 1},
        {0, 1, -1, 1, -1, 0, 0, 0, 0, 0, 0, -1, -1, -1, -1, 1, 1, 1, 1},
        {1, -2, -2, -2, -2, -2, -2, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1}};
    return t[k][i];
}

// N^a / den_a^2 for rows 10-18: N^a = 1 / sum_i w_i (m^a_i)^2 with
// m^a_i = mrt_hi(a - 10, i) / den_a, den = (3, 3, 3, 1, 1, 1, 2, 2, 6), so
// N = (27/2, 27/2, 27/2, 9/2, 9/2, 9/2, 3, 9, 18).
__host__ __device__ constexpr double mrt_scale(int k) {
    constexpr double t[9] = {1.5, 1.5, 1.5, 4.5, 4.5, 4.5, 0.75, 2.25, 0.5};
    return t[k];
}

// Coherent reads of a value this thread has just stored (no read-only path).
__device__ __forceinline__ double ld_own(const double* p, long long k) { return p[k]; }
__device__ __forceinline__ float ld_own(const float* p, long long k) { return p[k]; }
__device__ __forceinline__ float ld_own(const __half* p, long long k) { return __half2float(p[k]); }
__device__ __forceinline__ float ld_own(const __nv_bfloat16* p, long long k) { return __bfloat162float(p[k]); }

// Adds the MRT-minus-SRT difference to the populations site s has just
// stored: df are its pre-collision deviations f - w, rho, j, F its density,
// uncorrected momentum and total force (the corrected u of Eq. 57 enters
// f^eq).
template <typename FS, typename R>
__device__ __forceinline__ void mrt_correct(const StepArgs& a, long long s, const R* df, R rho, const R* j,
                                            const R* F) {
    using L = Lattice<3>;
    constexpr int Q = L::Q;
    const R irho = recip(rho);
    R u[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) u[c] = (j[c] + R(0.5) * F[c]) * irho;
    R feq[Q];
    Equilibrium<3, R>::dev(rho, u, feq);
    R omega, tau, T0;
    step_params(a, omega, tau, T0);
    (void)tau;
    (void)T0;
    const R s3 = mrt_rate(a, 0, R(0)), s4 = mrt_rate(a, 1, R(0));
    R c[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        R acc = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i)
            if (mrt_hi(k, i) != 0) acc += R(mrt_hi(k, i)) * (feq[i] - df[i]);
        c[k] = ((k < 6 ? s3 : s4) - omega) * R(mrt_scale(k)) * acc;
    }
    FS* __restrict__ fo = static_cast<FS*>(a.fout);
    const long long N = a.N;
    bool finite = true;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        R corr = R(0);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            if (mrt_hi(k, i) != 0) corr += R(mrt_hi(k, i)) * c[k];
        const R v = R(ld_own(fo, (long long)i * N + s)) + R(L::w(i)) * corr;
        finite = finite && isfinite(v);
        Store<FS>::st(fo, (long long)i * N + s, v);
    }
    // the corrected populations are the stored state: a non-finite one is
    // reported by this step, as site_collide reports its own
    if (!finite) atomicOr(a.flag, 1);
}

}  // namespace lbm
