// In-place time step of the bump-function lattice Boltzmann method (arXiv
// 2501.00620, Sec. II.C) with one population buffer: two passes per step over
// an "AA" access pattern, so that each site reads its incoming populations
// from exactly the slots it then overwrites with its emitted ones.
//
// Memory forms of the population buffer (periodic lattice):
//   form 0 (the emitted layout of the A-B kernels): plane i at x holds
//          f*_i(x), the population x emitted along e_i;
//   form 1: plane opp(i) at x holds f*_i(x - e_i), the population that
//          arrived at x along e_i.
// A step from form 0 reads f_i(x) = f*_i(x - e_i) at (i, x - e_i) (the pull
// of Eq. 49) and writes the new f*_i(x) to (opp(i), x + e_i): form 1.  A step
// from form 1 reads f_i(x) at (opp(i), x) and writes f*_i(x) to (i, x): form
// 0.  The slots a site writes are the slots it read, and no other site
// reads them in that step, so the update needs no second buffer.
//
// The gradient of rho b (Eqs. 59, 61, 68) needs the moments of the
// neighbours, which an in-place update would overwrite before a
// neighbouring block recomputed them; hence two passes:
//   pass 1 (aa_aux_kernel): pull and transport (Eq. 66), moments, and the
//     site's (u0, rho b) into an aux array;
//   pass 2 (aa_collide_kernel): pull and transport again (the site's own
//     rho, j0, Ebar, bbar), gradients from the neighbours' aux values,
//     collision (site_collide), store in place.
// The variance bbar stays in two buffers (its transport reads the emitted
// variance of all Q neighbours).  One thread per site; periodic boundary in
// every axis; FP64 or FP32 storage.
#pragma once

#include "lbm_site.cuh"

namespace lbm {

template <int D> struct AAGeom {
    int nx, ny, nz;
    long long N;
    int x, y, z;
    long long s;
    __device__ __forceinline__ AAGeom(const StepArgs& a, long long site)
        : nx(a.nx), ny(a.ny), nz(a.nz), N(a.N), s(site) {
        x = (int)(site % nx);
        const long long r = site / nx;
        y = (int)(r % ny);
        z = (int)(r / ny);
    }
    static __device__ __forceinline__ int wrap(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }
    // site x + sgn e_i (periodic)
    __device__ __forceinline__ long long nb(int i, int sgn) const {
        using L = Lattice<D>;
        const int xx = wrap(x + sgn * L::e(i, 0), nx);
        const int yy = (D >= 2) ? wrap(y + sgn * L::e(i, 1), ny) : 0;
        const int zz = (D == 3) ? wrap(z + sgn * L::e(i, 2), nz) : 0;
        return xx + (long long)nx * (yy + (long long)ny * zz);
    }
};

// Store map of pass 2: form 0 sends f*_i(x) to (opp(i), x + e_i), form 1 to
// (i, x).
template <int D> struct AADst {
    const AAGeom<D>* g;
    int form;
    __device__ __forceinline__ long long operator()(int i, long long N) const {
        return form == 0 ? (long long)opposite<D>(i) * N + g->nb(i, +1) : (long long)i * N + g->s;
    }
};

// Pull, transport and moments of one site (both passes).
template <int D, typename FS>
__device__ __forceinline__ void aa_site(const StepArgs& a, const AAGeom<D>& g, int form, typename Store<FS>::real* df,
                                        typename Store<FS>::real* bt, typename Store<FS>::real& rho,
                                        typename Store<FS>::real* j, typename Store<FS>::real& E,
                                        typename Store<FS>::real* u0, typename Store<FS>::real* rb) {
    using L = Lattice<D>;
    using real = typename Store<FS>::real;
    using breal = typename Store<FS>::breal;
    constexpr int Q = L::Q, NB = L::NB;
    const FS* __restrict__ fin = static_cast<const FS*>(a.fin);
    const breal* __restrict__ bin = static_cast<const breal*>(a.bin);
    const long long N = g.N;
    real bsum[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) bsum[k] = real(-0.0);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const long long src = g.nb(i, -1);  // x - e_i: the emitter of f_i(x)
        const real v = form == 0 ? Store<FS>::ld(fin, (long long)i * N + src)
                                 : Store<FS>::ld(fin, (long long)opposite<D>(i) * N + g.s);
        df[i] = v;
        const real fi = real(L::w(i)) + v;
#pragma unroll
        for (int k = 0; k < NB; ++k) bsum[k] += fi * real(__ldg(bin + BLayout<D, FS>::at(k, src, N)));
    }
    real omega, tau, T0;
    step_params(a, omega, tau, T0);
    (void)tau;
    site_moments<D, real>(df, bsum, omega, T0, a.thermal, bt, rho, j, E, u0, rb);
}

// Pass 1: (u0, rho b) of every site into aux (planes u0_0..u0_{D-1}, then
// rho b in the component order of sym<D>).
template <int D, typename FS>
__global__ void __launch_bounds__(256) aa_aux_kernel(const StepArgs a, int form, typename Store<FS>::real* aux) {
    using L = Lattice<D>;
    using real = typename Store<FS>::real;
    const long long s = blockIdx.x * 256ll + threadIdx.x;
    if (s >= a.N) return;
    const AAGeom<D> g(a, s);
    real df[L::Q], bt[L::NB], rho, j[D], E, u0[D], rb[L::NB];
    aa_site<D, FS>(a, g, form, df, bt, rho, j, E, u0, rb);
#pragma unroll
    for (int c = 0; c < D; ++c) aux[c * a.N + s] = u0[c];
#pragma unroll
    for (int k = 0; k < L::NB; ++k) aux[(D + k) * a.N + s] = rb[k];
}

// Pass 2: gradients from the neighbours' aux values, collision, in-place
// store; diagnostics as in the other kernels.
template <int D, typename FS>
__global__ void __launch_bounds__(256) aa_collide_kernel(const StepArgs a, int form,
                                                        const typename Store<FS>::real* __restrict__ aux) {
    using L = Lattice<D>;
    using real = typename Store<FS>::real;
    constexpr int Q = L::Q, NB = L::NB;
    __shared__ double red[32 * (D + 2)];
    const long long s = blockIdx.x * 256ll + threadIdx.x;
    DiagAcc<real, D + 2> acc;
    int bad = 0;
    if (s < a.N) {
        const AAGeom<D> g(a, s);
        real df[Q], bt[NB], rho, j[D], E, u0[D], rb[NB];
        aa_site<D, FS>(a, g, form, df, bt, rho, j, E, u0, rb);
        // the population buffer is read and written in place: keep every load
        // of this site before its stores to the same slots
        asm volatile("" ::: "memory");
        real F[D], G[NB];
#pragma unroll
        for (int c = 0; c < D; ++c) F[c] = real(-0.0);
#pragma unroll
        for (int k = 0; k < NB; ++k) G[k] = real(-0.0);
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const long long n = g.nb(i, +1);
            real rbn[NB], un[D];
#pragma unroll
            for (int k = 0; k < NB; ++k) rbn[k] = aux[(D + k) * a.N + n];
#pragma unroll
            for (int c = 0; c < D; ++c) un[c] = aux[c * a.N + n];
            fd_add<D, real>(i, rbn, un, F, G);
        }
#pragma unroll
        for (int c = 0; c < D; ++c) F[c] *= real(-3);
#pragma unroll
        for (int k = 0; k < NB; ++k) G[k] *= real(-3);
        site_collide<D, FS, real, long long, DiagAcc<real, D + 2>, AADst<D>>(a, s, df, bt, rho, j, E, F, G, acc,
                                                                              bad, -1.0, AADst<D>{&g, form});
    }
    if (bad) atomicOr(a.flag, bad);
    if (a.want_diag) block_diagnostics<D, 256>(a, acc, red);
}

// Emitted state of a buffer in form 1 as FP64 planes (f*_i(x) is at
// (opp(i), x + e_i)); the variance is stored per site as always.
template <int D, typename FS>
__global__ void aa_get_state_kernel(const StepArgs a, double* __restrict__ fo) {
    using L = Lattice<D>;
    const long long s = blockIdx.x * 256ll + threadIdx.x;
    if (s >= a.N) return;
    const AAGeom<D> g(a, s);
    const FS* __restrict__ f = static_cast<const FS*>(a.fin);
#pragma unroll
    for (int i = 0; i < L::Q; ++i)
        fo[i * a.N + s] = L::w(i) + double(Store<FS>::ld(f, (long long)opposite<D>(i) * a.N + g.nb(i, +1)));
}

}  // namespace lbm
