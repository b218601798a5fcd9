// Standard-lattice comparator: the textbook BGK scheme with the Hermite
// equilibrium of Eq. 4 (arXiv 2501.00620, Sec. I), written in lattice units
// with cs2 = c^2/3 and temperature T0:
//   f^eq_i = w_i rho [1 + 3 e.u + 9/2 ((e.u)^2 - |u|^2/3 + (T0 - 1/3)(|e|^2 - D/3))],
// whose moments are rho, rho u and rho (T0 I + u u) and whose third moment is
// fixed by the lattice.  One launch maps the emitted populations S(t) to
// S(t+1) on a periodic lattice: pull S_i(x - e_i), moments, relax with the
// same omega = 1/(tau + 1/2) as the bump scheme, store.  Same storage codec
// (populations as f - w_i), diagnostics and moment output as the bump
// kernels; there is no variance and no gradient correction, so the step is a
// single streaming pass of Q loads and Q stores per site.
//
// Layout: one thread per x, blocks of kStdNT sites along x; each block
// marches over `chunk` planes of the slowest axis (z in 3D, y in 2D), so the
// grid holds a few thousand blocks -- one diagnostics partial each -- and
// the rows a block reads at the previous and next plane were just read by
// itself or its neighbours and come from L2.  The loads of a warp are
// consecutive x.
#include "lbm_internal.h"

namespace lbm {

namespace {

constexpr int kStdNT = 128;

template <int D, typename FS, int NT>
__global__ void __launch_bounds__(NT) std_step_kernel(const StepArgs a) {
    using L = Lattice<D>;
    using real = typename Store<FS>::real;
    constexpr int Q = L::Q;
    __shared__ double red[(NT / 32) * (D + 2)];
    const FS* __restrict__ fin = static_cast<const FS*>(a.fin);
    const int x = blockIdx.x * NT + threadIdx.x;
    const int nx = a.nx, ny = a.ny, nz = a.nz;
    const int np = (D == 3) ? nz : (D == 2 ? ny : 1);
    const int p0 = (D == 1) ? 0 : ((D == 3) ? blockIdx.z : blockIdx.y) * a.chunk;
    const int p1 = (D == 1) ? 1 : min(p0 + a.chunk, np);
    const long long N = a.N;
    real omega, tau, T0;
    step_params(a, omega, tau, T0);
    (void)tau;
    DiagAcc<real, D + 2> acc;
    int bad = 0;
    for (int p = p0; p < p1 && x < nx; ++p) {
        const int y = (D == 3) ? (int)blockIdx.y : (D == 2 ? p : 0);
        const int z = (D == 3) ? p : 0;
        const long long s = x + (long long)nx * (y + (long long)ny * z);
        real df[Q];
        real drho = real(-0.0), j[D], e2 = real(-0.0);
#pragma unroll
        for (int c = 0; c < D; ++c) j[c] = real(-0.0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int sx = wrap1(x - L::e(i, 0), nx);
            const int sy = (D >= 2) ? wrap1(y - L::e(i, 1), ny) : 0;
            const int sz = (D == 3) ? wrap1(z - L::e(i, 2), nz) : 0;
            const real v = Store<FS>::ld(fin, (long long)i * N + sx + (long long)nx * (sy + (long long)ny * sz));
            df[i] = v;
            drho += v;
#pragma unroll
            for (int c = 0; c < D; ++c)
                if (L::e(i, c) != 0) j[c] += real(L::e(i, c)) * v;
            if (norm2<D>(i) != 0) e2 += real(norm2<D>(i)) * v;
        }
        // sum_i w_i = 1, sum_i w_i e_i = 0, sum_i w_i |e_i|^2 = D/3
        const real rho = real(1) + drho;
        const real E = real(D) * real(1.0 / 3.0) + e2;
        const real irho = real(1) / rho;
        real u[D], uu = real(-0.0);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            u[c] = j[c] * irho;
            uu += u[c] * u[c];
        }
        if (!(rho > real(0)) || !isfinite(E) || !isfinite(uu)) bad |= 1;
        if (a.want_diag) {
            acc.add(0, rho);
#pragma unroll
            for (int c = 0; c < D; ++c) acc.add(1 + c, j[c]);
            acc.add(D + 1, E);
        }
        if (a.mout) {
            a.mout[s] = double(rho);
#pragma unroll
            for (int c = 0; c < D; ++c) a.mout[(1 + c) * N + s] = double(u[c]);
            a.mout[(1 + D) * N + s] = double((E - rho * uu) * irho * real(1.0 / D));
        }
        if (a.write_state) {
            FS* __restrict__ fout = static_cast<FS*>(a.fout);
            const real dT = T0 - real(1.0 / 3.0);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                real eu = real(-0.0);
#pragma unroll
                for (int c = 0; c < D; ++c)
                    if (L::e(i, c) != 0) eu += real(L::e(i, c)) * u[c];
                const real second = eu * eu - uu * real(1.0 / 3.0) + dT * real(norm2<D>(i) - D / 3.0);
                // f^eq_i - w_i = w_i [(rho - 1) + rho (3 e.u + 9/2 second)]
                const real feq = real(L::w(i)) * (drho + rho * (real(3) * eu + real(4.5) * second));
                Store<FS>::st(fout, (long long)i * N + s, df[i] + omega * (feq - df[i]));
            }
        }
    }
    if (bad) atomicOr(a.flag, bad);
    if (a.want_diag) block_diagnostics<D, NT>(a, acc, red);
}

// Start: every site emits the comparator's equilibrium of (rho, u, T).
template <int D, typename FS>
__global__ void std_init_kernel(const double* __restrict__ rho, const double* __restrict__ u,
                                const double* __restrict__ T, FS* __restrict__ f, long long N) {
    using L = Lattice<D>;
    using real = typename Store<FS>::real;
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= N) return;
    const real r = real(rho[s]);
    real uu = real(0), uc[D];
#pragma unroll
    for (int c = 0; c < D; ++c) {
        uc[c] = real(u[c * N + s]);
        uu += uc[c] * uc[c];
    }
    const real dT = real(T[s]) - real(1.0 / 3.0);
#pragma unroll
    for (int i = 0; i < L::Q; ++i) {
        real eu = real(0);
#pragma unroll
        for (int c = 0; c < D; ++c) eu += real(L::e(i, c)) * uc[c];
        const real second = eu * eu - uu * real(1.0 / 3.0) + dT * real(norm2<D>(i) - D / 3.0);
        Store<FS>::st(f, i * N + s, real(L::w(i)) * ((r - real(1)) + r * (real(3) * eu + real(4.5) * second)));
    }
}

template <typename F>
cudaError_t by_dtype(int dtype, F&& f) {
    switch (dtype) {
        case DT_F64: return f(double{});
        case DT_F32: return f(float{});
        case DT_F16: return f(__half{});
        case DT_BF16: return f(__nv_bfloat16{});
        default: return cudaErrorInvalidValue;
    }
}

template <int D>
cudaError_t launch_d(int dtype, const StepArgs& a, cudaStream_t st) {
    if (a.chunk < 1) return cudaErrorInvalidValue;
    return by_dtype(dtype, [&](auto tag) {
        using FS = decltype(tag);
        std_step_kernel<D, FS, kStdNT><<<std_grid(D, a.nx, a.ny, a.nz, a.chunk), kStdNT, 0, st>>>(a);
        return cudaGetLastError();
    });
}

template <int D>
cudaError_t init_d(int dtype, const double* rho, const double* u, const double* T, void* f, long long N,
                   cudaStream_t st) {
    return by_dtype(dtype, [&](auto tag) {
        using FS = decltype(tag);
        const unsigned nb = (unsigned)((N + 255) / 256);
        std_init_kernel<D, FS><<<nb, 256, 0, st>>>(rho, u, T, static_cast<FS*>(f), N);
        return cudaGetLastError();
    });
}

}  // namespace

dim3 std_grid(int D, int nx, int ny, int nz, int chunk) {
    const unsigned gx = (unsigned)((nx + kStdNT - 1) / kStdNT);
    if (D == 3) return dim3(gx, (unsigned)ny, (unsigned)((nz + chunk - 1) / chunk));
    if (D == 2) return dim3(gx, (unsigned)((ny + chunk - 1) / chunk), 1u);
    return dim3(gx, 1u, 1u);
}

cudaError_t launch_std_step(int D, int dtype, const StepArgs& a, cudaStream_t st) {
    switch (D) {
        case 1: return launch_d<1>(dtype, a, st);
        case 2: return launch_d<2>(dtype, a, st);
        case 3: return launch_d<3>(dtype, a, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_std_init(int D, int dtype, const double* rho, const double* u, const double* T, void* f,
                            long long N, cudaStream_t st) {
    switch (D) {
        case 1: return init_d<1>(dtype, rho, u, T, f, N, st);
        case 2: return init_d<2>(dtype, rho, u, T, f, N, st);
        case 3: return init_d<3>(dtype, rho, u, T, f, N, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
