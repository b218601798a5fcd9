// Velocity sets, equilibria and forcing of the bump-function lattice
// Boltzmann method (arXiv 2501.00620), device side.
//
// Populations are handled as deviations from the rest-state weights,
// df_i = f_i - w_i (w_i = f^eq_i(rho = 1, u = 0)), and the variance tensor as
// bt = b + (c^2/3) I, the bump variance plus the lattice's own second moment
// per axis.  Both shifts are exact changes of variable; they keep the O(1)
// constants out of FP32/FP16 rounding, which matters when T << c^2/3 and the
// bump variance b ~ T - 1/3 nearly cancels the lattice's 1/3 (Sec. II.B).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <type_traits>

namespace lbm {

// ---------------------------------------------------------------------------
// Velocity sets.  D3Q19 follows the column order of the population-to-moment
// matrix of Appendix B; D2Q9 and D1Q3 use rest, +x, +y, -x, -y, then the
// diagonals (++, +-, -+, --).

template <int D> struct Lattice;

template <> struct Lattice<1> {
    static constexpr int D = 1, Q = 3, NB = 1;
    __host__ __device__ static constexpr int e(int i, int a) {
        return a != 0 ? 0 : (i == 1 ? 1 : (i == 2 ? -1 : 0));
    }
    __host__ __device__ static constexpr double w(int i) { return i == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
};

template <> struct Lattice<2> {
    static constexpr int D = 2, Q = 9, NB = 3;
    __host__ __device__ static constexpr int e(int i, int a) {
        constexpr int ex[9] = {0, 1, 0, -1, 0, 1, 1, -1, -1};
        constexpr int ey[9] = {0, 0, 1, 0, -1, 1, -1, 1, -1};
        return a == 0 ? ex[i] : (a == 1 ? ey[i] : 0);
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    }
};

template <> struct Lattice<3> {
    static constexpr int D = 3, Q = 19, NB = 6;
    __host__ __device__ static constexpr int e(int i, int a) {
        constexpr int ex[19] = {0, 1, 0, -1, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1, 0, 0, 0, 0};
        constexpr int ey[19] = {0, 0, 1, 0, -1, 0, 0, 1, -1, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1};
        constexpr int ez[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1};
        return a == 0 ? ex[i] : (a == 1 ? ey[i] : ez[i]);
    }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 1.0 / 3.0 : (i < 7 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};

// Symmetric-tensor component index: 1D (xx); 2D (xx, yy, xy);
// 3D (xx, yy, zz, xy, xz, yz).
template <int D> __host__ __device__ constexpr int sym(int a, int b) {
    return a == b ? a : (D == 2 ? 2 : ((a + b) == 1 ? 3 : ((a + b) == 2 ? 4 : 5)));
}

template <int D> __host__ __device__ constexpr int norm2(int i) {
    return Lattice<D>::e(i, 0) * Lattice<D>::e(i, 0) + Lattice<D>::e(i, 1) * Lattice<D>::e(i, 1) +
           Lattice<D>::e(i, 2) * Lattice<D>::e(i, 2);
}

// Index of the velocity -e_i.
template <int D> __host__ __device__ constexpr int opposite(int i) {
    using L = Lattice<D>;
    int r = -1;
    for (int k = 0; k < L::Q; ++k)
        if (L::e(k, 0) == -L::e(i, 0) && L::e(k, 1) == -L::e(i, 1) && L::e(k, 2) == -L::e(i, 2)) r = k;
    return r;
}

// ---------------------------------------------------------------------------
// Equilibrium deviations df^eq_i = f^eq_i(rho, u) - w_i.
//
// D3Q19: the closed forms of Appendix A grouped by velocity class.  With
// X, Y, Z = u_x^2, u_y^2, u_z^2, S = X + Y + Z, eu = e_i . u and
// q = sum_a e_ia^2 u_a^2, the printed polynomials P_i = f^eq_i / (rho w_i) are
//   rest:  P - 1 = -(2/3) S - 2 (XY + XZ + YZ)
//   axis:  P - 1 = 3 eu + 4 eu^2 - 2 S + 6 eu^2 (S - eu^2)
//   edge:  P - 1 = 3 eu + 3 eu^2 - q - (3/2)(eu^2 - q)^2
// D2Q9 and D1Q3: the equilibrium is defined by its discrete moments
// (Eqs. 32-35 plus the fourth-order moment the collapse of Appendix A
// fixes); it is recovered by the tensor-product inverse of the 1D moment
// basis {1, e, e^2}: f_0 = m_0 - m_2, f_+- = (+-m_1 + m_2)/2 per axis.

template <int D, typename R> struct Equilibrium;

template <typename R> struct Equilibrium<1, R> {
    __device__ __forceinline__ static void dev(R rho, const R* u, R* df) {
        const R dr = rho - R(1);
        const R m1 = rho * u[0];
        const R dm2 = (dr + R(2) * rho * u[0] * u[0]) * R(1.0 / 3.0);
        df[0] = dr - dm2;
        df[1] = R(0.5) * (m1 + dm2);
        df[2] = R(0.5) * (dm2 - m1);
    }
};

template <typename R> struct Equilibrium<2, R> {
    __device__ __forceinline__ static void dev(R rho, const R* u, R* df) {
        const R dr = rho - R(1);
        const R X = u[0] * u[0], Y = u[1] * u[1];
        // deviation moments m_pq - (rest-state m_pq), p,q in {0,1,2}
        const R m00 = dr, m10 = rho * u[0], m01 = rho * u[1];
        const R m20 = (dr + R(2) * rho * X) * R(1.0 / 3.0);
        const R m02 = (dr + R(2) * rho * Y) * R(1.0 / 3.0);
        const R m11 = R(2.0 / 3.0) * rho * u[0] * u[1];
        const R m21 = m01 * R(1.0 / 3.0), m12 = m10 * R(1.0 / 3.0);
        const R m22 = (dr + rho * (R(2) * (X + Y) - R(6) * X * Y)) * R(1.0 / 9.0);
        // inverse along x for q = 0, 1, 2 : g[a][q], a in {0, +, -}
        const R g00 = m00 - m20, gp0 = R(0.5) * (m10 + m20), gm0 = R(0.5) * (m20 - m10);
        const R g01 = m01 - m21, gp1 = R(0.5) * (m11 + m21), gm1 = R(0.5) * (m21 - m11);
        const R g02 = m02 - m22, gp2 = R(0.5) * (m12 + m22), gm2 = R(0.5) * (m22 - m12);
        // inverse along y; population order rest,+x,+y,-x,-y,++,+-,-+,--
        df[0] = g00 - g02;
        df[1] = gp0 - gp2;
        df[3] = gm0 - gm2;
        df[2] = R(0.5) * (g01 + g02);
        df[4] = R(0.5) * (g02 - g01);
        df[5] = R(0.5) * (gp1 + gp2);
        df[6] = R(0.5) * (gp2 - gp1);
        df[7] = R(0.5) * (gm1 + gm2);
        df[8] = R(0.5) * (gm2 - gm1);
    }
};

// Accumulators start at -0.0: x + (-0.0) == x for every x, so the compiler
// may drop that add (it may not drop 0.0 + x, which differs for x = -0.0).
// Products with compile-time zero velocity components are skipped for the
// same reason (0 * x is not foldable under IEEE rules).
template <typename R> struct Equilibrium<3, R> {
    __device__ __forceinline__ static void dev(R rho, const R* u, R* df) {
        using L = Lattice<3>;
        const R dr = rho - R(1);
        const R X = u[0] * u[0], Y = u[1] * u[1], Z = u[2] * u[2];
        const R S = X + Y + Z;
        df[0] = R(1.0 / 3.0) * (dr + rho * (R(-2.0 / 3.0) * S - R(2) * (X * Y + X * Z + Y * Z)));
#pragma unroll
        for (int i = 1; i < L::Q; ++i) {
            R eu = R(-0.0);
#pragma unroll
            for (int a = 0; a < 3; ++a)
                if (L::e(i, a) != 0) eu += R(L::e(i, a)) * u[a];
            const R eu2 = eu * eu;
            if (norm2<3>(i) == 1) {
                const R p = R(3) * eu + R(4) * eu2 - R(2) * S + R(6) * eu2 * (S - eu2);
                df[i] = R(1.0 / 18.0) * (dr + rho * p);
            } else {
                R q = R(-0.0);
                if (L::e(i, 0) != 0) q += X;
                if (L::e(i, 1) != 0) q += Y;
                if (L::e(i, 2) != 0) q += Z;
                const R h = eu2 - q;
                const R p = R(3) * eu + R(3) * eu2 - q - R(1.5) * h * h;
                df[i] = R(1.0 / 36.0) * (dr + rho * p);
            }
        }
    }
};

// ---------------------------------------------------------------------------
// Storage codecs.  Populations are stored as df = fbar* - w_i in the storage
// type; the variance as bt = bbar* + I/3 in `breal`.

template <typename S> struct Store;

template <> struct Store<double> {
    using real = double;
    using breal = double;
    template <typename I> __device__ __forceinline__ static double ld(const double* p, I k) { return __ldg(p + k); }
    template <typename I> __device__ __forceinline__ static void st(double* p, I k, double v) { p[k] = v; }
    __device__ __forceinline__ static void stb(double* p, unsigned b, double v) {
        *reinterpret_cast<double*>(reinterpret_cast<char*>(p) + b) = v;
    }
};

template <> struct Store<float> {
    using real = float;
    using breal = float;
    template <typename I> __device__ __forceinline__ static float ld(const float* p, I k) { return __ldg(p + k); }
    template <typename I> __device__ __forceinline__ static void st(float* p, I k, float v) { p[k] = v; }
    __device__ __forceinline__ static void stb(float* p, unsigned b, float v) {
        *reinterpret_cast<float*>(reinterpret_cast<char*>(p) + b) = v;
    }
};

template <> struct Store<__half> {
    using real = float;
    using breal = float;
    template <typename I> __device__ __forceinline__ static float ld(const __half* p, I k) {
        return __half2float(__ldg(p + k));
    }
    template <typename I> __device__ __forceinline__ static void st(__half* p, I k, float v) { p[k] = __float2half_rn(v); }
    __device__ __forceinline__ static void stb(__half* p, unsigned b, float v) {
        *reinterpret_cast<__half*>(reinterpret_cast<char*>(p) + b) = __float2half_rn(v);
    }
};

template <> struct Store<__nv_bfloat16> {
    using real = float;
    using breal = float;
    template <typename I> __device__ __forceinline__ static float ld(const __nv_bfloat16* p, I k) {
        return __bfloat162float(__ldg(p + k));
    }
    template <typename I> __device__ __forceinline__ static void st(__nv_bfloat16* p, I k, float v) {
        p[k] = __float2bfloat16_rn(v);
    }
    __device__ __forceinline__ static void stb(__nv_bfloat16* p, unsigned b, float v) {
        *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(p) + b) = __float2bfloat16_rn(v);
    }
};

// ---------------------------------------------------------------------------
// Layout of the variance planes of a state buffer (N sites).  FP64 storage and
// the D1/D2 lattices: component-major, component k of site s at k N + s.
// D3 with 32/16-bit storage: three planes of component pairs (xx, yy),
// (zz, xy), (xz, yz) interleaved per site, component k at (k/2) 2N + 2s + k%2,
// so that the transport reads a pair with one 8-byte access.
template <int D, typename FS> struct BLayout {
    static constexpr bool paired = D == 3 && !std::is_same<FS, double>::value;
    __host__ __device__ static constexpr long long at(int k, long long s, long long N) {
        return paired ? (long long)(k >> 1) * 2 * N + 2 * s + (k & 1) : (long long)k * N + s;
    }
};

}  // namespace lbm
