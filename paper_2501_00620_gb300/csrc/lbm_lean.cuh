// Device helpers shared by the staged step kernels (lbm_step_fast.cuh,
// lbm_step_strip.cuh): FP32 deviation-sum diagnostics, the site-major
// (u0, rho b) groups of the shared-memory gradient slots, and one neighbour's
// term of the lattice-weight gradients F = -div(rho b) (Eq. 59) and
// G = -div(rho u0 b + rho u0 b) (Eq. 61), all in FP32.
#pragma once

#include <type_traits>
#include <utility>

#include "lbm_site.cuh"

namespace lbm {

// FP32 accumulator of the conservation diagnostics (mass, momentum, energy)
// as deviations from the rest state: mass as rho - 1, energy as E - eref with
// eref = D T0.  get() adds the references back in FP64.
template <int K> struct DiagDev {
    static constexpr bool kFF = true;  // reduced as float-float pairs (block_diagnostics)
    float d[K];
    int n;
    float eref;
    __device__ __forceinline__ explicit DiagDev(float e) : n(0), eref(e) {
#pragma unroll
        for (int k = 0; k < K; ++k) d[k] = 0.0f;
    }
    __device__ __forceinline__ void add(int k, float x) {
        if (k == 0) {
            d[0] += x - 1.0f;
            ++n;
        } else if (k == K - 1) {
            d[k] += x - eref;
        } else {
            d[k] += x;
        }
    }
    __device__ __forceinline__ double get(int k) const {
        return double(d[k]) + (k == 0 ? double(n) : (k == K - 1 ? double(n) * double(eref) : 0.0));
    }
    // value k = (h + l) + cnt() * cref(k)
    __device__ __forceinline__ void ff(int k, float& h, float& l) const {
        h = d[k];
        l = 0.0f;
    }
    __device__ __forceinline__ int cnt() const { return n; }
    __device__ __forceinline__ float cref(int k) const { return k == 0 ? 1.0f : (k == K - 1 ? eref : 0.0f); }
};

// (u0, rho b) of one site as the float2 groups of the aux slots:
//   3D: (u_x, u_y), (rb_xx, rb_xy), (rb_xy, rb_yy), (rb_xz, rb_yz), (u_z, rb_zz)
//   2D: (u_x, u_y), (rb_xx, rb_xy), (rb_xy, rb_yy)
template <int D>
__device__ __forceinline__ void put_aux(float2* ax, const float* u0, const float* rb) {
    if constexpr (D == 3) {
        ax[0] = make_float2(u0[0], u0[1]);
        ax[1] = make_float2(rb[0], rb[3]);
        ax[2] = make_float2(rb[3], rb[1]);
        ax[3] = make_float2(rb[4], rb[5]);
        ax[4] = make_float2(u0[2], rb[2]);
    } else {
        ax[0] = make_float2(u0[0], u0[1]);
        ax[1] = make_float2(rb[0], rb[2]);
        ax[2] = make_float2(rb[2], rb[1]);
    }
}


// Gradient contribution of neighbour x + e_i (unscaled, sign of e_i folded
// in): v = e_i . (rho b); F += v; G_bc += u_c v_b + u_b v_c, the diagonal
// counted once (doubled at the end).  `n` points at the neighbour's aux.
template <int D, int I>
__device__ __forceinline__ void grad_term(const float2* n, float* F, float* G) {
    using L = Lattice<D>;
    constexpr int ex = L::e(I, 0), ey = L::e(I, 1), ez = L::e(I, 2);
    const float2 A0 = n[0];
    if constexpr (D == 3) {
        const float2 A3 = n[3], A4 = n[4];
        const float ux = A0.x, uy = A0.y, uz = A4.x;
        float vx = 0.0f, vy = 0.0f, vz = 0.0f;
        bool first = true;
        auto addrow = [&](int s, float rx_, float ry_, float rz_) {
            if (first) {
                vx = s * rx_;
                vy = s * ry_;
                vz = s * rz_;
                first = false;
            } else {
                vx += s * rx_;
                vy += s * ry_;
                vz += s * rz_;
            }
        };
        if constexpr (ex != 0) {
            const float2 A1 = n[1];
            addrow(ex, A1.x, A1.y, A3.x);  // row x: (xx, xy, xz)
        }
        if constexpr (ey != 0) {
            const float2 A2 = n[2];
            addrow(ey, A2.x, A2.y, A3.y);  // row y: (xy, yy, yz)
        }
        if constexpr (ez != 0) addrow(ez, A3.x, A3.y, A4.y);  // row z: (xz, yz, zz)
        F[0] += vx;
        F[1] += vy;
        F[2] += vz;
        G[0] = fmaf(ux, vx, G[0]);
        G[1] = fmaf(uy, vy, G[1]);
        G[2] = fmaf(uz, vz, G[2]);
        G[3] = fmaf(uy, vx, fmaf(ux, vy, G[3]));
        G[4] = fmaf(uz, vx, fmaf(ux, vz, G[4]));
        G[5] = fmaf(uz, vy, fmaf(uy, vz, G[5]));
    } else {
        const float ux = A0.x, uy = A0.y;
        float vx = 0.0f, vy = 0.0f;
        if constexpr (ex != 0) {
            const float2 A1 = n[1];
            vx = ex * A1.x;
            vy = ex * A1.y;
        }
        if constexpr (ey != 0) {
            const float2 A2 = n[2];
            if constexpr (ex != 0) {
                vx += ey * A2.x;
                vy += ey * A2.y;
            } else {
                vx = ey * A2.x;
                vy = ey * A2.y;
            }
        }
        F[0] += vx;
        F[1] += vy;
        G[0] = fmaf(ux, vx, G[0]);
        G[1] = fmaf(uy, vy, G[1]);
        G[2] = fmaf(uy, vx, fmaf(ux, vy, G[2]));
    }
}


}  // namespace lbm

namespace lbm {

// F and G at a site from the aux groups of its neighbours (Eqs. 59, 61 with
// the lattice-weight central difference): `nb(std::integral_constant<int, I>)`
// returns the aux groups of neighbour x + e_I.  The axis terms carry
// w_axis = (w_axis / w_edge) w_edge, so they are summed first and scaled by
// that ratio (2 on D3Q19, 4 on D2Q9), then the edge terms are added and
// everything is scaled by -3 w_edge (the diagonal of G: twice that).
template <int D, typename NbFn, int... Is>
__device__ __forceinline__ void gradients_seq(NbFn&& nb, float* F, float* G, std::integer_sequence<int, Is...>) {
    using L = Lattice<D>;
    constexpr int NB = L::NB;
#pragma unroll
    for (int c = 0; c < D; ++c) F[c] = 0.0f;
#pragma unroll
    for (int k = 0; k < NB; ++k) G[k] = 0.0f;
    ((norm2<D>(Is + 1) == 1 ? grad_term<D, Is + 1>(nb(std::integral_constant<int, Is + 1>{}), F, G) : void()), ...);
    constexpr float ratio = float(L::w(1) / L::w(L::Q - 1));
#pragma unroll
    for (int c = 0; c < D; ++c) F[c] *= ratio;
#pragma unroll
    for (int k = 0; k < NB; ++k) G[k] *= ratio;
    ((norm2<D>(Is + 1) == 2 ? grad_term<D, Is + 1>(nb(std::integral_constant<int, Is + 1>{}), F, G) : void()), ...);
    constexpr float sc = float(-3.0 * L::w(L::Q - 1));
#pragma unroll
    for (int c = 0; c < D; ++c) F[c] *= sc;
#pragma unroll
    for (int k = 0; k < NB; ++k) G[k] *= (k < D ? 2.0f * sc : sc);
}

template <int D, typename NbFn>
__device__ __forceinline__ void gradients(NbFn&& nb, float* F, float* G) {
    gradients_seq<D>(nb, F, G, std::make_integer_sequence<int, Lattice<D>::Q - 1>{});
}

}  // namespace lbm
