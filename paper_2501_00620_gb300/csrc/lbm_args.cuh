// Launch arguments shared by the step kernels.
#pragma once

namespace lbm {

struct StepArgs {
    const void* fin;      // Q planes, storage type: emitted df at t
    const void* bin;      // NB planes, breal: emitted bt at t
    void* fout;           // Q planes: emitted df at t+1 (write_state)
    void* bout;           // NB planes
    int nx, ny, nz;
    int chunk;            // planes per block along the march axis
    int halo;             // 0, or 2: the march axis (y in 2D, z in 3D) ends in two halo planes at each
                          // side that the step reads but does not update, and nothing wraps along it
                          // (a slab of a decomposed lattice)
    long long N;
    double omega, tau, T0;
    float omega_f, tau_f, T0_f;  // the same, rounded to FP32 on the host (FP32 arithmetic)
    int thermal;
    int fixed_x;          // 1: frozen reservoirs outside [0, nx)
    long long rows;       // ny * nz (reservoir rows)
    const void* gf;       // reservoirs, real: [2][Q][rows] df
    const void* gb;       // [2][NB][rows] bt
    const void* gaux;     // [2][D+NB][rows] u (D), rho*b (NB)
    int write_state;      // 1: collide and store S(t+1)
    double* mout;         // if non-null: rho (N), u (D*N), T (N) in FP64
    int want_diag;        // 1: reduce mass, momentum, energy of the state at t
    double* partial;      // [gridDim total][D+2] per-block sums
    unsigned int* ticket; // completion counter for the last-block reduction
    double* diag_out;     // if non-null: the D+2 global sums
    double* hist;         // history ring: records of D+3 doubles
    int hist_cap;
    long long* step_ctr;  // device step counter (history index)
    int* flag;            // bit 0: fatal (rho <= 0 or non-finite); bit 1: T <= 0 seen
    int walls;            // 1: half-way bounce-back walls normal to the march axis (D = 2, 3)
    int forced;           // 1: uniform body force of acceleration acc
    double acc[3];        // body-force acceleration (lattice units)
    float acc_f[3];       // the same, rounded to FP32 on the host
    int walls_moving;     // 1: a wall has a nonzero (tangential) velocity
    double uw[2][3];      // wall velocities: [0] lower, [1] upper wall
    float uw_f[2][3];
    int debug_missing_copy;  // 1: block (0,0,0) of a staged kernel arms its first variance-copy barrier
                             // without issuing the copy (exercises the bounded waits; nothing is left in flight)
    double small_t;       // > 0 (thermal, 32/16-bit storage): sites with T < small_t |u|^2 recover T in FP64
    float small_t_f;
    int mrt;              // 1: MRT collision (D3Q19, lbm_mrt.cuh)
    double mrt_s[2];      // its rates of the third- and fourth-order moments
    float mrt_s_f[2];
};

// Planes of the march axis a step updates: [halo, np - halo).
__host__ __device__ __forceinline__ int march_extent(const StepArgs& a, int D) {
    return (D == 3 ? a.nz : (D == 2 ? a.ny : 1)) - (D >= 2 ? 2 * a.halo : 0);
}

// Body-force acceleration in the arithmetic type R.
__host__ __device__ __forceinline__ double acc_param(const StepArgs& a, int c, double) { return a.acc[c]; }
__host__ __device__ __forceinline__ float acc_param(const StepArgs& a, int c, float) { return a.acc_f[c]; }
// MRT rate (0: third-order moments, 1: fourth-order) in the arithmetic type R.
__host__ __device__ __forceinline__ double mrt_rate(const StepArgs& a, int k, double) { return a.mrt_s[k]; }
__host__ __device__ __forceinline__ float mrt_rate(const StepArgs& a, int k, float) { return a.mrt_s_f[k]; }
// Wall velocity (side 0 lower, 1 upper) in the arithmetic type R.
__host__ __device__ __forceinline__ double uw_param(const StepArgs& a, int side, int c, double) { return a.uw[side][c]; }
__host__ __device__ __forceinline__ float uw_param(const StepArgs& a, int side, int c, float) { return a.uw_f[side][c]; }

// omega, tau, T0 in the arithmetic type R (no per-site conversion from FP64).
__host__ __device__ __forceinline__ void step_params(const StepArgs& a, double& omega, double& tau, double& T0) {
    omega = a.omega;
    tau = a.tau;
    T0 = a.T0;
}
__host__ __device__ __forceinline__ void step_params(const StepArgs& a, float& omega, float& tau, float& T0) {
    omega = a.omega_f;
    tau = a.tau_f;
    T0 = a.T0_f;
}

// Sets omega = 1/(tau + 1/2) (Eq. 55), tau, T0 and their FP32 copies.
inline void set_step_params(StepArgs& a, double tau, double T0) {
    a.omega = 1.0 / (tau + 0.5);
    a.tau = tau;
    a.T0 = T0;
    a.omega_f = (float)a.omega;
    a.tau_f = (float)tau;
    a.T0_f = (float)T0;
}

}  // namespace lbm
