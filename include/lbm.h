/*
 * lbm.h -- C ABI of the GB300 (sm_103a) library for the bump-function lattice
 * Boltzmann method of Afrasiabian & Denniston, "A Novel Velocity
 * Discretization for Lattice Boltzmann Method: Application to Compressible
 * Flow" (arXiv 2501.00620).
 *
 * The method (Sec. II.B-C): every discrete population f_i is a bump in velocity
 * space with mean e_i and a per-site variance tensor b (Eq. 23), which lets the
 * equilibrium match the Maxwell-Boltzmann moments through third order on the
 * nearest-neighbour lattices D1Q3, D2Q9 and D3Q19 (Eqs. 28-31, Appendix A).
 * One time step takes the moments of the auxiliary populations fbar and of
 * bbar, corrects the velocity with an isotropic finite-difference gradient of
 * rho*b (Eqs. 57, 59, 67-68), relaxes fbar with forcing (Eq. 55) and bbar
 * (Eqs. 63, 65), and streams fbar (Eq. 49) and the mass-weighted bbar (Eq. 66)
 * to the nearest neighbours.
 *
 * Conventions for every entry point:
 *  - Lattice units: dx = dt = c = 1.  tau is the continuous relaxation time of
 *    Sec. II.C, so the discrete relaxation factor is omega = 1/(tau + 1/2)
 *    (Eq. 55) and the shear viscosity is eta = rho T tau (Eq. 84).
 *  - Sites are numbered s = x + nx*(y + ny*z).  Scalar fields are arrays of N
 *    doubles; vector fields are d planes of N doubles (component a of site s
 *    at a*N + s); symmetric tensors (b) are nb planes in the component order
 *    1D (xx), 2D (xx, yy, xy), 3D (xx, yy, zz, xy, xz, yz).
 *  - Population order: D3Q19 is the column order of the transformation matrix
 *    of Appendix B (rest, +x, +y, -x, -y, +z, -z, then the 12 edge
 *    velocities); D2Q9 is rest, +x, +y, -x, -y, (++), (+-), (-+), (--);
 *    D1Q3 is rest, +x, -x.
 *  - Host pointers passed in are owned by the caller; the library copies from
 *    or into them and never keeps them.  All device memory of a simulation
 *    is owned by the library (or by the allocator the caller installs).
 *  - Every call returns a status.  On failure, lbm_last_error() gives a
 *    message for the calling thread.  No entry point faults or traps the
 *    GPU on purpose: an unstable state (non-positive density or a non-finite
 *    value) raises a device flag that lbm_sync, lbm_moments and
 *    lbm_diagnostics report as LBM_EUNSTABLE.  A non-positive moment
 *    temperature in thermal mode is not fatal (it makes b^eq more negative
 *    and occurs transiently at sharp fronts); lbm_flags reports it.
 *  - Thread safety: one simulation handle must not be used from two host
 *    threads at once; different handles are independent.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_EINVAL = 1,     /* invalid argument */
    LBM_ENOMEM = 2,     /* device or host allocation failed, or over budget */
    LBM_ECUDA = 3,      /* a CUDA runtime call failed */
    LBM_EUNSTABLE = 4,  /* the state became non-physical (rho <= 0, NaN/Inf) */
    LBM_ETIMEOUT = 5,   /* a bounded device-side wait gave up */
    LBM_EBUSY = 6,      /* result not ready yet (serving) */
    LBM_EIO = 7         /* checkpoint file error */
} lbm_status;

typedef enum {
    LBM_BC_PERIODIC = 0,    /* periodic on every axis */
    LBM_BC_FIXED_STATE = 1, /* x: frozen equilibrium reservoirs carrying the
                               initial state of the edge site of each row;
                               y and z periodic */
    LBM_BC_WALLS = 2        /* dim 2, 3: two stationary half-way bounce-back
                               walls (Sec. III.A) normal to the last axis (y in
                               2D, z in 3D), half a site outside the lattice;
                               the other axes periodic.  A population whose
                               source lies beyond a wall is the site's own
                               emission in the opposite direction, with the
                               site's bbar; the gradient stencil sees beyond a
                               wall the image of the facing site (same rho b,
                               reversed u0).  Runs on the generic kernel. */
} lbm_bc;

typedef enum {
    LBM_F64 = 0,          /* populations and arithmetic in FP64 */
    LBM_F32 = 1,          /* FP32 storage and arithmetic */
    LBM_F16_SHIFTED = 2,  /* populations stored as FP16 deviations from the
                             rest-state weight w_i; bbar in FP32; FP32 math */
    LBM_BF16_SHIFTED = 3  /* as above with BF16 */
} lbm_dtype;

typedef enum {
    LBM_MODEL_BUMP = 0,     /* the bump-function scheme (Sec. II) */
    LBM_MODEL_STANDARD = 1  /* comparator: the textbook BGK scheme with the
                               Hermite equilibrium of Eq. 4 in lattice units,
                               f^eq_i = w_i rho [1 + e.u/cs2 + (u u + (T0 -
                               cs2) I) : (e e - cs2 I) / (2 cs2^2)], cs2 = 1/3,
                               relaxed with the same omega = 1/(tau + 1/2);
                               no variance and no gradient correction, so its
                               shear viscosity is rho tau / 3 for any T0 (the
                               paper's contrast, Sec. I).  Periodic lattices,
                               no body force, ny and nz <= 65535; lbm_init's T
                               field sets the start equilibrium, T0 the
                               collision's; lbm_moments reports the moment
                               temperature (E - rho|u|^2)/(d rho) and
                               lbm_diagnostics mass, sum j, sum f|e|^2 */
} lbm_model;

/* Optional device allocator (e.g. a framework's caching allocator).  alloc
 * returns device memory of at least `bytes` on the current device or NULL;
 * free releases it. */
typedef void *(*lbm_alloc_fn)(size_t bytes, void *ctx);
typedef void (*lbm_free_fn)(void *ptr, size_t bytes, void *ctx);

typedef struct {
    lbm_dtype dtype;        /* default LBM_F64 */
    int thermal;            /* 0 (default): isothermal, T = T0 in b^eq, as in
                               the paper's analysis (Sec. II.D, P = rho T);
                               1: T from the trace of the full second moment,
                               which conserves energy */
    int device;             /* CUDA device ordinal, default 0 */
    void *stream;           /* cudaStream_t to run on; NULL: the library
                               creates its own non-blocking stream */
    lbm_alloc_fn alloc;     /* NULL: cudaMalloc / cudaFree */
    lbm_free_fn free;
    void *alloc_ctx;
    int tile;               /* kernel variant index; -1 (default): autotuned */
    int chunk;              /* planes per block along the march axis; 0: auto */
    int steps_per_launch;   /* 1D lattices, and 2D lattices of at most 2^18
                               sites without halo: steps per cooperative
                               launch (a grid-wide barrier between steps; 1D
                               and FP64 2D give the same bits as single steps,
                               FP32 2D the same up to FP32 rounding); 0
                               (default): the faster of 64 per launch and
                               CUDA-graph replays of single steps, timed at
                               the first lbm_step on scratch copies of the
                               state (2D: only with an autotuned tile); 1:
                               single steps */
    int diagnostics;        /* 1 (default): every step also reduces mass,
                               momentum and energy of the state it consumes
                               into a device history (lbm_diagnostics_history);
                               0: off */
    int use_graphs;         /* 1 (default): lbm_step replays CUDA graphs */
    int model;              /* LBM_MODEL_BUMP (default) or LBM_MODEL_STANDARD */
    int halo;               /* 0 (default); 2: the simulation is one slab of a
                               lattice decomposed along its slowest axis (y in
                               2D, z in 3D): that axis ends in 2 halo planes on
                               each side, which the step reads but does not
                               update, and nothing wraps along it.  The extent
                               passed to lbm_create_ex includes the 4 halo
                               planes.  The halo holds the neighbouring slabs'
                               emitted state (lbm_halo_exchange or
                               lbm_halo_pack / lbm_halo_unpack after every
                               step).  2D/3D bump scheme, periodic or
                               fixed-state boundary in x */
    int inplace;            /* 0 (default): A-B buffers of the populations
                               (one fused pass per step); 1: one population
                               buffer, updated in place (two passes per step:
                               pass 1 writes (u0, rho b) per site to an aux
                               array, pass 2 reads the neighbours' values for
                               the gradients, collides and writes each site's
                               new populations into the slots it read; the
                               slots alternate between the emitted layout
                               after an even number of steps and the arrived
                               populations in opposite planes after an odd
                               one).  Device memory per site: Q + 2 nb +
                               dim + nb values instead of 2 (Q + nb); HBM
                               traffic per step about 1.9x the A-B step's.
                               Bump scheme, periodic boundary, FP64 or FP32
                               storage; no body force, MRT or small-T
                               recovery; lbm_save after an even step count */
    int cluster;            /* multi-step launches of small periodic 2D
                               lattices with the whole state resident in the
                               shared memory of one thread-block cluster (up
                               to 16 blocks on 16 multiprocessors, neighbour
                               rows read through distributed shared memory;
                               FP32 or FP64 storage, bump scheme, no walls,
                               force, MRT or small-T recovery, no halo): 0
                               (default) the steps-per-launch autotuner
                               times it with the other forms; -1 never; 1 + v
                               forces cluster variant v (0: 16 blocks of 256
                               threads, 1: 16 x 512, 2: 8 x 512) with
                               steps_per_launch steps per launch (64 if not
                               > 1); lbm_step then fails with LBM_EINVAL if
                               the lattice does not fit that variant.  A
                               setting only the generic kernel has (body
                               force, MRT, small-T recovery) takes
                               precedence over a forced variant */
} lbm_opts;

typedef struct lbm_sim lbm_sim;

/* Fill *opts with the defaults listed above. */
void lbm_default_opts(lbm_opts *opts);

/* Create a simulation of a dim-dimensional lattice (dim 1: D1Q3, 2: D2Q9,
 * 3: D3Q19; Sec. II.B) of nx*ny*nz sites (unused extents must be 1), with
 * relaxation time tau > 0 (Eq. 55), reference temperature T0 > 0 and boundary
 * bc.  Allocates the two emitted-state buffers (A-B ping-pong) on the device.
 * The state is undefined until lbm_init.  *out receives the handle. */
lbm_status lbm_create(int dim, int nx, int ny, int nz, double tau, double T0,
                      lbm_bc bc, lbm_sim **out);
lbm_status lbm_create_ex(int dim, int nx, int ny, int nz, double tau, double T0,
                         lbm_bc bc, const lbm_opts *opts, lbm_sim **out);

typedef struct {
    const double *rho;  /* N values, > 0 */
    const double *u;    /* dim planes of N values */
    const double *T;    /* N values, > 0 */
} lbm_fields_in;

/* Set the state from host fields (rho, u, T): every site emits its local
 * equilibrium fbar* = f^eq(rho, u) (Appendix A) and bbar* = b^eq(u, T)
 * (Eq. 36); the state at t = 0 is what streams in.  For LBM_BC_FIXED_STATE the
 * reservoirs take the state of the edge site of each row.  Resets the step
 * counter.  Blocks until the copy is done. */
lbm_status lbm_init(lbm_sim *sim, const lbm_fields_in *fields);

/* Uniform body force (Sec. III.A drives Poiseuille flow by an acceleration):
 * `a` points at dim host doubles, the acceleration in lattice units (copied;
 * NULL or all zeros removes the force).  Each step adds the force density
 * rho a to the gradient force F (Eq. 59) and rho (u a + a u) to G (Eq. 61),
 * with the corrected u = (j0 + F/2)/rho of Eq. 57, before the collision; so
 * the reported u and the momentum diagnostic carry half a step of force.
 * A forced simulation runs on the generic kernel.  Waits for the
 * simulation's stream.  LBM_EINVAL for a NULL sim or a non-finite value. */
lbm_status lbm_set_force(lbm_sim *sim, const double *a);

/* MRT collision (Appendix B) for the D3Q19 bump scheme: moments in the basis
 * of Table M, M^a = sum_i m^a_i f_i, relax at their own rates,
 * M*^a = M^a + s_a (M^a_eq - M^a) + (1 - s_a/2) Phi^a, and populations come
 * back as f_i = w_i sum_a m^a_i N^a M^a with N^a = 1 / sum_i w_i (m^a_i)^2.
 * The conserved and second-order moments relax at omega (the viscosity
 * eta = rho T tau of the SRT step); s3 is the rate of the third-order rows
 * 10-15, s4 of the fourth-order rows 16-18; bbar keeps the single rate.
 * s3 = s4 = omega is the SRT step; s3 <= 0 and s4 <= 0 switch MRT off.
 * Runs on the generic kernel.  Waits for the simulation's stream.
 * LBM_EINVAL for another lattice or model, or rates outside (0, 2). */
lbm_status lbm_set_mrt(lbm_sim *sim, double s3, double s4);

/* FP64 recovery of the temperature where it is small (thermal mode, 32/16-bit
 * storage; the paper's T of Eq. 57 and the T_unc of Eq. 68 taken from the
 * moments).  T = (Ebar - rho |u|^2) / (d rho) is a difference of two nearly
 * equal numbers when T << |u|^2, so in FP32 its relative error grows like
 * |u|^2 / T.  With kappa > 0, a site whose FP32 T_unc is below
 * kappa |u0|^2 repeats its variance transport (Eq. 66), moments and rho b
 * (Eq. 68) in FP64, and its corrected T and b^eq (Appendix A) come from the
 * FP64 energy; the bump parameters are then rounded to the storage type.
 * lbm_moments reports that FP64 T.  kappa = 0 (the default) turns it off.
 * Runs on the generic kernel (the staged kernels do not carry FP64 values
 * between their stages); each recovered site costs about 150 FP64
 * operations, which on GB300 take the time of several thousand FP32 ones,
 * so kappa should select only the sites that need it (kappa = 1: T below
 * |u|^2).  No effect for FP64 storage or isothermal runs.  A setting of
 * the simulation, not of a checkpoint.  Waits for the simulation's stream.
 * LBM_EINVAL for kappa < 0 or not finite. */
lbm_status lbm_set_small_t(lbm_sim *sim, double kappa);

/* Velocities of the walls of an LBM_BC_WALLS lattice (Sec. III.D's Couette
 * flow): `lo` and `hi` point at dim host doubles each, the velocity of the
 * lower and upper wall (copied; NULL means at rest).  Walls move along
 * themselves: the component along the last axis must be 0.  A population
 * bounced at a moving wall gains 6 w_i rho e_i.u_w, rho the density of the
 * site at t (the odd part of the equilibrium), and the gradient stencil's
 * image velocity is 2 u_w - u0.  Takes effect at the next streaming: the
 * start state of lbm_init is an emission that the first lbm_step streams,
 * so velocities set before that step apply to it.  Waits for the
 * simulation's stream.  LBM_EINVAL without walls, for a normal component
 * or a non-finite value. */
lbm_status lbm_set_wall_velocity(lbm_sim *sim, const double *lo, const double *hi);

/* Advance n >= 0 time steps (Sec. II.C, Eqs. 49-68): asynchronous on the
 * simulation's stream. */
lbm_status lbm_step(lbm_sim *sim, long n);

/* Wait for the simulation's stream; reports LBM_EUNSTABLE if the device flag
 * is set. */
lbm_status lbm_sync(lbm_sim *sim);

typedef struct {
    double *rho;  /* N values or NULL */
    double *u;    /* dim planes of N values or NULL: corrected velocity
                     u = (sum fbar e + F/2)/rho (Eq. 57) */
    double *T;    /* N values or NULL: moment temperature
                     (E - rho|u|^2)/(dim rho), E = sum fbar|e|^2 + rho tr bbar
                     + tr(G)/2 */
} lbm_fields_out;

/* Macroscopic fields of the current state, copied to the host.  Blocking. */
lbm_status lbm_moments(lbm_sim *sim, lbm_fields_out *out);

/* Global mass, momentum (dim values) and energy of the current state, summed
 * in FP64: out[0] = sum rho, out[1..dim] = sum rho u, out[dim+1] = sum E.
 * Blocking. */
lbm_status lbm_diagnostics(lbm_sim *sim, double *out);

/* The per-step diagnostics recorded by lbm_step when opts.diagnostics = 1:
 * up to `cap` most recent records, oldest first, each dim+3 doubles
 * (step index, mass, momentum..., energy).  *count receives the number
 * written.  Blocking. */
lbm_status lbm_diagnostics_history(lbm_sim *sim, double *out, int cap, int *count);

/* The newest per-step record (step index, mass, momentum..., energy; dim+3
 * doubles) written by lbm_step when opts.diagnostics = 1: a read of d+3
 * doubles, the cheap per-step result.  Blocking.  LBM_EINVAL if no step has
 * recorded diagnostics since lbm_init. */
lbm_status lbm_last_diagnostics(lbm_sim *sim, double *out);

/* Emitted (post-collision, about to stream) state in FP64 on the host:
 * f: Q planes of N values (fbar*_i), b: nb planes of N values (bbar*).
 * Either pointer may be NULL.  Blocking. */
lbm_status lbm_get_state(lbm_sim *sim, double *f, double *b);

/* Replace the emitted state from FP64 host planes (same layout), encoded to
 * the storage dtype.  Reservoirs and the step counter are unchanged. */
lbm_status lbm_set_state(lbm_sim *sim, const double *f, const double *b);

/* Sticky status bits since lbm_init: bit 0 = a fatal state was seen (see
 * LBM_EUNSTABLE), bit 1 = a non-positive moment temperature was seen
 * (thermal mode).  Blocking. */
lbm_status lbm_flags(lbm_sim *sim, int *flags);

/* Number of steps taken since lbm_init. */
long lbm_step_count(const lbm_sim *sim);

/* The launch configuration of the step (library service, no counterpart in
 * the paper): *tile = the tile variant in use (0.. the generic fused kernel;
 * on D2Q9 3 = the strip kernel; 100.. the shared-memory-staged kernels;
 * 200.. the pair kernel; 300 + v the cluster-resident kernel's variant v;
 * 900 the in-place step), *chunk = planes per thread block along the slowest
 * axis, or steps per launch when several steps run per launch, *kernel =
 * name of the kernel template (static string; "step_multi_kernel" or
 * "step_cluster_kernel" when several steps run per launch).  Fixed by
 * opts.tile/opts.chunk/opts.cluster or by the autotuner at the first
 * lbm_step; before that *tile = *chunk = -1 and *kernel = "".  Any pointer
 * may be NULL.  Host only, never fails for a valid handle. */
lbm_status lbm_launch_config(const lbm_sim *sim, int *tile, int *chunk, const char **kernel);

/* Checkpoint: write / read the full state (emitted planes in the storage
 * dtype, reservoirs, step counter, parameters) as a raw file with a small
 * header.  lbm_load requires a simulation created with the same dim, extents,
 * dtype, boundary and model (lbm_opts.model; LBM_EINVAL otherwise), and
 * refuses with LBM_EIO a file whose header holds tau or T0 that are not
 * finite and > 0.  A run of n steps equals n/2 steps + save + load + n/2
 * steps bit for bit.  The body force, the wall velocities and the MRT rates
 * are settings of the simulation, not of the checkpoint: set them on the
 * simulation that loads it. */
lbm_status lbm_save(lbm_sim *sim, const char *path);
lbm_status lbm_load(lbm_sim *sim, const char *path);

/* Domain decomposition (slabs along the slowest axis; no counterpart in the
 * paper, whose step is a nearest-neighbour stencil).  A site's update reads
 * the emitted state of its neighbours (the pull, Eq. 49, and the transport,
 * Eq. 66) and, through the gradient of rho b (Eqs. 59, 61, 68), of the
 * neighbours of its neighbours: a slab needs the two planes beyond each of
 * its faces, refreshed after every step.  Slabs are simulations created with
 * lbm_opts.halo = 2: with h = 2 and n planes along the slowest axis, planes
 * [0, h) and [n - h, n) are the halo and [h, n - h) are owned.  lbm_init of
 * a slab takes fields for all n planes (the halo from the neighbouring
 * slabs, as the whole lattice's fields give them); lbm_moments writes the
 * owned planes only; lbm_diagnostics sums the owned sites (the lattice's
 * totals are the sums over slabs, one all-reduce of dim + 2 doubles).
 *
 * lbm_halo_bytes: bytes of one message -- h planes of every population and
 * variance plane in the storage type (0 for a simulation without halo).
 * lbm_halo_pack: copies the outermost h owned planes on `side` (0: low,
 * planes h .. 2h-1; 1: high, planes n-2h .. n-h-1) of the current state into
 * `dst` (device memory of lbm_halo_bytes bytes), asynchronously on the
 * simulation's stream.  lbm_halo_unpack: writes `src` (a message packed by
 * the neighbour on that side) into the halo planes on `side` (0: planes
 * 0 .. h-1, 1: planes n-h .. n-1).  Between processes a message travels from
 * one slab's pack to the next slab's unpack (point-to-point, e.g. NCCL
 * send / recv); both calls only enqueue copies.
 * lbm_halo_exchange: the same exchange among k slabs held by this process
 * (one or several devices), periodic along the slowest axis: slab i's low
 * halo receives slab i-1's top owned planes, its high halo slab i+1's
 * bottom ones (indices mod k).  Device-to-device copies ordered by events
 * after each slab's last step and before its next one; call it after every
 * lbm_step(sim, 1) of all slabs.  Slabs must agree in dim, cross-section,
 * storage and halo depth (LBM_EINVAL otherwise). */
size_t lbm_halo_bytes(const lbm_sim *sim);
lbm_status lbm_halo_pack(lbm_sim *sim, int side, void *dst);
lbm_status lbm_halo_unpack(lbm_sim *sim, int side, const void *src);
lbm_status lbm_halo_exchange(lbm_sim *const *sims, int k);

/* Test switches (library service, no counterpart in the paper): they
 * exercise the failure paths of the kernels without faulting the GPU.
 * LBM_DEBUG_MISSING_COPY: in the next steps, one thread block of the
 * shared-memory-staged kernels (launch variants 100.. and 200..) arms the
 * transaction barrier of its first variance-plane copy but issues no copy.
 * Every wait on that barrier gives up after its time limit (20 ms), the
 * block leaves without storing, after its copies in flight have completed,
 * and the step reports LBM_ETIMEOUT at the next lbm_sync / lbm_moments /
 * lbm_diagnostics.  The state is then not a valid step: lbm_init or lbm_load
 * it again (lbm_init also clears the device flag).  The generic kernel has
 * no staged copies and ignores the switch.  flags = 0 turns it off.  Waits
 * for the simulation's stream; drops the captured step graphs.
 * LBM_EINVAL for unknown flags. */
#define LBM_DEBUG_MISSING_COPY 1
lbm_status lbm_set_debug(lbm_sim *sim, int flags);

/* One time step that allocates no device memory, on device buffers the
 * caller owns.  The paper has no counterpart: this is a library service for
 * callers that may not allocate device memory while they run, such as
 * real-time loops that cannot take the synchronisation an allocator may
 * impose, or host frameworks and plugins that own every device allocation
 * and give a library none.  Such a caller allocates the state once, up front,
 * and advances it with this call.
 *
 * It runs the same fused step as lbm_step (periodic boundary in every
 * direction, FP64 storage) on the emitted state, in the kernel's own layout:
 *   f_in, f_out: Q planes of N doubles, plane i = fbar*_i - w_i
 *                (the emitted population minus its lattice weight);
 *   b_in, b_out: nb planes of N doubles, bbar* + I/3 (the diagonal planes
 *                shifted by 1/3, the off-diagonal planes unchanged);
 * with the plane and site order of lbm_get_state.  f_in/b_in hold the state
 * at step t, f_out/b_out receive step t+1.
 * diag_out (device pointer or NULL) receives dim+2 doubles: mass, momentum
 * and energy of the state at step t, as lbm_diagnostics gives them.
 * tau, T0 and thermal are those of lbm_create_ex; stream is a cudaStream_t
 * (NULL = legacy default stream).  The call is blocking: it waits for the
 * step on `stream` and returns LBM_EUNSTABLE if the new state is
 * non-physical (rho <= 0 or not finite).
 *
 * Scratch: the per-block partial sums of the diagnostics, the reduction's
 * completion ticket and the status flag live in one fixed 1 MiB device
 * array inside the library (present on every GPU the library is loaded on),
 * so the lattice may span at most (2^20 - 256) / (8 (dim+2)) thread blocks:
 * 43,680 in 1D (256 sites each, 11.1 M sites), 32,760 in 2D (128 x 64 sites
 * each, 268 M sites), 26,208 in 3D (32 x 8 x 64 sites each, 429 M sites).
 * A larger lattice is rejected with LBM_EINVAL and a message.  The call sets
 * the ticket and flag to zero on `stream` before each launch; the partial
 * sums need no clearing.  Every call looks up the array's device address
 * with cudaGetSymbolAddress (so a device reset between calls is harmless);
 * the first call on a device, and the first after a reset, also sets the
 * kernels' shared-memory attribute: make that first call before any stream
 * capture.  input and output must not overlap: an output range that overlaps
 * an input or the other output (byte ranges of Q*N and nb*N doubles) is
 * rejected with LBM_EINVAL; the two inputs may alias each other.  The array
 * is shared by all calls on one device, so
 * two calls that overlap in time on one device -- from two host threads, or
 * on two streams -- race on it and may return wrong diagnostics or flags. */
lbm_status lbm_step_noalloc(int dim, int nx, int ny, int nz, double tau, double T0, int thermal,
                            const double *f_in, const double *b_in, double *f_out, double *b_out,
                            double *diag_out, void *stream);

/* Free all device memory of the simulation. */
void lbm_destroy(lbm_sim *sim);

/* Message of the last failed call on this host thread ("" if none). */
const char *lbm_last_error(void);

/* Library version string. */
const char *lbm_version(void);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
