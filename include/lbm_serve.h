/*
 * lbm_serve.h -- continuous-batching service for many small simulations of
 * the bump-function lattice Boltzmann method (arXiv 2501.00620) on one GPU.
 *
 * The paper has no counterpart: this is a library service on top of the
 * method.  Each request is one simulation -- D1Q3 or D2Q9, periodic or
 * fixed-state boundary, given initial fields (rho, u, T) and a step count --
 * and its result is the macroscopic fields (rho, u, T; Eq. 57 and the moment
 * temperature) after those steps, the same quantities lbm_moments returns.
 *
 * Precision: FP32 storage and arithmetic, except for 1D fixed-state requests
 * (two-state Riemann problems), which run with FP64 storage and arithmetic:
 * in FP32 the rounding-size perturbations at a shock front of such a problem
 * grow until the state leaves the physical range (rho <= 0, measured after
 * about 1600 steps on the 4096-site problem), while requests may ask for
 * thousands of steps; from FP64 rounding they stay small over that span.
 *
 * Model:
 *  - lbm_server_submit copies the request's fields and queues it; a service
 *    thread inside the library admits queued requests, first come first
 *    served, while their state fits in the server's device memory pool (the
 *    HBM budget) and the number of active simulations is below the limit.
 *    Admitted simulations stay resident on the device until they finish.
 *  - One persistent cooperative kernel advances all active simulations,
 *    round after round, by up to K steps a round: its thread blocks walk a
 *    work list of tiles of every simulation, with a grid-wide barrier between
 *    steps.  The service thread posts each round through a mailbox in mapped
 *    host memory (after the round's work list and the admitted requests'
 *    fields have been copied to the device); the kernel computes the
 *    admitted simulations' start states itself at the start of their first
 *    round, runs the round, and reports it done in the mailbox.  K is chosen
 *    so that a round lasts about opts.round_ms, so that newly admitted
 *    requests join within a round.  Requests of uneven sizes share every
 *    round.  Every wait of the kernel is bounded: after opts.idle_ms without
 *    a posted round (or when the server stops) it leaves, and the service
 *    thread launches it again when work arrives.  The kernel holds every
 *    multiprocessor of the device while it runs: one server per device is
 *    the intended use (a second server's kernel starts only after the
 *    first's has left, at the latest idle_ms after its last round).
 *  - A simulation that finishes within a round has its moments computed in
 *    the same round, after its last step; they are copied to host memory
 *    held by the server until lbm_server_poll returns them.  The service
 *    thread posts round i before it waits for round i - 1 and copies that
 *    round's results out (copies only, on a second stream, while the kernel
 *    runs round i), so the device does not wait for the host between
 *    rounds.
 *  - Each result equals, bit for bit, that of the same request run alone
 *    through the server: tiles of different simulations never interact and
 *    the per-site arithmetic has no data-dependent ordering.
 *
 * Conventions as in lbm.h (lattice units, site numbering, field layout,
 * status codes and lbm_last_error).  All host pointers passed in are owned by
 * the caller and copied before the call returns.  One server may be used
 * from several host threads.
 */
#ifndef LBM_SERVE_H
#define LBM_SERVE_H

#include <stddef.h>
#include <stdint.h>

#include "lbm.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    size_t hbm_budget;  /* bytes of device memory for resident simulations;
                           0: half of the device's free memory at creation */
    int max_active;     /* simulations advanced together; 0: 4096 */
    int device;         /* CUDA device ordinal, default 0 */
    double round_ms;    /* target duration of one round of K steps; 0: 2 ms */
    double idle_ms;     /* the persistent kernel leaves after this long without
                           a round to run (it is launched again when work
                           arrives); 0: 50 ms */
} lbm_server_opts;

typedef struct {
    int dim;            /* 1 (D1Q3) or 2 (D2Q9) */
    int nx, ny;         /* sites; ny = 1 for dim 1 */
    double tau, T0;     /* as in lbm_create; tau > 0, T0 > 0 */
    int thermal;        /* as lbm_opts.thermal */
    lbm_bc bc;          /* LBM_BC_PERIODIC or LBM_BC_FIXED_STATE (x) */
    long steps;         /* >= 0 */
    const double *rho;  /* initial fields, host, layout of lbm_fields_in */
    const double *u;
    const double *T;
} lbm_request;

typedef struct {
    uint64_t submitted, completed;  /* requests so far */
    int active, queued;             /* now */
    double site_updates;            /* sum over completed requests of sites x steps */
    double busy_s;                  /* device time of the rounds (kernel clock) */
    uint64_t rounds;                /* rounds completed so far */
    double first_submit_s, last_done_s;  /* host clock (seconds since server creation) */
    size_t pool_bytes, pool_in_use;
    uint64_t kernel_launches;       /* launches of the persistent kernel so far */
} lbm_server_stats;

typedef struct lbm_server lbm_server;

void lbm_server_default_opts(lbm_server_opts *opts);

/* Create a server on opts->device: allocates the device pool, starts the
 * service thread.  opts may be NULL (defaults). */
lbm_status lbm_server_create(const lbm_server_opts *opts, lbm_server **out);

/* Queue one request; *ticket identifies it.  LBM_EINVAL for invalid
 * parameters; LBM_ENOMEM if the request alone can never fit the pool. */
lbm_status lbm_server_submit(lbm_server *srv, const lbm_request *req, uint64_t *ticket);

/* Result of a request: LBM_EBUSY while it is queued or running; LBM_OK once
 * done, after copying rho (N), u (dim x N) and T (N) into `out` (any pointer
 * may be NULL) and *latency_s (submit to completion; may be NULL).  The
 * ticket is released by the first LBM_OK (or LBM_EUNSTABLE: the simulation
 * became non-physical; its fields are still copied).  LBM_EINVAL for an
 * unknown ticket. */
lbm_status lbm_server_poll(lbm_server *srv, uint64_t ticket, lbm_fields_out *out, double *latency_s);

/* Block until the request is done or timeout_s passes (LBM_EBUSY), then as
 * lbm_server_poll. */
lbm_status lbm_server_wait(lbm_server *srv, uint64_t ticket, double timeout_s, lbm_fields_out *out,
                           double *latency_s);

lbm_status lbm_server_stats_get(lbm_server *srv, lbm_server_stats *out);

/* Stop the service thread (unfinished requests are dropped) and free all
 * device memory of the server. */
void lbm_server_destroy(lbm_server *srv);

#ifdef __cplusplus
}
#endif

#endif /* LBM_SERVE_H */
