/*
 * sph.h -- C ABI of the GB300 (sm_103a) SPH hot-path library, libsph_gb300.so.
 *
 * The library computes the data-parallel hot path of SWIFT (arXiv 1807.01341):
 * cell-based SPH neighbour interactions -- the density loop with the
 * smoothing-length iteration, then the hydro force loop -- restricted to the
 * particles that are active in the current power-of-two time bin, inside a
 * kick-drift-kick integrator with individual time steps (Sec. II-A, Eq. 2),
 * drifting only the particles of the cells that can interact with an active
 * particle (Sec. III-D).
 *
 * Conventions for every call:
 *   - Every pointer inside sph_particles is a DEVICE pointer to an array of
 *     length n, owned by the caller.  sph_build_cells reorders all of them in
 *     place into cell order; every later call works on that order.
 *   - Every call is asynchronous on `stream` (a cudaStream_t passed as void*;
 *     NULL = the legacy default stream) unless it says otherwise.
 *   - Return value: SPH_OK (0) or an SPH_ERR_* code.  Argument and CUDA errors
 *     are returned directly.  Errors that arise on the device (h that does not
 *     converge, a cell that became too small, a time step below dt_min, a
 *     bounded wait that timed out) are recorded in a device status word that
 *     sph_get_status reads; the device never traps.
 *   - Once a device error that invalidates the step (SPH_ERR_CELL_OVERFLOW)
 *     is recorded, the remaining kernels of the step return without writing;
 *     sph_step recovers by rebuilding the cells and redoing the step.
 *   - The library owns all scratch memory (sorting, cells, leaves, records,
 *     queues); it is allocated by sph_create and sph_build_cells.
 */
#ifndef SPH_GB300_H
#define SPH_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum sph_status_code {
  SPH_OK = 0,
  SPH_ERR_ARG = 1,           /* invalid argument or call order */
  SPH_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  SPH_ERR_H_NOCONV = 3,      /* smoothing length did not converge in h_max_iter */
  SPH_ERR_CELL_OVERFLOW = 4, /* a kernel support outgrew the cell width: rebuild */
  SPH_ERR_DT_TOO_SMALL = 5,  /* a CFL time step fell below dt_min (put on bin 0) */
  SPH_ERR_TIMEOUT = 6,       /* a bounded device wait gave up */
  SPH_ERR_NOMEM = 7,         /* device allocation failed */
  SPH_ERR_NOT_BUILT = 8,     /* sph_build_cells has not been called */
  SPH_ERR_BOUNDS = 9         /* a device bounds check failed (library built with
                                SPH_CHECKS only; see sph_get_check_report) */
};

/* Sites of the device bounds checks.  A library compiled with -DSPH_CHECKS
 * (libsph_gb300_checks.so) tests, before every access through an index that
 * a kernel reads from device data written by another kernel (queues, cell,
 * chunk, leaf and work-group ranges, the permutation of a cell build), that
 * the index lies inside its array.  A failed check records SPH_ERR_BOUNDS in
 * the status word and the site, index and bound in the check report, skips
 * the access and halts the step (its remaining kernels return without
 * writing); it never traps.  The checks change no result; the normal library
 * has none of them. */
enum sph_check_site {
  SPH_CHECK_NONE = 0,
  SPH_CHECK_GROUP = 1,           /* work group taken from a queue, against the group count */
  SPH_CHECK_GROUP_LEAVES = 2,    /* a work group's last leaf, against the leaf count */
  SPH_CHECK_GROUP_SIZE = 3,      /* a work group's particle count, against the room for its
                                    active particles in shared memory */
  SPH_CHECK_CELL_LEAVES = 4,     /* a neighbour cell's last leaf, against the leaf count */
  SPH_CHECK_LEAF = 5,            /* a leaf's last particle, against the particle count */
  SPH_CHECK_PARTICLE_LEAF = 6,   /* a particle's leaf, against the leaf count */
  SPH_CHECK_DRIFT_CHUNK = 7,     /* chunk taken from the drift queue, against the chunk count */
  SPH_CHECK_ACTIVE_LEAF = 8,     /* leaf taken from the active-leaf queue, against the leaf count */
  SPH_CHECK_SCATTER = 9,         /* destination of the cell build's permutation, against n */
  SPH_CHECK_WAKE = 10            /* particle taken from the limiter's wake queue, against n */
};

/* Parameters.  Defaults (sph_default_params): eta 1.2348, gamma 5/3,
 * alpha_visc 0.8, cfl 0.1, h_tol 1e-6, h_max_iter 30, bin_cap 20,
 * dt_min 1e-6, t_begin 0, box 1, cell_margin 2.0, leaf_max 8,
 * threads_per_particle 1, drift_all 0, n_cells_override 0, heavy_factor 2,
 * coop_max_groups -1, list_cap 512, search_margin 1.02, staging_depth 1,
 * wait_limit 0, test_stall 0, balsara 0, predict_inactive 0, limiter 0.
 * With threads_per_particle = 1 every sum of a particle is taken in an order
 * that depends on the particle alone, so SPH_FORM_PLAIN and SPH_FORM_BATCHED
 * give bit-identical results; with more lanes per particle they agree to
 * rounding. */
typedef struct {
  double box;        /* side of the periodic cube */
  double eta;        /* resolution: h solves h^3 n(h) = eta^3, n = sum_j W(r_ij, h) */
  double gamma;      /* adiabatic index of the density-entropy equation of state */
  double alpha_visc; /* artificial viscosity strength (signal-velocity form, beta = 3) */
  double cfl;        /* C of Eq. 1: dt_i = C h_i / v_sig,i */
  double h_tol;      /* convergence of the h iteration: |dh| / h < h_tol, tested in FP64 */
  int h_max_iter;    /* iterations before SPH_ERR_H_NOCONV */
  int bin_cap;       /* largest time bin (0 = one global step); at most 62 */
  double dt_min;     /* t_min of Eq. 2: one tick of the integer timeline */
  double t_begin;    /* time of tick 0 */
  double cell_margin;/* top-level cell width >= cell_margin * largest kernel support */
  int leaf_max;      /* most particles in one leaf (sub-cell) of the cell tree, 1..32 */
  int threads_per_particle; /* lanes that share one active particle: 1, 2, 4, 8, 16 or 32 */
  int drift_all;     /* 0: drift only cells next to active cells (Sec. III-D); 1: drift all */
  int n_cells_override; /* > 0: use this many top-level cells per axis (must keep the
                           cell width >= the largest support) */
  double heavy_factor;  /* > 0: a work group whose estimated search cost exceeds
                           heavy_factor times the mean is started first (by the first
                           warps of a persistent launch, so that it does not end the
                           launch's tail); <= 0: no group is treated so */
  int coop_max_groups;  /* with one lane per particle: a step with at most this many
                           active work groups hands every one, in the force loop, to the
                           8 warps of a block (0: never; -1: twice the persistent grid's
                           block count).  The density loop takes every group one per warp. */
  int list_cap;         /* density loop: entries of each active particle's neighbour list
                           (squared distance and mass of every candidate within
                           search_margin x its support, kept across the h iterations;
                           a gather that finds more runs in passes of list_cap); 32..4096.
                           The library holds 8 x list_cap bytes per lane of every warp
                           of the persistent density grid for them (2 blocks of 8 warps
                           per SM: 319 MB at 512 on 152 SMs), whatever the particle count.
                           Results do not depend on it. */
  double search_margin; /* density loop: a particle's candidates are gathered within
                           search_margin x its support H, and gathered again only once
                           its H outgrows that radius; 1..2 (the first density pass of a
                           run, whose h comes from the initial conditions, uses at least
                           1.05).  Results do not depend on it. */
  int staging_depth;    /* pair loops: staging buffers per warp (1, 2 or 3); with d > 1
                           the bulk copies of the next d - 1 batches of neighbour records
                           are in flight while a batch is evaluated.  Results do not
                           depend on it. */
  int wait_limit;       /* polls of every bounded device wait (0: 2^22, about half a
                           second); a wait that gives up records SPH_ERR_TIMEOUT */
  int test_stall;       /* testing only, 0 in normal use: the first test_stall density
                           launches make one warp wait on a staging barrier that no copy
                           completes, so that the wait gives up after wait_limit polls and
                           the step stops with SPH_ERR_TIMEOUT */
  int test_bad_group;   /* testing only, 0 in normal use; accepted only by a library built
                           with SPH_CHECKS (SPH_ERR_ARG otherwise): the first test_bad_group
                           density launches replace the first work group they take from
                           the queue by an index past the last group, which the
                           SPH_CHECK_GROUP check catches before any use (SPH_ERR_BOUNDS) */
  /* Variants of the scheme, as Gadget-2 (the paper's reference code) has them;
   * 0 = off (the base scheme), 1 = on.  They need threads_per_particle 1 and,
   * when balsara or predict_inactive is on, the div_v and curl_v arrays of
   * sph_particles; sph_step_bwd supports none of them (SPH_ERR_ARG). */
  int balsara;          /* viscosity of a pair scaled by the mean of the particles'
                           Balsara factors |div v| / (|div v| + |curl v| + 1e-4 c / h) */
  int predict_inactive; /* an inactive particle's density and smoothing length are
                           predicted from its last density with its velocity divergence:
                           rho exp(-div v dt), h exp(div v dt / 3), dt the time since its
                           last density; an active one starts its h iteration there */
  int limiter;          /* Saitoh & Makino (2009): a new time bin is at most 2 above the
                           smallest bin among the particle's force neighbours (dt <= 4
                           min_j dt_j), and an inactive force neighbour whose bin is more
                           than 2 above an active particle's is woken at the step's close:
                           its step is cut to end at the first multiple of 2^(bin_i + 2)
                           after the current tick, its bin becomes bin_i + 2 and its
                           opening half-kick is cut to the shorter step (as Durier & Dalla
                           Vecchia 2012 describe it; sph_counters.wakes counts them) */
} sph_params;

/* Particle state, structure of arrays, all device pointers of length n.
 * Between kicks v and A hold the half-step values of the kick-drift-kick
 * scheme; a, Adot are the rates from the last force evaluation of each
 * particle; h, rho, f, P, c, vsig are from its last density/force pass.
 * The integer timeline: a particle on bin b has a step of 2^b ticks,
 * [ti_begin, ti_end), and ti_drift is the tick its position refers to. */
typedef struct {
  int64_t n;
  double *x, *y, *z;    /* positions, wrapped into [0, box) by sph_build_cells */
  float *vx, *vy, *vz;  /* velocities */
  float *ax, *ay, *az;  /* accelerations */
  float *A, *Adot;      /* entropic function A = P / rho^gamma and its rate */
  float *h;             /* smoothing length (in: initial guess; out: solution) */
  float *rho, *f, *P, *c, *vsig; /* density, grad-h factor, pressure, sound speed, signal velocity */
  float *m;             /* masses */
  int8_t *bin;          /* time bin */
  int64_t *ti_begin, *ti_end, *ti_drift;
  uint8_t *active;      /* out: 1 for the particles active at the current tick */
  int32_t *ngb_density; /* optional (may be NULL): neighbours j != i with r < H_i */
  int32_t *ngb_force;   /* optional (may be NULL): neighbours j != i with r < max(H_i, H_j) */
  float *div_v, *curl_v;/* velocity divergence and |curl| at each particle's last density
                           (div v = -(1/rho) sum_j m_j v_ij . grad W(h_i), curl v =
                           (1/rho) sum_j m_j v_ij x grad W(h_i)); needed (else may be
                           NULL) with the balsara or predict_inactive variant */
} sph_particles;

typedef struct sph_ctx sph_ctx;

/* Counters accumulated on the device since sph_create or the last
 * sph_reset_counters (read by sph_get_counters, synchronising). */
typedef struct {
  int64_t pairs_density;   /* useful density pairs: i active, j != i, r_ij < H_i (final h) */
  int64_t pairs_force;     /* useful force pairs: i active, j != i, r_ij < max(H_i, H_j) */
  int64_t cand_density;    /* candidate pairs tested in the density loop: staged records x
                              unconverged particles of the round, all iterations */
  int64_t cand_force;      /* candidate pairs tested in the force loop (records x particles) */
  int64_t iters_density;   /* sum over active particles of h iterations */
  int64_t active_particles;/* sum over steps of the active particle count */
  int64_t steps;           /* completed sph_step / sph_step_graph steps */
  int64_t rebuilds;        /* sph_build_cells calls */
  int64_t redone_steps;    /* steps redone after a cell overflow */
  int64_t kernel_launches; /* kernels this process launched through the library so far
                              (graph replays count their kernel nodes) */
  int64_t gathers_density; /* density loop: particle gathers (a particle counted once in
                              every staging pass over its candidates) */
  int64_t list_overflows;  /* density loop: gathers whose neighbour list filled up (the
                              gather then ran further passes over the same leaves) */
  int64_t evals_density;   /* density loop: neighbour-list entries evaluated, all h
                              iterations (pair terms computed, in or beyond the support) */
  int64_t wakes;           /* limiter: inactive particles woken (their steps cut short
                              because an active neighbour's bin was more than 2 below) */
} sph_counters;

void sph_default_params(sph_params *p);

/* Create a context for up to n_max particles on the current CUDA device.
 * Allocates the library's scratch.  Errors: SPH_ERR_ARG, SPH_ERR_NOMEM. */
int sph_create(const sph_params *params, int64_t n_max, sph_ctx **ctx);
int sph_destroy(sph_ctx *ctx);

/* Top-level cells and leaves (Sec. III-A).  Wraps positions into the box,
 * chooses n_c = floor(box / (cell_margin * H_max)) (at least 3; H_max from the
 * current h) unless overridden, assigns each particle the cell
 * floor(x / w) per axis (w = box / n_c), sorts the particles stably by
 * (cell, 30-bit Morton code of the position inside the cell) -- ties keep
 * their previous order -- and permutes every array of `p` in place.  Each
 * cell is split into leaves: octree nodes of the Morton order holding at most
 * leaf_max particles.  Refreshes the FP32 cell-relative records every pair
 * loop reads, and finds whether every particle has the same mass (the density
 * loop then sums the kernel alone: rho = m sum w; masses are taken to stay
 * as they are until the next build).  Synchronises `stream` (to size the
 * grid and to check the input).  Errors: SPH_ERR_ARG (also when a position is not finite or an h
 * is not a positive finite number; nothing is reordered then),
 * SPH_ERR_CUDA. */
int sph_build_cells(sph_ctx *ctx, sph_particles *p, void *stream);

/* After sph_build_cells: permutation (device, int32, length n) with
 * perm[k] = index, in the order of the first sph_build_cells call, of the
 * particle now at position k.  Valid until the next sph_build_cells. */
const int32_t *sph_perm(const sph_ctx *ctx);
/* Number of top-level cells per axis and number of leaves of the last build. */
int sph_grid_info(const sph_ctx *ctx, int *n_cells_per_axis, int *n_leaves);

/* Active set at tick ti_current (Eq. 2): particle i is active when its step
 * ends there, i.e. when ti_current is a multiple of 2^bin_i (every particle is
 * active at tick 0).  ti_current < 0 uses the device-resident time (the tick
 * the last sph_timestep_bins computed as next).  Writes p->active, builds the
 * queue of leaves holding active particles and the list of cells within one
 * cell of an active cell (the particles that must be drifted, Sec. III-D). */
int sph_mark_active(sph_ctx *ctx, sph_particles *p, int64_t ti_current, void *stream);

enum sph_phase {
  SPH_DRIFT = 0,      /* drift to the current tick: positions of the relevant cells (all
                         cells when drift_all), predicted v and A, P and c of inactive
                         particles from their predicted entropy; refreshes records */
  SPH_KICK_CLOSE = 1, /* active particles: v += a dt_old / 2, A += Adot dt_old / 2 */
  SPH_KICK_OPEN = 2   /* active particles: v += a dt_new / 2, A += Adot dt_new / 2 */
};
/* One phase of the kick-drift-kick integrator (Sec. II-A) for the current
 * tick set by sph_mark_active. */
int sph_kick_drift(sph_ctx *ctx, sph_particles *p, int phase, void *stream);

enum { SPH_DENSITY_INIT_ENTROPY = 1 }; /* p->A holds u on input; set A from u and rho */
/* Density loop with the smoothing-length iteration ("ghost", Sec. III-B) for
 * the active particles: solves h^3 n(h) = eta^3 by a bracket-safeguarded
 * Halley iteration (each iteration one pass over the neighbour leaves), then
 * writes h, rho, f (grad-h factor), P and c (from the predicted entropy).
 * Cubic-spline kernel with support H = 1.825742 h.  FP32 pair arithmetic on
 * cell-relative coordinates, compensated accumulation, FP64 convergence test. */
int sph_density_active(sph_ctx *ctx, sph_particles *p, int flags, void *stream);

/* Hydro force loop for the active particles over j with r_ij < max(H_i, H_j):
 * writes a, Adot and vsig.  Pressure term with grad-h factors, Monaghan
 * signal-velocity viscosity Pi_ij (beta = 3, the form inside Eq. 1). */
int sph_force_active(sph_ctx *ctx, sph_particles *p, void *stream);

/* New time steps of the active particles: dt = C h / v_sig (Eq. 1), bin =
 * floor(log2(dt / dt_min)) capped at bin_cap (Eq. 2), increases accepted only
 * while the current tick is a multiple of the new step; sets ti_begin, ti_end
 * and the device-resident next tick (the earliest ti_end of all particles),
 * which is also written to *ti_next_dev when not NULL (device pointer). */
int sph_timestep_bins(sph_ctx *ctx, sph_particles *p, int64_t *ti_next_dev, void *stream);

enum sph_form {
  SPH_FORM_PLAIN = 0,   /* per time bin: one launch of each pair loop per active bin, grids
                           sized on the host after reading the queue lengths */
  SPH_FORM_BATCHED = 1, /* all active leaves of all bins in one persistent launch per loop,
                           the whole step replayed from one captured CUDA graph, no host
                           synchronisation inside the step */
  SPH_FORM_BATCHED_NOGRAPH = 2 /* the batched launches issued one by one (ablation) */
};

/* Start a new run on this context: tick 0, the next step sets the entropy
 * from u (p->A holds u), counters and status cleared.  Synchronising. */
int sph_begin_run(sph_ctx *ctx, void *stream);

/* Enqueue one full kick-drift-kick step at the device-resident current tick:
 * mark, drift, density, force, closing kick, bins, opening kick, advance to
 * the next tick.  Builds the cells first if needed.  The first step of a run
 * (tick 0) sets the entropy from u.  SPH_FORM_BATCHED replays a CUDA graph
 * captured on first use (p must keep the same pointers; it is recaptured when
 * they or the library's buffers change).  When drift or h growth has made the
 * cells too small, the step leaves the state as it was (its kernels return
 * without writing) and records SPH_ERR_CELL_OVERFLOW; sph_step_sync repairs
 * that.  SPH_FORM_PLAIN synchronises `stream` inside the step. */
int sph_step_async(sph_ctx *ctx, sph_particles *p, int form, void *stream);

/* Wait for the enqueued steps; *completed (may be NULL) = the number of them
 * that completed.  If one stopped on a cell overflow, the cells are rebuilt
 * (wider when h outgrew them) and the status cleared, so the caller enqueues
 * the missing steps again. */
int sph_step_sync(sph_ctx *ctx, sph_particles *p, int *completed, void *stream);

/* One step, repeated after a rebuild until it completes (async + sync). */
int sph_step(sph_ctx *ctx, sph_particles *p, int form, void *stream);

/* n_steps steps of SPH_FORM_BATCHED enqueued back to back, one
 * synchronisation at the end (plus one per recovery). */
int sph_step_graph(sph_ctx *ctx, sph_particles *p, int n_steps, void *stream);

/* Diagnostics (FP64): the state's total energy and momentum at tick ti
 * (ti < 0: the current tick), with each particle's velocity and entropy
 * predicted from its half-step state, v = v_half + a (t - t_mid) and
 * A + Adot (t - t_mid) (the KDK state of Sec. II-A), and its internal energy
 * u = A rho^(gamma-1) / (gamma-1) from its last density.  At a tick where
 * every particle's step ends this is the synchronised energy.  out (host,
 * 8 doubles): kinetic energy, thermal energy, momentum x, y, z, mass, the
 * number of particles without a density (rho <= 0, no thermal term), 0.
 * Summed in a fixed order (reproducible).  Synchronising.
 * Errors: SPH_ERR_ARG, SPH_ERR_CUDA. */
int sph_diagnostics(sph_ctx *ctx, const sph_particles *p, int64_t ti, double *out, void *stream);

/* Current and next tick of the device-resident timeline (synchronising). */
int sph_get_time(sph_ctx *ctx, int64_t *ti_current, int64_t *ti_next);
/* Set the device-resident current tick (asynchronous). */
int sph_set_time(sph_ctx *ctx, int64_t ti_current, void *stream);

/* Device status word (synchronising): *status = the first SPH_ERR_* recorded
 * on the device since the last sph_clear_status (SPH_OK if none), *detail = the
 * number of particles it concerned.  Either pointer may be NULL. */
int sph_get_status(sph_ctx *ctx, int *status, int64_t *detail);
int sph_clear_status(sph_ctx *ctx, void *stream);
/* 1 if this library was compiled with the device bounds checks (SPH_CHECKS),
 * 0 otherwise. */
int sph_built_with_checks(void);
/* The first failed device bounds check since the last sph_clear_status
 * (synchronising): *site = an sph_check_site (SPH_CHECK_NONE if none failed, and
 * always in a library built without checks), *index = the index that failed,
 * *bound = the size of the array it indexed.  Any pointer may be NULL.
 * Errors: SPH_ERR_ARG, SPH_ERR_CUDA. */
int sph_get_check_report(sph_ctx *ctx, int *site, int64_t *index, int64_t *bound);
int sph_get_counters(sph_ctx *ctx, sph_counters *out);
int sph_reset_counters(sph_ctx *ctx, void *stream);
/* Occupancy of the time bins (Eq. 2): counts[b] = the number of particles on
 * bin b, b < n_bins (at most 64), as of the last step or cell build (the
 * histogram of Fig. 1).  Synchronising: waits for the work queued on stream.
 * Errors: SPH_ERR_ARG, SPH_ERR_CUDA. */
int sph_get_bin_counts(sph_ctx *ctx, int64_t *counts, int n_bins, void *stream);

/* Device time of the pair-loop launches, measured with CUDA events recorded
 * on the launching stream around every density and force launch (inside the
 * captured graph for SPH_FORM_BATCHED).  Off by default; enabling it changes
 * no result.  Times accumulate until sph_reset_kernel_times; reading them
 * synchronises the device. */
typedef struct {
  double density_ms, force_ms;
  int64_t density_launches, force_launches;
} sph_kernel_times;
int sph_set_profiling(sph_ctx *ctx, int enable);
int sph_get_kernel_times(sph_ctx *ctx, sph_kernel_times *out);
int sph_reset_kernel_times(sph_ctx *ctx);

/* Allocation-free cell ordering, for callers that must not allocate device
 * memory: a host program that has handed all of the device's memory to its
 * own pool or runs under a fixed memory budget, or a latency-critical loop in
 * which cudaMalloc (and the device synchronisation it can imply) is not
 * allowed.  The paper has no counterpart; this is a variant of the ordering
 * step of sph_build_cells.
 * Writes to perm (device, int32, length n, caller-allocated) the stable order
 * of the n particles by (cell, Morton code inside the cell) in an
 * n_cells_per_axis^3 grid of the periodic box of side `box` -- exactly the
 * order sph_build_cells produces for that grid from the same positions.  x, y,
 * z (device, FP64) are read, not modified; they must be finite (sph_build_cells
 * rejects a non-finite position; this call does not check, returns SPH_OK and
 * leaves the order of such input unspecified).  No allocation: the sort buffers are
 * one 1.6 MB array in device memory that the library defines statically, held
 * by every GPU that loads the library until the process exits.
 * Limits and errors: n <= 65536 and 1 <= n_cells_per_axis <= 255, else
 * SPH_ERR_ARG before anything is launched; SPH_ERR_CUDA if a launch or copy
 * fails.  The first call on a device looks up the array's device address
 * (with that device current) and keeps it for the life of the process; make
 * that first call before any stream capture, and make no call on a device
 * after cudaDeviceReset there (the array goes with the context, and the kept
 * address with it).  Every call on a device uses the same array, so calls whose work
 * overlaps on the GPU (different streams, or host threads) race and must be
 * serialised by the caller; each call writes every part of the array it reads,
 * so a call needs nothing cleared from the last one.  Asynchronous on
 * `stream`. */
int sph_cell_order_noalloc(const double *x, const double *y, const double *z, int64_t n,
                           double box, int n_cells_per_axis, int32_t *perm, void *stream);

/* ---------------------------------------------------------------------------
 * Differentiation.  The paper has no adjoint: these calls give the gradient
 * of a loss on a later state of a run with respect to an earlier state (up to
 * the initial positions, velocities and internal energies), by running the
 * steps above (Sec. II-A integration, Eq. 1 and Eq. 2 bins, the Sec. III
 * density and force loops) backwards.  Time bins, active sets and which pairs
 * are neighbours are piecewise constant: the backward pass takes them from
 * the forward run.  Pair arithmetic is FP32 as in the forward loops; every
 * adjoint accumulator is FP64.
 * ------------------------------------------------------------------------- */

/* Adjoint of a particle state (caller-owned device arrays, FP64, length n, in
 * the same particle order as the states handed to sph_step_bwd): the
 * derivative of the loss with respect to each field of the state. */
typedef struct {
  int64_t n;
  double *x, *y, *z;    /* positions */
  double *vx, *vy, *vz; /* velocities (the half-step velocities of the state) */
  double *ax, *ay, *az; /* accelerations */
  double *A, *Adot;     /* entropic function and its rate; before the first step
                           of a run (where A holds u) A is d loss / d u */
  double *h, *rho, *f;  /* smoothing length, density, grad-h factor */
} sph_adjoint;

/* Copy every array of src into dst (both caller-owned, same n, asynchronous).
 * to_input_order = 0: plain copy.  to_input_order = 1: src is the state ctx
 * works on (sorted by its cell builds) and dst receives it in the order of
 * the first sph_build_cells call (dst[sph_perm[k]] = src[k]); src and dst must
 * not overlap.  NULL optional arrays (ngb_*) are skipped.  Used for checkpoints. */
int sph_state_copy(const sph_ctx *ctx, const sph_particles *src, sph_particles *dst,
                   int to_input_order, void *stream);

/* Continue a run from a state held in p: the arrays of p are taken as a new
 * input order (the next step rebuilds the cells and sph_perm restarts from the
 * identity), the current tick becomes ti_current, and first = 1 makes the
 * next step the initial one (p->A holds u), first = 0 a later one.  Clears
 * the status.  A run resumed from a state saved (in input order) before some
 * step, on a context with the same parameters, repeats that step and the
 * following ones bit for bit when the saved run also resumed there and
 * threads_per_particle is 1.  Synchronising. */
int sph_resume(sph_ctx *ctx, sph_particles *p, int64_t ti_current, int first, void *stream);

/* SPH density of a state sampled on the centres of an n_grid^3 grid of the
 * periodic box (point (a, b, c) at ((a, b, c) + 1/2) box / n_grid, index
 * a + n_grid (b + n_grid c)): rho_g = sum_j m_j W(|x_g - x_j|, h_j) with each
 * particle's own h, every particle taken at tick ti (x + v (ti - ti_drift)
 * dt_min).  rho_grid (device, FP64, n_grid^3) is overwritten.  Requires
 * GAMMA_K h < box / 2.  FP64 arithmetic.  Errors: SPH_ERR_ARG. */
int sph_grid_density(sph_ctx *ctx, const sph_particles *p, int n_grid, int64_t ti,
                     double *rho_grid, void *stream);
/* Its adjoint: given rho_grid_bar = d loss / d rho_g (device, FP64), adds
 * d loss / d x, d h and (through the drift to ti) d v to adj. */
int sph_grid_density_bwd(sph_ctx *ctx, const sph_particles *p, int n_grid, int64_t ti,
                         const double *rho_grid_bar, sph_adjoint *adj, void *stream);

/* One kick-drift-kick step backwards.  pre and post are the states before and
 * after a step of sph_step at tick ti (the step's current tick), both in one
 * particle order (e.g. saved with sph_state_copy(..., 1)); first = 1 for the
 * initial step of a run.  On entry adj holds d loss / d post; on return
 * d loss / d pre.  pre, post and adj are read-only apart from adj.  Uses a
 * second internal context of ctx (its own cells over internal copies), so ctx
 * may be the one that ran the forward steps.  Synchronising.  Errors:
 * SPH_ERR_ARG, SPH_ERR_NOMEM, SPH_ERR_CUDA, SPH_ERR_TIMEOUT (a bounded wait in
 * a pair kernel gave up). */
int sph_step_bwd(sph_ctx *ctx, const sph_particles *pre, const sph_particles *post, int64_t ti,
                 int first, sph_adjoint *adj, void *stream);

const char *sph_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* SPH_GB300_H */
