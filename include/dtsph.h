/*
 * dtsph.h - C ABI of the GB300 (sm_103a) library for the inner pseudo-time
 * iteration of the dual-time EDAC-SPH scheme with particles frozen in pseudo-time
 * (Ramachandran, Muta & Ramakrishna, arXiv:1904.00861, Algorithm 2), or moved in
 * pseudo-time (Algorithm 1, dtsph_params.moving).
 *
 * Conventions shared by every entry point:
 *  - Return value: DTSPH_OK (0) on success, a negative DTSPH_E_* code otherwise;
 *    dtsph_last_error() then holds a one-line message. A failed call leaves the
 *    context usable unless it returned DTSPH_E_CUDA.
 *  - Host arrays are owned by the caller and only read (inputs) or written
 *    (outputs) during the call. Particle arrays are row-major AoS in FP64:
 *    positions and velocities are n x dim, pressures n. Particle i of every
 *    output is particle i of the last dtsph_set_particles call (the library
 *    sorts particles internally and undoes the permutation on output).
 *  - *_device variants take device pointers (for example torch data_ptr());
 *    the caller keeps those buffers alive until the stream has consumed them.
 *  - All GPU work of a context is ordered on the stream passed to dtsph_create
 *    (NULL = the legacy default stream). A context is not thread-safe.
 *  - Non-convergence of the pseudo-time loop is not an error: it is reported in
 *    dtsph_step_stats.reason, following the stop rules of Sec. 3.4.
 *  - Two environment variables serve tests of the failure paths and are unset
 *    in normal use; both are read when a context allocates its particle state.
 *    DTSPH_TEST_ALLOC_LIMIT (bytes): device allocations of the context beyond
 *    it fail with DTSPH_E_OOM. DTSPH_TEST_BARRIER_WAIT_NS: give-up time of the
 *    persistent loop's grid barrier (default one second); a step whose barrier
 *    gave up is reported by dtsph_sync as DTSPH_E_TIMEOUT.
 *  - DTSPH_TUNE_CACHE (a file name, optional): the autotuner's choices persist
 *    there across processes, keyed by device, dim, precision, slots, instances
 *    and loop driver; a shape found in the file is not timed again.
 */
#ifndef DTSPH_H
#define DTSPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DTSPH_VERSION "0.1.0"

enum {
    DTSPH_OK = 0,
    DTSPH_E_ARG = -1,         /* invalid argument (null pointer, size, parameter) */
    DTSPH_E_STATE = -2,       /* call out of order, e.g. dtsph_step before dtsph_set_particles */
    DTSPH_E_CUDA = -3,        /* a CUDA runtime call failed */
    DTSPH_E_OOM = -4,         /* a device allocation failed */
    DTSPH_E_CAPACITY = -5,    /* a particle had more than max_neighbors neighbours */
    DTSPH_E_DOMAIN = -6,      /* a particle left the box of a non-periodic axis */
    DTSPH_E_UNSUPPORTED = -7, /* parameter combination not implemented on the GPU */
    DTSPH_E_TIMEOUT = -8,     /* a device-side wait gave up (persistent loop barrier) */
    DTSPH_E_SKIN = -9         /* moving = 2: a particle moved farther than skin/2 from r^0 in
                                 pseudo-time, so the lists may miss a neighbour */
};

typedef enum {
    DTSPH_FP64 = 0,   /* every floating-point operation in IEEE double */
    DTSPH_FP32C = 1   /* pair sums in FP32 with Kahan compensation; positions, the
                         real-time BDF2 source term, the velocity iterate and the
                         residual reduction in FP64 */
} dtsph_precision;

/* Parameters of one simulation (Sec. 3.4 and the test cases of Sec. 4). Derived values:
 * c = beta * v_ref, nu_e = h c / 16 (Eq. nu_edac), dtau = dt / beta. */
typedef struct {
    int32_t dim;              /* 2 or 3 */
    int32_t precision;        /* dtsph_precision */
    int32_t periodic[3];      /* 1 = periodic axis; a periodic axis needs hi - lo >= 9h */
    int32_t pad0;
    double lo[3], hi[3];      /* domain box; on a periodic axis positions are kept in
                                 [lo, hi) (input positions outside it are brought in by
                                 whole box lengths); on the other axes every particle
                                 must stay inside */
    double h;                 /* smoothing length; the quintic kernel has support 3h */
    double m;                 /* particle mass (uniform) */
    double rho0;              /* density, held fixed (Sec. 3) */
    double beta;              /* artificial-compressibility factor, c = beta * v_ref */
    double v_ref;             /* reference speed of Eq. (conv) */
    double nu;                /* kinematic viscosity */
    double dt;                /* real time step */
    double eta;               /* regulariser of r^2 + eta h^2 (0.01) */
    double alpha;             /* Monaghan artificial viscosity (0 = off) */
    double g[3];              /* body force */
    double eps;               /* tolerance of Eq. (conv) */
    double stag_tol;          /* stagnation threshold (0.05) */
    int32_t stag_window;      /* stagnation window in iterations (4; 0 = off) */
    int32_t max_iter;         /* iteration cap (1000) */
    int32_t edac;             /* 1: EDAC pressure diffusion on (Eq. dp-dtau-frozen-edac) */
    int32_t edac_h2_literal;  /* 1: EDAC denominator r^2 + h^2 as printed; 0: r^2 + eta h^2 */
    int32_t fixed_iters;      /* > 0: run exactly this many iterations per step, no stop rules */
    int32_t max_neighbors;    /* neighbour capacity per particle (0 = derived from h and m) */
    int32_t graph;            /* how the pseudo-time loop is driven. 1: each real step is a
                                 CUDA graph whose loop is a conditional while node (one
                                 launch per iteration); 2: each real step is a CUDA graph whose
                                 loop is one persistent cooperative kernel (grid barrier per
                                 iteration); 0: plain launches, host polls every 8 iterations */
    int32_t lanes;            /* lanes per particle in the pseudo-iteration kernel: 1, 2, 4
                                 or 8; 0 = picked by the built-in autotuner when the particles
                                 are first set (timed candidates, cached per shape in the
                                 process). With moving != 0, the lanes of the moving pass; 0 =
                                 one on FP32C, up to four on FP64 (no tuning) */
    int32_t stages;           /* staging depth of the one-lane kernel (lanes = 1): pair-cache
                                 chunks in flight per warp in shared memory, 2..8; 0 = 3, or
                                 picked by the autotuner together with lanes */
    int32_t shifting;         /* 1: particle shifting after every real step (Sec. 3.5, Eqs.
                                 shift-deltar, shift-correct): at the new positions,
                                 dr_i = -(h^2/2) sum_j V_j (1 + W_ij / W(h)) gradW_ij over every
                                 neighbour (wall particles included), then p_i += gradp_i . dr_i,
                                 V_i += (gradV_i) dr_i with grad f_i = sum_j V_j (f_j - f_i)
                                 gradW_ij over fluid neighbours, r_i += dr_i;
                                 0 = off. Instances of a batch share it. */
    int32_t steady;           /* 1: steady-state mode (Sec. 2.3 "Steady state solutions", Eq.
                                 mom-steady): the particles never move; each dtsph_step runs one
                                 pseudo-time solve from the current state with no real-time
                                 (BDF2) term, the pressure rate of Eq. (dp-dtau-frozen) without
                                 the EDAC term, and the convection term V_i . sum_j (V_i m/rho0 +
                                 V_j m/rho0) gradW_ij in the momentum rate; dt only scales the
                                 residuals and sets dtau = dt / beta. Shifting must be off.
                                 Instances of a batch share it. */
    int32_t free_surface;     /* 1: free-surface run: the Adami wall pressure is kept >= 0
                                 (Sec. 3.2), and with shifting a fluid particle with
                                 div r_i = -sum_j V_j r_ij . gradW_ij < dim - 1/2 (fluid and wall
                                 neighbours; Lind et al.'s test, Sec. 3.5) is not shifted.
                                 Instances of a batch share it. */
    int32_t moving;           /* particles in pseudo-time. 0: fixed (Algorithm 2). 1 or 2:
                                 moved (Algorithm 1): r^{k+1/2} = r^k + dtau/2 V~^k
                                 (Eq. rkstar), rates at r^{k+1/2} with the advective terms
                                 V~_i . sum_j m (p_i + p_j)/rho0^2 gradW_ij in dp/dtau (Eq.
                                 dp-dtau) and sum_j m/rho0 (V_i + V_j) (V~_i . gradW_ij) in the
                                 momentum rate (Eq. discrete_ME), V~^{k+1} = dt dV/dtau
                                 (Eq. vtilde), r^{k+1} = r^{k+1/2} + dtau/2 V~^{k+1} (Eq. rkp1),
                                 V~^0 = 0; walls stay; r^{n+1} still from Eq. (r-update).
                                 1: over the neighbour lists of r^0; 2: neighbours updated at
                                 every pass (lists with the cutoff 3h + skin; a particle that
                                 moves farther than skin/2 from r^0 ends the step with
                                 DTSPH_E_SKIN). Not with steady. With graph = 2 the loop runs
                                 as in graph = 1. Instances of a batch share it. */
    int32_t form;             /* the pair terms of the pseudo-time loop. 1: from the pair-
                                 coefficient cache, written once per real step by a pass over
                                 the lists at r^0 (gradW_ij and F_ij per pair). 2: recomputed
                                 in every pseudo-iteration from the lists at r^0 with the same
                                 operations (no cache; the cheaper form when a step takes few
                                 iterations). Both forms give the same bits. 0 (default):
                                 chosen per real step on the device from the measured costs
                                 of both forms and the previous step's iteration count, a
                                 step without the cache switching to it after kstar
                                 iterations (graph = 2; the cache otherwise;
                                 dtsph_form_stats). Form 2 only without walls,
                                 particles fixed in pseudo-time (DTSPH_E_UNSUPPORTED
                                 otherwise). Instances of a batch share it. */
    double skin;              /* list skin for moving = 2 (a length > 0; the lists then hold
                                 every pair within 3h + skin, dtsph_get_neighbors included);
                                 ignored otherwise. Instances of a batch share it. */
    double cell_scale;        /* side of the binning cells in list cutoffs (3h, + skin): 0 or
                                 1 (default) the smallest cells the 3^dim stencil allows,
                                 up to 4 wider ones (more candidates per list; the lists
                                 hold the same sets, in another order, so the last bits of
                                 the sums can differ). Instances of a batch share it. */
    double list_skin;         /* > 0: the lists at r^0 of each step are built to 3h + list_skin
                                 and also serve the next step's pass at r^n (one list build,
                                 one binning per step instead of two; pairs beyond 3h add
                                 exact zeros, the kernel gradient vanishing there). When a
                                 particle's r^{n+1} lies farther than list_skin / 2 from its
                                 r^0, the next step bins and lists at r^n as without it (on
                                 the device, in the step graph); a new state of the same
                                 particles set between steps keeps the lists on the same
                                 terms. Only with the persistent
                                 loop (graph = 2), no walls, particles fixed in pseudo-time,
                                 no shifting and no steady mode (DTSPH_E_UNSUPPORTED
                                 otherwise). 0 (default): two builds per step. The instances
                                 of a batch all set it (each its own length) or none does. */
} dtsph_params;

typedef struct {
    int32_t iters;    /* pseudo-time iterations taken in this real step */
    int32_t reason;   /* 0 converged, 1 stagnated, 2 iteration cap, 3 non-finite residual,
                         4 fixed iteration count reached */
    double rp;        /* mean|dp/dtau| dt / (rho0 c^2) of the last iteration, Eq. (conv) */
    double rv;        /* mean|dt dV/dtau| / v_ref of the last iteration, Eq. (conv) */
    double vmax;      /* max |V^{n+1}| over the fluid particles at the end of the step
                         (before shifting): the decay diagnostic of the Taylor-Green
                         runs (Sec. 4.1) */
    int32_t form;     /* the pair terms the step's loop used (dtsph_params.form): 1 the pair
                         cache, 2 recomputed from the lists, 3 recomputed for floor(kstar)
                         iterations, then the cache built and used for the rest */
    int32_t pad;
} dtsph_step_stats;

enum {
    DTSPH_FIELD_POS = 0,      /* r^n, n x dim */
    DTSPH_FIELD_VEL = 1,      /* V^n, n x dim */
    DTSPH_FIELD_P = 2,        /* p^n, n */
    DTSPH_FIELD_VEL_PREV = 3  /* V^{n-1}, n x dim */
};

typedef struct dtsph_ctx dtsph_ctx;

/* Creates a context on the current CUDA device. stream: a cudaStream_t, or NULL.
 * Allocates nothing on the device until dtsph_set_particles. */
int dtsph_create(const dtsph_params *params, void *stream, dtsph_ctx **out);

/* Frees every device buffer, graph and stream of the context (NULL is a no-op). */
void dtsph_destroy(dtsph_ctx *ctx);

/* Fluid state at real time t^n (Algorithm 2 starts from it): nf particles with
 * positions x (nf x dim), velocities V^n (nf x dim), pressures p^n (nf) and the
 * previous velocities V^{n-1} for the BDF2 term (NULL: V^{n-1} = V^n, as the
 * paper does without an exact solution, Sec. 3.1). Host pointers, each holding
 * its full size: on a device that reads pageable host memory itself
 * (cudaDevAttrPageableMemoryAccess, as Grace-based systems do over NVLink-C2C) a
 * kernel reads them in place, otherwise they are copied with cudaMemcpyAsync.
 * Allocates the device state (sized for nf plus the current walls); resets the
 * step counter. Must come after dtsph_set_boundary if there are walls. A
 * coordinate on a periodic axis outside [lo, hi) is brought into it by whole box
 * lengths (walls too); a non-finite position gives DTSPH_E_ARG (a non-finite
 * velocity or pressure is not an error here: the first step stops with reason 3). */
int dtsph_set_particles(dtsph_ctx *ctx, int64_t nf, const double *x, const double *v,
                        const double *p, const double *v_prev);

/* As dtsph_set_particles with device pointers; enqueued on the context stream
 * (a non-finite position is then reported by dtsph_sync as DTSPH_E_ARG). */
int dtsph_set_particles_device(dtsph_ctx *ctx, int64_t nf, const double *x, const double *v,
                               const double *p, const double *v_prev);

/* Fixed solid-wall particles (Sec. 3.2, Adami et al. 2012): nw positions
 * (nw x dim) and prescribed velocities (nw x dim, NULL = at rest). Their
 * pressure and ghost velocity are extrapolated from the fluid in every
 * pseudo-iteration. Host pointers. Call before dtsph_set_particles. */
int dtsph_set_boundary(dtsph_ctx *ctx, int64_t nw, const double *x, const double *v_wall);

/* Enqueues nsteps real steps of Algorithm 2 (neighbour rebuild, state-n rates
 * and predictor Eqs. v0/r0, pseudo-time loop Eqs. pkstar_frozen..pkp1_frozen
 * with Eq. dv_dtau_exact until Eq. conv or a stop rule holds, Eq. r-update).
 * Asynchronous: returns once the work is enqueued. Per-step statistics go to a
 * device log read by dtsph_read_stats. With list_skin > 0, the first call after
 * the particle set's binning or lists were rebuilt otherwise (a new particle set,
 * dtsph_eval_rates, dtsph_build_neighbors) first bins and lists at r^n. */
int dtsph_step(dtsph_ctx *ctx, int32_t nsteps);

/* Batches: one context advancing ninst independent simulations together (each
 * with its own particles, parameters, walls and pseudo-time loop; they share dim,
 * precision, graph and lanes). Every step runs all instances in the same
 * launches; an instance whose loop has stopped skips the remaining iterations.
 * Results of an instance are bit-identical to running it alone. Fields read back
 * concatenate the instances' fluid particles in instance order.
 * dtsph_batch_create: params points to ninst parameter sets (1 <= ninst <= 65535). */
int dtsph_batch_create(int32_t ninst, const dtsph_params *params, void *stream, dtsph_ctx **out);

/* Walls of instance inst (as dtsph_set_boundary). Call before dtsph_batch_set_particles. */
int dtsph_batch_set_boundary(dtsph_ctx *ctx, int32_t inst, int64_t nw, const double *x, const double *v_wall);

/* Fluid state of every instance: nf[i] particles for instance i; x, v, p and
 * v_prev (NULL: = v) hold the instances one after the other (host arrays). */
int dtsph_batch_set_particles(dtsph_ctx *ctx, const int64_t *nf, const double *x, const double *v,
                              const double *p, const double *v_prev);

/* dtsph_read_stats for instance inst. */
int dtsph_batch_read_stats(dtsph_ctx *ctx, int32_t inst, int64_t first, int32_t count, dtsph_step_stats *out);

/* Waits for the stream, then reports a device-side error of the work enqueued
 * so far (DTSPH_E_ARG for a non-finite input position, DTSPH_E_CAPACITY,
 * DTSPH_E_DOMAIN, DTSPH_E_TIMEOUT, DTSPH_E_SKIN) or DTSPH_OK. */
int dtsph_sync(dtsph_ctx *ctx);

/* Number of real steps taken since dtsph_set_particles (host-side count). */
int64_t dtsph_step_count(const dtsph_ctx *ctx);

/* Copies the statistics of steps first .. first+count-1 (0-based since
 * dtsph_set_particles) to out. Waits for the stream. Only the last 65536 steps
 * are kept. */
int dtsph_read_stats(dtsph_ctx *ctx, int64_t first, int32_t count, dtsph_step_stats *out);

/* Copies one field of the fluid particles (DTSPH_FIELD_*) into the host array
 * out (nf x comps doubles), in the caller's particle order: on a device that
 * writes pageable host memory itself a kernel writes out in place, otherwise
 * cudaMemcpyAsync does. Waits for the stream. */
int dtsph_read_field(dtsph_ctx *ctx, int32_t field, double *out);

/* The whole fluid state in the caller's particle order into host arrays: r^n and
 * V^n (nf x dim), p^n (nf), V^{n-1} (nf x dim); a null pointer skips that field.
 * One call instead of four dtsph_read_field calls: the fields go through one
 * device scratch buffer and the call waits for the stream once. Host arrays are
 * written as by dtsph_read_field. */
int dtsph_read_state(dtsph_ctx *ctx, double *x, double *v, double *p, double *v_prev);

/* As dtsph_read_field into device memory; enqueued on the context stream. */
int dtsph_read_field_device(dtsph_ctx *ctx, int32_t field, double *out);

/* Test entry: the two rates of Eqs. (dp-dtau-frozen-edac, mom-sph-frozen) at
 * the current state (positions r^n, V^n, p^n; walls extrapolated first), for
 * every fluid particle in caller order: ap (nf) and F (nf x dim), host arrays.
 * Does not change the state. Waits for the stream. */
int dtsph_eval_rates(dtsph_ctx *ctx, double *ap, double *F);

/* Test entry: builds the neighbour lists N(i) = {j != i : |r_i - r_j| < 3h} at the
 * current positions (all particles, walls after fluid in the numbering) and
 * keeps them until the next call. */
int dtsph_build_neighbors(dtsph_ctx *ctx);

/* Test entry: after dtsph_build_neighbors, writes the neighbours of particle i
 * (0..nf+nw-1, caller numbering, ascending) to out (capacity cap) and their
 * number to *count (which may exceed cap; out then holds the first cap). */
int dtsph_get_neighbors(dtsph_ctx *ctx, int64_t i, int64_t *out, int64_t cap, int64_t *count);

/* Measurement entry: after at least one dtsph_step, re-runs the pseudo-time
 * iteration kernel of the last step `launches` times (1..256) on its frozen pair
 * cache (with moving != 0: the moving pass, wall kernel included, on the lists
 * of the last step), each launch bracketed by CUDA events on the context stream, and
 * returns the mean launch duration in milliseconds, the algorithmic bytes one
 * launch must move (particle state read and written once, every cached pair
 * read once; the layout is described in the design notes) and the number of
 * cached fluid pairs. With shifting on, the shifting pass has replaced the
 * step's lists by its own, so the kernel runs on a pair cache built for the
 * current positions instead (DTSPH_E_STATE with moving != 0). The state r^n,
 * V^n, p^n is not changed. Waits for the stream. */
int dtsph_probe_iterate(dtsph_ctx *ctx, int32_t launches, float *ms_per_launch, double *bytes_per_launch,
                        int64_t *pairs);

/* Device time (ms) of the pseudo-time loop of real steps first .. first+count-1
 * (steps are numbered from 0 since dtsph_set_particles; each must be among the
 * last 256 taken), from CUDA events recorded just before and after the loop of
 * every step: event nodes of the step graph (graph = 1, 2) or events on the
 * stream (graph = 0). Waits for those steps to finish. The paper has no
 * counterpart; it serves measurement (the loop's share of a step). */
int dtsph_loop_times(dtsph_ctx *ctx, int64_t first, int32_t count, float *ms);

/* Measurement entry: the vector FMA throughput of the current device in FLOP/s
 * (an FMA counts two), FP64 (precision = DTSPH_FP64) or FP32 (DTSPH_FP32C): every
 * SM runs eight 256-thread blocks of eight independent multiply-add chains per
 * thread, timed with CUDA events on a private stream, best of three launches of
 * about 50 ms each. Allocates and frees a few KB of device memory; waits for its
 * work. The paper has no counterpart; it is the compute ceiling of the roofline
 * for kernels bound by FP32 or FP64 arithmetic. */
int dtsph_fma_peak(int32_t precision, double *flop_per_s);

/* Autotuner report: the lanes per particle the iterate kernel uses, and (if
 * ms_by_lanes is not NULL, 4 floats) the best time measured for 1, 2, 4 and 8
 * lanes when this context tuned (per launch, or per loop iteration with
 * graph = 2; for one lane the best staging depth; -1 where it did not
 * measure, e.g. when the shape was already tuned in this process or lanes was
 * fixed). */
int dtsph_tuning(const dtsph_ctx *ctx, int32_t *lanes, float *ms_by_lanes);

/* Every candidate the autotuner timed when this context tuned, in the order
 * timed: lanes per particle, staging depth (0 for lanes > 1) and mean ms per
 * launch of the pseudo-iteration kernel (graph = 0, 1) or per iteration of the
 * persistent loop kernel over four fixed iterations (graph = 2). Writes min(cap, count) entries of
 * the three arrays (each may be NULL when cap is 0); *count = candidates timed
 * (0 when the shape's choice came from the process cache or lanes was fixed);
 * *stages = staging depth in use (0 when lanes > 1). */
int dtsph_tuning_candidates(const dtsph_ctx *ctx, int32_t cap, int32_t *lanes, int32_t *stages, float *ms,
                            int32_t *count, int32_t *stages_in_use);

/* Report of the pair-term form (dtsph_params.form). With form = 0, the
 * persistent loop (one instance, or a batch's decoupled loop), no walls and
 * particles fixed in pseudo-time, the context measured at dtsph_set_particles
 * (or took from the process cache or the DTSPH_TUNE_CACHE file) the costs
 * ms[0] = one pair-cache pass, ms[1] = one pseudo-iteration with the cache,
 * ms[2] = one without it (milliseconds, at the lanes and staging depth in use),
 * and *kstar = ms[0] / (ms[2] - ms[1]) (1e9 when the uncached iteration is not
 * slower). The step graph then holds both forms and picks one per step on the
 * device, in stream order: without the cache when the previous step took at
 * most kstar iterations (in a batch: the instances' iteration counts averaged
 * with their fluid counts as weights; an instance with no finished step since
 * the particle set's allocation counts one), else with it. A loop without the
 * cache pauses after floor(kstar) iterations if no stop rule holds; the step
 * then builds the cache and goes on with it from that iteration (form 3 in
 * dtsph_step_stats), so a wrong guess costs about one cache pass. All forms
 * give the same bits. *kstar < 0 and ms[i] < 0 when nothing was measured.
 * *steps_cache, *steps_nocache and *steps_switched count the steps run in each
 * form since dtsph_set_particles (with form = 0 this waits for the context's
 * stream). Any pointer may be NULL. */
int dtsph_form_stats(const dtsph_ctx *ctx, double *kstar, float *ms, int64_t *steps_cache, int64_t *steps_nocache,
                     int64_t *steps_switched);

/* Allocation-free rate evaluation, for callers that cannot allocate device
 * memory when they need the rates: code running while a stream capture it does
 * not own is open, solvers that reserved their whole device budget up front, and
 * code called where a synchronous allocation could stall the host thread. The
 * paper has no counterpart; it computes what dtsph_eval_rates computes (the two
 * rates of Eqs. dp-dtau-frozen-edac and mom-sph-frozen for every fluid particle,
 * walls extrapolated first, with the same reading of every parameter: steady,
 * free_surface, alpha, edac, moving's list cutoff) without a context and without
 * any device allocation.
 *   params     simulation parameters, checked as by dtsph_create
 *   nf, x, v, p   fluid positions (nf x dim), velocities (nf x dim), pressures (nf):
 *              device pointers, row-major AoS, FP64
 *   nw, xw, vw wall positions and prescribed velocities (device; vw may be NULL)
 *   ap, F      outputs, device: dp/dtau (nf) and the momentum right-hand side
 *              (nf x dim), in the caller's particle order
 *   status     optional device int32 (may be NULL): after the call's GPU work it
 *              holds DTSPH_OK, DTSPH_E_CAPACITY (a particle had more neighbours
 *              than the neighbour capacity; its list was cut there and its rates
 *              are wrong) or DTSPH_E_DOMAIN (a particle lay outside the box of a
 *              non-periodic axis)
 *   stream     cudaStream_t or NULL; it must belong to the current device. The
 *              call only enqueues work and returns.
 * All work happens in one fixed scratch array of about 30 MB that is part of the
 * library image and that every GPU using the library holds until the process
 * exits. Limits: nf + nw <= 16384 particles, at most 32768 cells of side 3h, and
 * at most 16384 x 192 neighbour-list entries (nf + nw rounded up to 256, times the
 * neighbour capacity: max_neighbors, or the one derived from h and m), else
 * DTSPH_E_CAPACITY and nothing is enqueued. The first call on a device looks
 * up the array's device address (once per device, with that device current): make
 * that first call before any stream capture. Every call reuses the same array, so
 * calls whose GPU work can overlap (different streams or threads) race and corrupt
 * each other; calls ordered on one stream are safe. Returns DTSPH_E_ARG for a
 * stream of another device. */
int dtsph_eval_rates_noalloc(const dtsph_params *params, int64_t nf, const double *x, const double *v,
                             const double *p, int64_t nw, const double *xw, const double *vw, double *ap,
                             double *F, int32_t *status, void *stream);

/* Kernel launches this context has made so far (counted on the host; a graph
 * launch counts the kernels it runs, pseudo-iterations included). */
int64_t dtsph_kernel_launches(const dtsph_ctx *ctx);

/* Message of the last failed call, or "" (never NULL; valid until the next call). */
const char *dtsph_last_error(const dtsph_ctx *ctx);

/* DTSPH_VERSION. */
const char *dtsph_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DTSPH_H */
