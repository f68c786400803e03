/*
 * symba.h -- C ABI of the GB300 SyMBA hot path (arXiv:2304.07325, SyMBAp).
 *
 * One call of symba_step advances a system of N bodies around a central mass m0 by SyMBA steps
 * (Duncan, Levison & Lee 1998) with the SyMBAp structure of the paper:
 *   - every interaction of the right-angled trapezoid i < N_m, j > i (Sec. 2, the nested loop),
 *     split into a rectangle plus a triangle folded into a rectangle (Sec. 2);
 *   - the close-encounter check, whose flagged pairs are grouped into independent groups that
 *     are integrated separately (Sec. 2, the encounter paragraph);
 *   - recursive sub-stepping with subdivision factor M, shell ratio R_k/R_{k+1} and the
 *     partition function f_l (Sec. 3, first paragraph: M = 4, 2.08, l = 3);
 *   - per-particle Kepler and sun drifts (Sec. 2, the simple loops).
 * All computation runs in CUDA kernels for sm_103a on the calling process's current device.
 *
 * Conventions shared by every entry point
 *   - Units are the caller's; the defaults are AU, yr, solar masses (G = 4 pi^2, m0 = 1).
 *   - Particle arrays are indexed 0..n-1, massive bodies first (indices < n_massive), field
 *     (massless) particles after.  Vectors are n x 3 row-major doubles: x0 y0 z0 x1 y1 z1 ...
 *   - A pointer argument may be host memory or device memory of the current device; the library
 *     detects which.  A pointer into another GPU's memory is rejected with SYMBA_E_INVAL.  The
 *     library copies what it needs and never keeps the caller's pointer.
 *   - The state the library keeps is democratic heliocentric: heliocentric positions and
 *     barycentric velocities.
 *   - Return values: SYMBA_OK (0), a negative SYMBA_E_* code, or SYMBA_COLLISION (positive,
 *     informational: at least one merger happened).  Errors detected on the device inside an
 *     asynchronous call are sticky and reported by the next synchronising call (symba_sync,
 *     symba_energy, symba_get_state, symba_enc_groups, symba_get_stats); the state is then
 *     undefined until symba_set_state.
 *   - No call uses hidden global state; separate contexts may be used from separate threads.
 */
#ifndef SYMBA_H
#define SYMBA_H

#ifdef __cplusplus
extern "C" {
#endif

#define SYMBA_OK 0
#define SYMBA_E_INVAL (-1)     /* bad argument */
#define SYMBA_E_NOMEM (-2)     /* device allocation failed, or a pool has no room */
#define SYMBA_E_CUDA (-3)      /* a CUDA runtime call failed */
#define SYMBA_E_KEPLER (-4)    /* Kepler's equation did not converge */
#define SYMBA_E_DEPTH (-5)     /* recursion deeper than max_depth, or sub-step budget exhausted */
#define SYMBA_E_CAPACITY (-6)  /* more level-0 encounter pairs than pair_capacity */
#define SYMBA_E_NONFINITE (-7) /* NaN or Inf in the state */
#define SYMBA_COLLISION 1      /* informational: bodies merged during the last steps */

#define SYMBA_PRECISION_FP64 0 /* every operation in FP64 */
#define SYMBA_PRECISION_MIXED 1 /* FP32 pair kick (Kahan into FP64); FP64 state, drifts, check, energy */

/* Method parameters (Sec. 3 gives dt, M, shell_ratio and l for the benchmark). */
typedef struct {
  double dt;           /* full step tau */
  double shell_ratio;  /* R_k / R_{k+1} (2.08) */
  double hill_scale;   /* lambda: level-0 critical radius lambda (rH_i + rH_j) (6.5) */
  double G;            /* gravitational constant (4 pi^2) */
  double m0;           /* central mass (1) */
  int M;               /* time-step subdivision factor (4) */
  int l;               /* order of the partition function f_l (3) */
  int max_depth;       /* deepest recursion level (20) */
  int precision;       /* SYMBA_PRECISION_FP64 or SYMBA_PRECISION_MIXED */
  int pair_capacity;   /* level-0 encounter pairs per step; 0 = max(4096, 4 n) */
  int max_substeps;    /* sub-step budget per group and step; 0 = 1 << 22 */
  double rmin;         /* removal (the paper names no rule; SWIFT-style discard): after the      */
  double rmax;         /* closing kick of a step, a live body with heliocentric distance below   */
                       /* rmin (it hit the star) or above rmax (ejected) leaves the system: its  */
                       /* mass and radii become 0 and it no longer takes part; 0 = no limit     */
} symba_params;

/* Per-step diagnostics of the last step (summed over a multi-step call where stated). */
typedef struct {
  int n_pairs;              /* level-0 encounter pairs of the last step */
  int n_groups;             /* encounter groups of the last step */
  int max_depth;            /* deepest level entered during the last call */
  int status;               /* sticky device status (SYMBA_OK or SYMBA_E_*) */
  long long merges;         /* mergers since the context was created */
  long long substeps;       /* recursion sub-steps (E_k calls, k >= 1) during the last call */
  long long steps;          /* steps taken since the context was created */
  long long max_chain;      /* most sub-steps of one group in one step during the last call: the
                               dependent chain that bounds the recursion's time */
  long long removals;       /* bodies removed by rmin / rmax since the context was created */
  long long pair_substeps;  /* of the sub-steps of the last call, those the single-pair path took
                               (a pair alone in F_{k-1}, its two bodies packed across the warp) */
} symba_stats;

typedef struct symba_ctx symba_ctx;
typedef struct symba_pool symba_pool;

/* Fills *p with the paper's benchmark parameters: dt 0.5, M 4, shell ratio 2.08, l 3,
 * lambda 6.5, G 4 pi^2, m0 1, max_depth 20, FP64.  Never fails. */
void symba_default_params(symba_params *p);

/* Creates a context for one system and uploads it (Sec. 2: N particles, the first N_m massive and
 * the rest massless field particles that interact only with massive ones; Sec. 3: the method's
 * parameters in *p).  The velocities are turned into the democratic-heliocentric state the
 * SyMBA step keeps (barycentric v = v_hel - sum m v_hel / (m0 + sum m)).
 * n, n_massive: particle counts (0 <= n_massive <= n, n >= 1).
 * x, v: n x 3 heliocentric positions and velocities; m, radius: n masses (0 for field particles)
 * and physical radii (contact detection); rhill: n Hill radii, or NULL to compute them as
 * a (m / 3 m0)^{1/3} from the osculating heliocentric orbit.
 * cuda_stream: a cudaStream_t every later call of this context is ordered on (NULL = a stream
 * the context creates).  Returns SYMBA_OK and *out, or SYMBA_E_INVAL / E_NOMEM / E_CUDA. */
int symba_init(symba_ctx **out, const symba_params *p, int n, int n_massive, const double *x,
               const double *v, const double *m, const double *radius, const double *rhill,
               void *cuda_stream);

/* Enqueues nsteps SyMBA steps E(tau) on the context's stream and returns without waiting
 * (Sec. 2: the trapezoid kick, the encounter check with grouping, the groups integrated
 * separately, the simple per-particle loops; Sec. 3: M, R_k/R_{k+1}, l).
 * Each step: sun drift tau/2; level-0 check fused into kick tau/2 over the trapezoid; grouping;
 * Kepler drift tau of bodies in no encounter and M-fold recursion of every group; kick tau/2;
 * removal by rmin / rmax (when set); sun drift tau/2.  Returns SYMBA_OK, SYMBA_E_INVAL (nsteps < 0) or SYMBA_E_CUDA. */
int symba_step(symba_ctx *c, int nsteps);

/* Waits for the context's stream; returns the sticky device status (or SYMBA_COLLISION if
 * bodies merged since the last synchronising call and no error happened). */
int symba_sync(symba_ctx *c);

/* Advances n independent contexts by nsteps steps each and waits for all of them.  The systems
 * are not stepped in lock-step: each context keeps exactly one step in flight on its own stream,
 * and its next step is launched as soon as the last one has completed, so the systems' chains of
 * recursion sub-steps overlap on the device and none waits for a slower one (a pool, by
 * contrast, steps every system by the same launches).  Every context must be distinct.  The
 * calling thread polls completion (short sleeps) until the last step is done.  Returns the worst
 * status over the contexts as symba_sync does, SYMBA_E_INVAL for a NULL array or context or
 * negative counts, or the first launch error (contexts may then still have a step in flight). */
int symba_step_many(symba_ctx *const *ctxs, int n, int nsteps);

/* Total energy E and angular momentum L[3] of the current state (democratic heliocentric, equal
 * to the barycentric totals; Sec. 3 accuracy test).  Each is the correctly rounded sum of its
 * terms.  Synchronises.  E and L are host pointers. */
int symba_energy(symba_ctx *c, double *E, double L[3]);

/* The level-0 encounter pairs of the last step in ascending (i, j) order (i < j) and, for each,
 * the index of its group; groups are numbered by ascending smallest member (Sec. 2, encounter
 * paragraph: pairs found by the check join groups that are integrated independently).  pairs: 2 x cap
 * ints, group_of_pair: cap ints (host or device).  *n_pairs and *n_groups receive the full
 * counts even when they exceed cap (then only cap entries are written).  Synchronises. */
int symba_enc_groups(symba_ctx *c, int *pairs, int *group_of_pair, int cap, int *n_pairs,
                     int *n_groups);

/* Copies the integrator's state out (the democratic-heliocentric split of SyMBA, which the paper
 * parallelises without changing; Sec. 2): x (n x 3 heliocentric), v (n x 3 barycentric; the
 * heliocentric velocity is v + P / m0 with P = sum m v), and optionally m,
 * radius (n) and alive (n ints, 0 for a body merged into another or removed).  Any output may be NULL.
 * Synchronises. */
int symba_get_state(symba_ctx *c, double *x, double *v, double *m, double *radius, int *alive);

/* Copies out the n Hill radii the context uses (host or device array of n doubles): those given
 * to symba_init, or a_i (m_i / 3 m0)^{1/3} computed there from the osculating heliocentric orbit
 * (vis-viva with mu = G (m0 + m_i); r_i if unbound; 0 for field particles) with a correctly
 * rounded cube root, then rescaled by (m / m_i)^{1/3} when body i grows by a merger.  They set
 * the critical radii lambda (rH_i + rH_j) of the encounter check (Sec. 2, the encounter
 * paragraph; Sec. 3 for the shell ratio).  Synchronises; returns the sticky status. */
int symba_get_rhill(symba_ctx *c, double *rhill);

/* Replaces positions (heliocentric) and barycentric velocities -- the state symba_get_state
 * returns, so a get/set round trip is exact (checkpoint and resume); masses, radii and Hill radii
 * stay.  Enqueued on the context's stream.  Also clears the sticky status. */
int symba_set_state(symba_ctx *c, const double *x, const double *v);

/* Diagnostics of the last call (encounter pairs and groups, Sec. 2; recursion depth and sub-steps,
 * Sec. 3); synchronises. */
int symba_get_stats(symba_ctx *c, symba_stats *s);

/* Phase timing (tracing; the paper times whole runs, Sec. 3): runs nsteps steps like symba_step, launching the kernels one by one
 * with CUDA events between them on the context's stream, then synchronises and writes the
 * summed device time of each phase in milliseconds to phase_ms[0..SYMBA_NPHASES-1] (host):
 * 0 sun drift + step prologue, 1 kick 1 with the fused encounter check, 2 kick-1 reduction,
 * 3 grouping, 4 Kepler drift, 5 group recursion, 6 kick 2, 7 kick-2 reduction,
 * 8 total momentum, 9 closing sun drift.  Returns the sticky status like symba_sync. */
#define SYMBA_NPHASES 10
int symba_profile_step(symba_ctx *c, int nsteps, double *phase_ms);

/* Releases the context and all its device memory (after waiting for its stream). */
void symba_free(symba_ctx *c);

/* ---------------------------------------------------------------------------------------- */
/* Pools: many independent systems (a parameter scan, Sec. 1) stepped together, every kernel  */
/* of a step launched once for all of them.  Results of a system do not depend on which other */
/* systems share the pool.                                                                     */
/* ---------------------------------------------------------------------------------------- */

/* Creates a pool that can hold up to max_systems systems with at most max_particles bodies in
 * total and max_tiles 32 x 32 trapezoid tiles in total (the pair-kick scratch: 1.5 KiB each).
 * precision: SYMBA_PRECISION_FP64 or SYMBA_PRECISION_MIXED for every system of the pool. */
int symba_pool_create(symba_pool **out, int max_systems, long long max_particles,
                      long long max_tiles, int precision, void *cuda_stream);

/* Device bytes a system of n bodies (n_massive massive) occupies in a pool. */
long long symba_pool_footprint(int n, int n_massive, const symba_params *p);

/* Admits one system (arguments as symba_init) into a free slot; *slot receives its id.
 * Returns SYMBA_E_NOMEM if the pool has no room for it (slots, bodies, tiles or pairs). */
int symba_pool_admit(symba_pool *pool, const symba_params *p, int n, int n_massive,
                     const double *x, const double *v, const double *m, const double *radius,
                     const double *rhill, int *slot);

/* Enqueues nsteps steps of every admitted system.  Asynchronous. */
int symba_pool_step(symba_pool *pool, int nsteps);

/* Waits; returns the worst sticky status over the pool's systems. */
int symba_pool_sync(symba_pool *pool);

/* Per-system state, energy, Hill radii, encounter list and diagnostics (synchronising) and
 * set-state (enqueued), with the arguments, meaning and errors of the single-system forms
 * symba_get_state, symba_energy, symba_get_rhill, symba_enc_groups, symba_set_state and
 * symba_get_stats; slot is the id symba_pool_admit returned (SYMBA_E_INVAL otherwise). */
int symba_pool_get_state(symba_pool *pool, int slot, double *x, double *v, double *m,
                         double *radius, int *alive);
int symba_pool_energy(symba_pool *pool, int slot, double *E, double L[3]);
int symba_pool_get_rhill(symba_pool *pool, int slot, double *rhill);
int symba_pool_enc_groups(symba_pool *pool, int slot, int *pairs, int *group_of_pair, int cap,
                          int *n_pairs, int *n_groups);
int symba_pool_set_state(symba_pool *pool, int slot, const double *x, const double *v);
int symba_pool_get_stats(symba_pool *pool, int slot, symba_stats *s);

/* Removes a system; its slot, bodies and scratch become free for later admissions. */
int symba_pool_evict(symba_pool *pool, int slot);

void symba_pool_free(symba_pool *pool);

/* ---------------------------------------------------------------------------------------- */
/* Launch schedules and their autotuner.  The pair kick (Sec. 2's trapezoid loop) is a queue   */
/* of 32 x 32 tiles taken by persistent warps; the encounter groups (Sec. 2: each group is     */
/* integrated independently) are a queue of groups taken by persistent warps.  How the queues  */
/* are cut and ordered changes no result -- per-tile partials are reduced in a fixed order and  */
/* groups touch disjoint bodies -- only the time.                                              */
/* ---------------------------------------------------------------------------------------- */
typedef struct {
  int kick_blocks_per_sm;   /* persistent kick CTAs (4 warps each) per multiprocessor, >= 1 */
  int kick_tiles_per_item;  /* tiles a warp takes per grab from the tile queue, 1..64 */
  int rec_blocks_per_sm;    /* recursion CTAs (4 warps, one per SM quadrant) per SM, 1 or 2 */
  int group_order;          /* 0: groups in label order; 1: longest estimated chain first
                               (M^k for the deepest shell k the pair's straight-line closest
                               approach reaches, times the share of the step it stays inside;
                               up to 16,384 groups per step are ordered, more keep label order) */
} symba_schedule;

typedef struct {
  symba_schedule chosen;        /* the schedule in effect when the call returns */
  double kick_ms;               /* its second-kick time, mean over the repetitions */
  double recursion_ms;          /* its group-recursion time on the trial step */
  double kick_ms_before;        /* the same two for the schedule in effect before the call */
  double recursion_ms_before;
  int kick_candidates;          /* kick schedules timed */
  int recursion_candidates;     /* recursion schedules timed */
  int identical;                /* 1: every recursion trial ended in a bit-identical state */
  int pad;
} symba_tune_result;

/* Current schedule of a pool (host struct). */
int symba_pool_get_schedule(symba_pool *pool, symba_schedule *s);

/* Sets a schedule; SYMBA_E_INVAL for fields outside their ranges (kick_blocks_per_sm above the
 * kernel's occupancy limit included).  Takes effect at the next step. */
int symba_pool_set_schedule(symba_pool *pool, const symba_schedule *s);

/* Times candidate schedules on the pool's current systems and keeps the fastest; synchronises.
 * Kick: every kick_blocks_per_sm up to the occupancy limit x kick_tiles_per_item in
 * {1, 2, 4, 8, 16}, each timed over reps (>= 1) launches of the second kick, which writes only
 * per-tile scratch that every step overwrites.  Recursion: rec_blocks_per_sm in {1, 2} x
 * group_order in {0, 1}, each timed on the same trial step, run from a device copy of the
 * pool's state (positions, velocities, masses, radii, flags, momenta, statistics) that is put
 * back before every trial and after the last, so the call leaves every system as it found it.
 * The copy is allocated for the call (SYMBA_E_NOMEM if it does not fit) and freed.  With no
 * system admitted it returns SYMBA_OK and leaves the schedule unchanged.  A trial step that
 * sets an error status does not change the pool's status (it is restored); CUDA failures
 * return SYMBA_E_CUDA.  out (host) may be NULL. */
int symba_pool_autotune(symba_pool *pool, int reps, symba_tune_result *out);

/* The same for the pool behind a context. */
int symba_autotune(symba_ctx *c, int reps, symba_tune_result *out);

/* Human-readable name of a status code. */
const char *symba_status_string(int status);

/* Measures, on the current device, the rates that bound this path (measurement infrastructure:
 * the paper reports only wall-clock times, Sec. 3; the pair kick of Sec. 2 is FP64-pipe bound
 * and the per-group recursion is bound by one warp's dependent FP64 work).  Writes out[0..5]
 * (host): 0 the device's FP64 FLOP/s (independent fused multiply-adds on every SM, an FMA
 * counting 2 flops); 1 cycles per FMA of one warp's dependent FMA chain; 2 cycles per FMA of one
 * warp running four independent chains; 3 cycles per round trip of a value between two warps of
 * a CTA through shared memory and two named barriers; 4 multiprocessors; 5 the device's nominal
 * SM clock in Hz (0 if the runtime does not report it).  Allocates and frees a few bytes, runs
 * for a few milliseconds on the legacy default stream and synchronises.  Returns SYMBA_OK,
 * SYMBA_E_INVAL (NULL out), SYMBA_E_NOMEM or SYMBA_E_CUDA. */
#define SYMBA_NRATES 6
int symba_measure_rates(double *out);

/* ---------------------------------------------------------------------------------------- */
/* Energy without device allocation.  The paper has no counterpart: this entry point exists    */
/* for callers that cannot allocate device memory -- a host loop with a hard per-iteration      */
/* latency budget (cudaMalloc and cudaFree may synchronise the device) or a process whose       */
/* device memory belongs to another allocator (a framework's caching allocator, a fixed memory  */
/* budget).  It computes the same E and L[3] as symba_energy, bit for bit, for n bodies given as */
/* caller-owned DEVICE arrays: x (n x 3 heliocentric), v (n x 3 barycentric), m (n); out      */
/* receives E, Lx, Ly, Lz (4 doubles, device).  Every body counts (pass only live ones); bodies */
/* n_massive..n-1 are field particles.  Enqueued on cuda_stream (NULL = the legacy default      */
/* stream); returns without waiting.                                                           */
/* It calls no allocating routine: its exact-sum scratch is a 3,864-byte file-scope device     */
/* array that every GPU which loads the library holds until the process exits.  Each call asks */
/* the runtime for that array's device address on the current device (no allocation); the     */
/* first call on a device may load the library's device code, so make it before any stream    */
/* capture.  All calls share the array and it keeps the last call's contents (each call       */
/* clears it first), so calls that overlap on the GPU -- on different streams, or from         */
/* different host threads -- race and must be serialised by the caller.                        */
/* Sizes: one accumulator sums at most 2^31 - 1 terms and the energy of n bodies takes         */
/* n (n - 1)/2 + 2n + 1, so n > SYMBA_ENERGY_STATIC_MAX_N is rejected with SYMBA_E_INVAL, as   */
/* are n < 1, host pointers and pointers into another GPU's memory.                            */
/* ---------------------------------------------------------------------------------------- */
#define SYMBA_ENERGY_STATIC_MAX_N 65534
int symba_energy_static(int n, int n_massive, const double *x, const double *v, const double *m,
                        double G, double m0, double *out, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* SYMBA_H */
