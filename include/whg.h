/*
 * whg.h -- C ABI of libwhg, a GB300 (sm_103a) FP64 ensemble integrator for the
 * WHFast512 timestep (Javaheri, Rein & Tamayo 2023).
 *
 * The library advances S independent planetary systems (a star plus 1..8
 * planets each) with the Wisdom-Holman map in democratic heliocentric (DH)
 * coordinates:
 *     K(dt/2) . J(dt/2) . I(dt) . J(dt/2) . K(dt/2)           (Sec. 3.1, Eq. 2)
 * with the Kepler drift K (Sec. 3.2, Eq. 3), the jump J (Sec. 3.4, Eq. 6), the
 * interaction kick I (Sec. 3.3, Eq. 5) and the optional 1/r^2 GR term
 * (Sec. 3.3).  Adjacent half drifts of consecutive steps are fused; output
 * calls synchronize a copy and leave the live state unsynchronized
 * ("keep unsynchronized", Sec. 3.5 list), so results are bitwise identical
 * whatever the number of outputs or the way step counts are split into calls.
 *
 * Conventions (Sec. 3.5 list): G = 1; dt > 0 and fixed per system (integrate
 * backwards by flipping velocities); masses are constant (call whg_init again
 * to change masses or dt).  Massless planets are allowed.
 *
 * Arrays (row-major, FP64 unless stated; S = n_systems, N = max_planets,
 * body 0 of every system is the star, bodies 1..n_planets[s] its planets,
 * slots above n_planets[s] are ignored on input and zero on output):
 *     masses [S][1+N]        pos [S][1+N][3]        vel [S][1+N][3]
 * Positions and velocities are inertial-frame.  Raw state (DH, unsynchronized):
 *     Q [S][N][3] heliocentric positions, v [S][N][3] barycentric velocities.
 *
 * Errors: every int-returning call returns WHG_OK (0) or a negative WHG_E*
 * code and records a message retrievable with whg_last_error().  Numerical
 * trouble inside one system is not an error: it sets that system's status
 * bits (WHG_STATUS_*), rolls the system back to the start of the failing step
 * and freezes it; all other systems continue.  The optional stop rules
 * (close encounter, ejection) end a system the same way.
 *
 * Threads and streams: a context is not thread-safe.  All device work of a
 * context is ordered on the stream given to whg_create / whg_set_stream (NULL =
 * the legacy default stream): the adjoint's work on its own side streams and
 * SM partitions starts after what was issued on that stream before the call,
 * and the stream waits for it before anything issued after the call.  Calls
 * marked "async" return after enqueueing; calls taking host buffers block
 * until their data has been copied.
 */
#ifndef WHG_H
#define WHG_H

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define WHG_OK 0
#define WHG_EINVAL (-1)      /* invalid argument or input value */
#define WHG_ECUDA (-2)       /* a CUDA runtime call or kernel launch failed */
#define WHG_ENOMEM (-3)      /* device or host allocation failed */
#define WHG_ESTATE (-4)      /* call out of order (e.g. step before init) */

/* per-system status bits (frozen systems keep their last good state) */
#define WHG_STATUS_NONFINITE 1   /* a step produced a non-finite coordinate */
#define WHG_STATUS_HYPERBOLIC 2  /* a Kepler drift started with beta = 2 m0/r - v^2 <= 0
                                    (unbound orbit: outside the fixed solver's domain, Sec. 3.2) */
#define WHG_STATUS_INVALID 4     /* rejected input (device-pointer init only) */
#define WHG_STATUS_CLOSE_ENCOUNTER 8  /* stop rule: a pair closer than close_encounter_hill
                                         mutual Hill radii during an interaction step */
#define WHG_STATUS_EJECTED 16    /* stop rule: a planet beyond eject_factor x the system's
                                    largest initial semi-major axis at the start of a step */

#define WHG_MAX_PLANETS 8

typedef struct whg_ctx whg_ctx;

typedef struct {
    int gr_mode;              /* 0: no GR term.  1 (default): kick v_i by dt*a_GR(Q_i),
                                 a_GR(Q) = -6 (G m0)^2 Q / (c^2 |Q|^4), the force of the
                                 potential -3 (G m0)^2/(c^2 r^2) centred on the star
                                 (Sec. 3.3, GR paragraph).  2: additionally subtract
                                 sum_j (m_j/m0) a_GR(Q_j) from every planet (the
                                 paper's back-reaction sentence read literally). */
    double c_light;           /* speed of light in code units (AU, Msun, yr/2pi);
                                 default 10065.32 */
    int newton_terms;         /* Stumpff series terms in the Newton phase: 8 (default,
                                 Sec. 3.2) or 6 (Appendix A).  The Halley phase always
                                 uses 4 terms; 2 Halley + 2 Newton iterations (Sec. 3.2).
                                 T terms: c_2, c_3 summed through the z^T term,
                                 c_n(z) ~ sum_{k=0..T} (-z)^k / (n+2k)!.  The initial
                                 guess is X = h/r0. */
    int lanes_per_system;     /* 0 = auto: systems are grouped by planet count n and a
                                 system gets n warp lanes (8 for n = 7), floor(32/n)
                                 systems per warp, all groups in one launch.  1..8
                                 (>= max_planets): that many lanes for every system */
    int block_size;           /* CUDA threads per block, 0 = auto (multiple of 32) */
    long long steps_per_launch; /* 0 = auto; bounds one kernel launch's length */
    double close_encounter_hill; /* ensemble stop rule (not in the paper's map), 0 = off:
                                 stop a system when a pair comes closer than this many
                                 mutual Hill radii ((m_i+m_j)/(3 m0))^(1/3) (a_i+a_j)/2,
                                 a_i = initial osculating heliocentric semi-major axes */
    double eject_factor;      /* ensemble stop rule, 0 = off: stop a system when a planet
                                 is farther from the star than this factor times the
                                 system's largest initial a at the start of a step */
    int graph_launches;       /* 0 = off; else whg_step replays a CUDA graph of this many
                                 step launches (captured once per init and launch length)
                                 for the whole multiples, and launches the rest directly.
                                 Results are bitwise those of direct launches. */
    int merge_jumps;          /* 1: without the GR term, one J(dt) followed by I(dt) per step
                                 instead of J(dt/2) I(dt) J(dt/2): J and I commute when there
                                 is no GR term (Sec. 3.1), so this is the same map up to
                                 rounding, one jump cheaper.  Ignored when gr_mode != 0. */
    int halley_fp32;          /* 1: the Kepler solver's initial guess and its 2 Halley steps
                                 (Sec. 3.2) run in FP32; the 2 Newton steps, the f and g
                                 functions and everything else stay FP64.  The Halley phase
                                 only supplies the Newton phase's start, and two FP64 Newton
                                 steps from a start within ~1e-7 converge quadratically to
                                 FP64 rounding, so inside the solver's domain (Fig. 1) the
                                 results match the all-FP64 solver to rounding.  Outside it
                                 (pericentre timescale below ~2 steps) both are inaccurate and
                                 may stop differently.  Default 0: the whole solver in FP64
                                 (the paper's arithmetic). */
    int repack_frozen;        /* -1 (default): on when a stop rule is on
                                 (close_encounter_hill > 0 or eject_factor > 0), else off.
                                 1: every graph_launches step launches (every 16 without
                                 graphs; inside the captured graph with them) regroup the
                                 systems of each planet count so that running systems come
                                 first and stopped ones (status != 0) last.  A warp whose
                                 systems have all stopped skips its steps, so stopped
                                 systems stop costing time.  Each system's arithmetic uses
                                 only its own lanes: results are bitwise those without
                                 repacking.  Costs a second copy of the state in device
                                 memory (allocated by whg_create).  Not part of the
                                 paper's method.  Ignored by whg_integrate_noalloc.
                                 0: off. */
    int interaction_schedule; /* 0 (default): pairs at lane distance k < L/2 evaluated once
                                 with the reaction passed back (Newton's third law, Sec. 3.3),
                                 distance L/2 by both lanes: 4 reciprocal square roots per lane
                                 for 8 planets.  1: all L-1 rotations, every lane summing its
                                 own pairs (7 per lane for 8 planets).  Same map; the summation
                                 order, and so the rounding, differs.  A tuning dimension. */
    int queue_steps;          /* 1..10000 (default 100): a persistent work queue; resident
                                 warps take (warp-group, queue_steps steps) units in order,
                                 each waiting for its group's previous unit, so work moves
                                 between SMs and no SM finishes late because it holds one warp
                                 more than another (+3.5 % at 4096 8-planet systems, +7 % at
                                 8192).  Used for launches of at least 4 units per warp-group
                                 (shorter ones run as plain launches); queue launches use
                                 one-warp blocks (block_size does not apply).  0: one warp per
                                 warp-group for the whole launch.
                                 Results are bitwise the same either way.  A wait that exceeds
                                 its limit (seconds; only possible after a fault) makes the
                                 next whg_synchronize or whg_read_state return WHG_ECUDA.  Not
                                 part of the paper's method.  Ignored by
                                 whg_integrate_noalloc (plain launches). */
} whg_options;

/* Fill *opt with the defaults above. */
void whg_default_options(whg_options* opt);

/* Create a context for n_systems systems of at most max_planets (1..8)
 * planets on the current CUDA device; allocates all device memory the
 * context needs (owned by the library until whg_destroy).  opt may be NULL
 * (defaults).  cuda_stream is a cudaStream_t or NULL.  On failure *out is
 * NULL and whg_last_error(NULL) describes why. */
int whg_create(whg_ctx** out, int n_systems, int max_planets, const whg_options* opt,
               void* cuda_stream);

/* Set the stream used by all later calls on ctx. */
int whg_set_stream(whg_ctx* ctx, void* cuda_stream);

/* Initialise every system from HOST arrays (layouts above): converts to DH
 * coordinates (Sec. 3.1: Q_i = x_i - x_0, v_i = u_i - V_cm) on the device and
 * marks the state synchronized (the next step starts with K(dt/2)).
 * n_planets [S] (int32) may be NULL (all systems have max_planets planets);
 * dt [S] > 0.  Inputs are copied; the caller keeps ownership.  Returns
 * WHG_EINVAL (nothing changed) if any system has m0 <= 0, a negative or
 * non-finite mass, dt <= 0, n_planets outside 1..max_planets, a non-finite
 * coordinate, or a planet at the star's position.  Blocks until copied. */
int whg_init(whg_ctx* ctx, const double* masses, const double* pos, const double* vel,
             const int* n_planets, const double* dt);

/* As whg_init, but all pointers are DEVICE pointers (same layouts) on ctx's
 * device, read on ctx's stream.  With lanes_per_system = 0 and n_planets
 * given, the planet counts are copied back to the host once to lay the
 * ensemble out.  Returns after the init kernel has run.  Invalid systems are
 * not reported by the return value: they get WHG_STATUS_INVALID and stay
 * frozen. */
int whg_init_device(whg_ctx* ctx, const double* masses, const double* pos, const double* vel,
                    const int* n_planets, const double* dt);

/* Advance every live system by n_steps Wisdom-Holman steps (Eq. 2, drifts
 * fused; async).  n_steps >= 0.  The split of work into kernel launches never
 * changes results.  WHG_ESTATE before the first init. */
int whg_step(whg_ctx* ctx, long long n_steps);

/* Synchronized inertial state into HOST buffers pos, vel [S][1+N][3];
 * status [S] (int32) and t [S] (time = steps done * dt) may be NULL.
 * The pending K(dt/2) (Sec. 3.5 list) is applied to a copy; the live state is
 * unchanged.  Blocks. */
int whg_read_state(whg_ctx* ctx, double* pos, double* vel, int* status, double* t);

/* As whg_read_state, into DEVICE buffers (async). */
int whg_read_state_device(whg_ctx* ctx, double* pos, double* vel, int* status, double* t);

/* Total energy H = H_0 + H_K + H_I + H_J (Eq. 1) of each system's
 * synchronized state, plus sum_i m_i Phi_GR(Q_i) when gr_mode != 0; E [S] HOST
 * buffer.  Blocks. */
int whg_energy(whg_ctx* ctx, double* E);

/* As whg_energy, into a DEVICE buffer (async). */
int whg_energy_device(whg_ctx* ctx, double* E);

/* Raw unsynchronized DH state for bitwise checkpoint / resume, HOST buffers:
 * Q, v [S][N][3]; nstep [S] (int64, steps done; 0 = synchronized);
 * status [S] (int32).  get blocks; set copies and returns (async after copy).
 * set requires a prior init (masses, dt and barycentre come from it). */
int whg_get_raw(whg_ctx* ctx, double* Q, double* v, long long* nstep, int* status);
int whg_set_raw(whg_ctx* ctx, const double* Q, const double* v, const long long* nstep,
                const int* status);

/* ---- adjoint (reverse mode) --------------------------------------------- */

/* Forward half of a gradient computation for the loss
 *     L_s = sum_i |Q_i(T) - target_i|^2        (one value per system s)
 * with Q_i(T) the heliocentric positions of the synchronized state after
 * n_steps Wisdom-Holman steps (Eq. 2).  Needs a context initialised with
 * whg_init / whg_init_device and not stepped since.  Advances the state by
 * n_steps exactly as whg_step does (without repacking stopped systems, so
 * that every checkpoint has the same layout), keeping the state every
 * checkpoint_every steps in device memory owned by ctx (kept until
 * whg_destroy): (n/K + 1) * 48 B per planet lane of checkpoints and
 * K * 592 B per planet lane for each tape buffer (three, or with a tape
 * budget of whg_adjoint_schedule up to one per segment; the per-step values
 * of a segment that the backward half consumes).  target [S][N][3] and
 * loss [S] are DEVICE pointers; target is copied.  Async. */
int whg_adjoint_forward(whg_ctx* ctx, long long n_steps, int checkpoint_every, const double* target,
                        double* loss);

/* Backward half: gradients of sum_s w_s L_s with respect to the inputs of the
 * last init (inertial positions and velocities [S][1+N][3], masses [S][1+N],
 * star included), w_s = loss_weight[s] (DEVICE [S], NULL = all 1).  Each K-step
 * segment is recomputed from its checkpoint while a per-step tape is kept,
 * and the vector-Jacobian products of J, I (+GR), J and K (the Kepler flow
 * through the implicit function theorem at the converged universal variable)
 * are applied in reverse.  Output pointers are DEVICE pointers (any may be
 * NULL);
 * systems that froze during the forward half get NaN.  May be called again
 * with other weights.  Async. */
int whg_adjoint_backward(whg_ctx* ctx, const double* loss_weight, double* grad_pos, double* grad_vel,
                         double* grad_mass);

/* Scheduling of the adjoint; not part of the paper's method.  Results are
 * bitwise the same under every setting.  Takes effect at the next
 * whg_adjoint_forward.
 * sm_split: -1 (default): split the SMs into two green contexts when the
 *   ensemble's warps need at most half of the SMs at one warp per SM
 *   sub-partition (about 1200 8-planet systems or fewer on a 152-SM GPU).
 *   In the backward half the back kernels, its critical path, then run on
 *   ceil(warps / 4) SMs (rounded up to the partition granularity, 8 SMs on
 *   this GPU), one warp per sub-partition, and the tape kernels on the
 *   remaining SMs, so that the two never share a sub-partition.  The forward
 *   half runs on all SMs except for its last two segments, which move to the
 *   back kernels' SMs while the tape kernels compute the first two tapes the
 *   backward half needs.
 *   0: no split; the tape kernels run on two side streams beside the back
 *   kernels, wherever the block scheduler puts them.
 *   n > 0: split with n SMs for the back kernels.
 *   Where green contexts are unavailable the adjoint runs unsplit.
 * tape_bytes: tape buffers (K * 592 B per planet lane each, kept until
 *   whg_destroy).  0 (default): three; each segment's tape is recomputed
 *   during the backward half, two segments ahead of the back kernels.
 *   With the split, a budget makes the tapes of the segments already passed
 *   be recomputed during the forward half instead, beside it, into up to one
 *   buffer per segment; the forward half then runs on the back kernels' SMs.
 *   -1: as many buffers as fit in half of the free device memory at
 *   whg_adjoint_forward; n > 0: at most n bytes (at least 3 buffers).
 *   Segments without a buffer of their own get their tapes recomputed during
 *   the backward half.
 * Returns WHG_EINVAL for values below -1. */
int whg_adjoint_schedule(whg_ctx* ctx, int sm_split, long long tape_bytes);

/* After whg_adjoint_forward: SMs of the partition that runs the back kernels
 * (and the forward half's last segments, or all of it with a tape budget) and
 * of the one that runs the tape kernels (both 0 when unsplit), and the number
 * of tape buffers.  Any pointer may be NULL. */
int whg_adjoint_layout(const whg_ctx* ctx, int* chain_sms, int* tape_sms, int* tape_buffers);

/* Wait until all work issued on ctx's stream has finished. */
int whg_synchronize(whg_ctx* ctx);

/* Number of the library's kernel launches issued on ctx so far. */
long long whg_launch_count(const whg_ctx* ctx);

/* Message for the last error on ctx (or of the last failed whg_create, ctx
 * NULL).  Valid until the next call on ctx. */
const char* whg_last_error(const whg_ctx* ctx);

/* Free all resources of ctx (NULL is a no-op).  Synchronizes its stream. */
void whg_destroy(whg_ctx* ctx);

/* ---- allocation-free variant -------------------------------------------- */

/* The paper has no counterpart of this call: it exists for callers that
 * cannot allocate device memory, such as frameworks that reserve the GPU's
 * memory up front and only hand out buffers from their own pool, host
 * programs or plugins that forbid device allocation once running, and loops
 * that cannot afford cudaMalloc's implicit device-wide synchronization.
 *
 * Does what whg_create + whg_init_device + whg_step(n_steps) +
 * whg_read_state_device would do, with the same kernels and results, but
 * calls no cudaMalloc, cudaFree or other allocating routine: the working state
 * lives in one fixed array of 10 MiB in the library's device memory,
 * which every GPU that loads the library holds until the process exits.
 * All array pointers are DEVICE pointers with the layouts above (n_planets,
 * status_out and t_out may be NULL); work is issued on cuda_stream (NULL =
 * legacy default stream) and the call returns after enqueueing it.
 *
 * Every system gets the same lane group (opt->lanes_per_system, or by default
 * the group a context would use for max_planets planets), so results match a
 * context created with that lanes_per_system.
 * Limit: the warps needed (floor(32 / lanes) systems each) must not exceed
 * WHG_NOALLOC_MAX_LANES / 32 lanes' worth, e.g. 8192 systems of 7 or 8
 * planets; larger requests fail with WHG_EINVAL.
 * Every call looks up the array's device address (no allocation); the first
 * lookup on a device may load the library's device image, so make the first
 * call on each device before any stream capture.
 * Every call reuses the same array and leaves its contents behind; each call
 * rewrites everything it reads before reading it.  Calls whose GPU work
 * overlaps (other streams, other host threads) race on the array: order them.
 * Errors are reported by the return code and whg_last_error(NULL). */
#define WHG_NOALLOC_MAX_LANES 65536
int whg_integrate_noalloc(int n_systems, int max_planets, const whg_options* opt,
                          const double* masses, const double* pos, const double* vel,
                          const int* n_planets, const double* dt, long long n_steps,
                          double* pos_out, double* vel_out, int* status_out, double* t_out,
                          void* cuda_stream);

/* ---- diagnostics (not part of the integration path) -------------------- */

/* FP64 FMA-stream throughput: runs a loop of independent dependent-FMA
 * chains on every SM of the current device for about `seconds` and returns
 * the achieved FP64 TFLOP/s (FMA = 2 flops).  Blocks.  A diagnostic, not a
 * peak: on GB300 a pure stream of DFMA, DMUL or DADD instructions issues at
 * about 1.68 FP64 lanes per clock per SM however many warps and chains run,
 * while the step kernel, whose FP64 instructions are interleaved with
 * integer, shuffle and MUFU work, sustains about 1.8. */
int whg_measure_fp64_tflops(double seconds, double* tflops);

/* Solver search of Appendix A: n massless particles (DEVICE q, v [n][3]) each
 * drifted `steps` times by time h around a central mass mu with its own
 * solver configuration cfg [n][4] = (Halley iterations, Halley series terms,
 * Newton iterations, Newton series terms), terms 1..12 (series through z^T,
 * as newton_terms above), initial guess h/r0; G_n after the last
 * iteration evaluated at the final X with the Newton series length.  Plain
 * per-particle loops (a validation tool, not the integration path).
 * Writes q_out, v_out (DEVICE).  Blocks. */
int whg_kepler_sweep(const double* q, const double* v, const int* cfg, int n, double mu, double h,
                     long long steps, double* q_out, double* v_out);

/* FP64 pipe probe (no counterpart in the paper; it backs the lane layout):
 * times, with CUDA events on the legacy default stream, one launch of
 * warps_per_sm x (SM count) one-warp blocks running iters x 8 independent
 * dependent-DFMA chains in the first active_lanes lanes of each warp (the
 * others skip the loop).  *ms receives the kernel time.  warps_per_sm 1..64,
 * active_lanes 1..32, iters 1..2^24; allocates and frees a small buffer;
 * blocks.  On GB300 the time does not depend on active_lanes, so masked
 * lanes cost full FP64 pipe time. */
int whg_probe_fp64_lanes(int warps_per_sm, int active_lanes, int iters, float* ms);

/* FP64 issue rate by instruction kind (no counterpart in the paper; it backs
 * the choice of the roofline's denominator): warps_per_sm x (SM count)
 * one-warp blocks, each lane running iters x 8 independent chains of one
 * kind: 0 DFMA, 1 DMUL, 2 DADD, 3 DFMA plus one integer multiply-add per
 * DFMA, 4 DFMA plus one FP32 FMA per DFMA.  *lanes_per_clk receives the FP64
 * lane-operations per SM clock over the slowest block (clock64 around the
 * loop, so independent of the clock frequency; all blocks are resident at
 * once).  kind 0..4, warps_per_sm 1..32, iters 1..2^24; allocates and frees
 * a small buffer; blocks. */
int whg_probe_fp64_kind(int kind, int warps_per_sm, int iters, double* lanes_per_clk);

/* Failure-path test of the work queue (no counterpart in the paper): one
 * queue launch on ctx (initialized, queue_steps > 0) whose unit counter starts
 * past every warp-group's first unit, so each unit waits for a predecessor
 * that never runs.  Every wait gives up after spin_limit polls (>= 1; ~100 ns
 * or more each) and sets the queue's error flag; no step runs, so the state
 * is untouched.  *flag receives the flag (1 = a wait gave up), which is then
 * cleared.  Blocks.  Returns WHG_EINVAL if the queue is off. */
int whg_test_queue_timeout(whg_ctx* ctx, long long spin_limit, int* flag);

/* Index checks (no counterpart in the paper; the stand-in for a device memory
 * checker): in the debug build of the library (libwhg_debug.so, compiled with
 * WHG_DEBUG_BOUNDS) every kernel checks its lane, system, bucket, permutation,
 * repack and work-queue indices against the context's sizes and records a
 * failed check as a bit in a flag word (1 lane, 2 system, 4 caller index,
 * 8 bucket, 16 repack order, 32 queue unit) instead of trapping.  Synchronizes
 * ctx's stream, writes the bits set since the last call to *flag and clears
 * them.  In the release build: *flag = 0 and WHG_EINVAL. */
int whg_debug_bounds(whg_ctx* ctx, unsigned* flag);

/* The same index-check flags for whg_integrate_noalloc, whose checks record
 * into one flag word of its own (no context): synchronizes the current
 * device, writes the bits set by all calls since the last read to *flag and
 * clears them.  Allocates nothing.  In the release build: *flag = 0 and
 * WHG_EINVAL (message in whg_last_error(NULL)). */
int whg_noalloc_debug_bounds(unsigned* flag);

/* The library's own reciprocal, reciprocal square root and FP64 <-> FP32
 * conversions next to CUDA's, for testing: out [12][n] DEVICE buffer receives
 * rcp_own(x), 1/x (CUDA, IEEE), rsqrt_own(x), rsqrt(x) (CUDA) (0 < x < 4e307
 * for the square roots, else 0), the own FP64 -> FP32 -> FP64 round trip of
 * x, CUDA's round-toward-zero FP64 -> FP32 conversion of x widened to FP64,
 * then the own routines' FP64-only reference forms: rcp, rsqrt, the own
 * x^(-3/2) and its reference (0 <= x < 4e307, else 0), then the own 1/x^2
 * and the square of CUDA's 1/x (0 <= x < 4e307, else 0), for the n DEVICE
 * inputs x.
 * Blocks. */
int whg_test_special(const double* x, int n, double* out);

#ifdef __cplusplus
}
#endif

#endif /* WHG_H */
