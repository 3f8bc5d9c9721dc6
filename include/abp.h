/*
 * abp.h -- C ABI of the GB300 active-Brownian-particle ensemble integrator.
 *
 * The library integrates many independent trajectories of the energy-depot
 * Langevin model of arXiv 1104.2499, Sec. 2 (Zabicki, "OpenCL/OpenGL approach
 * for studying active Brownian motion"):
 *
 *   Eq. (ereservoir)  de/dt = q - c e - d e v^2
 *   Eq. (velocity)    dv/dt = F0 + d e v - gamma0 v - U'(x) + sqrt(2 D) xi(t)
 *   Eq. (pot)         U(x)  = h [0.499 - 0.453 (sin phi + a sin 2 phi)],
 *                     phi = 2 pi (x / L + 0.1903)
 *                     dx/dt = v
 *
 * across sets of parameters and initial conditions (Sec. 2: one work item per
 * parameter value, results averaged over noise realisations and over time),
 * with explicit Euler-Maruyama steps (Fig. 1: per iteration, draw uniforms,
 * Box-Muller them into a Gaussian, update velocity and energy), and reduces
 * the ensemble on the device to the mean velocity (ratchet current), the
 * diffusion coefficient and position / velocity histograms.
 *
 * Noise.  Step n of global trajectory t under seed s uses the Philox4x32-10
 * block with key (s_lo, s_hi) and counter (m_lo, m_hi, t_lo, t_hi), m = n >> 2
 * (Salmon et al., SC'11).  Words (w0, w1) give steps 4m and 4m+1, (w2, w3)
 * steps 4m+2 and 4m+3, through Box-Muller with u1 = (w_a + 1/2) 2^-32 and
 * u2 = floor(w_b / 2^9) 2^-23: z_even = r cos(2 pi u2), z_odd = r sin(2 pi u2),
 * r = sqrt(-2 ln u1).  The initial condition uses counter m = 2^63:
 * x0 = L floor(w0 / 2^8) 2^-24, v0 = 0 or sqrt(D) r(w1) cos(2 pi u2(w2)), e0 = 0.
 * Global trajectory ids number the sets' ensembles consecutively in set order.
 *
 * Arithmetic.  State is FP32.  The position is an integer cell index plus an
 * FP32 fraction of the period, and the per-step increments v dt are summed in
 * a separate small accumulator that is folded into the fraction every 64 steps
 * with its rounding error kept (compensated FP32), so that long runs lose no
 * precision (the paper's precision section warns against adding small
 * increments to large values).  Because the scheme advances x by v_n dt, the
 * time average of v over n steps is (x_n - x_0) / (n dt), taken from this
 * compensated displacement in FP64.  All ensemble sums are FP64.
 *
 * Conventions for every entry point:
 *   - Returns ABP_OK or an error code; the message of the last error of a
 *     context is available from abp_last_error().  Nothing is printed.
 *   - Work is enqueued asynchronously on the context's CUDA stream; a device
 *     side failure recorded by a kernel (an expired bounded wait, or in the
 *     checked build, compiled with ABP_DEBUG_CHECKS=1, an index outside its
 *     buffer) surfaces as ABP_ETIMEOUT / ABP_ESTATE from abp_synchronize() or
 *     from the next call that synchronises.
 *   - Output pointers documented as "host or device" may point to either; the
 *     library inspects them with cudaPointerGetAttributes and copies device ->
 *     host itself when they are host memory (pinned or pageable), in which case
 *     the call returns after the copy has completed.  Device memory must belong
 *     to the context's device (or be managed memory); another GPU's memory is
 *     rejected with ABP_EINVAL, since kernels may write the outputs directly.
 *   - The context owns every device buffer it allocates (state, histograms,
 *     checkpoints, scratch); callers own the buffers they pass in.
 *   - Calls on one context must not run concurrently from several host threads.
 */
#ifndef ABP_H
#define ABP_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define ABP_API __attribute__((visibility("default")))
#else
#define ABP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct abp_ctx abp_ctx;

typedef enum {
    ABP_OK = 0,
    ABP_EINVAL = 1,   /* an argument is out of range, inconsistent or NULL */
    ABP_ENOMEM = 2,   /* a device or host allocation failed */
    ABP_ECUDA = 3,    /* a CUDA runtime call failed (message has the CUDA error) */
    ABP_ETIMEOUT = 4, /* a bounded device-side wait expired; results are invalid */
    ABP_ESTATE = 5    /* the call is out of order (e.g. abp_reduce before abp_set_params) */
} abp_status;

/* Parameters of one set, Sec. 2: Eqs. (ereservoir), (velocity), (pot).
 * asym is the weight a of the second harmonic of Eq. (pot) (1/4 in the paper;
 * a = 0 gives a symmetric potential).  Requirements: L > 0, D >= 0, finite. */
typedef struct {
    double q, c, d, gamma0, F0, D, h, L, asym;
} abp_params;

/* Context-wide configuration. */
typedef struct {
    uint64_t seed;               /* Philox key */
    double dt;                   /* Euler-Maruyama time step, > 0 */
    int32_t v0_mode;             /* 0: v0 = 0; 1: v0 ~ N(0, sqrt(D)) */
    int32_t state_fp64;          /* 0: FP32 state (production path); 1: FP64 state and FP64
                                    arithmetic throughout (precision reference; slow on GB300) */
    int32_t hist_x_bins;         /* bins of x mod L over [0, L); 0 = no position histogram */
    int32_t hist_v_bins;         /* bins of v over [v_lo, v_hi); 0 = none (+2 out-of-range counters) */
    double v_lo, v_hi;           /* velocity histogram range, v_hi > v_lo */
    int64_t snapshot_every;      /* S > 0: histograms of the state after steps S, 2S, ...;
                                    0: one snapshot after each set's last step */
    int64_t checkpoint_every;    /* K > 0: keep the state every K steps for abp_backward;
                                    0: no checkpoints (abp_backward returns ABP_ESTATE) */
    int32_t particles_per_thread;/* 1, 2 or 4 trajectories per CUDA thread; 0 = autotuned */
    int32_t schedule;            /* 0: chosen by the autotuner; 1: lockstep -- one launch per window
                                    of steps_per_launch steps over all tiles; 2: work queue -- one
                                    persistent launch whose blocks pop (tile, round) items, so
                                    uneven sets balance across SMs.  The autotuner times every
                                    (schedule, particles_per_thread) pair once per device and
                                    library build on a synthetic batch (table kept in
                                    abp_tune_cache.txt beside the library, or in the file the
                                    environment variable ABP_TUNE_FILE names; empty: none),
                                    predicts every (schedule, particles_per_thread,
                                    steps_per_launch in {10^3, 10^4, 10^5}) candidate's time on
                                    the batch of abp_set_params from the fraction of the SMs
                                    the batch keeps busy (abp_plan_efficiency) and the state
                                    traffic of its launches, then, when both schedules are
                                    allowed, times every candidate within 3% of its schedule's
                                    best on the first steps of the batch itself and keeps the
                                    fastest prediction (abp_tuning_report shows the record) */
    int64_t steps_per_launch;    /* lockstep: steps per launch; work queue: steps per work item
                                    (round); 0 = chosen by the autotuner from 10^3, 10^4, 10^5 */
    uint64_t traj_base;          /* added to every global trajectory id: a process that runs
                                    one shard of a larger ensemble passes the id of its first
                                    trajectory, so every trajectory keeps its own noise */
    int32_t scheme;              /* 0: explicit Euler-Maruyama, the step of Fig. 1 (all
                                    right-hand sides at step n); 1: stochastic Heun -- predictor
                                    s~ = s + a(s) dt + w, corrector s' = s + (a(s) + a(s~)) dt/2 + w
                                    with the same noise increment w of the step (weak order 2 for
                                    this additive noise; a variant the paper does not use).
                                    Heun needs state_fp64 = 0 and checkpoint_every = 0 (no adjoint) */
    int32_t noise;               /* 0: counter-based Philox4x32-10 keyed by (seed, trajectory, step);
                                    1: Marsaglia's xorshift (shifts 11, 8, 19), the RNG of Fig. 1:
                                    one 128-bit state per trajectory, seeded from the Philox block
                                    of counter 2^63 + 1, two words and one Box-Muller cosine per
                                    step.  Xorshift keeps 16 more bytes of state per trajectory and
                                    needs scheme 0, state_fp64 = 0 and checkpoint_every = 0 */
} abp_config;

/* Create a context on the current CUDA device.  cuda_stream is a cudaStream_t
 * (NULL = the legacy default stream) on which all work of the context runs.
 * The configuration is copied.  On success *out owns a context to be released
 * with abp_destroy. */
ABP_API abp_status abp_create(abp_ctx **out, const abp_config *cfg, void *cuda_stream);

/* Define the batch: n_sets parameter sets (host array, copied), set i with
 * n_traj[i] >= 0 trajectories of n_steps[i] >= 0 steps (host arrays, copied;
 * n_steps[i] < 2^34).  Allocates the trajectory state (28 bytes per FP32
 * trajectory, plus histograms and checkpoints), draws the initial condition on
 * the device and zeroes all accumulators.  May be called again to start a new
 * batch; the previous one is discarded. */
ABP_API abp_status abp_set_params(abp_ctx *ctx, int32_t n_sets, const abp_params *sets, const int64_t *n_traj,
                          const int64_t *n_steps);

/* Start the current batch over: redraw the initial condition with the given
 * seed (the parameters, sizes and device buffers are kept), zero the time sums
 * and histograms and set every set back to step 0.  Only kernels and memsets
 * are enqueued; nothing is copied from the host. */
ABP_API abp_status abp_reset(abp_ctx *ctx, uint64_t seed);

/* Advance every set by min(max_steps, remaining) Euler-Maruyama steps
 * (max_steps < 0: to completion).  Steps run on the device, trajectory state
 * stays resident in HBM between calls, and splitting a run into several calls
 * gives bitwise the same result as one call.  Snapshot histograms are filled
 * as their steps are reached; checkpoints are stored when checkpoint_every > 0. */
ABP_API abp_status abp_integrate(abp_ctx *ctx, int64_t max_steps);

/* Number of steps every set has completed so far (host output, n_sets values). */
ABP_API abp_status abp_progress(const abp_ctx *ctx, int64_t *steps_done);

/* Ensemble reduction (Sec. 2: results averaged over realisations and time).
 * moments (host or device, may be NULL): [n_sets][8] doubles per set:
 *   0 mean_v  = (1/M) sum_i vbar_i, vbar_i = (1/n) sum_{k<n} v_k = (x_n - x_0)/(n dt)
 *             (n = steps done)
 *   1 se_v    = sqrt(sum_i (vbar_i - mean_v)^2 / ((M-1) M))
 *   2 msd     = (1/M) sum_i (x_n - x_0)^2
 *   3 d_eff   = ((1/M) sum_i dx_i^2 - ((1/M) sum_i dx_i)^2) / (2 n dt)
 *   4..7      = sum_i vbar_i, sum_i vbar_i^2, sum_i dx_i, sum_i dx_i^2
 * hist_x (host or device, may be NULL): uint32 [n_snap][n_sets][hist_x_bins]
 * hist_v (host or device, may be NULL): uint32 [n_snap][n_sets][hist_v_bins + 2],
 *   the last two entries counting v < v_lo and v >= v_hi.
 * n_snap = max over sets of (n_steps / snapshot_every), or 1 when
 * snapshot_every == 0; snapshots not reached yet are zero.  The sums are taken
 * in a fixed order, so results are bitwise reproducible.  Asynchronous on the
 * context's stream when every output is device memory (the reduction kernels
 * write device moments directly); with a host output the call returns once it
 * is filled (small page-locked moment outputs are written by the kernels
 * through their device mapping, others copied). */
ABP_API abp_status abp_reduce(abp_ctx *ctx, double *moments, uint32_t *hist_x, uint32_t *hist_v);

/* Number of snapshot slots of the current batch (host output): the longest
 * set's step count divided by snapshot_every when snapshot_every > 0; else 1
 * when there are histograms (the final state) and 0 without. */
ABP_API abp_status abp_num_snapshots(const abp_ctx *ctx, int64_t *n_snap);

/* Live results while the integration runs (the headless counterpart of the
 * results the paper shows during a run, Sec. 3.2 and Table 1).  After this
 * call, abp_integrate stops its launches at every snapshot step k S (S =
 * snapshot_every > 0), computes the ensemble moments at that step on the
 * device, and copies snapshot k -- its moments and its histogram rows -- into
 * the caller's host buffers on a second stream, while the next steps are
 * already integrating.  Buffers (page-locked host memory, from cudaMallocHost
 * or cudaHostRegister; any may be NULL; owned by the caller, who keeps them
 * alive until abp_live_ready reports the last snapshot or the context is
 * synchronised):
 *   moments  [n_snap][n_sets][8] doubles, the layout of abp_reduce at step k S
 *   hist_x   [n_snap][n_sets][hist_x_bins] uint32 (needs hist_x_bins > 0)
 *   hist_v   [n_snap][n_sets][hist_v_bins + 2] uint32 (needs hist_v_bins > 0)
 * n_snap = abp_num_snapshots.  All three NULL switches live results off.
 * Requires abp_set_params first (the buffers are sized by the batch) and
 * snapshot_every > 0; pageable memory is rejected (ABP_EINVAL), because a copy
 * from it would stall the integration.  Snapshots completed before this call
 * are not sent. */
ABP_API abp_status abp_live(abp_ctx *ctx, double *moments, uint32_t *hist_x, uint32_t *hist_v);

/* How many snapshots, counted from the first, have fully arrived in the live
 * host buffers (host output; never waits). */
ABP_API abp_status abp_live_ready(abp_ctx *ctx, int64_t *n_ready);

/* Final (current) state of every trajectory, in global trajectory order
 * (host or device outputs, each of sum(n_traj) doubles; any may be NULL):
 * x = unwrapped position, x0 = initial position, v, e, vbar = time-averaged
 * velocity so far. */
ABP_API abp_status abp_get_state(abp_ctx *ctx, double *x, double *x0, double *v, double *e, double *vbar);

/* Checkpoint / resume of a batch on the host side.  abp_save writes the
 * context's current batch -- step counter, seed, the per-trajectory state
 * (28 bytes per FP32 trajectory) and the histograms -- into buf (host or device
 * memory, caller-owned); with buf == NULL it only stores the size needed in
 * *bytes.  abp_load restores such an image into a context whose batch was set
 * with the same sets, sizes and state type (checked; ABP_EINVAL otherwise);
 * integrating on then gives bitwise the same results as an uninterrupted run.
 * The adjoint checkpoints are not part of the image: abp_backward after
 * abp_load returns ABP_ESTATE until the batch is integrated again from step 0.
 * Both calls return after their copies have completed. */
ABP_API abp_status abp_save(abp_ctx *ctx, void *buf, size_t *bytes);
ABP_API abp_status abp_load(abp_ctx *ctx, const void *buf, size_t bytes);

/* Pathwise adjoint.  With the noise held fixed, returns for every set
 * grad[s][j] = dJ/dtheta_j, J = sum_s dJ_dmean_v[s] * mean_v[s], theta =
 * (D, q, c, d, gamma0, asym) of that set.  dJ_dmean_v: host or device, n_sets
 * doubles (NULL = all ones); grad: host or device, [n_sets][6] doubles.
 * Requires a completed abp_integrate with checkpoint_every > 0 (otherwise
 * ABP_ESTATE); recomputes each checkpoint interval forward and sweeps it in
 * reverse, accumulating in FP64.  Device scratch (context-owned, kept for the
 * next call): 32 bytes per trajectory per 8 steps of checkpoint_every plus 64
 * bytes per trajectory; when checkpoint_every is a multiple of 8, also 8 bytes
 * per trajectory per step of checkpoint_every for handing the noise of each
 * interval's first re-run to its reverse sweep, if that fits in the budget the
 * environment variable ABP_ADJ_HANDOFF_BYTES gives (0: never), by default half
 * the free device memory -- else the noise is drawn again.  The results are the
 * same bit for bit either way. */
ABP_API abp_status abp_backward(abp_ctx *ctx, const double *dJ_dmean_v, double *grad);

/* Windowed pathwise adjoint: as abp_backward, with the adjoint state restarted
 * from zero at steps window, 2 window, ... -- each window's contribution to
 * the time-averaged velocity differentiated with the state at the window's
 * start held fixed.  Over long horizons the frozen-noise dynamics of Sec. 2 is
 * chaotic and the full pathwise derivative grows exponentially with time; the
 * windowed derivative stays bounded (a truncated sensitivity: it leaves out
 * the effect of a parameter change that outlasts a window).  window must be a
 * positive multiple of checkpoint_every (else ABP_EINVAL); window >= the run
 * length gives abp_backward's result. */
ABP_API abp_status abp_backward_windowed(abp_ctx *ctx, const double *dJ_dmean_v, double *grad, int64_t window);

/* Per-trajectory derivatives of the last abp_backward / abp_backward_windowed call:
 * dvbar (host or device, [total_traj][6] doubles, global trajectory order) receives
 * d vbar_i / d theta_j for every trajectory i, vbar_i its time-averaged velocity and
 * theta = (D, q, c, d, gamma0, asym) of its set, noise held fixed (windowed if the last
 * call was).  The set gradient of abp_backward with unit weights is the mean of these
 * over the set's trajectories.  ABP_ESTATE when no backward call has run since the
 * batch was last set, reset or loaded. */
ABP_API abp_status abp_backward_traj(abp_ctx *ctx, double *dvbar);

/* Upper bound, in nanoseconds, of every device-side wait: in the work-queue
 * schedule (schedule 2) a work item waiting for the previous round of its tile,
 * in a warp-specialised narrow lockstep launch (a batch with fewer tiles than
 * SMs) a stepping warp waiting for its producer warps' noise or a producer
 * waiting for a free slot; 0 restores the default
 * of 60 s.  An expired wait ends the launch with ABP_ETIMEOUT
 * (reported by abp_synchronize); the context stays usable after abp_reset. */
ABP_API abp_status abp_set_wait_limit(abp_ctx *ctx, int64_t wait_limit_ns);

/* Test hook for failure detection: tile `tile` (index in the tile table, -1 to
 * clear) never publishes the completion of its rounds in later work-queue
 * launches, so the items that depend on it wait until the wait limit expires;
 * in warp-specialised narrow lockstep launches its producer warps never hand
 * their noise over, so its stepping warps wait until the limit expires.
 * Nothing faults or hangs: the launch ends and reports ABP_ETIMEOUT. */
ABP_API abp_status abp_test_hold_tile(abp_ctx *ctx, int32_t tile);

/* The autotuner's choices for the current batch (host outputs, any may be NULL):
 * schedule (1 lockstep, 2 work queue), particles per thread, steps per launch
 * (lockstep) or per work item (work queue), and the blocks of the chosen schedule's
 * integrator kernel resident on the GPU at once (the work queue's grid). */
ABP_API abp_status abp_tuning(const abp_ctx *ctx, int32_t *schedule, int32_t *particles_per_thread,
                              int64_t *steps_per_item, int32_t *blocks);

/* The autotuner's record for the current batch, as JSON text: every candidate
 * (schedule, particles per thread, steps per launch) with its model prediction, the
 * measured time of the probe on the batch's first steps and the prediction used, and
 * the choice.  buf (host, len bytes, may be NULL) receives it NUL-terminated and cut to
 * fit; *needed (may be NULL) the size with the terminator.  "{\"fixed\": true}" when
 * the configuration fixed every choice. */
ABP_API abp_status abp_tuning_report(const abp_ctx *ctx, char *buf, size_t len, size_t *needed);

/* Tiling of the current batch (host outputs, any may be NULL): tiles in all, how
 * many of them are packed (several small sets sharing one block), and the block
 * width of a narrow lockstep launch (a batch with fewer tiles than SMs runs its
 * tiles as several blocks of `narrow` threads each; 0 when not narrow).  The
 * tiling never changes a result: state, moments and histograms are the same bits. */
ABP_API abp_status abp_tiles(const abp_ctx *ctx, int32_t *n_tiles, int32_t *n_packed, int32_t *narrow);

/* Host-only planning, the logic abp_set_params applies (no device work, usable
 * without a GPU).  abp_plan: the tiling of a batch of n_sets sets (n_traj,
 * n_steps host arrays) for `schedule` (1 lockstep, 2 work queue),
 * particles_per_thread (1, 2, 4), adjoint checkpoints on (checkpoints != 0) or
 * off, on a device of sm_count SMs.  Outputs (host, any may be NULL): tiles in
 * all, packed tiles among them, narrow block width (0 if not narrow); and, when
 * max_tiles >= the tile count, every tile's first trajectory, trajectory count
 * and set (a packed tile: its first non-empty set).  A negative count or a
 * schedule / particles_per_thread out of range gives ABP_EINVAL.
 * abp_plan_efficiency: the fraction of `units` parallel units, each running one
 * tile of 256 * particles_per_thread trajectories at a time, that the batch keeps
 * busy, in particle-steps (lockstep: whole waves of tiles per window; work queue:
 * ceil(items / units) equal items when every tile has the same step count and
 * the items divide it, else the tile-steps spread over the units plus half an
 * item; never less than the longest tile).  The autotuner passes the SM count,
 * since one resident block already draws an SM's full integration rate, and
 * predicts a candidate's time on a batch as its trial time x the trial batch's
 * fraction / the batch's fraction (plus the state traffic and fixed costs of its
 * launches);  steps_per_launch = the lockstep window or the work queue's item
 * size, 0 = a window of about 2e10 particle-steps (lockstep) or the largest of
 * 10^5, 10^4, 10^3 steps that gives every unit 32 items (work queue). */
ABP_API abp_status abp_plan(int32_t n_sets, const int64_t *n_traj, const int64_t *n_steps, int32_t schedule,
                            int32_t particles_per_thread, int32_t checkpoints, int32_t sm_count, int32_t *n_tiles,
                            int32_t *n_packed, int32_t *narrow, int64_t *tile_first, int32_t *tile_count,
                            int32_t *tile_set, int32_t max_tiles);
ABP_API abp_status abp_plan_efficiency(int32_t n_sets, const int64_t *n_traj, const int64_t *n_steps,
                                       int32_t schedule, int32_t particles_per_thread, int32_t checkpoints,
                                       int64_t steps_per_launch, int64_t units, double *efficiency);

/* Number of kernels this context has enqueued since it was created (host output). */
ABP_API abp_status abp_kernel_launches(const abp_ctx *ctx, int64_t *launches);

/* Wait for the context's stream (and its live-result copies) and report any
 * device-side failure. */
ABP_API abp_status abp_synchronize(abp_ctx *ctx);

/* Release the context and every buffer it owns.  NULL is allowed. */
ABP_API void abp_destroy(abp_ctx *ctx);

/* Message of the last failed call on ctx ("" if none; static text if ctx is NULL). */
ABP_API const char *abp_last_error(const abp_ctx *ctx);

/* --- building blocks exposed for verification ---------------------------- */

/* Philox4x32-10 blocks on the device: out[i][0..3] = Philox(key = seed,
 * ctr = (m[i]_lo, m[i]_hi, traj[i]_lo, traj[i]_hi)).  traj, m: device arrays of
 * n uint64; out: device array of 4n uint32.  Runs on cuda_stream. */
ABP_API abp_status abp_philox(uint64_t seed, const uint64_t *traj, const uint64_t *m, int64_t n, uint32_t *out,
                      void *cuda_stream);

/* The FP32 standard normals z_k, k = n0 .. n0 + count - 1, that drive the steps
 * of trajectory traj (device output of count floats). */
ABP_API abp_status abp_normals(uint64_t seed, uint64_t traj, uint64_t n0, int64_t count, float *out,
                       void *cuda_stream);

/* The first `count` words of the xorshift stream of global trajectory `traj`
 * under `seed` (noise = 1), written to device memory out[count] on
 * cuda_stream: the verification entry of the xorshift option. */
ABP_API abp_status abp_xorshift(uint64_t seed, uint64_t traj, int64_t count, uint32_t *out, void *cuda_stream);

/* --- allocation-free entry point ------------------------------------------ */

/* The paper has no counterpart to this call; it serves callers that cannot
 * allocate device memory: code embedded in a host framework that owns all
 * device memory through its own pool and forbids cudaMalloc / cudaFree (both
 * also synchronise the device), or a latency-critical loop that must never
 * stall on an allocation.
 *
 * abp_run_set_noalloc integrates ONE parameter set (n_traj trajectories of
 * n_steps steps, configuration cfg; cfg->traj_base offsets the trajectory ids)
 * to completion and reduces it, exactly like abp_set_params + abp_integrate +
 * abp_reduce on a context, but allocates nothing: the trajectory state, tile
 * table and reduction partials live in one static device array of
 * ABP_NOALLOC_SCRATCH_BYTES bytes that every GPU which loads the library holds
 * until the process exits.  Limits: 0 <= n_traj <= ABP_NOALLOC_MAX_TRAJ, FP32
 * state only (state_fp64 = 0), no checkpoints (checkpoint_every = 0); anything
 * else returns ABP_EINVAL with a message in err (err_len bytes, may be NULL).
 * It runs the lockstep schedule (one block per tile, cfg->particles_per_thread
 * trajectories per thread, 0 meaning 1; never the narrow small-batch launch) in
 * launches of cfg->steps_per_launch steps (0: one launch); cfg->schedule must be
 * 0 or 1 (the work queue needs per-tile counters this call has no room for).
 * Outputs, all memory of the CURRENT device owned by the caller (host memory or
 * another GPU's memory is rejected): moments [8] doubles as in abp_reduce;
 * hist_x [n_snap][hist_x_bins] and hist_v [n_snap][hist_v_bins + 2] uint32
 * (required when their bins are > 0, zeroed by the call), n_snap as in
 * abp_num_snapshots for one set of n_steps steps.  The caller sizes them: the
 * call cannot see their extent.
 * The call only enqueues work on cuda_stream; results are ready when the stream
 * is.  The first call on a device looks up the array's device address (with
 * that device current) and keeps it for the life of the process; make that
 * first call before any stream capture, and do not use the call again on a
 * device after cudaDeviceReset (the array may then live at another address).
 * All calls share the one array, so calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller. */
#define ABP_NOALLOC_MAX_TRAJ 65536
#define ABP_NOALLOC_SCRATCH_BYTES 1848064
ABP_API abp_status abp_run_set_noalloc(const abp_params *params, const abp_config *cfg, int64_t n_traj,
                                       int64_t n_steps, double *moments, uint32_t *hist_x, uint32_t *hist_v,
                                       void *cuda_stream, char *err, size_t err_len);

/* Moments of an ensemble integrated in shards.  A batch may be split into
 * trajectory ranges run by several processes (one GPU each, abp_config.traj_base =
 * the global id of each range's first trajectory).  The averages of Sec. 2 over
 * noise realisations are sums over trajectories divided by their number, so adding
 * the per-set sums (columns 4..7 of abp_reduce) of all shards gives the sums of the
 * whole ensemble; this call then forms its moments:
 *   moments: [n_sets][8] doubles, host or device memory, read and written in place;
 *     on entry columns 4..7 hold the combined sums, on return columns 0..3 hold
 *     mean_v, se_v, msd and d_eff as abp_reduce defines them (bitwise the values
 *     abp_reduce gives for the same sums);
 *   n_traj, n_steps: host arrays of n_sets values -- the trajectories of set s in
 *     all shards together and the steps they have run; dt: the time step.
 * Device memory (of the current device) is processed by a kernel on cuda_stream
 * (the call returns at once; results are ready with the stream); host memory is
 * processed before the call returns and needs no GPU.  No context is needed.
 * ABP_EINVAL for n_sets < 0, NULL arrays, negative counts, dt not finite and > 0,
 * or moments in another GPU's memory. */
ABP_API abp_status abp_combine_moments(int32_t n_sets, double *moments, const int64_t *n_traj,
                                       const int64_t *n_steps, double dt, void *cuda_stream);

/* Library version string. */
ABP_API const char *abp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ABP_H */
