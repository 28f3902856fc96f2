/*
 * mlmc.h -- C ABI of the GB300 nested-MLMC level library (libmlmc_gb300.so).
 *
 * The library simulates, on one CUDA GPU, the per-sample coupled fine/coarse
 * Geometric Brownian Motion paths of one or more MLMC levels and reduces them
 * to per-level sums of Y and Y^2, as described in Haas & Giles, "A nested MLMC
 * framework for efficient simulations on FPGAs" (arXiv 2502.07123):
 *   - Sec. 2.1, eq. classic_MLMC_iden: level differences Y = P_l - P_{l-1}
 *     with fine and coarse paths driven by the same Normal increments;
 *   - Sec. 2.2, eq. chap:nested_exp: the nested split into an approximate
 *     level difference dP~_l and the correction dP_l - dP~_l;
 *   - Sec. 3: exact Normals Z = Phi^{-1}(U) and approximate Normals Z~ from a
 *     table indexed by the top d bits of the same uniform integer J;
 *   - Sec. 4.1, Algorithm 1: the low-precision path step in fixed point.
 *
 * Conventions for every entry point:
 *   - Host pointers are caller-owned and only read or written during the call.
 *     Pointers documented as "device" must point to CUDA device memory of the
 *     current device that stays valid until the enqueued work has finished.
 *   - Every call returns an mlmc_status; no call aborts the process.  On an
 *     error the output arguments are left unspecified.
 *   - Sums are of discounted sample values: the factor exp(-rT) is applied.
 *   - A `void *stream` argument is a cudaStream_t (NULL = legacy default stream).
 *   - The library allocates its own device memory (tables, work lists, scratch)
 *     lazily on the current CUDA device and keeps it until process exit.
 *   - Calls may come from several host threads: the entry points that use the
 *     library's shared state (context, tables, caches, engines) take one
 *     process-wide lock, so such calls run one at a time (a call that waits
 *     for the GPU, like mlmc_engine_step, holds it while it waits).
 *   - There is no CPU fallback: without a usable CUDA device every compute
 *     entry point returns MLMC_ECUDA.
 */
#ifndef MLMC_GB300_H
#define MLMC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MLMC_OK = 0,
  MLMC_EINVAL = 1,     /* an argument is out of range or inconsistent        */
  MLMC_ENOMEM = 2,     /* a device or host allocation failed                 */
  MLMC_ECUDA = 3,      /* a CUDA runtime call failed (or no device)          */
  MLMC_ETIMEOUT = 4,   /* a bounded wait ran out                             */
  MLMC_EOVERFLOW = 5,  /* a constant does not fit its fixed-point format     */
  MLMC_ENOTREADY = 6   /* results requested before the work was launched     */
} mlmc_status;

typedef enum { MLMC_EULER = 0, MLMC_MILSTEIN = 1 } mlmc_scheme;

/* Payoffs (undiscounted form; the library discounts the sums):
 *   EURO     max(S_N - K, 0)
 *   DIGITAL  1[S_N > K]
 *   ASIAN    max(A - K, 0), A = trapezoidal time average on the path's own grid
 *   LOOKBACK S_N - min_i S_i (floating-strike call, minimum over the path's grid) */
typedef enum { MLMC_EURO = 0, MLMC_DIGITAL = 1, MLMC_ASIAN = 2, MLMC_LOOKBACK = 3 } mlmc_payoff;

/* Estimator variants.  "EXACT" = plain level difference dP_l with exact Normals
 * (Sec. 2.1); "APPROX" = dP~_l with approximate Normals and low-precision
 * arithmetic (eq. GBM_sde_fi); "NESTED_CORR" = dP_l - dP~_l on shared uniforms
 * (eq. chap:nested_exp), exact part in FP32. */
typedef enum {
  MLMC_FP64_EXACT = 0,
  MLMC_FP32_EXACT = 1,
  MLMC_FP16_APPROX = 2,
  MLMC_BF16_APPROX = 3,
  MLMC_FIXED_APPROX = 4,
  MLMC_NESTED_CORR_FIXED = 5,
  MLMC_NESTED_CORR_FP16 = 6,
  MLMC_NESTED_CORR_BF16 = 7,
  /* binary16 / bfloat16 increments (one rounding per operation, as above)
   * with S, its running average and minimum in FP32: mul2 = fl32(S sum1),
   * S = fl32(S + mul2) */
  MLMC_FP16S_APPROX = 8,
  MLMC_BF16S_APPROX = 9,
  MLMC_NESTED_CORR_FP16S = 10,
  MLMC_NESTED_CORR_BF16S = 11
} mlmc_variant;

/* Fixed-point format of the Algorithm-1 variables on one level (Sec. 4.1):
 * value = n 2^-f[i], |n| <= 2^(e[i]+f[i]) - 1, i in the order
 * {Z~, con1, con2, mul1, sum1, mul2, S}.  The GPU path requires
 * e+f <= 31 for the first five and e+f <= 62 for mul2 and S, and that every
 * exact product and alignment fits 62 bits (checked; MLMC_EINVAL otherwise). */
typedef struct {
  int8_t e[7];
  int8_t f[7];
} mlmc_format;

typedef struct {
  double S0, K, r, sigma, T;    /* GBM dS = r S dt + sigma S dW, maturity T      */
  int32_t payoff;               /* mlmc_payoff                                   */
  int32_t scheme;               /* mlmc_scheme                                   */
  int32_t icdf_method;          /* 1: piecewise constant on uniform intervals (Sec. 3.1);
                                   2: sum of n table variables of d/n bits with the
                                      least-squares / permutation optimisation (Sec. 3.2;
                                      n = icdf_fields); the correction estimators' exact
                                      path then uses the uniform in interval pi(j),
                                      U = 2^-d pi(j) + 2^-32 ((J mod 2^(32-d)) + 1/2);
                                   3: piecewise linear on dyadic intervals (Sec. 3.3) */
  int32_t icdf_bits;            /* d in [2, 14]: bits of J used by the table      */
  const mlmc_format *formats;   /* host array indexed by level, or NULL for the
                                   library's default schedule (mlmc_default_format) */
  int32_t n_formats;            /* entries in formats                            */
  uint32_t request_id;          /* enters the Philox counter (independent streams) */
  int32_t rng_pack;             /* 1: approximate-only estimators read 3 table indices
                                   from each 32-bit Philox word (d = 9 or 10 only):
                                   sample s = 3P + L takes bits [32-d(L+1), 32-dL) of
                                   the word its pack P reads at each step; 0: one word
                                   per step.  Ignored by exact and correction estimators,
                                   which need all 32 bits of J (Sec. 3.1 coupling). */
  int32_t icdf_fields;          /* Method 2: n, the number of fields (0 means 2); n
                                   divides d with at least 2 bits per field.  Must be 0
                                   for methods 1 and 3. */
} mlmc_params;

/* Per-level result.  sum/sum2 are discounted FP64 sums of Y and Y^2.  When
 * exact_int is 1 (approximate-only estimators, whose samples are integers)
 * isum and isum2 hold the exact undiscounted integer sums in units 2^-unit
 * and 2^-2unit; sum = exp(-rT) 2^-unit isum rounded once. */
typedef struct {
  double sum, sum2;
  uint64_t n;
  double seconds;               /* device time of the launch that produced it    */
  uint64_t saturations;         /* samples on which a fixed-point value saturated */
  int64_t isum;
  uint64_t isum2_lo, isum2_hi;
  int32_t unit, exact_int;
} mlmc_sums;

/* One simulated sample, written by mlmc_level_dump (for parity testing). */
typedef struct {
  double pf, pc;     /* exact-path payoffs (undiscounted); pc = 0 on level 0   */
  double sf, sc;     /* exact-path terminal values                             */
  double af, ac;     /* approximate-path terminal values                       */
  int64_t qf, qc;    /* approximate-path payoffs, integers in units 2^-unit    */
  double y;          /* the sample value accumulated into the sums (undiscounted) */
  uint32_t sat, pad; /* sat = 1 if a fixed-point value saturated              */
} mlmc_sample;

/* Chunking of the level kernels.  threads: CTA size (32..128, multiple of 32);
 * steps_per_thread: target fine path-steps per thread (>= 1); zero = the
 * library's launch-shape table (128 / 256 unless mlmc_autotune changed it). */
typedef struct {
  int32_t threads;
  int32_t steps_per_thread;
} mlmc_tuning;

/* One unit of work: samples [first_sample, first_sample + N) of one level. */
typedef struct {
  const mlmc_params *params;    /* host pointer, copied at plan creation         */
  int32_t level;                /* l in [0, 20]: 2^l fine steps of size T 2^-l   */
  int32_t variant;              /* mlmc_variant                                  */
  uint64_t first_sample;
  uint64_t N;
  int32_t stream;               /* Philox stream id 0..255, or -1 for the default
                                   (1 for APPROX variants, 0 otherwise)          */
  int32_t flags;                /* bit 0 (MLMC_WORK_ENUMERATE): instead of random
                                   draws, sample s of an approximate-only estimator
                                   on level 0 or 1 takes table index
                                   j_i = (s >> (d i)) mod 2^d at fine step i, so
                                   samples [0, 2^(d 2^l)) cover every combination of
                                   table cells once and their mean is E[dP~_l]
                                   exactly; needs first_sample = 0 and
                                   N = 2^(d 2^l) <= 2^24 */
} mlmc_work;
#define MLMC_WORK_ENUMERATE 1

typedef struct mlmc_plan mlmc_plan;

/* ---- single level (Sec. 2.1 / 2.2 level estimator) ----------------------
 * Simulates samples [first_sample, first_sample + N) of `level` with variant v
 * and writes their sums to *out (host).  Blocks until the result is on the host.
 * Sample s, fine step i draws J = word (w mod 4) of Philox4x32-10 with key
 * (seed_lo, seed_hi) and counter (q_lo, q_hi, level | stream << 8, request_id),
 * w = s 2^level + i, q = w div 4.  N = 0 gives zero sums.
 * Errors: MLMC_EINVAL (bad level/variant/params/formats), MLMC_EOVERFLOW (a
 * constant outside its format), MLMC_ECUDA, MLMC_ENOMEM. */
mlmc_status mlmc_level(int level, uint64_t N, const mlmc_params *p, mlmc_variant v,
                       uint64_t seed, uint64_t first_sample, mlmc_sums *out);

/* As mlmc_level, with an explicit Philox stream (-1 = default), and also writes
 * every sample to d_samples (device array of N mlmc_sample, caller-owned). */
mlmc_status mlmc_level_dump(int level, uint64_t N, const mlmc_params *p, mlmc_variant v,
                            uint64_t seed, uint64_t first_sample, int32_t stream,
                            mlmc_sample *d_samples, mlmc_sums *out);

/* ---- single level without device allocation -------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * must not allocate device memory while they run: a process whose device
 * memory is owned by another allocator (a framework's caching pool, or memory
 * reserved up front), a latency-critical loop in which a cudaMalloc would
 * synchronise the device, or code whose memory budget has been fixed ahead.
 * It computes exactly what mlmc_level computes: the work item is built and
 * chunked by the same code (same kernels, chunking and packed-draw layout,
 * hence the same sums), and it calls no cudaMalloc, cudaFree or other
 * allocating routine.  Its scratch (per-CTA partial sums, the work item, the
 * tables and the result record) is one file-scope device array of about
 * 0.9 MiB that every GPU which loads the library keeps until exit; its device
 * address is looked up on every call.  CUDA loads a kernel's code on its first
 * launch on a device (lazy module loading), which takes device memory once:
 * a caller that must see no change at all makes one call of each kind of
 * estimator up front.  The first call for each table size d also reads the
 * FP64 table back to the host, which synchronises the stream midway.
 * Limits: at most 16384 CTAs per call -- larger sample counts return
 * MLMC_EINVAL; icdf_bits <= 14; icdf_method 1 or 3 (Method 2's tables are
 * built on the host and need allocation: MLMC_EINVAL).  All work is enqueued
 * on `stream` (a cudaStream_t, NULL = legacy default stream) and the call
 * returns after synchronising it; seconds = 0.  Every call writes every part
 * of the array that it reads, and calls are serialised by the library lock
 * and each returns after its stream has finished, so they cannot overlap on
 * the GPU.  Errors as mlmc_level. */
mlmc_status mlmc_level_noalloc(int level, uint64_t N, const mlmc_params *p, mlmc_variant v,
                               uint64_t seed, uint64_t first_sample, mlmc_sums *out, void *stream);

/* ---- batched work lists ---------------------------------------------------
 * A plan holds a device-resident work list; launching it enqueues one level
 * kernel per kernel configuration (concurrently, on forked streams joined
 * back to `stream`; in each, the CTA that finishes an item's last chunk sums
 * the item's chunk partials in chunk order), with no host synchronisation and
 * no host <-> device copy.  Results stay on the device until mlmc_plan_results.
 * Work items are simulated in order of decreasing cost per CTA.
 * Errors as mlmc_level; a plan with n_work = 0 is MLMC_EINVAL. */
mlmc_status mlmc_plan_create(mlmc_plan **plan, const mlmc_work *work, int n_work,
                             uint64_t seed, const mlmc_tuning *tuning);
mlmc_status mlmc_plan_launch(mlmc_plan *plan, void *stream);
/* Synchronises with the last launch and copies one mlmc_sums per work item
 * (host array of n_work).  seconds = device time of the last launch.
 * MLMC_ENOTREADY if the plan was never launched. */
mlmc_status mlmc_plan_results(mlmc_plan *plan, mlmc_sums *out);
/* Number of level-kernel launches and CTAs one launch of the plan issues, the
 * fine path-steps it simulates (sum of N 2^level), and the bytes the plan
 * copies host->device at creation and device->host per mlmc_plan_results.
 * Any output pointer may be NULL. */
mlmc_status mlmc_plan_info(const mlmc_plan *plan, int *kernels, uint64_t *ctas,
                           uint64_t *path_steps, uint64_t *h2d_bytes, uint64_t *d2h_bytes);
/* Device time (ms, CUDA events on the kernel's own stream) of level kernel k of
 * the last launch, and its family (0 exact FP32, 1 exact FP64, 2 approximate
 * fixed, 3 approximate binary16, 4 approximate bfloat16, 5/6/7 correction with
 * fixed / binary16 / bfloat16; 8-16 the same estimators' other datapaths
 * (fast fixed point, packed draws), 17 the merged nested launch (24: the same
 * with the pre-scaled product, when every item's increment fits it), 18-23
 * binary16 / bfloat16 with FP32 S: approximate 18 / 19, correction 20 / 21,
 * approximate with packed draws 22 / 23).  Waits for that kernel.  MLMC_ENOTREADY before
 * the first launch, MLMC_EINVAL for k out of range. */
mlmc_status mlmc_plan_kernel_time(const mlmc_plan *plan, int k, int *family, double *ms);
/* Device time (ms) of the whole last launch of the plan: CUDA events recorded
 * on the launch stream right before its first kernel and after its last one
 * (joined streams included); for a one-kernel plan, the same events as
 * mlmc_plan_kernel_time(plan, 0).  Waits for the launch.  MLMC_ENOTREADY
 * before the first launch, MLMC_EINVAL for a NULL plan or ms. */
mlmc_status mlmc_plan_elapsed(const mlmc_plan *plan, double *ms);
/* Level-kernel launch k of the plan (0 <= k < kernels of mlmc_plan_info):
 * its kernel family, work items, CTAs and fine path-steps (sum of N 2^l over
 * its items); any output may be NULL.  MLMC_EINVAL for k out of range. */
mlmc_status mlmc_plan_launch_info(const mlmc_plan *plan, int k, int *family, int *items, uint64_t *ctas,
                                  uint64_t *path_steps);
/* Work items of level-kernel launch k: their positions in the work list given
 * to mlmc_plan_create, in launch order, written to work_index (host array of
 * cap entries; at most cap are written) and their number to *n.  MLMC_EINVAL
 * for k out of range, a NULL n, or cap > 0 with a NULL work_index. */
mlmc_status mlmc_plan_launch_items(const mlmc_plan *plan, int k, int32_t *work_index, int cap, int *n);
void mlmc_plan_destroy(mlmc_plan *plan);

/* Host-buffer convenience: create, launch on `stream`, read results, destroy. */
mlmc_status mlmc_run(const mlmc_work *work, int n_work, uint64_t seed,
                     const mlmc_tuning *tuning, mlmc_sums *out, void *stream);

/* ---- launch-shape autotuner ----------------------------------------------
 * The level kernels' launch shape (CTA threads; fine path-steps, hence paths,
 * per thread) is chosen per kernel class: (kernel family, scheme, payoff class,
 * level class {0}, {1}, {2..4}, {5..7}, {>= 8}).  mlmc_autotune runs one
 * pass of coordinate descent over the classes present in `work` (largest
 * model work first): each class in turn tries every distinct chunking from
 * threads {128, 96, 64} x steps_per_thread {256, 64, 128, 512, 1024, 2048}
 * while the other classes keep their shapes, timing the whole work list as
 * one plan (median of `reps` launches by CUDA events, after one untimed
 * launch; a candidate must beat the best so far by 2%), and installs the
 * fastest in the process-wide table that every later call without an
 * mlmc_tuning uses (plans, mlmc_run, mlmc_level, mlmc_level_noalloc,
 * mlmc_estimate, engine admissions).  chosen (host, n_work entries, or NULL)
 * receives each item's shape.  The shape changes the chunking only: integer
 * sums are unchanged, FP32 sums may change in their last bits.  Synchronous;
 * runs the work (1 + reps) times per candidate.  Errors as mlmc_plan_create,
 * MLMC_EINVAL for reps outside [1, 1000]. */
mlmc_status mlmc_autotune(const mlmc_work *work, int n_work, uint64_t seed, int reps, mlmc_tuning *chosen);
/* Restore the default shape (128 threads, 256 path-steps per thread) for every class. */
void mlmc_tuning_reset(void);

/* ---- adaptive MLMC (Sec. 2.1-2.2 sample allocation, on-line phase of Sec. 6) ----
 * Estimates E[P] to root-mean-square error eps with the adaptive algorithm of
 * Giles (2008): variance target eps^2/2, bias target eps/sqrt(2), weak order 1,
 * L from 2 up to max_level, 10^4 initial samples per level and estimator,
 * sample counts N = ceil(lambda sqrt(V/C)) with lambda = (eps^2/2)^-1 sum sqrt(V C)
 * over every (level, estimator) term.  Each round runs every term's pending
 * samples and recomputes the counts; once every remaining top-up is at most
 * 1% of its term's samples (the form of the loop in Giles 2015) the bias test
 * runs, and a new level's first samples run in the same round as those
 * top-ups; the result is returned when nothing is pending and the bias test
 * passed or L = max_level.  mode: 0 plain FP64, 1 plain FP32,
 * 2 nested fixed point, 3 nested binary16, 4 nested bfloat16, 7 and 8 nested
 * binary16 / bfloat16 increments with S in FP32; 5, 6, 9 and 10 nested
 * fixed point / binary16 / binary16 with FP32 S / bfloat16 with FP32 S whose
 * approximate terms on levels 0 and 1 (when
 * d 2^l <= 20) are computed exactly, by enumerating the 2^(d 2^l) combinations
 * of table cells (MLMC_WORK_ENUMERATE), and then carry no variance and take no
 * further samples (the approximate Normal has finitely many values; the
 * corrections stay Monte Carlo).  The cost model
 * is C = 2^l c_kind with c_kind from mlmc_cost_model (deterministic).
 * Outputs (host): *price, *stderr_out, *L; N_l[l * 2 + k] = samples of
 * estimator k on level l (k = 0: plain or approximate, k = 1: correction), for
 * l <= *L (caller array of 2 * cap_levels).  Errors as mlmc_level, MLMC_EINVAL
 * if cap_levels <= max_level, MLMC_ETIMEOUT after 100000 rounds. */
mlmc_status mlmc_estimate(double eps, const mlmc_params *p, int mode, uint64_t seed,
                          int max_level, double *price, double *stderr_out, int *L,
                          uint64_t *N_l, int cap_levels);

/* ---- continuous-batching engine (many adaptive requests per launch) --------
 * Requests (params, eps, mode, seed) queue on submit and are admitted into free
 * slots; each slot keeps its adaptive state (sums of Y and Y^2, sample counts,
 * pending counts per level and estimator) in FP64 in device memory, with one
 * work-item template per (level, estimator) built at admission.  One engine
 * iteration is device work only: a scheduler kernel chunks every active
 * slot's pending (level, estimator) work and groups it by launch class, one
 * persistent level-kernel launch per class runs it (fixed grid of resident
 * CTAs, chunks taken in turn), an accumulate kernel adds each item's sums to
 * its slot in chunk order, and a decide kernel recomputes level variances,
 * N = ceil(lambda sqrt(V/C)) (Sec. 2.1 / 2.2), the bias test, a new level or
 * completion -- the same algorithm and arithmetic as mlmc_estimate, so a
 * request's result is the same whatever else runs beside it.  The iteration
 * is captured once as a CUDA graph (again when a new launch class appears)
 * and replayed; mlmc_engine_step admits waiting requests (host), launches the
 * graph once (iters_per_launch iterations), waits for it and retires
 * completed requests.  Slots are limited by max_slots and by
 * device_bytes_budget (0 = no budget): a slot needs its state, templates and
 * work-list space, about 30 KB at max_level 10.  The per-chunk partial array
 * (48 bytes a chunk) starts at max(4 chunks per template, 65536) and grows
 * when an iteration needs more.
 * Requests that share a seed must have distinct request_id values in their
 * params.  Errors: MLMC_EINVAL for bad arguments (params->formats, when
 * given, must cover levels 0..max_level), MLMC_ENOMEM, MLMC_ECUDA; a request
 * that cannot be admitted (for instance a format its constants do not fit,
 * or more than 32 launch classes among the requests holding slots) completes
 * with that status from
 * mlmc_engine_poll and a NaN price. */
typedef struct {
  int32_t max_slots;             /* concurrent requests (0 = 256)                 */
  int32_t max_level;             /* L_max of every request, 2..20                 */
  uint64_t device_bytes_budget;  /* bytes of per-slot device memory, 0 = any      */
  int32_t iters_per_launch;      /* engine iterations per graph launch, 1..64 (0 = 1);
                                    -n (n <= 4096): one launch iterates on the device
                                    (a conditional WHILE graph node) until no admitted
                                    request is left running, at most n iterations */
  int32_t reserved;              /* must be 0 */
} mlmc_engine_config;
typedef struct mlmc_engine mlmc_engine;
mlmc_status mlmc_engine_create(mlmc_engine **e, const mlmc_engine_config *cfg);
/* Copies *p (and its format table); mode as mlmc_estimate. */
mlmc_status mlmc_engine_submit(mlmc_engine *e, const mlmc_params *p, double eps, int mode, uint64_t seed,
                               uint64_t *req_id);
/* One graph launch on `stream` (synchronous; NULL = the default stream); with
 * a negative iters_per_launch the launch runs until every request admitted
 * by this step has completed (or the partial array must grow, or the
 * iteration cap is reached), so requests submitted meanwhile wait for the
 * next step.
 * *active = requests holding a slot after the step, *queued = requests
 * waiting for one (either may be NULL). */
mlmc_status mlmc_engine_step(mlmc_engine *e, void *stream, int *active, int *queued);
/* *done = 1 once the request has completed; then price, standard error, final
 * level and latency (seconds from submit to completion) are filled in.
 * Returns the request's status (MLMC_OK unless its admission failed). */
mlmc_status mlmc_engine_poll(mlmc_engine *e, uint64_t req_id, double *price, double *stderr_out, int *L,
                             int *done, double *latency_s);
/* Drains the ids of requests that completed since the last call, in the order
 * they completed (admission failures included): up to cap ids into the host
 * array ids, their count in *n; the rest stay queued for the next call.  A
 * serving loop reads only what finished instead of polling every request;
 * mlmc_engine_poll still answers for any id.  MLMC_EINVAL for a NULL engine
 * or n, a negative cap, or cap > 0 with ids NULL. */
mlmc_status mlmc_engine_completed(mlmc_engine *e, uint64_t *ids, int cap, int *n);
/* The schedule and bias test of a completed request: N_l[l * 2 + k] = samples
 * of estimator k on level l (k = 0: plain or approximate, k = 1: correction;
 * host array of 2 * cap_levels, zero beyond the final level L) and
 * *bias_estimate (may be NULL) = the remaining-bias estimate of the final
 * bias test, max(|m_L|, |m_{L-1}| / 2) with the level means floored as in
 * mlmc_estimate; a request that stopped at max_level with this above
 * eps / sqrt(2) did not reach its bias target.  MLMC_ENOTREADY before the
 * request has completed; a request whose admission failed returns its status. */
mlmc_status mlmc_engine_request_info(mlmc_engine *e, uint64_t req_id, uint64_t *N_l, int cap_levels,
                                     double *bias_estimate);
/* Engine counters: steps taken, graph launches, fine path-steps simulated, slots. */
mlmc_status mlmc_engine_stats(const mlmc_engine *e, uint64_t *steps, uint64_t *launches,
                              uint64_t *path_steps, int *slots);
/* Captured iteration: launch classes in the graph, captures so far,
 * iterations per launch, partial-array capacity in chunks (any may be NULL). */
mlmc_status mlmc_engine_graph_info(const mlmc_engine *e, int *groups, int *captures, int *iters_per_launch,
                                   uint64_t *partial_capacity);
void mlmc_engine_destroy(mlmc_engine *e);

/* Batched adaptive MLMC: n independent requests (params[i], eps[i]), all in
 * `mode` with `seed` (distinct params[i].request_id), run to completion in one
 * engine of n slots: every graph launch covers iters_per_launch iterations of
 * all requests (negative: the whole run in one launch, a device-side loop;
 * see mlmc_engine_config).  Outputs (host arrays of n; stderr_out and L may be NULL):
 * price, standard error, final level; *launches = graph launches (may be
 * NULL).  Each result equals what mlmc_estimate returns for that request.
 * Errors as the engine functions; MLMC_ETIMEOUT after 100000 launches. */
mlmc_status mlmc_batch_estimate(const mlmc_params *params, const double *eps, int n, int mode, uint64_t seed,
                                int max_level, int iters_per_launch, double *price, double *stderr_out, int *L,
                                int *launches, void *stream);

/* ---- error model and bit-width optimisation (Sec. 4-6) ----------------------
 * mlmc_sensitivities: statistics of the level difference DeltaP_l = P_f - P_c
 * (discounted European call, Euler-Maruyama, exact FP64 Normals from the
 * correction estimator's uniforms, stream 0) for samples [first_sample,
 * first_sample + N), with every intermediate variable of Algorithm 1 -- con1
 * (and the coarse constant r 2h), con2, Z_j, mul1_k, sum1_k, mul2_k, S_k on the
 * fine and coarse path, and S0 -- as an instance whose sensitivity
 * xbar = d DeltaP / d x is computed by adjoint (algorithmic) differentiation:
 *   A[t]      = E[sum over the instances of type t of xbar^2]  (V_indep, eq. optimistic)
 *   B[t]      = sum over the instances of sqrt(E[xbar^2])      (V_corr, eq. pessimistic)
 *   maxabs[t] = max |x| over instances and samples            (exponents, Sec. 4.1)
 *   mean, var = of DeltaP_l;  n_instances = 2^l + 2^(l-1) + 1 (l >= 1; 2 on level 0).
 * Type order t: Z, con1, con2, mul1, sum1, mul2, S (the mlmc_format order).
 * inst (host, 7 x n_instances doubles, type-major, or NULL) receives E[xbar^2]
 * per instance: mul1 / sum1 / mul2: fine step k at k, coarse step k at
 * 2^l + k; S: S_{k+1} fine at k, coarse at 2^l + k, S0 last; Z: Z_j at j;
 * con1: fine 0, coarse 1; con2: 0.  level 0..10, European payoff and Euler
 * scheme only (MLMC_EINVAL otherwise).  Synchronous; allocates scratch. */
typedef struct {
  double A[7];
  double B[7];
  double maxabs[7];
  double mean, var;
  uint64_t n;
  int32_t n_instances;
  int32_t reserved;
} mlmc_sensitivity;
mlmc_status mlmc_sensitivities(int level, uint64_t N, const mlmc_params *p, uint64_t seed,
                               uint64_t first_sample, mlmc_sensitivity *out, double *inst);

/* mlmc_optimise_level: optimal bit-widths of one level (host only, no GPU).
 * Minimises the level cost sqrt(V C~(d)) + sqrt(V_indep(d) C) (eq.
 * level_cost2) with V = s->var, C = 2^l c_rng, C~(d) = steps (1/2 sum M_t
 * d_t^2 + sum M'_t d_t) (eq. cost_sq, steps = fine + coarse steps): for a
 * Lagrange multiplier lambda every d_t solves (ln 4 / 12) A_t 4^(e_t - d_t) =
 * lambda steps (M_t d_t + M'_t) (eq. Lagr), and a golden-section search over
 * log(lambda) finds the optimum (Sec. 6.1); the real widths are then rounded
 * down and bits added greedily by variance decrease per unit cost until
 * V_indep is back at or below the real solution's (Sec. 6.2).  e_t is the
 * smallest integer with maxabs_t < 2^e_t.  With cfg->lut_mse (MSE of the
 * approximate Normal for table bits d, indexed by d) the smallest d_lut in
 * [2, lut_max_bits] with A_Z MSE(d_lut) <= V_indep is chosen (Sec. 4.3). */
typedef struct {
  double c_rng;              /* cost of one full-precision path-step; <= 0: 1e4 (Sec. 6.1) */
  double mul[7], add[7];     /* M_t, M'_t per time step; all zero: Algorithm 1's counts */
  const double *lut_mse;     /* host array indexed by table bits, or NULL */
  int32_t lut_max_bits;      /* 0: 16 */
  int32_t reserved;
} mlmc_opt_config;
typedef struct {
  int32_t e[7];              /* exponents */
  int32_t d[7];              /* integer bit-widths */
  double d_real[7];          /* real solution */
  double lambda;
  double v_indep, v_indep_real, v_corr;
  double cost_lp, cost_exact;
  double level_cost_ratio;   /* sqrt(C~/C) + sqrt(V_indep/V) (the paper's Fig. 5 quantity) */
  double mse_term;           /* A_Z MSE(lut_bits) */
  int32_t lut_bits;          /* 0: not chosen */
  int32_t reserved;
  mlmc_format format;        /* e and f = max(0, d - e), ready for mlmc_params.formats */
} mlmc_opt_result;
mlmc_status mlmc_optimise_level(int level, const mlmc_sensitivity *s, const mlmc_opt_config *cfg,
                                mlmc_opt_result *out);

/* Cost per fine path-step of each estimator kind used by mlmc_estimate
 * (relative units; defaults: exact FP32 1.0, exact FP64 8.0, approximate 0.5,
 * correction 1.5).  kind: 0 exact FP64, 1 exact FP32, 2 approximate, 3 correction.
 * Setting a value <= 0 restores the default.  Host only; no GPU needed. */
mlmc_status mlmc_cost_model(int kind, double cost_per_step);

/* ---- host helpers (no GPU needed) ---------------------------------------- */
/* The default fixed-point schedule for a level (used when params->formats is NULL).
 * Fractional bits f = {12, 16+l, 14+l, 12+l, 12+l, 12+l, 14+l} clamped to [10, 24]
 * (one more bit per level, Sec. 6.3), then f_S capped at 21 and f_mul2 at f_S,
 * and where e_S + f_S would exceed 30, f_S = max(10, 30 - e_S) (e_S then
 * recomputed).  Integer bits e are the smallest with
 * |x| < 2^e (and e + f >= 1) for these bounds, h = T 2^-l (for con1, con2 and
 * S, whose bounds include rounded constants: x + 2^-(f+1) < 2^e):
 *   Z~ 8;  con1 max(|r| 2h, sigma^2 h / 2);  con2 sigma sqrt(h);
 *   mul1 M = max(16 sigma sqrt(h), 128 sigma^2 h);  sum1 |r| 2h + M;
 *   S max(S0 exp(|r| T + 6 sigma sqrt(T)), K);  mul2 e_S + e_sum1. */
mlmc_status mlmc_default_format(const mlmc_params *p, int level, mlmc_format *out);

/* Approximate-Normal table built on the GPU (for parity testing): writes the
 * value of every index k < 2^(d-1) as doubles (host array of 2^(d-1)).
 * rep: 0 fp64, 1 fp32, 2 fp16, 3 bf16, 4 fixed with fZ fractional bits.
 * method 3 values are the a + b k evaluations the kernels use. */
mlmc_status mlmc_icdf_table(int method, int d, int rep, int fZ, double *out);
/* Method 2 (Sec. 3.2) with n fields (0 means 2) of b = d/n bits, the first
 * field the top bits of j: the optimised small table x (host array of
 * 2^(b-1) doubles, or NULL), the interval rank pi(j) of every j < 2^d (host
 * array of 2^d, or NULL) and the number of least-squares fits made.  Z~_j is
 * sum_k c_k x_k, c_k the net count of +x_k minus -x_k among j's fields (the
 * Method-1 sign rule per field), over the nonzero c_k in ascending k.  The
 * small table starts as the b-bit Method-1 table / sqrt(n); each fit solves the
 * normal equations for sum_j (Z_{pi(j)} - Z~_j)^2 with Z_k the d-bit Method-1
 * values, then the 2^d sums are ranked again (ascending, ties by j); the fits
 * stop when pi equals the previous or any earlier permutation (for n > 2 the
 * iteration can alternate between permutations), at most 1000.  MLMC_EINVAL
 * unless n divides d, d/n >= 2 and d <= 14. */
mlmc_status mlmc_icdf_method2(int d, int n, double *x, uint32_t *perm, int *iterations);
/* Method-2 values of every index k < 2^(d-1) in a representation (as
 * mlmc_icdf_table): each x rounded once, then sum_k c_k x_k exactly (fixed
 * point, fZ fractional bits) or with one rounding per product and per
 * addition (fp32 / fp16 / bf16); rep 0 gives the FP64 sums.  mlmc_icdf_table
 * with method 2 is this with n = 2. */
mlmc_status mlmc_icdf_method2_table(int d, int n, int rep, int fZ, double *out);

/* The FP32 exact Normal of the level kernels (Sec. 3.1): z[i] = Phi^{-1}(u_i),
 * u_i = 2^-32 (J[i] + 1/2), as every FP32 exact path and correction estimator
 * computes it -- the upper half folded by Phi^{-1}(1 - u) = -Phi^{-1}(u), then
 * a cubic in each of 512 parts of (0, 1/2) (the float's exponent and top four
 * significand bits; coefficients fitted in FP64).  Error about 1e-7 (1 + |z|).
 * J and z are device arrays of n elements (caller-owned); the call enqueues on
 * `stream` (NULL = legacy default stream) and returns after synchronising it.
 * MLMC_EINVAL for a NULL array with n > 0; MLMC_ECUDA on a CUDA error. */
mlmc_status mlmc_exact_normal_f32(const uint32_t *J, float *z, uint64_t n, void *stream);

/* Mean square error E[(Z - Z~)^2] of the approximate Normal with d table bits
 * (Sec. 3.4, eq. mse_dyadic), from the library's FP64 Method-1 table Z_k (the
 * mean of Phi^{-1} over interval k, built on the GPU):
 *   method 1: 1 - 2^(1-d) sum_{k < 2^(d-1)} Z_k^2;
 *   method 3: the Method-1 value plus 2^(1-d) sum_k (a_c + b_c k - Z_k)^2 with
 *             the FP64 least-squares lines of the dyadic classes;
 *   method 2: the Method-1 value plus 2^-d sum_{j < 2^d} (Z_pi(j) - Z~_j)^2 for
 *             the coupled uniform drawn in interval pi(j) (fields n, 0 means 2).
 * fields must be 0 for methods 1 and 3.  *out (host) receives the MSE.
 * MLMC_EINVAL for d outside [2, 14] or a bad method / field count;
 * MLMC_ECUDA without a GPU. */
mlmc_status mlmc_icdf_mse(int method, int d, int fields, double *out);

/* Philox4x32-10 words computed on the GPU for n counters (for parity testing):
 * ctr is a host array of 4n words, out a host array of 4n words. */
mlmc_status mlmc_philox(const uint32_t *ctr, uint64_t n, uint64_t seed, uint32_t *out);

/* Human-readable message of a status (static string). */
const char *mlmc_strerror(mlmc_status s);

/* Library version string (static). */
const char *mlmc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MLMC_GB300_H */
