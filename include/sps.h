/*
 * sps.h -- C ABI of the B300 (sm_103a) sequential posterior simulator for logit models.
 *
 * The method is the sequential posterior simulator (SPS) of Geweke, Durham & Xu (2013),
 * "Bayesian Inference for Logistic Regression Models using Sequential Posterior Simulation":
 * J groups of N particles are moved through the data in cycles, each a correction (C) phase
 * that reweights particles by the likelihood of new observations, a selection (S) phase that
 * resamples within each group, and a mutation (M) phase of Metropolis steps (Algorithms 1-2,
 * Sec. 2.2-2.3). The model is the multinomial logit of Eq. (1) with base outcome 0 (theta_0 = 0).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every call returns sps_status; none aborts, traps or prints. sps_last_error(ctx) keeps a
 *   message for the last failure on that context.
 * - The caller owns every buffer it passes. sps_init copies and encodes X and y to the device;
 *   the context owns its device memory until sps_destroy.
 * - Parameter vectors are FP64 and class-major: theta[p*D + (c-1)*k + i] is the coefficient of
 *   covariate i for outcome c (c = 1..C-1) of particle p; D = k*(C-1).
 * - Pointers marked "mem" are host pointers when mem == SPS_MEM_HOST (the call copies, runs and
 *   synchronises before returning) or device pointers when mem == SPS_MEM_DEVICE (the call only
 *   enqueues work on the context's stream and returns; results are ready when that stream is).
 * - One context per stream; calls on one context must not run concurrently from several host
 *   threads.
 * - Library errors: SPS_ERR_INVALID_ARG for shapes, ranges or non-finite inputs;
 *   SPS_ERR_CUDA for a failed CUDA runtime call or kernel launch (the CUDA error string is kept);
 *   SPS_ERR_OOM when device memory cannot be allocated; SPS_ERR_DEGENERATE when the proposal
 *   covariance h*V is not positive definite (the failure of Algorithm 2 step 2(c)i described in
 *   Sec. 4.2) or all of a group's resampling weights vanish; SPS_ERR_NONFINITE when a
 *   log-likelihood is not finite; SPS_ERR_TIMEOUT when a bounded device wait gave up;
 *   SPS_ERR_STATE for a call out of order (e.g. an S phase before any C phase).
 */
#ifndef SPS_H_
#define SPS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sps_status {
  SPS_OK = 0,
  SPS_ERR_INVALID_ARG = 1,
  SPS_ERR_CUDA = 2,
  SPS_ERR_OOM = 3,
  SPS_ERR_DEGENERATE = 4,
  SPS_ERR_NONFINITE = 5,
  SPS_ERR_TIMEOUT = 6,
  SPS_ERR_STATE = 7,
  SPS_ERR_UNSUPPORTED = 8
} sps_status;

typedef enum sps_mem { SPS_MEM_HOST = 0, SPS_MEM_DEVICE = 1 } sps_mem;

/* Arithmetic of the log-likelihood kernel.
 * SPS_PREC_SPLIT: X and theta as BF16 hi+lo pairs (exact 0/1 and integer columns as one BF16),
 *   tcgen05 tensor-core products with FP32 accumulation, FP32 log-sum-exp, FP64 sums across
 *   observation tiles.
 * SPS_PREC_FP32: plain FP32 SIMT dot products and log-sum-exp, FP64 sums across tiles. */
typedef enum sps_precision { SPS_PREC_SPLIT = 0, SPS_PREC_FP32 = 1 } sps_precision;

/* M-phase transition kernel. RW is the Gaussian random walk of Algorithm 2 step 2(c);
 * MALA adds the drift (h/2) V grad log p(theta | y) and the matching proposal-density ratio. */
typedef enum sps_mkernel { SPS_MKERNEL_RW = 0, SPS_MKERNEL_MALA = 1 } sps_mkernel;

/* S-phase resampling scheme (Sec. 2.2 allows multinomial or residual resampling). */
typedef enum sps_resampling { SPS_RESAMPLE_MULTINOMIAL = 0, SPS_RESAMPLE_RESIDUAL = 1 } sps_resampling;

typedef enum sps_prior_kind {
  SPS_PRIOR_ISO = 0,   /* cov = sd^2 I, cov_or_sd points to 1 value (sd) */
  SPS_PRIOR_DIAG = 1,  /* cov = diag(sd^2), cov_or_sd points to D values (sd) */
  SPS_PRIOR_FULL = 2   /* cov_or_sd points to a D x D row-major covariance */
} sps_prior_kind;

/* Gaussian prior on the normalised parameter vector (Eq. 16 with theta_0 = 0; Sec. 3.1).
 * mean: D values, or NULL for the zero vector. Host pointers, copied by sps_init. */
typedef struct sps_prior {
  int32_t kind;
  const double* mean;
  const double* cov_or_sd;
} sps_prior;

/* The design constants of Algorithm 2 (Sec. 2.3 calls them hard-wired but user-changeable)
 * and the library's own settings. sps_options_default fills the paper's values. */
typedef struct sps_options {
  double ess_fraction;     /* 0.5: the C phase ends when ESS/(J N) < ess_fraction (Eq. 14) */
  double h_init;           /* 0.5: h_11 */
  double h_step;           /* 0.01 */
  double h_min;            /* 0.1 */
  double h_max;            /* 1.0 */
  double target_accept;    /* 0.25 (RW); the step-size rule compares alpha_lr > target */
  double rne_cycle;        /* 0.35: K when s < T */
  double rne_final;        /* 0.9: K when s = T */
  int32_t r_max;           /* 200: cap on M steps per cycle (not in the paper) */
  int32_t precision;       /* sps_precision, default SPS_PREC_SPLIT */
  int32_t mkernel;         /* sps_mkernel, default SPS_MKERNEL_RW */
  int32_t cphase_block;    /* observations per C-phase block launch, default 64 */
  double mala_target_accept; /* 0.5: step-size target when mkernel == MALA (not in the paper) */
  uint64_t seed;           /* Philox key for sps_run's random numbers */
  int32_t resampling;      /* sps_resampling, default SPS_RESAMPLE_MULTINOMIAL */
  int32_t graphs;          /* 1 (default): after its first step, an adaptive M phase of sps_run or
                              sps_mphase runs as one captured CUDA graph (a conditional loop whose
                              body is one M step and a device-side step-size and RNE rule), with one
                              host synchronisation per phase; in sps_run_batched, the lockstep M
                              phase of all models likewise (per-model conditional nodes); results
                              are identical to graphs = 0, which issues and reads back every step
                              from the host */
} sps_options;

typedef struct sps_ctx sps_ctx;
typedef struct sps_state sps_state;

/* Recorded schedule of an adaptive run, the input of the second pass of the two-pass
 * simulator (Algorithm 3, Sec. 2.4): t_l, R_l and Sigma_lr. Caller-allocated arrays with the
 * stated capacities; sps_run writes n_cycles and the used entries, or returns
 * SPS_ERR_INVALID_ARG when a capacity is too small. When passed as the schedule argument of
 * sps_run, the run replays it (C phases end at t[l], M phases take R[l] steps with the recorded
 * Sigma matrices). */
typedef struct sps_schedule {
  int32_t n_cycles;
  int32_t cap_cycles;
  int64_t* t;              /* [cap_cycles] t_l */
  int32_t* R;              /* [cap_cycles] R_l */
  int64_t cap_steps;       /* capacity of sigma/h/accept in steps (sum of R_l) */
  double* sigma;           /* [cap_steps * D * D] Sigma_lr, row-major, steps in order; may be NULL
                              when only recording t and R */
  double* h;               /* [cap_steps] h_lr, may be NULL */
  double* accept;          /* [cap_steps] alpha_lr, may be NULL */
} sps_schedule;

/* Output of sps_run. All arrays are caller-allocated host memory.
 * Moments are for the D coordinates of theta followed by the C-1 log-odds theta_c' xbar
 * (Eq. 15 at the covariate mean xbar over all T observations): m = D + C - 1 entries each. */
typedef struct sps_result {
  double* mean;            /* [m] grand mean, Eq. (5) */
  double* sd;              /* [m] posterior SD from the pooled particles */
  double* nse;             /* [m] numerical standard error, (v-hat / (J N))^(1/2), Eqs. (6)-(7) */
  double* rne;             /* [m] relative numerical efficiency, Eq. (10) */
  double* log_ml_group;    /* [J] per-group log marginal likelihood */
  double log_ml;           /* mean over groups of log_ml_group */
  double log_ml_nse;       /* sd over groups / sqrt(J) */
  double log_ml_pooled;    /* log of the mean over groups of the group marginal likelihoods */
  int32_t n_cycles;        /* L */
  int64_t m_steps;         /* sum of R_l */
  double seconds;          /* wall time of the run on the host clock */
  double* log_pred;        /* [n] or NULL: log predictive likelihoods log p(y_s | y_1:s-1), the
                              mean over groups of log sum_n w_jn(s) - log sum_n w_jn(s-1) within
                              the cycle containing s (Sec. 6 calls them a by-product of SPS);
                              over a cycle they sum to the log-ML increment */
  double* log_pred_nse;    /* [n] or NULL: their sd over groups / sqrt(J) */
  int64_t graph_steps;     /* M steps that ran inside captured graphs (options.graphs) */
} sps_result;

/* ------------------------------------------------------------------ lifecycle */

/* Fill *opt with the paper's Algorithm 2 constants and the library defaults. */
void sps_options_default(sps_options* opt);

/* Prior of the normalised parameters from independent class priors (Sec. 3.1, Eq. 17):
 * theta_c ~ N(mu_c, Sigma_c), c = 0..C-1; with outcome 0 as the base the D = k (C-1) vector of
 * theta_j - theta_0 has block mean mu_j - mu_0, diagonal blocks Sigma_j + Sigma_0 and
 * off-diagonal blocks Sigma_0. Host arrays: mu [C x k], Sigma [C x k x k] row-major;
 * mean_out [D], cov_out [D x D]. Pure host arithmetic (setup, not on the simulator's path). */
sps_status sps_prior_normalize(int32_t k, int32_t n_outcomes, const double* mu, const double* Sigma,
                               double* mean_out, double* cov_out);

/* Create a context for the data (X, y) and prior (Sec. 2.1, Eq. 1; Sec. 3.1, Eq. 16).
 *   X: host FP64 [n x k] row-major covariates; y: host int32 [n], values 0..n_outcomes-1.
 *   n >= 1, 1 <= k <= 256, 2 <= n_outcomes <= 4 for the tensor-core path (the FP32 path
 *   accepts up to 16 outcomes). prior: Gaussian on the D = k*(n_outcomes-1) free coefficients.
 *   opt may be NULL (defaults). Copies and encodes X and y to the current CUDA device.
 *   For binary logits whose tiles are bound by their tensor-core products (many covariates) the
 *   fused split-precision kernel runs on CTA pairs (tcgen05 MMAs of 256 particles over two CTAs,
 *   each holding half of every X tile) when the device can co-schedule them, else on single
 *   CTAs; the environment variable SPS_TC_CLUSTER, read here, overrides the choice: "1" single
 *   CTAs, "2" CTA pairs wherever they can be co-scheduled (same results either way).
 * Errors: SPS_ERR_INVALID_ARG for bad sizes, y out of range, non-finite X or a prior covariance
 * that is not positive definite; SPS_ERR_OOM; SPS_ERR_CUDA. *out is NULL on failure. */
sps_status sps_init(sps_ctx** out, const double* X, int64_t n, int32_t k, const int32_t* y,
                    int32_t n_outcomes, const sps_prior* prior, const sps_options* opt);

/* Release every device and host resource of the context (NULL is a no-op). States created on
 * it must be destroyed first. */
void sps_destroy(sps_ctx* ctx);

/* Run the context's work on `stream` (a cudaStream_t; NULL = the legacy default stream). */
sps_status sps_set_stream(sps_ctx* ctx, void* stream);

/* Message for a status code, and the last error message recorded on ctx (never NULL). */
const char* sps_status_string(sps_status s);
const char* sps_last_error(const sps_ctx* ctx);

/* Sizes of the context: n, k, C, D. Any pointer may be NULL. */
sps_status sps_get_dims(const sps_ctx* ctx, int64_t* n, int32_t* k, int32_t* C, int32_t* D);

/* Replace the context's prior (same rules as sps_init); states created later draw from it. */
sps_status sps_set_prior(sps_ctx* ctx, const sps_prior* prior);

/* Zellner's g-prior of the paper for the context's data (Sec. 3.1, Eq. 18): Sigma_c = g n (X'X)^-1
 * and mu_c = 0 for every outcome, normalised on outcome 0 (sps_prior_normalize). X'X is summed
 * on the device in FP64; its inverse (k x k) is taken on the host by Cholesky. mean_out [D]
 * (zeros) and cov_out [D x D] are host arrays; pass them to sps_set_prior as SPS_PRIOR_FULL.
 * SPS_ERR_DEGENERATE when X'X is singular. */
sps_status sps_gprior(sps_ctx* ctx, double g, double* mean_out, double* cov_out);

/* Instrumentation (the paper has no counterpart). sps_set_timing(ctx, 1) records CUDA events on
 * the context's stream around every launch of the fused log-likelihood kernel from then on.
 * sps_counters synchronises the stream and reports, since the last reset: the number of kernels
 * the library launched on ctx, the number of timed fused-kernel launches and their total device
 * time in milliseconds (any output may be NULL); reset != 0 then clears the counts. */
sps_status sps_set_timing(sps_ctx* ctx, int32_t on);
sps_status sps_counters(sps_ctx* ctx, int32_t reset, int64_t* launches, int64_t* hot_launches,
                        double* hot_ms);

/* Diagnostics of the failure path (the paper has no counterpart). Every wait of the fused
 * split-precision log-likelihood kernel on its pipeline barriers is bounded by a wall-clock
 * limit, after which the kernel stops its CTAs cleanly and the call reports SPS_ERR_TIMEOUT.
 * timeout_ns sets that limit for later launches on ctx (0 restores the default, 2 s);
 * stall_producer != 0 makes the kernel's TMA producer issue no copy at all, so that every
 * consumer wait runs out after timeout_ns and the call returns SPS_ERR_TIMEOUT with nothing left
 * in flight; 0 restores normal operation. The context stays usable. */
sps_status sps_set_debug(sps_ctx* ctx, int32_t stall_producer, uint64_t timeout_ns);

/* ------------------------------------------------------------------ the likelihood hot path */

/* Log-likelihood of every particle over the first t observations (Eq. 1, product form of
 * Sec. 2.1): ll[p] = sum_{s<=t} log P(Y_s = y_s | x_s, theta_p).
 *   theta: [P x D] FP64 class-major (mem); ll: [P] FP64 output (mem); 1 <= P; 0 <= t <= n.
 *   precision: sps_precision (the context's option is only the default of sps_run).
 * Deterministic: the same theta always gives the same bits. With mem = SPS_MEM_HOST the call
 * returns after the results are in ll; split-precision calls of at least 32 768 particles copy
 * theta in up to eight particle slices on a second stream of the library, overlapping the copy
 * with the kernel, and agree with a device-memory call up to the order of partial sums. */
sps_status sps_loglik(sps_ctx* ctx, const double* theta, int64_t P, int64_t t, double* ll,
                      int32_t precision, int32_t mem);

/* Allocation-free form of sps_loglik (split precision, device pointers only). The paper has no
 * counterpart: it serves callers that cannot let the library call cudaMalloc during a call,
 * for example code whose device memory is owned by another allocator (a framework's memory
 * pool or a fixed arena) or loops that cannot accept the device synchronisation that cudaMalloc
 * and cudaFree may cause. Its per-call scratch (theta operand rows, partial sums, a flag) lives in
 * one 32 MiB device array that every GPU loading the library holds until the process exits;
 * the call allocates nothing.
 *   theta: [P x D] device FP64; ll: [P] device FP64 output; work is enqueued on the context's
 *   stream (the call returns before it completes). Same results as sps_loglik(SPS_PREC_SPLIT),
 *   bit for bit (the same kernels and summation order).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress) with
 * the context's device current; make that first call before any stream capture. All calls share
 * the array: calls whose GPU work overlaps race and must be serialised by the caller.
 * Limit: with k16 = k rounded up to 16, kt = 2 k16 rounded up to 64, P' = P rounded up to the
 * particles of one work item (128, or 256 when the context's kernel runs on CTA pairs) and c the
 * call's observation chunks (at most ceil(t / 64)), the call needs 2 kt (C-1) P' bytes of operand
 * rows plus 32 c P' bytes of partial sums plus 256 bytes, each
 * part rounded up to 256 bytes, within 32 MiB: the binary workload with 65 536 particles,
 * k = 30 and n = 20 000 needs about 18 MiB. Larger calls return SPS_ERR_INVALID_ARG, with the
 * required size in sps_last_error, and launch nothing.
 * Timeouts: when the fused kernel gives up on a bounded wait (see sps_set_debug) this call cannot
 * report it in its status, which is returned before the kernel runs; every ll[p] is then set to
 * NaN instead. Other errors as sps_loglik. */
sps_status sps_loglik_noalloc(sps_ctx* ctx, const double* theta, int64_t P, int64_t t, double* ll);

/* Log-likelihoods of M nested models in one fused-kernel launch (split precision): model m uses
 * the first k_models[m] covariates of the context's X (1 <= k_m <= k) with D_m = k_m (C-1)
 * parameters, P_models[m] particles and the prefix t_models[m] (0 <= t_m <= n). Each model's
 * tiles use the model's own encoding of X[:, :k_m] (its continuous columns first; built on the
 * device at the first call with that k_m and kept by the context, n x 64 or more BF16 values
 * per model), so they load the X bytes and issue the MMAs of the model's own launch, and the
 * results equal sps_loglik on a context built from X[:, :k_m] (within the split tolerance).
 *   theta: device FP64, the models' [P_m x D_m] class-major blocks concatenated in model order;
 *   ll: device FP64 [sum P_m]; k_models, P_models, t_models: host [M], 1 <= M <= 1024.
 * Work is enqueued on the context's stream. The paper runs one model at a time; batching the
 * candidate models of a marginal-likelihood comparison into one launch fills the GPU. */
sps_status sps_loglik_batched(sps_ctx* ctx, int32_t M, const int32_t* k_models, const int64_t* P_models,
                              const int64_t* t_models, const double* theta, double* ll);

/* Tile-shape autotuner of the fused split-precision kernel. Times every candidate launch shape
 * on P particles at prefix t (1 <= t <= n) with CUDA events: observation rows per tile (the two
 * widths the outcome count allows, where the pipeline fits shared memory), single CTAs or CTA
 * pairs (256-particle MMAs over two CTAs, each holding half of every X tile), and work items of
 * 512 to 65536 observations. The fastest is kept
 * in the context and used by every later split-precision call (results change only by the
 * order of FP32/FP64 partial sums). Each candidate runs 1 untimed and 3 timed launches on zero
 * particles; the call synchronises the context's stream.
 *   out (optional): the chosen shape, its time per launch in ms and the candidates tried. */
typedef struct sps_tune_result {
  int32_t tile_rows;       /* observations per tile */
  int32_t cluster;         /* CTAs per cluster */
  int32_t chunk_obs;       /* observations per work item */
  int32_t n_candidates;
  double ms;               /* time per launch of the chosen shape */
  double ms_default;       /* time per launch of the shape chosen at sps_init */
} sps_tune_result;
sps_status sps_autotune(sps_ctx* ctx, int64_t P, int64_t t, sps_tune_result* out);

/* Log-likelihood and its gradient d ll / d theta_c = sum_{s<=t} (1[y_s = c] - p_{s,c}) x_s
 * (the derivative of Eq. 1; the paper prints no gradient).
 *   grad: [P x D] FP64 output, class-major like theta (mem).
 * With options.precision = SPS_PREC_SPLIT and C - 1 <= 3 (and gradient accumulators that fit
 * TMEM: k16 + kc16 <= 256 for C = 2, (k16 + kc16) 2 <= 240 for C = 3, (k16 + kc16) 3 <= 400 for
 * C = 4; k16 / kc16 the covariate counts rounded up to 16): tensor cores, the forward products
 * as in sps_loglik and sum_s q_s x_s as a second BF16 hi + lo MMA (q = p - 1/2 for C = 2, p_c
 * for C > 2) with FP32 accumulation per work item and FP64 across items. Otherwise: FP32 SIMT
 * products and residuals, FP64 sums across 128-observation tiles.
 * One context always uses the same form for the same shape. */
sps_status sps_loglik_grad(sps_ctx* ctx, const double* theta, int64_t P, int64_t t, double* ll,
                           double* grad, int32_t mem);

/* ------------------------------------------------------------------ simulator state and phases */

/* Create the particle state of J groups of N particles and draw them iid from the prior
 * (Algorithm 1 step 1) with Philox key `seed`. 2 <= J, 2 <= N <= 4096. t = 0, h = h_init. */
sps_status sps_state_create(sps_ctx* ctx, int32_t J, int32_t N, uint64_t seed, sps_state** out);
void sps_state_destroy(sps_state* st);

/* Copy the state's particles [J*N x D], cached log-likelihoods [J*N] and log weights [J*N]
 * (host pointers, any may be NULL) and its scalars (t, h; any may be NULL). The call waits for
 * the context's stream only when one of the three arrays is requested (t and h live on the host). */
sps_status sps_state_get(sps_ctx* ctx, const sps_state* st, double* theta, double* ll,
                         double* logw, int64_t* t, double* h);
/* Overwrite particles and cached log-likelihoods (host pointers, [J*N x D] and [J*N]; ll may be
 * NULL to recompute it at the state's t) and set t (0 <= t <= n). */
sps_status sps_state_set(sps_ctx* ctx, sps_state* st, const double* theta, const double* ll,
                         int64_t t);
/* Outputs of the state's particles as sps_run reports them at the end of a run: mean, SD, NSE and
 * RNE (Eqs. 5-7, 10, over the J groups) of every coordinate of theta and of the log-odds
 * theta_c' xbar (Eq. 15; D + C - 1 values each), and the per-group log marginal likelihoods
 * accumulated by the state's C phases with their mean, NSE and pooled value. out: caller
 * arrays as for sps_run; n_cycles = S phases run, m_steps = M steps run (log_pred ignored).
 * Waits for the context's stream. */
sps_status sps_state_result(sps_ctx* ctx, sps_state* st, sps_result* out);

/* C phase (Algorithm 1 step 2(a), Eq. 11, ended by the ESS rule of Algorithm 2 step 1, Eq. 14):
 * from the state's t, multiply the weights by p(y_s | theta) for s = t+1, ... until
 * ESS(s)/(J N) < ess_fraction or s = n; with t_target > 0 stop at s = t_target instead
 * (a recorded schedule). Adds log N^-1 sum_n w_jn to each group's log marginal likelihood,
 * updates the cached log-likelihoods and sets t. Outputs (host, may be NULL): t_new, ess at
 * t_new, logml_inc [J], log_pred [(t_new - t) x J] row-major: the per-group log predictive
 * likelihoods of the observations taken in (capacity (n - t) x J; FP32 exponentials of the
 * running log weights, FP64 sums). Without a target the call reads the ESS of every block back
 * (one synchronisation per block); with a target and no log_pred it waits for the stream only
 * when ess or logml_inc is requested, once. */
sps_status sps_cphase(sps_ctx* ctx, sps_state* st, int64_t t_target, int64_t* t_new,
                      double* ess, double* logml_inc, double* log_pred);

/* S phase (Algorithm 1 step 2(b)): resampling of each group from its C-phase weights (the
 * context's sps_options.resampling scheme, see sps_resample), then the gather of particles and
 * cached log-likelihoods.
 *   uniforms: [J*N] FP64 on [0,1) (mem) to use instead of the state's Philox stream, or NULL.
 *   idx_out: [J*N] int32 (mem) receives the selected index within the group, or NULL. */
sps_status sps_sphase(sps_ctx* ctx, sps_state* st, const double* uniforms, int32_t* idx_out,
                      int32_t mem);

/* Diagnostics of one M step. */
typedef struct sps_mstep_info {
  double h;                /* step-size factor used by this step */
  double accept_rate;      /* alpha_lr */
  double rne_min;          /* smallest RNE of the monitoring set after the step */
  double h_next;           /* h after the +-h_step rule */
} sps_mstep_info;

/* One M step (Algorithm 2 step 2(c)): V = pooled particle covariance (divisor J N - 1),
 * Sigma = h V (or the given sigma [D x D] host, row-major, e.g. from a recorded schedule),
 * theta' = theta + chol(Sigma) z, Metropolis accept with log u < log alpha; then the step-size
 * rule and the RNE of the monitoring set {ll, theta_c' xbar}. kernel: sps_mkernel.
 *   sigma_used: [D x D] host output of the Sigma used (may be NULL).
 * The state's h is updated to info.h_next unless sigma was given. */
sps_status sps_mstep(sps_ctx* ctx, sps_state* st, int32_t kernel, const double* sigma,
                     double* sigma_used, sps_mstep_info* info);

/* M phase (Algorithm 2 step 2): M steps until the smallest RNE of the monitoring set reaches
 * K (rne_cycle if t < n, rne_final if t == n) or r_max steps; with fixed_steps > 0, exactly that
 * many steps. Outputs (host, may be NULL): steps taken, last acceptance rate, last RNE min. */
sps_status sps_mphase(sps_ctx* ctx, sps_state* st, int32_t kernel, int32_t fixed_steps,
                      int32_t* steps, double* accept_rate, double* rne_min);

/* The whole simulator: adaptive Algorithm 2 with J groups of N particles, or, when `schedule`
 * is non-NULL with n_cycles > 0, the replay of that schedule (Algorithm 3 pass 2). When
 * `record` is non-NULL the run's schedule is written into it. Results in *out (caller arrays). */
sps_status sps_run(sps_ctx* ctx, int32_t groups, int32_t particles_per_group,
                   const sps_schedule* schedule, sps_schedule* record, sps_result* out);

/* Batched model comparison: the adaptive simulator (Algorithm 2, with the context's M kernel,
 * random walk or MALA) for M nested models of the context's data at once, model m using the
 * first k_models[m] covariates (1 <= k_m <= k) with J groups x N particles and the context's
 * options. Prior of model m: with g > 0 the paper's g-prior for its own covariates (Sec. 3.1,
 * Eq. 18, as sps_gprior); else the marginal of the context's prior on its coordinates
 * (theta_c,i for i < k_m). (A diffuse prior on many coordinates can leave fewer distinct
 * particles than parameters after the first S phase; the step then fails with
 * SPS_ERR_DEGENERATE, as the paper notes in Sec. 4.) Each model has its own particles, C and S
 * phases and step size (a context of its own, built from the context's data, on the context's
 * stream, with the Philox key options.seed + m-dependent offset). Their M phases run in
 * lockstep: in every M step the proposals of all models still moving are evaluated, each at its
 * model's t, with one batched fused-kernel launch (sps_loglik_batched, in which each model's
 * tiles use the model's own encoding of its covariates); FP32 precision: one launch per model;
 * MALA: each model's own gradient launch, which also gives the log-likelihoods. A model that
 * has met its stopping rule leaves the phase: its kernels stop and the batched launch skips its
 * particle tiles (keeping the launch's work decomposition, so each model's sums round the same
 * way in every step). With options.graphs, a cycle is two CUDA graph launches: the C and S
 * phases of all models (a conditional loop over C-phase blocks with the ESS stopping rule and
 * the next block decided on the device, each model under conditional nodes of its own, then
 * the S phases), and, after the M phase's first step, the rest of the lockstep M phase (a
 * conditional loop whose body holds each moving model's kernels under its own conditional
 * nodes, the batched launch between them and device-side step-size and RNE rules per model).
 * The models' kernels run concurrently; the results are identical to graphs = 0.
 * Marginal likelihoods for comparing the models (Sec. 2.3) are in out[m].log_ml.
 *   out: [M] caller-allocated results as for sps_run (log_pred ignored).
 * A model's error is returned with its message. */
sps_status sps_run_batched(sps_ctx* ctx, int32_t M, const int32_t* k_models, double g, int32_t groups,
                           int32_t particles_per_group, sps_result* out);

/* ------------------------------------------------------------------ building blocks */

/* Resampling by integer CDFs, each of J groups of N independently (the S phase of Algorithm 1):
 * q_n = floor(w_n 2^40) with w the group's FP64 weights divided by their maximum (w is given
 * already divided: max w_n = 1 in each group), Q = sum q.
 *   SPS_RESAMPLE_MULTINOMIAL: cumulative sums of q in uint64, tau_i = min(floor(u_i * Q), Q - 1),
 *     idx_i = first n with cumulative q > tau_i.
 *   SPS_RESAMPLE_RESIDUAL: c_n = floor(N q_n / Q) copies of n placed first in particle order,
 *     then R = N - sum c draws i = 0..R-1 multinomial as above on r_n = (N q_n mod Q) >> 12,
 *     using u_i.
 *   w, u: [J*N] FP64 (mem); idx: [J*N] int32 within-group indices (mem). N <= 4096.
 * SPS_ERR_DEGENERATE (host memory only) when a group's weights all quantise to zero. */
sps_status sps_resample(sps_ctx* ctx, const double* w, const double* u, int32_t J, int32_t N,
                        int32_t scheme, int32_t* idx, int32_t mem);

/* Philox4x32-10 blocks (Salmon et al., SC'11) for counters (ctr0 + i, ctr1, ctr2, ctr3),
 * i = 0..count-1, key (key0, key1): out [count x 4] uint32 (mem). */
sps_status sps_philox(sps_ctx* ctx, uint32_t key0, uint32_t key1, uint32_t ctr0, uint32_t ctr1,
                      uint32_t ctr2, uint32_t ctr3, int64_t count, uint32_t* out, int32_t mem);

/* ESS (Eq. 14) of P log weights and log N^-1 sum exp(logw) of each of J groups of N = P/J
 * (the per-cycle log marginal likelihood increment). logw: [P] (mem); ess: 1 value (mem);
 * lme: [J] (mem). */
sps_status sps_ess(sps_ctx* ctx, const double* logw, int64_t P, int32_t J, double* ess,
                   double* lme, int32_t mem);

/* Pooled sample covariance of P particles (divisor P - 1), V: [D x D] FP64 (mem). */
sps_status sps_particle_cov(sps_ctx* ctx, const double* theta, int64_t P, double* V, int32_t mem);

/* One random-walk Metropolis step with given randomness, for step-level parity:
 * theta' = theta + L z with L the lower Cholesky factor of sigma (host [D x D]); log alpha =
 * ll(theta'; y_1:t) - ll + log p(theta') - log p(theta); accept when log u < log alpha.
 *   theta [P x D], ll [P] are updated in place (mem); z [P x D], u [P] (mem);
 *   log_alpha [P], accepted [P] (int32) outputs (mem, may be NULL). */
sps_status sps_rw_step_given(sps_ctx* ctx, double* theta, double* ll, int64_t P, int64_t t,
                             const double* sigma, const double* z, const double* u,
                             int32_t precision, double* log_alpha, int32_t* accepted,
                             int32_t mem);

/* One MALA step with given randomness, for step-level parity (the MALA M kernel is not in the
 * paper; it is an exact Metropolis-Hastings kernel for the posterior given y_1:t, Eq. 13, beside
 * the random walk of Algorithm 2 step 2(c)i). With L the lower Cholesky factor of sigma (host
 * [D x D]) and g the gradient of the log posterior (log-likelihood and log prior) at theta:
 * theta' = theta + sigma g(theta) / 2 + L z; log alpha = ll(theta') - ll(theta) + log p(theta')
 * - log p(theta) + log q(theta | theta') - log q(theta' | theta), q(. | a) = N(a + sigma g(a) / 2,
 * sigma); accept when log u < log alpha. The log-likelihood and gradient at theta and theta' come
 * from the function of sps_loglik_grad; the drift and the proposal ratio are formed with FP32
 * products of L and g (as in the simulator's MALA steps).
 *   theta [P x D] is updated in place; ll [P] receives the log-likelihood of the returned
 *   particles (mem); z [P x D], u [P] (mem); log_alpha [P], accepted [P] (int32) outputs (mem, may
 *   be NULL). 1 <= t <= n. SPS_ERR_DEGENERATE when sigma is not positive definite. */
sps_status sps_mala_step_given(sps_ctx* ctx, double* theta, double* ll, int64_t P, int64_t t,
                               const double* sigma, const double* z, const double* u,
                               double* log_alpha, int32_t* accepted, int32_t mem);

#ifdef __cplusplus
}
#endif

#endif /* SPS_H_ */
