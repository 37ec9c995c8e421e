/*
 * oais.h -- C ABI of the GB300 (sm_103a) Optimised Annealed Importance Sampling engine.
 *
 * Method: Syed, Bouchard-Cote, Chern, Doucet, "Optimised Annealed Sequential Monte
 * Carlo Samplers" (arXiv 2408.12057).  N particles move through an annealing
 * schedule 0 = beta_0 < ... < beta_T = 1 on the geometric path
 * pi_beta ∝ eta(x) L(x)^beta (Sec. 2), eta = N(0, s^2 I) the normalised reference.
 * Each step adds the incremental weight (beta_t - beta_{t-1}) log L(x) at the
 * pre-move state, reduces the moment statistics g_hat_{t,0:2} (Alg. 1), and applies
 * K Metropolis-Hastings moves targeting pi_{beta_t}.  log Z_hat is a logsumexp of the
 * final weights (eq. estimator_Z).  Between rounds the cumulative barrier
 * Lambda_hat_t = sum_{s<=t} sqrt(D_hat_s) is inverted into the next schedule
 * (Alg. 2, Alg. 3).  asmc_run adds ESS-triggered systematic resampling (Sec. 2.1.3).
 *
 * Conventions for every entry point:
 *   - every call returns an oais_status; nothing aborts, throws or exits;
 *   - "device pointer" arguments must be CUDA device memory of the current device;
 *     "host pointer" arguments must be host memory; sizes are element counts;
 *   - stream arguments are cudaStream_t passed as void*; NULL means the legacy
 *     default stream.  Calls are ordered on that stream.
 *   - a context is used by one host thread at a time.
 *   - after OAIS_ECUDA the CUDA error text is in oais_last_error(ctx) (or
 *     oais_last_error(NULL) for calls without a context).
 */
#ifndef OAIS_H_
#define OAIS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    OAIS_OK = 0,
    OAIS_EINVAL = 1,        /* bad argument: sizes, schedule not strictly increasing 0..1, ... */
    OAIS_ENOMEM = 2,        /* device allocation failed or workspace too small */
    OAIS_ECUDA = 3,         /* a CUDA runtime call failed */
    OAIS_ENONFINITE = 4,    /* a log-weight or log-likelihood became NaN or +inf (-inf is a zero weight) */
    OAIS_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    OAIS_EUNSUPPORTED = 6   /* combination not built (dimension, family, move) */
} oais_status;

/* Target families (Sec. 2 geometric path; likelihood L, reference eta = N(0, s^2 I)). */
typedef enum {
    OAIS_T_GAUSS = 0,   /* L(x) = exp(-|x - mu|^2 / (2 p0^2)); X = mu[d]                   */
    OAIS_T_LOGREG = 1,  /* L(x) = prod_r Bern(y_r | sigmoid(X_r . x)); X[n][d], y[n] in {0,1} */
    OAIS_T_GMM = 2,     /* L(x) = p(x)/eta(x), p = (1/n) sum_k N(X_k, p0 I); X[n][d] means   */
    OAIS_T_LINREG = 3,  /* L(x) = prod_r N(y_r; X_r . x, p0^2); X[n][d], y[n]               */
    OAIS_T_UNID = 4     /* the unidentifiable product model of the paper's model appendix and
                           GPU experiments: X, Y ~ Uniform(0, p0), K ~ Binomial(m, X Y) observed
                           at k.  State z in R^2 under eta = N(0, I) (ref_scale must be 1), with
                           X = p0 Phi(z_1), Y = p0 Phi(z_2); L(z) = Binom(k; m, X Y), 0 where
                           X Y >= 1 (log L = -inf: such states get weight 0).  X = (m, k) as
                           float64, d = 2, n = 0; fp64 throughout, CUDA-core form only */
} oais_target_kind;

typedef enum { OAIS_DT_F64 = 0, OAIS_DT_F32 = 1 } oais_dtype;

typedef struct {
    int32_t kind;       /* oais_target_kind */
    int32_t d;          /* state dimension, 1 <= d <= 32 (GAUSS: <= 16); LOGREG and LINREG up to
                           d = 256 (the tiled fp32 form and the streamed tensor-core form) */
    int32_t n;          /* rows of X (LOGREG, LINREG), mixture components (GMM, <= 16); 0 for GAUSS, UNID */
    int32_t dtype;      /* oais_dtype of X and y: GAUSS and UNID run in F64 and take F64 X;
                           the other families run in F32 and take F32 or F64 input */
    const void* X;      /* row-major, see kind; host or device per on_device */
    const void* y;      /* [n] (LOGREG, LINREG), else NULL */
    double ref_scale;   /* s > 0 */
    double p0;          /* GAUSS: likelihood sigma; GMM: component variance; LINREG: noise sigma;
                           UNID: upper end of the uniform priors */
    int32_t on_device;  /* 0: X, y are host memory, copied at init.  1: device memory, also copied
                           (to the padded device layout); the caller may free them after init */
    int32_t contraction;/* how X x is computed (oais_contraction):
                           OAIS_CONTRACT_FP32: CUDA cores, fp32 data.  Up to d = 32 one thread
                             per particle keeps the particle in registers for the whole sweep;
                             LOGREG and LINREG with 32 < d <= 256 run the tiled fp32 form: a CTA
                             per tile of 64 particles evaluates log L and its gradient as two
                             fp32 contractions over X streamed through shared memory, with the
                             particle vectors in device memory (OAIS rounds, the shard calls and
                             oais_potential; not oasmc_round, oais_zja_round or oais_ctx_sweep).
                           OAIS_CONTRACT_BF16_TC: tcgen05 tensor cores with X rounded once to
                             bf16 (the sampler targets that X~).  LOGREG with d <= 32,
                             n <= 2048 and MALA runs with X~ resident in shared memory (states
                             and residuals split into two bf16 terms); every other LOGREG
                             (MALA) or LINREG (MALA, HMC) problem with d <= 256 runs the
                             streamed form below.
                           OAIS_CONTRACT_BF16_TC_STREAM: always the streamed form: X~ is
                             streamed from device memory in chunks, held as f16 (exact for
                             bf16 values of magnitude >= 2^-17; smaller ones take the nearest
                             f16), states and residuals split into two f16 terms (relative
                             error ~2^-22); any n, d <= 256, LOGREG (MALA) or LINREG (MALA,
                             HMC).
                           OAIS_CONTRACT_FP8_TC_STREAM: the streamed form with X stored as
                             FP8 e4m3 with one scale per row: s_r = max_j |X_rj| / 448 (fp32;
                             1 for a zero row), q_rj = e4m3(X_rj / s_r) rounded to nearest
                             even, and the sampler targets X~_rj = s_r q_rj.  The chunks are
                             expanded to f16 on chip (exact), so the contraction keeps the
                             accuracy of the f16 form; LINREG only.
                           The tensor-core forms run the OAIS sweep (oais_round and the shard
                           calls); the streamed kernel also runs resampling rounds (oasmc_round:
                           one launch per step over its stored particle state) and
                           oais_potential, for streamed and resident contexts alike (a resident
                           context keeps the streamed form's image and state for them).
                           oais_ctx_sweep and oais_zja_round use the one-thread-per-particle
                           CUDA-core form, which exists for d <= 32 (they return
                           OAIS_EUNSUPPORTED above that).  Other combinations return
                           OAIS_EUNSUPPORTED at init. */
} oais_target;

typedef enum {
    OAIS_CONTRACT_FP32 = 0,
    OAIS_CONTRACT_BF16_TC = 1,
    OAIS_CONTRACT_BF16_TC_STREAM = 2,
    OAIS_CONTRACT_FP8_TC_STREAM = 3
} oais_contraction;

typedef enum { OAIS_RWMH = 0, OAIS_MALA = 1, OAIS_HMC = 2 } oais_move_kind;

typedef struct {
    int32_t kind;       /* oais_move_kind; each is a pi_beta-invariant MH kernel (Sec. 2.1.1) */
    int32_t moves;      /* K >= 1 moves per annealing step */
    int32_t leapfrog;   /* HMC leapfrog steps (>= 1) */
    int32_t cycle;      /* RWMH only: proposal std cycles 0.1, 1, 10 by global move index
                           (the alternation of the paper's GPU experiments, App. E.3) */
    int32_t adapt;      /* 1: between rounds rescale step sizes toward a target acceptance
                           (App. on propagation-kernel adaptation); 0: keep them */
} oais_move;

typedef struct {
    double logZ;        /* log Z_hat of the round (eq. estimator_Z with R = 1) */
    double se;          /* delta-method standard error of log Z_hat: sqrt(1/ESS - 1/N) */
    double Lambda_hat;  /* Lambda_hat_T = sum_t sqrt(D_hat_t) (Alg. 3) */
    double ess;         /* ESS of the final weights, (sum w)^2 / sum w^2 */
    double sweep_ms;    /* device time of the sweep kernel, CUDA events */
    int32_t T;          /* steps run this round */
    int32_t round;      /* 0-based index of the round */
    int32_t n_resample; /* asmc_run: intermediate resampling events; 0 for OAIS */
    int32_t pad;
    double elbo;        /* ELBO estimate sum_t sum_n W_{t-1}^n log g_t^n with the normalised
                           weights since the last resampling (Sec. on the KL divergence of a
                           schedule: log Z = ELBO + KL); NaN for a sharded round */
    double kl;          /* logZ - elbo: the accumulated-KL estimate, >= 0 up to rounding (per
                           step, log sum_n W g >= sum_n W log g by Jensen) */
} oais_round_result;

typedef struct oais_ctx oais_ctx;

/* Device bytes oais_init needs for this problem when it is given a workspace.
 * N particles, schedules of at most T_max steps. */
oais_status oais_workspace_bytes(const oais_target* target, const oais_move* move, int64_t N,
                                 int32_t T_max, size_t* bytes);

/* Create a context (Alg. 2 state).  beta: host [T+1], 0 = beta_0 < ... < beta_T = 1, the
 * schedule of the first round (the paper's Alg. 2 starts from T = 1, beta = (0, 1)).
 * eps: host [T] step sizes per step (RWMH proposal std, MALA/HMC step), or NULL for
 * 0.5/sqrt(d).  workspace: device memory of at least oais_workspace_bytes(), owned by the
 * caller and kept alive until oais_destroy; NULL lets the library cudaMalloc its own.
 * stream: cudaStream_t for all work of this context (NULL: default stream).
 * Errors: EINVAL (bad sizes, schedule), EUNSUPPORTED (d/kind/move not built), ENOMEM, ECUDA. */
oais_status oais_init(oais_ctx** ctx, const oais_target* target, const oais_move* move,
                      int64_t N, const double* beta, int32_t T, int32_t T_max, const double* eps,
                      uint64_t seed, void* workspace, size_t workspace_bytes, void* stream);

/* One round of OAIS (Alg. 2 body): run the loop-swapped sweep with the current schedule,
 * merge the per-step moments, form log Z_hat, then install
 * OptimiseSchedule(T_next, B_T, g_hat) (Alg. 3) as the schedule of the next round.  Its step
 * sizes are carried from the round's: each step size is held as its ratio to the shape
 * 1 / sqrt(1/s^2 + beta kappa) of the starting rule (oais_default_step_sizes), the logarithm of
 * that ratio interpolated linearly in beta (constant beyond the round's first and last steps),
 * and with move.adapt each step nudged toward the move's target acceptance.
 * T_next <= T_max.  Synchronises the context's stream.  On error the previous round's
 * results and the current schedule are left unchanged (anytime property, Sec. 1) and the round
 * counter does not advance; the particle buffers of oais_particles then hold the failed
 * round's values. */
oais_status oais_round(oais_ctx* ctx, int32_t T_next, oais_round_result* out);

/* One round of optimised ASMC (Alg. 2 with Alg. 1's adaptive resampling): particles
 * advance in lock-step, one launch sequence per annealing step.  After the reweight of
 * step t the ESS (eq. sample_size_IS) of w_{t^-} is reduced on the device; if
 * ESS < ess_frac * N (and always at t = T) the segment closes, log Z_hat += LSE(log w) - log N
 * (eq. estimator_Z), and for t < T the particles are resampled systematically (Sec. 2.1.3):
 * fp64 inclusive scan C of the normalised weights, a^n = min{m : C_m > (n + U)/N} with one
 * uniform U per event, gather into the second buffer, weights reset to 1.  ess_frac = 0 gives
 * AIS in lock-step form; ess_frac = 1 resamples at every step (SIR).  The moments g_hat use
 * w_{t-1}, i.e. the weights since the last resampling event.  Then installs
 * OptimiseSchedule(T_next, ...) like oais_round.  Same errors as oais_round. */
oais_status oasmc_round(oais_ctx* ctx, int32_t T_next, double ess_frac, oais_round_result* out);

/* The online conditional-ESS comparator of the paper's section on the connection to online
 * CESS optimisation (Zhou, Johansen & Aston 2016, "ZJA"; the method the paper's GPU
 * experiments compare against): like oasmc_round, but before step t the next annealing
 * parameter is chosen on the device so that CESS_t / N = (sum_n W_n g_n)^2 / sum_n W_n g_n^2
 * = cess_frac, g_n = L(X_{t-1}^n)^(beta_t - beta_{t-1}), W the normalised weights since the last
 * resampling (the paper matches budgets with cess_frac = exp(-Lambda^2 / T^2)).  The line
 * search refines a bracket of beta_t - beta_{t-1} in a geometric scan and five linear passes of 32 candidates, keeping the
 * last candidate meeting the target.  The run ends at beta = 1 or after T_max steps (the last
 * forced to beta = 1); step sizes are the current schedule's, log eps interpolated linearly
 * in beta.  ess_frac as in oasmc_round.  The schedule that ran becomes the round's
 * (oais_get_stats), and OptimiseSchedule(T_next, ...) of its moments the next one.  CUDA-core
 * form only (EUNSUPPORTED otherwise); not on a shard (EUNSUPPORTED). */
oais_status oais_zja_round(oais_ctx* ctx, double cess_frac, double ess_frac, int32_t T_next, oais_round_result* out);

/* Resampling record of the last oasmc_round: ess [T] (ESS of w_{t^-} at every step),
 * resampled [T] (1 where a segment closed, including t = T), ancestors [N] (int64, the
 * ancestor indices of the last intermediate event; undefined if there was none).
 * Host arrays, each may be NULL.  EINVAL if the last round was an OAIS round. */
oais_status oais_get_resampling(const oais_ctx* ctx, double* ess, int32_t* resampled, int64_t* ancestors);

/* Stand-alone ASMC(N, B_T) (Alg. 1) with adaptive resampling at threshold ess_frac on the
 * schedule beta [T+1] (host) with step sizes eps [T] (host, NULL for 0.5/sqrt(d)).  Allocates
 * its own device memory (cudaMalloc) for the call.  Outputs (host, may be NULL): out,
 * log_ghat [T][3], ess_trace [T], resampled [T]. */
oais_status asmc_run(const oais_target* target, const oais_move* move, int64_t N, const double* beta,
                     int32_t T, const double* eps, double ess_frac, uint64_t seed, void* stream,
                     oais_round_result* out, double* log_ghat, double* ess_trace, int32_t* resampled);

/* Sharding across processes (OAIS particles are independent within a round, Sec. 5.1.2):
 * this context's N particles are [n_offset, n_offset + N) of a run of N_total; particle n
 * draws from counter n, so the union of the shards is the same sample as one context with
 * N_total particles.  A round is then split in two:
 *   oais_round_local:  the sweep of this shard and its reductions; returns host arrays
 *     log_ghat [T][3] (log g_hat_{t,i} over this shard), accepted [T] (accepted-move counts)
 *     and lse [2] (log sum w_T, log sum w_T^2 over this shard), T in *T.
 *   oais_round_commit: takes the statistics merged over all shards -- log_ghat and lse by
 *     log-sum-exp over shards, accepted by summing -- forms log Z_hat = lse[0] - log N_total,
 *     ESS and SE, and installs OptimiseSchedule(T_next, ...) exactly as oais_round does.
 * The exchange itself (an all-gather of 4T + 2 doubles per shard) is the caller's.
 * ASMC resamples across all particles and is not sharded (oasmc_round returns
 * EUNSUPPORTED on a shard); oais_round returns EINVAL on a shard. */
oais_status oais_set_shard(oais_ctx* ctx, int64_t n_offset, int64_t N_total);
oais_status oais_round_local(oais_ctx* ctx, double* log_ghat, double* accepted, double* lse, int32_t* T);
oais_status oais_round_commit(oais_ctx* ctx, int32_t T_next, const double* log_ghat, const double* accepted,
                              const double* lse, oais_round_result* out);

/* Checkpoint / resume between rounds.  The state of Alg. 2 between rounds is the round
 * counter, the next schedule and its step sizes, the seed and the shard; the particles are
 * redrawn every round, and the counter-based random numbers make a resumed round
 * bit-identical to an uninterrupted one.  oais_state_bytes gives the size of the blob;
 * oais_save_state writes it into host memory; oais_load_state restores it into a context
 * created for the same target, move and N (EINVAL otherwise, the context unchanged).  A blob
 * is checked as the setters check their arguments (schedule as oais_set_schedule, step sizes
 * finite and > 0, shard block as oais_set_shard); a successful load discards the results of
 * any round run before it (oais_logZ and the other last-round queries return EINVAL until the
 * next round completes). */
oais_status oais_state_bytes(const oais_ctx* ctx, size_t* bytes);
oais_status oais_save_state(const oais_ctx* ctx, void* buf, size_t bytes);
oais_status oais_load_state(oais_ctx* ctx, const void* buf, size_t bytes);

/* log Z_hat and its delta-method SE from the last completed round. EINVAL if none. */
oais_status oais_logZ(const oais_ctx* ctx, double* logZ, double* se);

/* Statistics of the last completed round, host arrays sized by *T (query with NULLs):
 * log_ghat [T][3] = log g_hat_{t,i}; D_hat [T]; beta [T+1] (the schedule that ran);
 * accept [T] mean MH acceptance per step.  Any output pointer may be NULL. */
oais_status oais_get_stats(const oais_ctx* ctx, double* log_ghat, double* D_hat, double* beta,
                           double* accept, int32_t* T);

/* ELBO terms of the last completed round, host [T] (query *T with elbo_terms = NULL):
 * elbo_terms[t-1] = sum_n W_{t-1}^n log g_t^n, the step-t term of the ELBO estimator of the
 * paper's section on the KL divergence of a schedule, with W_{t-1} the normalised weights
 * since the last resampling.  Reading of the printed estimator: its weights are the
 * normalised W of Alg. 1, so no further 1/N factor applies.  EINVAL before the first round
 * and after a sharded round (the terms are per shard there). */
oais_status oais_get_elbo(const oais_ctx* ctx, double* elbo_terms, int32_t* T);

/* The schedule the next round will run (host [*T + 1]; query *T with beta = NULL) and
 * its step sizes (host [*T], may be NULL). */
oais_status oais_get_schedule(const oais_ctx* ctx, double* beta, double* eps, int32_t* T);

/* Replace the next round's schedule and step sizes (host arrays; eps may be NULL to keep
 * the rule 0.5/sqrt(d)). */
oais_status oais_set_schedule(oais_ctx* ctx, const double* beta, const double* eps, int32_t T);

/* Final particles of the last round: logw [N] (log w_T), ell [N] (log L(X_T)) as double,
 * x [d][N] structure-of-arrays in the family's precision (double for GAUSS, float otherwise).
 * Device pointers of the context's workspace, valid until the next round or oais_destroy. */
oais_status oais_particles(const oais_ctx* ctx, const double** logw, const double** ell,
                           const void** x);

/* Fisher-identity gradient of log Z with respect to theta = (log s, log p0):
 * grad_theta log Z = E_pi[grad_theta log gamma(x; theta)] (not in the paper; the weighted
 * expectation estimator of eq. estimator_pi_t with the final weights and states of the last
 * round).  grad[0] = sum_n W_n (|x_n|^2 / s^2 - d)  (reference scale s),
 * grad[1] = sum_n W_n d log L(x_n)/d log p0 for the Gaussian (-2 log L) and linear-regression
 * (-n - 2 log L - n log(2 pi p0^2)) families, NaN for the others.  grad: host [2].
 * A ratio estimator: consistent, biased at finite N.  Synchronises the context's stream. */
oais_status oais_grad_logZ(oais_ctx* ctx, double* grad);

/* The target's potential for a batch of states (the forward and backward of the likelihood
 * used inside MALA and HMC): ell[n] = log L(x_n) and, if d_grad != NULL,
 * grad[i][n] = d log L / d x_i at x_n.  d_x, d_grad: device [d][N] in the family's precision
 * (double for GAUSS, float otherwise); d_ell: device [N] doubles.  Ordered on `stream`.
 * With the streamed tensor-core contraction the evaluation is the streamed kernel's own
 * (X~, two-term f16 operands) and the call waits for it; with the resident tensor-core form
 * it is the fp32 CUDA-core evaluation of X. */
oais_status oais_potential(oais_ctx* ctx, const void* d_x, int64_t N, double* d_ell, void* d_grad,
                           void* stream);

void oais_destroy(oais_ctx* ctx);
const char* oais_last_error(const oais_ctx* ctx);
const char* oais_status_string(oais_status s);

/* Alg. 3 OptimiseSchedule on the host: D_hat_t = log g2 - 2 log g1 + log g0 (clamped at 0),
 * Lambda_hat_t = cumulative sum of sqrt(D_hat), a monotone cubic Hermite interpolant through
 * the knots (Lambda_hat_t, beta_t) (equal Lambda_hat knots dropped, the first kept), and
 * beta*_t' = interp(Lambda_hat_T t'/T').  All host arrays: beta [T+1], log_ghat [T][3],
 * beta_next [T_next+1], D_hat [T] and Lambda [T+1] (both may be NULL).  No device work. */
oais_status oais_optimise_schedule(int32_t T, const double* beta, const double* log_ghat,
                                   int32_t T_next, double* beta_next, double* D_hat,
                                   double* Lambda);

/* Merge of per-shard round statistics for oais_round_commit (Sec. 5.1.2: within a round the
 * particles are independent, so a sum over all particles is the sum of the shards' sums).
 * Inputs are the P shards' outputs of oais_round_local, stacked in rank order (host arrays):
 * log_ghat [P][T][3], accepted [P][T], lse [P][2].  Outputs (host): log_ghat_out [T][3] and
 * lse_out [2], each the log-sum-exp over shards of the inputs at that position (maximum, then
 * the sum of exp(a_p - maximum) in rank order: every rank given the same inputs gets the same
 * bits; -inf entries are zero sums), and accepted_out [T], the sums of the counts.  No device
 * work.  EINVAL for P < 1, T < 1 or a null pointer. */
oais_status oais_merge_shard_stats(int32_t P, int32_t T, const double* log_ghat, const double* accepted,
                                   const double* lse, double* log_ghat_out, double* accepted_out,
                                   double* lse_out);

/* A starting rule for the per-step sizes of a first round (the paper fixes none; App. on
 * propagation-kernel adaptation tunes them between rounds): eps[t-1] = c / sqrt(1/s^2 +
 * beta[t] kappa), t = 1..T, i.e. the scale of pi_beta_t along a typical direction under a
 * Gaussian approximation whose precision is the reference's plus beta_t times a diagonal
 * curvature estimate kappa of -log L, times the kernel's dimension scaling c (RWMH 2.38/sqrt(d),
 * MALA 1.2 d^(-1/6), HMC d^(-1/4)).  kappa: GAUSS 1/p0^2; LOGREG sum_rj X_rj^2 / (4 d); LINREG
 * sum_rj X_rj^2 / (d p0^2); GMM 1/p0; UNID m q (1 - q)^-1 q^2 with q = k/m.  target as for
 * oais_init (X read from host or device memory per on_device; contraction ignored); beta: host
 * [T+1]; eps: host [T].  No device work beyond reading a device-resident X. */
oais_status oais_default_step_sizes(const oais_target* target, int32_t move_kind, const double* beta, int32_t T,
                                    double* eps);

/* ---------------------------------------------------------------------------------
 * Kernel-level entry points (device pointers only, no host synchronisation).
 * --------------------------------------------------------------------------------- */

/* Number of StepPartial records per step the sweep writes for N particles (one per CTA). */
int32_t oais_sweep_blocks(int64_t N);

/* Bytes of one StepPartial record: shift m[3] (double), sum s[3] (double), accepted (u32). */
int32_t oais_step_partial_bytes(void);

/* The loop-swapped OAIS sweep (Alg. 1 with the particle loop outside, Sec. 5.1.2) over
 * particles n_offset .. n_offset+N-1 of the counter space.
 * d_data: the padded device layout built by oais_prepare_target (opaque, from the context) --
 * use oais_ctx_sweep instead unless you manage it yourself.  Outputs (device):
 * logw [N], ell [N] doubles, x [d][N], partials [T][oais_sweep_blocks(N)] records,
 * status (u32, bit 0 set on a non-finite value; the caller zeroes it).
 * tag = round | (problem << 16) selects the random streams. */
oais_status oais_ctx_sweep(oais_ctx* ctx, int32_t T, const double* d_beta, const double* d_eps,
                           uint64_t seed, uint32_t tag, int64_t n_offset, int64_t N,
                           double* d_logw, double* d_ell, void* d_x, void* d_partials,
                           uint32_t* d_status, void* stream);

/* Merge the per-CTA records of every step in a fixed order (deterministic):
 * log_ghat [T][3] = log g_hat_{t,i}, accept [T] = accepted / (N * moves).  Device pointers. */
oais_status oais_merge_stats(const void* d_partials, int32_t nblocks, int32_t T, int64_t N,
                             int32_t moves, double* d_log_ghat, double* d_accept, void* stream);

/* out[0] = log sum_n exp(a_n), out[1] = log sum_n exp(2 a_n), deterministic two-pass
 * reduction.  d_scratch: device memory of oais_logsumexp_scratch_bytes(n). */
size_t oais_logsumexp_scratch_bytes(int64_t n);
oais_status oais_logsumexp(const double* d_a, int64_t n, double* d_out, void* d_scratch,
                           void* stream);

/* ---------------------------------------------------------------------------------
 * Allocation-free log-sum-exp.  No counterpart in the paper: this is a service for
 * callers that cannot call cudaMalloc or take scratch memory from elsewhere -- code
 * running inside a CUDA-graph capture that must not allocate, under another allocator
 * that owns all device memory, or in a fixed-budget loop that may only hand over its
 * input and output buffers.  Same result as oais_logsumexp (out[0] = log sum exp a,
 * out[1] = log sum exp 2a, deterministic), but the scratch lives in a fixed device array
 * inside the library (128 KiB per GPU that loads the library, held until the process
 * exits), so no allocation happens and the caller passes no scratch.
 *   d_a: device [n] doubles; d_out: device [2] doubles; stream as above.
 *   n: 1 .. OAIS_LOGSUMEXP_NOALLOC_MAX_N, else OAIS_EINVAL (nothing launched).
 *   All calls on a device share the array and it keeps the last call's contents; calls
 *   whose kernels overlap on the GPU (unordered streams or threads) race and may give
 *   wrong results -- order them on one stream.
 *   The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make it before any stream capture.
 *   The cached address is only valid for the device's current primary context: do not call
 *   this entry point on a device after cudaDeviceReset in the same process.
 *   Errors: OAIS_EINVAL (null pointer, n out of range), OAIS_ECUDA (no device, lookup or
 *   launch failed; an error left pending by an earlier call is cleared first), with the text
 *   in oais_last_error(NULL).
 *   Calls no cudaMalloc/cudaFree and no allocating library routine. */
#define OAIS_LOGSUMEXP_NOALLOC_MAX_N 16777216LL
oais_status oais_logsumexp_noalloc(const double* d_a, int64_t n, double* d_out, void* stream);

/* ------------------------------------------------------------------------------------------
 * Many independent problems in one launch.
 *
 * A batch holds P independent OAIS runs (Alg. 2 each, Sec. 5.1.2 sweeps) of one family
 * (LOGREG with MALA, or LINREG with MALA or HMC), each with its own data (n and d <= 128 may
 * differ), particles, statistics and schedule; problem p draws its random numbers with
 * problem index p in the counter tag (round | p << 16), so its round is the same computation
 * as a single context given oais_set_problem(ctx, p).  Every problem uses the streamed
 * tensor-core contraction (X~ = f16(bf16(X)), see oais_target.contraction).
 *
 * oais_batch_round runs one round of every problem: the sweeps of all (problem, tile)
 * items go through ONE persistent kernel (one CTA per SM taking items from a queue ordered
 * by decreasing cost, so long problems start first and short ones fill the tail), then each
 * problem's moment records are merged and its schedule re-optimised (Alg. 3) as in
 * oais_round.  The device work of a round is captured once as a CUDA graph and replayed
 * while the schedule length stays the same.  All problems must hold schedules of the same
 * length (they do when every round is given the same T_next).
 *
 *   targets   [P] target descriptions (copied at init, as oais_init)
 *   beta      [T+1] first schedule, shared; eps [P][T] step sizes or NULL (0.5 / sqrt(d))
 *   workspaces, ws_bytes  [P] caller-owned device workspaces of problem p (size from
 *             oais_workspace_bytes with contraction OAIS_CONTRACT_BF16_TC_STREAM), or NULL:
 *             the batch allocates them
 *   results   [P] per-problem round results (may be NULL)
 * oais_batch_autotune chooses the tile shape of the batched kernel for each width class
 * present (d_pad 16, 32, 64, 128; classes 0..3): it times the class's largest problem over
 * T_probe steps through the batched kernel for every candidate pair of rows per X chunk (the
 * K extent of the backward contraction and the N extent of the forward one: 64, and 128 for
 * logistic problems with d_pad <= 64, which have one forward accumulator instead of two) and
 * ring depth (X chunk buffers in shared memory: 2,
 * 3, 4, 6, 8 as far as shared memory holds them), and keeps the fastest pair; chosen [4]
 * receives the depths (0 = class absent).  The probe sweeps overwrite the problems' particle
 * buffers (the next round redraws them).  The ring depth changes no result; the chunk size
 * changes the order of the fp32 partial sums of log L (rows are split differently between a
 * particle's two threads), so a run is reproducible for a given shape, and the shape the
 * autotuner chose can be read and pinned:
 * oais_batch_tile_shape writes the chunk rows and ring depth the class's problems run with
 * (0, 0 for an absent class); oais_batch_set_tile_shape sets them (chunk_rows 0 = 64, 64 or
 * 128, else OAIS_EINVAL; stages
 * 0 = the deepest ring that fits), OAIS_EUNSUPPORTED when a problem of the class cannot take
 * the chunk size (linear regression, d_pad 128: their chunk images depend on it).
 * oais_batch_context lends problem p's context (owned by the batch) for the per-problem
 * queries (oais_logZ, oais_get_stats, oais_particles, ...).
 * Errors: OAIS_EINVAL / OAIS_EUNSUPPORTED for bad lists (mixed families, d > 128), the
 * single-context errors otherwise; oais_batch_last_error gives the detail.  No counterpart in
 * the paper: a way of running its method on many posteriors at once.
 * ------------------------------------------------------------------------------------------ */
typedef struct oais_batch oais_batch;
oais_status oais_batch_init(oais_batch** out, int32_t P, const oais_target* targets, const oais_move* move,
                            int64_t N, const double* beta, int32_t T, int32_t T_max, const double* eps,
                            uint64_t seed, void* const* workspaces, const size_t* ws_bytes, void* stream);
oais_status oais_batch_round(oais_batch* b, int32_t T_next, oais_round_result* results);
oais_status oais_batch_autotune(oais_batch* b, int32_t T_probe, int32_t* chosen);
oais_status oais_batch_tile_shape(const oais_batch* b, int32_t width_class, int32_t* chunk_rows, int32_t* stages);
oais_status oais_batch_set_tile_shape(oais_batch* b, int32_t width_class, int32_t chunk_rows, int32_t stages);
oais_status oais_batch_context(oais_batch* b, int32_t p, oais_ctx** ctx);
const char* oais_batch_last_error(const oais_batch* b);
void oais_batch_destroy(oais_batch* b);

/* Budget (Alg. 2; the paper's rule for increasing N and T between rounds): multiply the
 * particle count and the schedule length by sqrt(2) until the particle count reaches N_cap
 * (the step that would pass it stops at N_cap), then keep N and double T; T never exceeds
 * T_cap.  N_next is rounded to the nearest multiple of 128 (at least 128, at most N_cap),
 * T_next to the nearest integer (at least T + 1 while T < T_cap).  Pure host arithmetic; OAIS_EINVAL for N, T < 1 or caps below them. */
oais_status oais_budget(int64_t N, int32_t T, int64_t N_cap, int32_t T_cap, int64_t* N_next, int32_t* T_next);

/* Final reweighting to the data X for the tensor-core forms (on = 1; 0 switches it off, the
 * default).  Those forms sample the posterior of the rounded data X~ (bf16, or f16 of bf16, or
 * FP8 with row scales), whose log Z differs from that of X by the quantisation shift.  With the
 * reweighting each OAIS round appends one more target to its annealing sequence, gamma(.; X) at
 * beta = 1 after gamma(.; X~), reached without a move: every particle's weight is multiplied
 * by L(x_T; X) / L(x_T; X~), L(.; X) evaluated in fp32 on the CUDA cores (Alg. 1's
 * incremental weight for that step), so log Z_hat estimates log Z of X and stays unbiased for Z.
 * The round's moments, D_hat and next schedule are those of the beta path (the extra step is not
 * part of it); log w and log L of oais_particles include the step, and its contribution to the
 * KL estimate goes into the round result's kl (elbo covers the beta path).  EUNSUPPORTED for the
 * CUDA-core form (which samples X already) and for d > 32 (no fp32 copy of X is kept). */
oais_status oais_set_exact_data(oais_ctx* ctx, int32_t on);

/* Active particle count of the next rounds (1 <= N <= the count the context was created
 * with; unsharded contexts): a round with more particles needs no new workspace as long as
 * the context was created with the largest count (Budget). */
oais_status oais_set_particles(oais_ctx* ctx, int64_t N);

/* Problem index p (0 <= p <= 65535) of a single context: its random numbers use the tag
 * round | p << 16, as problem p of a batch does.  Default 0. */
oais_status oais_set_problem(oais_ctx* ctx, int32_t p);

/* ------------------------------------------------------------------------------------------
 * Test support: failure paths without a GPU fault.  No counterpart in the paper.
 *
 * oais_arm_fault arms one fault, made on the host side, for the next round of the context
 * (oais_round, oasmc_round or oais_round_local), so that a test can drive a round into each of
 * its failure paths while the GPU stays healthy; the fault is disarmed when that round ends.
 *   OAIS_FAULT_NONE: disarm.
 *   OAIS_FAULT_NAN_DATA: before the round, element 0 of every device copy of the data X that
 *     the context holds (the CUDA-core layout, the resident bf16 image, the streamed f16 image)
 *     is overwritten with a quiet NaN by a host-to-device copy, and its value is copied back
 *     when the round ends.  Every log-likelihood is then NaN and the round returns
 *     OAIS_ENONFINITE.  EUNSUPPORTED for FP8 storage.
 *   OAIS_FAULT_WITHHOLD_HANDOFF: a tensor-core sweep that runs as a persistent grid (more tiles
 *     of 128 particles than the resident groups or CTAs of one wave) raises none of its hand-off
 *     flags, so every resumed tile's bounded wait for its flag gives up after wait_seconds
 *     (0: the default limit of 2 s), the CTA stops its work and releases its tensor memory, and
 *     the round returns OAIS_ETIMEOUT.  A sweep that fits in one wave hands nothing over and is
 *     not affected.  EUNSUPPORTED for the CUDA-core form.
 * wait_seconds: in [0, 60], used by OAIS_FAULT_WITHHOLD_HANDOFF only.  A failed round leaves
 * the last completed round's results and the next round's schedule as they were (the anytime
 * property, Sec. 1), and does not advance the round counter: the next round draws the random
 * numbers the failed one drew.  The particle buffers (oais_particles) hold the failed round's
 * values.  EINVAL for an unknown kind. */
typedef enum { OAIS_FAULT_NONE = 0, OAIS_FAULT_NAN_DATA = 1, OAIS_FAULT_WITHHOLD_HANDOFF = 2 } oais_fault;
oais_status oais_arm_fault(oais_ctx* ctx, int32_t kind, double wait_seconds);

#ifdef __cplusplus
}
#endif
#endif /* OAIS_H_ */
