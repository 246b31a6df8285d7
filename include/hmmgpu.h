/*
 * hmmgpu -- C ABI of the GB300 (sm_103a) hidden-Markov-model hot path.
 *
 * The library implements, on one GPU, the data-parallel hot path of the HMM
 * method of "libhmm: A Modern C++20 Library for Hidden Markov Models with
 * Correct MLE Emission M-Steps" (arXiv 2605.29208):
 *   - emission log-densities log b_j(y_t)              (paper Sec. 4.1-4.5)
 *   - log-space forward / backward recursions           (Sec. 3.2, Eq. 1-2)
 *   - posteriors gamma_t(j), xi_t(i,j)                  (Sec. 3.1, 3.4)
 *   - weighted sufficient statistics and the M-steps    (Sec. 4, Eq. 5-24)
 *   - Baum-Welch iterations (fit)
 *   - max-plus Viterbi with backpointer traceback       (Sec. 3.3, Eq. 3-4)
 *
 * Conventions (every entry point):
 *   - Returns hmm_status; never throws or aborts across the ABI.  On error
 *     hmm_last_error() gives a thread-local message.
 *   - Pointers named d_* / inside hmm_batch are DEVICE pointers owned by the
 *     caller (e.g. torch.Tensor.data_ptr()); pointers named h_* are host
 *     pointers owned by the caller.  Handles (hmm_ctx, hmm_model, hmm_stats,
 *     hmm_plan) are owned by the library: create/destroy pairs.
 *   - Work is enqueued on the given CUDA stream (0 = legacy default stream);
 *     device outputs are valid once that stream has synchronised.  Calls
 *     that return host data synchronise the stream themselves.
 *   - Asynchronous numeric problems (NaN observations, zero-probability
 *     sequences) are reported through the per-sequence log-likelihood
 *     (-inf or NaN) and hmm_ctx_status().
 *
 * Layouts:
 *   - Packed ragged batch: values[total_T * dim] row-major float32 (all
 *     sequences concatenated), offsets[n_seq + 1] int64 (sequence s covers
 *     rows offsets[s] .. offsets[s+1]-1; offsets[0] = 0,
 *     offsets[n_seq] = total_T, non-decreasing), model_id[n_seq] int32 in
 *     [0, n_models).  Empty sequences (length 0) are allowed and get
 *     log-likelihood 0.
 *   - Per-time-step outputs (gamma, logb) are [total_T][n_states] row-major
 *     float32 in the same row order as the batch.
 *   - Parameter blob (float64, host): the models one after another; model m
 *     holds pi[N], A[N][N] (row-stochastic, a_ij = P(q_{t+1}=j | q_t=i)),
 *     then for each state j its family parameters (hmm_family_param_count).
 */
#ifndef HMMGPU_H
#define HMMGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HMM_OK = 0,
  HMM_E_ARG = 1,          /* invalid argument (null pointer, bad size, bad family) */
  HMM_E_NOMEM = 2,        /* device or host allocation failed                       */
  HMM_E_CUDA = 3,         /* a CUDA runtime call failed (message has the details)   */
  HMM_E_NUMERIC = 4,      /* non-finite result detected                              */
  HMM_E_TIMEOUT = 5,      /* a bounded device wait expired                           */
  HMM_E_BUSY = 6,         /* server queue full                                       */
  HMM_E_NOTREADY = 7,     /* server request still pending                            */
  HMM_E_UNSUPPORTED = 8   /* valid request outside what this library implements      */
} hmm_status;

/* Emission families (paper Sec. 4).  Parameters per state, in blob order:
 *   HMM_GAUSS       mu, sigma2                          (Sec. 4.1)
 *   HMM_POISSON     lambda                              (Sec. 4.1)
 *   HMM_GAMMA       alpha (shape), beta (RATE)          (Sec. 4.2, Eq. 7-8)
 *   HMM_BETA        a, b                                (Sec. 4.2, Eq. 9-10)
 *   HMM_WEIBULL     k (shape), lambda (scale)           (Sec. 4.2, Eq. 11)
 *   HMM_NEGBIN      r, p     (mean r(1-p)/p)            (Sec. 4.2)
 *   HMM_STUDENT_T   mu, sigma2, nu                      (Sec. 4.3, Eq. 13-19)
 *   HMM_VONMISES    mu, kappa                           (Sec. 4.1-4.2, Eq. 12)
 *   HMM_DIAG_GAUSS  mu[D], var[D]                       (Sec. 4.5, Eq. 20-21)
 *   HMM_FULL_GAUSS  mu[D], cov[D][D]                    (Sec. 4.5, Eq. 22-24)
 *   HMM_DISCRETE    p[K] symbol probabilities            (Sec. 4, "Discrete
 *                   (categorical)"): the model's `dim` is the number of
 *                   symbols K (2..1024); observations are the symbol indices
 *                   0..K-1, one float per step (a batch's dim is 1)
 *   HMM_LOGNORMAL   mu, sigma2 of log y                 (Sec. 4.1 "Log-normal")
 *   HMM_EXPONENTIAL lambda (rate)                       (Sec. 4.1 "Exponential")
 *   HMM_RAYLEIGH    sigma2                              (Sec. 4.1 "Rayleigh")
 *   HMM_UNIFORM     a, b (a < b; closed interval)       (Sec. 4.1 "Uniform")
 *   HMM_CHISQ       nu (degrees of freedom)             (Sec. 4.2 "Chi-squared")
 *   HMM_PARETO      xm, alpha (scale, shape)            (Sec. 4.2 "Pareto")
 * Observations outside a family's support (y <= 0 for Gamma/Weibull/
 * log-normal/chi-squared, y < 0 for exponential/Rayleigh, y outside (0,1)
 * for Beta, outside [a, b] for uniform, y < xm for Pareto, non-integer or
 * negative counts) have density 0.  The last six families (and the
 * discrete one) evaluate their densities into a log b table; a model set
 * holds families of one group only: the first eight scalar families, the
 * two multivariate ones, the discrete one, or the last six. */
typedef enum {
  HMM_GAUSS = 0, HMM_POISSON = 1, HMM_GAMMA = 2, HMM_BETA = 3, HMM_WEIBULL = 4,
  HMM_NEGBIN = 5, HMM_STUDENT_T = 6, HMM_VONMISES = 7, HMM_DIAG_GAUSS = 8,
  HMM_FULL_GAUSS = 9, HMM_DISCRETE = 10, HMM_LOGNORMAL = 11, HMM_EXPONENTIAL = 12,
  HMM_RAYLEIGH = 13, HMM_UNIFORM = 14, HMM_CHISQ = 15, HMM_PARETO = 16,
  HMM_INDEP = 17          /* independent components: see hmm_model_create_indep */
} hmm_family;

typedef struct hmm_ctx_s* hmm_ctx;       /* device + workspace            */
typedef struct hmm_model_s* hmm_model;   /* M models x N states on device */
typedef struct hmm_stats_s* hmm_stats;   /* FP64 sufficient statistics    */
typedef struct hmm_plan_s* hmm_plan;     /* host-side schedule of a batch */

typedef struct {
  const float* values;        /* device [total_T * dim]                        */
  const int64_t* offsets;     /* device [n_seq + 1]                            */
  const int32_t* model_id;    /* device [n_seq]                                */
  int64_t n_seq;
  int64_t total_T;
  int32_t dim;                /* 1 for scalar families, D for multivariate     */
  hmm_plan plan;              /* optional (may be NULL): a plan made by
                                 hmm_plan_create for exactly this batch; without
                                 one each call copies offsets/model_id to the
                                 host and plans on the fly (synchronous).     */
} hmm_batch;

/* Options of the M-step (paper Sec. 4).  Zero-initialised fields take the
 * defaults given in brackets. */
typedef struct {
  double collapse_eps;   /* [1e-8]  Sec. 4.4: N_j below this keeps theta_j      */
  double tikhonov_eps;   /* [1e-6]  Sec. 4.5: Sigma + eps I                     */
  int32_t newton_maxit;  /* [50]    Newton iterations (Gamma/Beta/Weibull/...)  */
  double newton_tol;     /* [1e-10] |d theta| <= tol * max(1, |theta|)          */
  int32_t nu_mode;       /* [0]     Student-t nu equation: 0 = ECM equation with
                                    the E[log U] constant, 1 = Eq. 18 as printed */
  int32_t update_transitions; /* [1 when the struct is NULL] 0 keeps pi and A    */
  double dirichlet_A;    /* [0]     MAP Baum-Welch (the MAP trainer the paper
                                    names, Sec. 5.6; reading): symmetric
                                    Dirichlet concentration of every row of A;
                                    the update adds dirichlet_A - 1 pseudo-counts
                                    to each row's transitions (values <= 1: none) */
  double dirichlet_pi;   /* [0]     the same for pi                              */
} hmm_mstep_opts;

typedef struct {
  int32_t max_iter;      /* number of Baum-Welch iterations                      */
  double tol;            /* stop when |dlogL| <= tol * |logL| (0: run max_iter)  */
  hmm_mstep_opts mstep;
  int32_t trainer;       /* [0] Baum-Welch; 1 Viterbi training (hmm_estep_viterbi
                            as the E-step; the trace then holds the sums of the
                            best paths' log-probabilities)                     */
} hmm_fit_opts;

/* ---------------------------------------------------------------- basics */
const char* hmm_status_string(hmm_status s);
/* Thread-local text of the last error raised by a call on this thread. */
const char* hmm_last_error(void);
/* Library version string. */
const char* hmm_version(void);

/* Number of float64 parameters of ONE state of a family with dimension dim
 * (see hmm_family); -1 for an unknown family. */
int32_t hmm_family_param_count(int32_t family, int32_t dim);
/* Total size in float64 values of the parameter blob of n_models models. */
int64_t hmm_param_blob_size(int32_t n_models, int32_t n_states, int32_t dim,
                            const int32_t* h_family);
/* Model-selection criteria of one fitted model (the paper names AIC, BIC and
 * AICc for model comparison, Sec. 5.6 and the multivariate example, without
 * formulas; these are the textbook forms).  Host-only arithmetic, no device
 * work.  k = the number of free parameters: (N - 1) initial probabilities,
 * N (N - 1) transition probabilities and N times the free emission
 * parameters of the family (the count of hmm_family_param_count, except
 * discrete K - 1 and full covariance D + D (D + 1) / 2);
 *   h_out[0] = k, h_out[1] = AIC = 2 k - 2 logL,
 *   h_out[2] = BIC = k ln(n_obs) - 2 logL,
 *   h_out[3] = AICc = AIC + 2 k (k + 1) / (n_obs - k - 1)  (+inf when
 *              n_obs <= k + 1).
 * loglik: the model's total log-likelihood (natural log); n_obs: its number
 * of observations (time steps).  HMM_E_ARG for an unknown family, n_states
 * < 1, n_obs < 1 or a NULL h_out. */
hmm_status hmm_information_criteria(int32_t family, int32_t n_states, int32_t dim, double loglik,
                                    int64_t n_obs, double* h_out);

/* ------------------------------------------------------------ context */
/* Context options (hmm_ctx_set_option). */
typedef enum {
  HMM_OPT_PROFILE = 1,        /* 1: time every kernel launch with CUDA events on
                                 its stream (read with hmm_ctx_profile_read)     */
  HMM_OPT_ESTEP_LANES = 2,    /* lanes per chain of the small-N E-step, 0 = auto */
  HMM_OPT_VITERBI_LANES = 3,  /* lanes per chain of the small-N Viterbi, 0 = auto */
  HMM_OPT_PLAIN_ESTEP = 4,    /* 1: run E-steps with the plain float32 log-space
                                 kernels (straight log-sum-exp of Sec. 3.2, N^2
                                 exponentials per step) -- the GPU baseline     */
  HMM_OPT_TENSOR_RECURRENCE = 5, /* 1: padded N in {64, ..., 512} run the forward
                                 and backward recursions (Eq. 2 in the shifted
                                 exp-space form) as tcgen05 GEMMs with FP16
                                 operands and FP32 accumulation; the shift and
                                 the log-likelihood stay in float64.  0 (default):
                                 float32 CUDA-core recursions.  2: the same with
                                 TF32 operands (10 significant bits as FP16, the
                                 float32 exponent range) where padded N <= 256;
                                 at 512 the FP16 recursion runs.  The FP16 and
                                 TF32 paths' error against float64 is larger than
                                 the float32 path's (about 1e-3 absolute on
                                 gamma).                                          */
  HMM_OPT_TIME_PARALLEL = 6     /* forward-backward without statistics at padded
                                 N <= 32: 0 (default) runs the time-parallel form
                                 (chunk transfer matrices, boundary vectors,
                                 chunks recomputed in parallel) when the batch
                                 has at most as many sequences as the GPU has
                                 SMs and a sequence of at least 2048 steps;
                                 1 always; -1 never.                             */
} hmm_option;

/* Kernel timing slots of hmm_ctx_profile_read. */
typedef enum {
  HMM_KT_ESTEP = 0,           /* fused E-step kernel                     */
  HMM_KT_REDUCE = 1,          /* fixed-order statistic reductions        */
  HMM_KT_MSTEP = 2,           /* M-step + derived tables                 */
  HMM_KT_VITERBI = 3,         /* Viterbi forward + traceback             */
  HMM_KT_EMISSION = 4,        /* emission log-density tables             */
  HMM_KT_PLAIN = 5,           /* plain float32 log-space E-step kernels  */
  HMM_KT_XI = 6,              /* tensor-core xi GEMM (inside HMM_KT_REDUCE) */
  HMM_KT_SLOTS = 8
} hmm_kernel_slot;

/* Creates a context on CUDA device `device`.  workspace_bytes is an initial
 * reservation (0: grow on demand).  The context owns its scratch memory. */
hmm_status hmm_ctx_create(int device, size_t workspace_bytes, hmm_ctx* out);
hmm_status hmm_ctx_destroy(hmm_ctx ctx);
/* Sticky device-side status word (HMM_OK or the first error raised by a
 * kernel since the last call); synchronises `stream`, then clears it. */
hmm_status hmm_ctx_status(hmm_ctx ctx, void* stream);

/* Failure-detection self-test of the bounded device waits (the paper has no
 * counterpart; it checks the library's own error path).  Every mbarrier wait
 * of the tensor-core kernels gives up after a cycle limit and records
 * HMM_E_TIMEOUT in the context's sticky status instead of hanging the GPU.
 * This call launches one thread that waits, with that same bounded wait, on
 * an mbarrier phase nothing ever completes, with a limit of limit_cycles SM
 * clock cycles (1 .. the library's own limit, about 4e9), then returns;
 * hmm_ctx_status afterwards reports HMM_E_TIMEOUT and the context stays
 * usable.  h_waited (may be NULL; then the call does not synchronise)
 * receives the cycles the wait took.  HMM_E_ARG for a limit out of range. */
hmm_status hmm_ctx_wait_selftest(hmm_ctx ctx, int64_t limit_cycles, int64_t* h_waited, void* stream);

/* Sets a context option (hmm_option); unknown keys give HMM_E_ARG. */
hmm_status hmm_ctx_set_option(hmm_ctx ctx, int32_t key, int64_t value);
/* Accumulated device milliseconds and launch counts per timing slot
 * (h_ms / h_launches [n_slots], either may be NULL) of the launches recorded
 * while HMM_OPT_PROFILE was on; waits for the recorded events.  reset != 0
 * clears the totals.  Launches inside a graph capture are not timed. */
hmm_status hmm_ctx_profile_read(hmm_ctx ctx, double* h_ms, int64_t* h_launches,
                                int32_t n_slots, int32_t reset);

/* -------------------------------------------------------------- models */
/* n_models models of n_states states with observation dimension dim; the
 * family of model m is h_family[m] (host array).  Multivariate families need
 * dim >= 1, scalar families dim == 1.  State counts up to 1024. */
hmm_status hmm_model_create(hmm_ctx ctx, int32_t n_models, int32_t n_states,
                            int32_t dim, const int32_t* h_family, hmm_model* out);
/* Independent-components models (paper Sec. 4.5, "Independent
 * components"): every state of model m emits y_t in R^dim with density
 * b_j(y_t) = prod_d phi_{m,d,j}(y_td), where component d of model m is the
 * scalar family h_comp[m * dim + d] with its own parameters per state, and
 * the M-step runs each component's scalar update with the same occupancy
 * weights gamma_t(j).  Component families: HMM_GAUSS, HMM_POISSON,
 * HMM_GAMMA, HMM_BETA, HMM_STUDENT_T, HMM_VONMISES, HMM_LOGNORMAL,
 * HMM_EXPONENTIAL, HMM_RAYLEIGH, HMM_CHISQ (others: HMM_E_UNSUPPORTED);
 * 1 <= dim <= 32; state counts up to 1024.  Batches have dim = `dim`
 * (values [total_T][dim]).  Parameter blob per model: pi[N], A[N][N], then
 * per state j the parameters of component 0, component 1, ... in the order
 * of hmm_family (hmm_model_blob_size gives the total).  Statistics
 * (hmm_stats_get) per state j of an independent-components model: W, then
 * per component its sums (weights gamma_t(j)): GAUSS Wy, Wy^2; POISSON Wy;
 * GAMMA Wy, W log y, Wy^2; BETA Wy, Wy^2, W log y, W log(1-y); STUDENT_T
 * Wu, Wuy, Wuy^2, W(log u - u); VONMISES W cos y, W sin y; LOGNORMAL
 * W log y, W (log y)^2; EXPONENTIAL Wy; RAYLEIGH Wy^2; CHISQ W log y. */
hmm_status hmm_model_create_indep(hmm_ctx ctx, int32_t n_models, int32_t n_states, int32_t dim,
                                  const int32_t* h_comp, hmm_model* out);
/* Number of float64 values of `model`'s parameter blob (any family). */
int64_t hmm_model_blob_size(hmm_model model);
hmm_status hmm_model_destroy(hmm_model model);
/* Copies the float64 parameter blob (layout above, n_values entries) to the
 * device and refreshes the derived single-precision tables. */
hmm_status hmm_model_set_params(hmm_model model, const double* h_blob, int64_t n_values);
/* Copies the current parameters back (synchronises the model's last stream). */
hmm_status hmm_model_get_params(hmm_model model, double* h_blob, int64_t n_values);

/* k-means++ seeding and Lloyd iterations for R restarts at once, on the
 * device (the initialisation the paper names for Baum-Welch, Sec. 4.5,
 * without constants; the rules are the library's reading).  d_x [T][F]
 * float32 features (device, caller-owned); distances, sums and centres are
 * float64.  h_u [R][K] (host) uniforms in [0, 1) drawn by the caller: the
 * first centre of restart r is observation floor(u[r][0] T), centre j the
 * first observation whose running sum of D2 (squared distance to the
 * nearest centre so far) exceeds u[r][j] times the total (total 0:
 * floor(u[r][j] T)).  Then at most max_iter Lloyd passes: every observation
 * to its nearest centre (lowest index at ties), every non-empty cluster's
 * centre to the mean of its observations, until a pass changes no
 * assignment.  Outputs: d_centres [R][K][F] float64, d_labels [R][T] int32
 * (the last pass's assignments; untouched when max_iter is 0) and h_passes
 * [R] (host, may be NULL) the assignment passes run.  1 <= F <= 16,
 * 1 <= K <= 64, 1 <= R <= 65535; HMM_E_ARG otherwise or for a uniform
 * outside [0, 1).  Results are bitwise reproducible.  Synchronises
 * `stream` every 8 passes to stop once every restart has converged. */
hmm_status hmm_kmeans(hmm_ctx ctx, const float* d_x, int64_t T, int32_t F, int32_t K, int32_t R,
                      const double* h_u, int32_t max_iter, double* d_centres, int32_t* d_labels,
                      int32_t* h_passes, void* stream);

/* ---------------------------------------------------------------- plans */
/* Builds the schedule of a batch (processing order by family and length,
 * the per-model sequence lists used for the deterministic reductions).
 * h_offsets / h_model_id are host copies of the batch arrays. */
hmm_status hmm_plan_create(hmm_ctx ctx, hmm_model model, const hmm_batch* batch,
                           const int64_t* h_offsets, const int32_t* h_model_id,
                           hmm_plan* out);
hmm_status hmm_plan_destroy(hmm_plan plan);
/* Autotuner: times the fused E-step and the Viterbi kernel at every chain
 * width compiled for the model's state count on this batch (CUDA events on
 * `stream`, one warm-up and one timed run each) and stores the fastest widths
 * in batch->plan (which must be set), where every later call with that plan
 * uses them.  hmm_fit runs it by itself on a caller's plan that was never
 * tuned.  Synchronises `stream`.  h_ms (may be NULL) receives the measured
 * E-step and Viterbi milliseconds of the chosen widths. */
hmm_status hmm_plan_autotune(hmm_ctx ctx, hmm_model model, const hmm_batch* batch,
                             double* h_ms, void* stream);

/* ------------------------------------------------------------ inference */
/* Emission log-densities log b_j(y_t) (natural log) of every row of the batch
 * under the model of its sequence: d_logb [total_T][n_states].
 * Paper Sec. 4.1-4.5 (densities), used by Eq. 1-4. */
hmm_status hmm_emission_logpdf(hmm_ctx ctx, hmm_model model, const hmm_batch* batch,
                               float* d_logb, void* stream);

/* Forward-backward in log space (Sec. 3.2, Eq. 1-2): per-sequence
 * log-likelihood d_loglik[n_seq] (float64, natural log), and optionally the
 * occupancies gamma_t(j) (d_gamma [total_T][n_states], may be NULL) and the
 * posterior decoding argmax_j gamma_t(j) (Sec. 3.4; d_post_path [total_T]
 * int32, may be NULL; ties -> lowest j).  d_logb may be NULL (emissions
 * evaluated in the kernel from the model) or a [total_T][n_states] natural-log
 * table that replaces the model's emissions. */
hmm_status hmm_forward_backward(hmm_ctx ctx, hmm_model model, const hmm_batch* batch,
                                const float* d_logb, float* d_gamma,
                                int32_t* d_post_path, double* d_loglik, void* stream);

/* Forward-backward for callers that cannot allocate device memory at call
 * time (a caller-managed memory pool that must not be bypassed, a real-time
 * loop that cannot afford cudaMalloc's implicit synchronisation, a process
 * that has already claimed the free memory).  The paper has no counterpart:
 * this is an operational variant of hmm_forward_backward, with the same
 * outputs (d_loglik [n_seq] and d_gamma [total_T][n_states], both required),
 * but its scratch lives in a fixed 32 MiB array inside the library and the
 * call makes no device allocation of any kind.  Limit: total_T * padded
 * states * 4 + n_seq * 4 + 512 bytes must fit in 32 MiB (padded states:
 * n_states rounded up to a power of two, at most 32), else HMM_E_ARG.  The
 * batch's plan is ignored (sequences run in input order).  The array is
 * shared by every call in the process and kept between calls: calls whose
 * GPU work overlaps race on it, so order them on one stream.  The first call
 * on a device looks up the array's address; make it before any stream
 * capture.  Sizes, pointers and the family are checked on the host
 * (HMM_E_ARG / HMM_E_UNSUPPORTED); the contents of the device arrays are
 * checked on the device (offsets[0] = 0, non-decreasing, offsets[n_seq] =
 * total_T, model ids in [0, n_models)): a malformed batch processes no
 * sequence, writes NaN to every d_loglik entry and leaves HMM_E_ARG in the
 * context's sticky status (hmm_ctx_status).  The caller's current device is
 * restored before the call returns. */
hmm_status hmm_forward_backward_static(hmm_model model, const hmm_batch* batch,
                                       const float* d_logb, float* d_gamma,
                                       double* d_loglik, void* stream);

/* Max-plus Viterbi (Sec. 3.3, Eq. 3-4) with backpointer traceback:
 * d_path [total_T] int32 states, d_score [n_seq] float64 (natural log of the
 * best path's joint probability).  Ties: lowest predecessor index, lowest
 * final state.  d_logb as in hmm_forward_backward; with a table the decode
 * uses only float32 additions, subtractions and comparisons of that table and
 * the model's float32 log pi / log A. */
hmm_status hmm_viterbi(hmm_ctx ctx, hmm_model model, const hmm_batch* batch,
                       const float* d_logb, int32_t* d_path, double* d_score,
                       void* stream);

/* ------------------------------------------------------------ training */
hmm_status hmm_stats_create(hmm_ctx ctx, hmm_model model, hmm_stats* out);
hmm_status hmm_stats_destroy(hmm_stats stats);
/* Layout of the canonical statistics returned by hmm_stats_get, per model m
 * (float64): n_seq, sum of logL, then per state j: gamma1_j (sum over
 * sequences of gamma_1(j)), then the N x N matrix sum_t xi_t(i,j), then per
 * state j the family sums (Sec. 4, weights gamma_t(j)):
 *   GAUSS     W, Wy, Wy^2         POISSON  W, Wy
 *   GAMMA     W, Wy, W log y, Wy^2
 *   BETA      W, Wy, Wy^2, W log y, W log(1-y)
 *   WEIBULL   W, W log y, W (log y)^2
 *   NEGBIN    W, Wy, Wy^2
 *   STUDENT_T W, Wu, Wuy, Wuy^2, W(log u - u)   (u of Eq. 14, current params)
 *   VONMISES  W, W cos y, W sin y
 *   DIAG_GAUSS W, Wy_d (D), Wy_d^2 (D)
 *   FULL_GAUSS W, Wy_d (D), Wy_d y_e (D*D)
 *   DISCRETE  W 1[y = k] (K)
 *   LOGNORMAL W, W log y, W (log y)^2     EXPONENTIAL W, Wy
 *   RAYLEIGH  W, Wy^2                     CHISQ       W, W log y
 *   UNIFORM   W, min y, max y             PARETO      W, W log y, min y
 * where W = sum_t gamma_t(j) (x) and x the named function of y_t; the
 * uniform / Pareto min and max run over the rows of the model's sequences
 * that lie in the state's current support (b_j(y_t) > 0). */
int64_t hmm_stats_size(hmm_stats stats);
hmm_status hmm_stats_get(hmm_stats stats, double* h_out, int64_t n_values);

/* Device view of the raw float64 statistic record behind `stats`
 * (*d_values, *n_values).  Its layout is internal, but every entry is a sum
 * over sequences, so records of the same model made on different GPUs from
 * different sequences can be added element-wise (e.g. an all-reduce of
 * data-parallel E-steps) before hmm_mstep.  The memory stays owned by the
 * library and lives as long as `stats`. */
hmm_status hmm_stats_device_buffer(hmm_stats stats, double** d_values, int64_t* n_values);

/* ---------------------------------------------- data-parallel exchange
 * Sequences are independent in the E-step (Sec. 3), and every statistic the
 * M-step of Sec. 4 reads is a sum over sequences (Eq. 5 and the family sums
 * above), a minimum or maximum over rows (the uniform / Pareto supports),
 * or, for the Newton steps that re-read the data (Weibull shape, Eq. 11;
 * negative-binomial r), a sum over rows per Newton pass.  A data-parallel
 * fit therefore gives each process a shard of the sequences and combines
 * these records across processes before the M-step reads them; every
 * process then runs the same M-step and keeps the same model.
 *
 * The library does not talk to other processes itself: the caller installs
 * an all-reduce callback on the stats object, and the library calls it on
 * its device records at the points where the M-step needs the combined
 * values.  d_values: device memory of n elements, reduced in place; op:
 * hmm_reduce_op (float64 sum, or int32 minimum); the reduction must be
 * ordered on `stream` (work enqueued on it before the call is complete
 * before the reduction reads the data, and work enqueued after the call
 * sees the result).  Every process calls it the same number of times with
 * the same sizes and ops.  A nonzero return makes the library call fail with
 * HMM_E_CUDA. */
typedef enum {
  HMM_REDUCE_SUM_F64 = 0,  /* element-wise sum of float64 values            */
  HMM_REDUCE_MIN_I32 = 1   /* element-wise minimum of int32 values          */
} hmm_reduce_op;
typedef int32_t (*hmm_allreduce_fn)(void* d_values, int64_t n, int32_t op, void* stream, void* user);

/* Installs (fn != NULL) or removes (fn == NULL) the exchange of `stats`.
 * With it, hmm_estep_stats ends by reducing each record of
 * hmm_stats_record (index order 0, 1, 2; records of size 0 are skipped) and
 * hmm_mstep reduces the sums of each Newton data pass before the update
 * that reads them (float64 sums, n = n_models x padded states x 3; a fixed
 * number of passes, the same on every process).  An empty shard (n_seq = 0)
 * is allowed and contributes zeros / the identity of the minimum. */
hmm_status hmm_stats_set_allreduce(hmm_stats stats, hmm_allreduce_fn fn, void* user);

/* Device view of record `index` of `stats` after an E-step, and the
 * reduction that combines it across processes:
 *   0  the statistic record (the layout behind hmm_stats_get: counts,
 *      log-likelihood sums, gamma_1, xi and the family sums of the first
 *      eight families), HMM_REDUCE_SUM_F64;
 *   1  the feature / moment sums of the table families (multivariate,
 *      discrete, log-normal .. Pareto), HMM_REDUCE_SUM_F64; n = 0 when the
 *      model has none;
 *   2  the support extremes of the uniform and Pareto states, int32 keys
 *      whose order is the order of the float32 values (the maximum stored
 *      complemented, so that both combine with a minimum),
 *      HMM_REDUCE_MIN_I32; n = 0 when the model has none.
 * The memory stays owned by the library.  HMM_E_ARG for another index. */
hmm_status hmm_stats_record(hmm_stats stats, int32_t index, void** d_values, int64_t* n_values, int32_t* op);

/* E-step over a batch (Sec. 3.2 + Sec. 4, Eq. 5): fills `stats` with the
 * weighted sufficient statistics of every model and writes per-sequence
 * log-likelihoods to d_loglik [n_seq] (may be NULL).  The reductions are in
 * a fixed order (bitwise reproducible). */
hmm_status hmm_estep_stats(hmm_ctx ctx, hmm_model model, const hmm_batch* batch,
                           hmm_stats stats, double* d_loglik, void* stream);

/* Viterbi-training E-step (the Viterbi trainer the paper names, Sec. 5.6;
 * reading: hard EM / segmental k-means).  Decodes every sequence's Viterbi
 * path q* (Eq. 3-4, as hmm_viterbi) and fills `stats` with the statistics of
 * the paths: occupancies gamma_t(j) = 1[q*_t = j], transition counts
 * n_ij = #{t : q*_t = i, q*_{t+1} = j} (in place of the expected ones) and
 * first states, so that hmm_mstep then runs the Baum-Welch M-step on these
 * hard weights.  The statistic record's log-likelihood entry holds the sum
 * of the paths' log-probabilities max_q log P(q, y), the objective that
 * Viterbi training does not decrease, and hmm_stats_get reports the
 * transition counts in place of the expected transitions.  d_score [n_seq] (may be NULL)
 * receives them per sequence.  The installed all-reduce (if any) runs as
 * after hmm_estep_stats. */
hmm_status hmm_estep_viterbi(hmm_ctx ctx, hmm_model model, const hmm_batch* batch, hmm_stats stats,
                             double* d_score, void* stream);

/* M-step (Sec. 4, Eq. 6 with the closed forms, Newton-Raphson and ECM
 * steps of Sec. 4.1-4.5, the Sec. 4.4 collapse guard, and the transition /
 * initial-distribution update) from `stats`, in place on `model`.
 * `batch` is needed only by families whose Newton step re-reads the data
 * (Weibull shape, negative-binomial r); it may be NULL otherwise.  opts may
 * be NULL for the defaults. */
hmm_status hmm_mstep(hmm_ctx ctx, hmm_model model, hmm_stats stats,
                     const hmm_batch* batch, const hmm_mstep_opts* opts, void* stream);

/* max_iter Baum-Welch iterations (the EM of Sec. 3-4: the E-step of Sec. 3.2
 * and Eq. 5, then the M-step of Sec. 4, Eq. 6; the paper's Baum-Welch, MAP
 * Baum-Welch and Viterbi trainers, Sec. 5.6, select with opts) on the batch,
 * in place on `model`.  h_loglik_trace (host, may be NULL) receives, for every
 * iteration k, the sum of log-likelihoods of each model under the parameters
 * entering iteration k: [max_iter][n_models].  *iters_done (may be NULL) gets
 * the number of iterations run.  The iterations run as one captured CUDA
 * graph replay per iteration when tol == 0. */
hmm_status hmm_fit(hmm_ctx ctx, hmm_model model, const hmm_batch* batch,
                   const hmm_fit_opts* opts, double* h_loglik_trace,
                   int32_t* iters_done, void* stream);

/* ------------------------------------------------------------ serving
 * A request server on one GPU: decode (Viterbi), posterior (forward-backward)
 * and fit (Baum-Welch) requests, each carrying its own model and one
 * observation sequence, are queued by hmm_serve_submit and run by a
 * dispatcher with continuous batching: whenever a slot is free and the
 * device-memory budget allows, the oldest pending request and the pending
 * requests of the same kind, family, N, dim (and iteration count) are packed
 * into one multi-model batch (one model per request) and launched on that
 * slot's stream, while earlier batches still run on the other slots.  Models,
 * EM state and scratch stay on the device for the whole request; only the
 * inputs go up and the results come down.  The paper describes no serving
 * system: the batching follows from its problem statement (independent
 * sequences and models, Sec. 3), the entry points from the request kinds of
 * Sec. 3.3-3.4 and Sec. 4. */
typedef struct hmm_server_s* hmm_server;

typedef enum {
  HMM_REQ_DECODE = 0,      /* Viterbi path and score                         */
  HMM_REQ_POSTERIOR = 1,   /* gamma rows and log-likelihood                  */
  HMM_REQ_FIT = 2          /* n_iter Baum-Welch iterations from `params`     */
} hmm_request_kind;

typedef struct {
  int32_t n_slots;         /* concurrent batches (streams), 0: 4               */
  int32_t max_batch;       /* requests per batch, 0: 16                       */
  int32_t max_queue;       /* pending requests before HMM_E_BUSY, 0: 4096      */
  size_t mem_budget;       /* admission budget in bytes, 0: half of free memory */
} hmm_serve_opts;

typedef struct {
  int32_t kind;            /* hmm_request_kind                                */
  int32_t family;          /* hmm_family of the request's model              */
  int32_t n_states;
  int32_t dim;
  const double* params;    /* host blob of one model (hmm_param_blob_size)    */
  int64_t n_params;
  const float* values;     /* host observations [T][dim]                      */
  int64_t T;
  int32_t n_iter;          /* HMM_REQ_FIT: iterations                         */
} hmm_request;

typedef struct {
  int32_t status;          /* hmm_status of the request                       */
  int32_t kind;
  int64_t T;
  double loglik;           /* POSTERIOR: log-likelihood; FIT: under the final
                              parameters' predecessor (last trace entry)     */
  double score;            /* DECODE: log probability of the best path        */
  const int32_t* path;     /* DECODE: [T]                                     */
  const float* gamma;      /* POSTERIOR: [T][n_states]                        */
  const double* params;    /* FIT: fitted blob                                 */
  const double* trace;     /* FIT: [n_iter] log-likelihood entering each iteration */
  int32_t n_iter;
  double latency_ms;       /* submit to completion                           */
  const char* error;       /* message of a failed request, else ""            */
} hmm_result;

/* Starts the server's dispatcher and slot threads on ctx's device (each slot
 * owns a context, a stream and cached device buffers; ctx must outlive the
 * server).  opts may be NULL. */
hmm_status hmm_serve_create(hmm_ctx ctx, const hmm_serve_opts* opts, hmm_server* out);
/* Copies the request's host inputs and queues it; *ticket identifies it.
 * HMM_E_BUSY when max_queue requests are pending, HMM_E_ARG for an invalid
 * request, HMM_E_NOMEM when its footprint exceeds the whole budget. */
hmm_status hmm_serve_submit(hmm_server server, const hmm_request* req, uint64_t* ticket);
/* HMM_E_NOTREADY while the request is pending or running; then fills *out
 * (pointers owned by the server, valid until hmm_serve_release) and returns
 * HMM_OK (out->status carries the request's own status). */
hmm_status hmm_serve_poll(hmm_server server, uint64_t ticket, hmm_result* out);
/* Blocks until the request completes (or timeout_ms passes: HMM_E_TIMEOUT). */
hmm_status hmm_serve_wait(hmm_server server, uint64_t ticket, double timeout_ms, hmm_result* out);
/* Frees a completed request's results. */
hmm_status hmm_serve_release(hmm_server server, uint64_t ticket);
/* h_out[10]: submitted, completed, p50 ms, p99 ms, mean ms, completed per
 * second since the first submission, pending, running, batches run, mean
 * slot occupancy (time the slots spent running batches / (slots x span)). */
hmm_status hmm_serve_stats(hmm_server server, double* h_out);
/* Finishes the running batches, drops pending requests, frees everything. */
hmm_status hmm_serve_destroy(hmm_server server);

#ifdef __cplusplus
}
#endif
#endif /* HMMGPU_H */
