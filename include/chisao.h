/*
 * chisao.h -- C ABI of the GB300 (sm_103a) ChiSao population step.
 *
 * ChiSao ("Convergence-Halt-Invert-Stick-And-Oscillate") looks for every
 * significant mode of f on a box Theta (Section 3.1, Eq. 1) by running a
 * population of N samples through oscillation cycles of six phases
 * (Algorithm 1): batched L-BFGS ascent (Phase 1, Eq. 2), stick detection
 * (Phase 2, Eq. 3), L-infinity deduplication (Phase 3, Eq. 4), Repulse Monkey /
 * Golden Rooster reseeding (Phase 4, Sec. 3.2.4), Hands Like Clouds smoothed
 * ascent (Phase 5, Eq. 5) and momentum anti-convergence (Phase 6, Eq. 6).
 * The last cycle runs Phases 1-3 only.
 *
 * One context owns the device state of one or more independent problems.
 * Every phase runs in hand-written CUDA kernels on the context's stream;
 * nothing here falls back to the CPU.
 *
 * Conventions
 *   - Every call returns a chisao_status; none aborts.  On failure the
 *     context (when there is one) keeps a message for chisao_last_error().
 *   - "host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the context's device.  The library never keeps a
 *     caller pointer past the call that received it.
 *   - Populations are row-major float32 [n][d].
 *   - Calls on one context are not thread-safe; distinct contexts are
 *     independent.
 */
#ifndef CHISAO_H
#define CHISAO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CHISAO_MAX_DIM 64        /* largest supported dimension d            */
#define CHISAO_MAX_MEMORY 10     /* largest L-BFGS memory m                  */

typedef enum {
  CHISAO_OK = 0,
  CHISAO_ERR_ARG = 1,        /* invalid argument (sizes, pointers, ranges)   */
  CHISAO_ERR_CUDA = 2,       /* a CUDA runtime call failed                    */
  CHISAO_ERR_OOM = 3,        /* device allocation or arena too small         */
  CHISAO_ERR_CAPACITY = 4,   /* output buffer smaller than the result        */
  CHISAO_ERR_STATE = 5,      /* call not valid in the context's state         */
  CHISAO_ERR_TIMEOUT = 6     /* a device-side wait ran out of its time budget
                                (reported once by chisao_get_counters, which
                                clears the flag; the context stays usable)     */
} chisao_status;

/* Objective families (built-in device objectives). */
typedef enum {
  /* log sum_k w_k N(x; mu_k, diag(sigma_k^2))   (Appendix D mixture)       */
  CHISAO_OBJ_MIXTURE_DIAG = 1,
  /* log sum_k w_k N(x; mu_k, L_k L_k^T), L_k lower-triangular Cholesky     */
  CHISAO_OBJ_MIXTURE_FULL = 2,
  /* -(x - c)^T Q^T diag(lam) Q (x - c), a log-concave target (Prop. 1)     */
  CHISAO_OBJ_QUADRATIC = 3,
  /* Appendix D benchmark functions, negated for maximisation; no parameter
   * arrays.  Coordinates i = 1..d.  Where a function is not differentiable
   * the adjoint gradient takes the zero subgradient of the offending term.  */
  /* -sum_i (x_i^2 - 10 cos(2 pi x_i) + 10), App. D domain [-5.12, 5.12]^d   */
  CHISAO_OBJ_RASTRIGIN = 10,
  /* 20 exp(-0.2 sqrt(sum x_i^2 / d)) + exp(sum cos(2 pi x_i) / d) - 20 - e,
   * domain [-32.768, 32.768]^d                                              */
  CHISAO_OBJ_ACKLEY = 11,
  /* sum_i x_i sin(sqrt|x_i|) - 418.9829 d, domain [-500, 500]^d              */
  CHISAO_OBJ_SCHWEFEL = 12,
  /* -(1/2) sum_i (x_i^4 - 16 x_i^2 + 5 x_i), domain [-5, 5]^d                */
  CHISAO_OBJ_STYBLINSKI_TANG = 13,
  /* sum_i sin(x_i) sin(i x_i^2 / pi)^20, domain [0, pi]^d                    */
  CHISAO_OBJ_MICHALEWICZ = 14,
  /* -sum_i (x_i - 1)^2 + sum_{i>=2} x_i x_{i-1}, domain [-d^2, d^2]^d        */
  CHISAO_OBJ_TRID = 15,
  /* -100 sqrt|x_2 - x_1^2 / 100| - |x_1 + 10| / 100, d = 2,
   * domain [-15, -5] x [-3, 3]                                              */
  CHISAO_OBJ_BUKIN6 = 16,
  /* A caller-supplied batched evaluator (chisao_objective.eval below): the
   * cycle runs Phases 1, 5 and 6 as per-sample kernels around batched calls
   * to it, as in the tensor-core mode.  Needs grad_mode CHISAO_GRAD_ADJOINT
   * (the evaluator returns exact gradients), noise_sigma 0, hlc_value_only 0. */
  CHISAO_OBJ_EXTERNAL = 20
} chisao_objective_kind;

/* Batched evaluator of a CHISAO_OBJ_EXTERNAL objective (Sec. 3.1: f is a
 * black box and its gradient is supplied).  Every pointer is device memory.
 * The points are rows of x (row r starts at x + r * ldx, its first d floats
 * are the coordinates).  The rows to evaluate are 0 .. rows-1 when idx is NULL,
 * else idx[k] for k < *count (idx and count on the device, *count <= rows,
 * every idx[k] < rows).  For each such row write f[r] (when f is not NULL) and
 * the exact gradient of f, g[r * ldg + j] for j < d (when g is not NULL);
 * writing other rows is allowed and ignored.  All work must go onto `stream`
 * (a cudaStream_t) and may finish after the call returns.  With use_graph = 1
 * the call happens while the stream is being captured into a CUDA graph, so
 * it must be capture-safe (no synchronization, no reading *count on the
 * host); the graph then replays the captured work every cycle.  Return 0 on
 * success; any other value aborts the step with CHISAO_ERR_CUDA and a message
 * naming that value. */
typedef int32_t (*chisao_batch_eval_fn)(void *user, const float *x, int32_t ldx, int64_t rows,
                                        const int32_t *idx, const int32_t *count, float *f,
                                        float *g, int32_t ldg, void *stream);

/* How gradients are obtained (Section 3.1: central differences of the values,
 * or an exact gradient where one is available). */
typedef enum {
  /* central differences at absolute step h; stencil coordinates and every
   * stencil evaluation in FP64, quotient in FP64, result stored FP32       */
  CHISAO_GRAD_FD64 = 0,
  /* central differences at h_j = h_rel * max(1, |x_j|), evaluations FP32   */
  CHISAO_GRAD_FD32 = 1,
  /* exact gradient from the objective's hand-written adjoint, FP32         */
  CHISAO_GRAD_ADJOINT = 2,
  /* full-covariance mixtures: value and exact gradient of the mixture whose
   * precision factors are L_k^-1 rounded to BF16, on the tcgen05 tensor
   * cores (BF16 operands, FP32 accumulation and log-sum-exp; the input split
   * into two BF16 terms; component centres kept exact).  chisao_eval only. */
  CHISAO_GRAD_ADJOINT_TC = 3
} chisao_grad_mode;

/* Objective description.  All arrays are host FP64, row-major, read during
 * chisao_create only.  Unused fields may be NULL.
 *   MIXTURE_DIAG: weights[K], means[K][d], sigmas[K][d]  (sigma > 0)
 *   MIXTURE_FULL: weights[K], means[K][d], chol[K][d][d] (lower, diag > 0)
 *   QUADRATIC:    center[d], Q[d][d], lam[d]             (K ignored)
 *   RASTRIGIN .. BUKIN6: no arrays (K ignored; BUKIN6 requires d = 2)      */
typedef struct {
  int32_t kind;            /* chisao_objective_kind                          */
  int32_t n_comp;          /* K for mixtures                                 */
  const double *weights;
  const double *means;     /* mixtures: means; quadratic: unused             */
  const double *sigmas;
  const double *chol;
  const double *center;
  const double *Q;
  const double *lam;
  /* Additive evaluation noise f~ = f + eps, eps ~ N(0, noise_sigma^2)
   * (Sec. 5.6); 0 for none.  Each evaluation point gets its own draw, keyed
   * by the point's binary32 coordinates and the Philox seed.  Exact (adjoint)
   * gradients are those of the noise-free f. */
  double noise_sigma;
  /* CHISAO_OBJ_EXTERNAL: the evaluator and its opaque argument (the caller
   * keeps both valid until chisao_destroy). */
  chisao_batch_eval_fn eval;
  void *user;
} chisao_objective;

/* One problem: dimension, population size, the box Theta and the initial
 * population (host, float32 [n][d], copied at create). */
typedef struct {
  int32_t d;               /* 1 .. CHISAO_MAX_DIM                           */
  int64_t n;               /* population size, >= 1                          */
  const double *lo;        /* host [d] lower corner of Theta                 */
  const double *hi;        /* host [d] upper corner, hi > lo                 */
  const float *x0;         /* host [n][d] initial population                 */
  chisao_objective objective;
} chisao_problem;

/* Hyperparameters: Table 1 of the paper plus the values that fix details
 * the paper leaves open (line search, FD step, step-size rule). */
typedef struct {
  int32_t n_osc;           /* oscillation cycles (Table 1: 3)                */
  int32_t n_conv;          /* L-BFGS steps per Phase 1; 0: max(10, ceil(3 log2 d)) */
  int32_t n_anti;          /* anti-convergence steps (5)                      */
  int32_t n_cloud;         /* Hands Like Clouds steps (3)                     */
  int32_t M;               /* perturbations per smoothed gradient (Eq. 5)    */
  int32_t m;               /* L-BFGS memory, 1 .. CHISAO_MAX_MEMORY (10)     */
  int32_t T_ls;            /* backtracking trials per line search (20)       */
  int32_t grad_mode;       /* chisao_grad_mode                                */
  double eps_grad;         /* stick threshold on |grad f|_inf (Eq. 3)        */
  double eps_dup;          /* dedup L-inf radius (Eq. 4)                      */
  double delta;            /* quality threshold, stuck iff f >= f_max + log delta */
  double mu;               /* momentum (Eq. 6)                                */
  double alpha;            /* anti/HLC step; <= 0: alpha_scale * s / g_rms    */
  double sigma;            /* HLC smoothing scale; <= 0: c_sigma * s          */
  double c_sigma;          /* 0.1                                             */
  double alpha_scale;      /* 0.1                                             */
  double h;                /* FD64 absolute step (1e-5)                       */
  double h_rel;            /* FD32 relative step (2^(-23/3))                  */
  double c1;               /* Armijo constant (1e-4)                          */
  double curv_eps;         /* keep (s, y) iff s^T y > curv_eps |s| |y|        */
  uint64_t seed;           /* Philox key                                      */
  int32_t rm_min_unfrozen; /* Repulse Monkey iff >= this many unfrozen (5)    */
  int32_t gr_patience;     /* Golden Rooster off after this many idle generations (2) */
  int32_t use_graph;       /* 1: capture each cycle in a CUDA graph           */
  int32_t n_refine;        /* CHISAO_GRAD_ADJOINT_TC: FP32 L-BFGS steps on the
                              survivors after the last cycle (exact objective) */
  int32_t hlc_value_only;  /* 0: Phase 5 averages gradients at x + sigma z_k (Eq. 5);
                              1: the value-only estimator (1/M) sum_k
                              (f(x + sigma z_k) - f(x)) z_k / sigma (the Gaussian-
                              smoothing estimator Sec. 3.2.5 cites; a variant, not
                              Eq. 5), M + 1 evaluations per step in every grad_mode */
} chisao_params;

/* Per-problem counters accumulated on the device since create. */
typedef struct {
  uint64_t evals;          /* objective evaluations (value computations)      */
  uint64_t grads;          /* gradient computations (FD or adjoint)           */
  uint64_t ls_trials;      /* line-search trial points                         */
  uint64_t ls_fail;        /* line searches with no acceptable step            */
  int64_t cycles;          /* completed cycles                                  */
  int64_t n_stuck;         /* stuck samples after the last deduplication        */
  int64_t k_lost;          /* samples removed by the last deduplication         */
  int64_t n_unfrozen;      /* unfrozen samples counted for the last reseeding   */
  int32_t last_reseed;     /* 0 none, 1 Repulse Monkey, 2 Golden Rooster, 3 uniform */
  int32_t gr_enabled;      /* Golden Rooster still enabled                      */
  float f_max;             /* max_i f(x_i) of the last Phase 2                   */
  float sigma;             /* last HLC smoothing scale                           */
  float alpha_hlc;         /* last HLC step                                      */
  float alpha_anti;        /* last anti-convergence step                         */
  int32_t device_error;    /* device error flag: 0 none, 2 a bounded wait timed out */
} chisao_counters;

typedef struct chisao_ctx chisao_ctx;

/* Fill *p with the defaults of Table 1 (n_osc 3, n_anti 5, n_cloud 3,
 * eps_grad 1e-6, eps_dup 1e-3, delta 0.1, mu 0.9, sigma/alpha auto) and the
 * stated readings (M 8, m 10, T_ls 20, h 1e-5, c1 1e-4). */
void chisao_default_params(chisao_params *p);

/* Bytes of device memory a context for these problems needs.  Returns
 * CHISAO_ERR_ARG for invalid problems or parameters. */
chisao_status chisao_arena_bytes(const chisao_problem *probs, int32_t n_probs,
                                 const chisao_params *params, size_t *bytes);

/* Create a context.  Its inputs are those of Algorithm 1: the objective f
 * over the bounded domain Theta (Sec. 3.1, the problem statement), an initial
 * population that the caller provides (Sec. 3.1: arbitrary), and the
 * hyperparameters of Table 1 (chisao_params); several independent problems may
 * share one context.  Validates everything (CHISAO_ERR_ARG, with a message),
 * carves the device state out of `arena` (device, >= chisao_arena_bytes,
 * 256-byte aligned; it stays owned by the caller and must outlive the
 * context) or, when arena is NULL, allocates it with cudaMalloc
 * (CHISAO_ERR_OOM on failure); copies objectives and initial populations;
 * binds `cuda_stream` (a cudaStream_t, NULL for the legacy default stream).
 * *out receives the context (NULL on failure).  Synchronous. */
chisao_status chisao_create(const chisao_problem *probs, int32_t n_probs,
                            const chisao_params *params, void *arena,
                            size_t arena_bytes, void *cuda_stream,
                            chisao_ctx **out);

/* chisao_create with the library allocating its own device memory: the
 * initialisation of Algorithm 1 (the problems of Sec. 3.1, the population
 * given by the caller, the Table 1 parameters) under its short name.  Same
 * arguments, errors and ownership as chisao_create with arena = NULL. */
chisao_status chisao_init(const chisao_problem *probs, int32_t n_probs,
                          const chisao_params *params, void *cuda_stream,
                          chisao_ctx **out);

/* One oscillation cycle (Algorithm 1, one iteration of its outer loop) for
 * every problem: asynchronous on the context's stream.  The n_osc-th call runs
 * the last cycle (Phases 1-3 only); calls after it return CHISAO_ERR_STATE. */
chisao_status chisao_step(chisao_ctx *c);

/* Replace problem `prob`'s population by host x[n][d] (float32) and reset its
 * per-sample state (history, stuck flags, counters) and the context's cycle
 * count.  The copy is ordered on the context's stream: x_host must stay
 * unchanged until the stream has passed it (any later synchronizing call
 * such as chisao_modes, or a stream synchronize). */
chisao_status chisao_load_population(chisao_ctx *c, int32_t prob, const float *x_host);

/* Initial population generated on the device.  method 0: uniform in the box Theta
 * (counter-based Philox, keyed by the context seed, the problem and the sample);
 * method 1: Carry Tiger (Sec. 5.1 describes it only as rays toward the box's corners,
 * edges and faces, so this is a reading) - sample i lies on the ray from the box
 * centre to a face centre, an edge midpoint or a vertex (the class cycles with i,
 * face centres round-robin, edge free axis round-robin, signs random), at a
 * uniform position along it.  Resets the per-sample state and the cycle count as
 * chisao_load_population does.  Asynchronous on the context's stream. */
typedef enum { CHISAO_SEED_UNIFORM = 0, CHISAO_SEED_CARRY_TIGER = 1 } chisao_seed_method;
chisao_status chisao_seed(chisao_ctx *c, int32_t prob, int32_t method);

/* The estimated mode set {x_i : stuck_i} of problem `prob` after the last
 * deduplication (Algorithm 1's return value), in sample-index order:
 * x_out host [cap][d], f_out host [cap] (may be NULL).  *count receives the
 * number of modes; CHISAO_ERR_CAPACITY (nothing written) when cap < count.
 * Synchronizes the stream. */
chisao_status chisao_modes(chisao_ctx *c, int32_t prob, float *x_out,
                           float *f_out, int64_t cap, int64_t *count);

/* Measured FMA throughput of this GPU, the denominator of the ALU rooflines the
 * benchmark reports: *flops receives FLOP/s (two per FMA) of independent FMA chains
 * filling every SM, binary32 (precision 0; packed two-lane FMAs, as the objective
 * kernels issue them) or binary64 (precision 1).  Runs on the given stream (NULL:
 * the default stream) and synchronizes it; a few milliseconds. */
chisao_status chisao_measure_fma_peak(int32_t precision, void *cuda_stream, double *flops);

/* Measured instruction rate of the tensor core for the small MMAs the full-covariance
 * objective issues (tcgen05.mma kind::f16, M = 128, K = 16, width n a multiple of 16 up
 * to 256 with one issuer, 128 with two, 64 with three or four): `threads` issuing
 * threads (1 .. 4, in different warps) each run 2048 MMAs into their own accumulator,
 * the last tmem_a (0 .. threads) of them reading A from tensor memory;
 * *clk_per_mma receives SM clocks per MMA with all of them together.  One CTA, zero
 * operands; runs on the given stream (NULL: the default stream) and synchronizes it.
 * CHISAO_ERR_ARG for other arguments; CHISAO_ERR_CUDA if the kernel fails or its
 * bounded completion wait runs out. */
chisao_status chisao_measure_mma_rate(int32_t n, int32_t threads, int32_t tmem_a, void *cuda_stream,
                                      double *clk_per_mma);

/* Result of chisao_autotune. */
typedef struct {
  int32_t n_branch;        /* branch streams chosen (contexts of several problems)  */
  int32_t grouped;         /* 1: Phases 1, 5, 6 and the scale passes run as grouped
                              launches per (objective kind, padded dimension)        */
  int32_t trials;          /* configurations timed                                    */
  float ms_per_cycle;      /* the chosen configuration's time per non-final cycle     */
  float ms_default;        /* the configuration the context had before              */
  int32_t ck[5];           /* grouped diagonal mixtures of padded dimension 4 << k: the
                              components taken per step by their kernels (a compile-time
                              tile shape: 2, 4 or 8); 0 where the context has no such group */
} chisao_tuning;

/* Launch-shape autotuner for contexts of several problems: for each candidate (8, 16,
 * 32 or 64 branch streams, times grouped launches over all problems or per-problem
 * launches) it captures a non-final cycle of the context itself in a CUDA graph, runs
 * it once untimed and then cycles_per_trial (1 .. 100) times under CUDA events, and
 * keeps the fastest; with grouped launches it then tries, group by group, the
 * compiled tile shapes of the diagonal mixture's kernels (2, 4 or 8 components per
 * step) the same way.  Every candidate computes the same
 * results bit for bit, and the context's state is saved before and restored after
 * each trial (one device copy of the arena, needing arena-sized free memory), so the
 * tuning changes no result and no trajectory.  A context of one problem, or one with
 * an external objective (whose evaluator need not be capture-safe), is left as it is
 * (trials = 0).  Synchronous. */
chisao_status chisao_autotune(chisao_ctx *c, int32_t cycles_per_trial, chisao_tuning *out);

/* Laplace widths of the modes chisao_modes returns (same order).  Phase 3
 * (Sec. 3.2.3) keeps each surviving sample's inverse-Hessian estimate for width
 * estimation; the paper gives no formula, and the reading here is the Laplace
 * approximation at the mode: the covariance is H, the L-BFGS inverse-Hessian
 * estimate of F = -f that the two-loop recursion applies (H_0 = gamma I, gamma =
 * s^T y / y^T y of the newest pair; H = I with no stored pairs), computed column
 * by column as H e_j in binary32.
 *   w_out    [cap][d]: w[r][j] = sqrt(max(H_jj, 0)) of mode r;
 *   cov_out  [cap][d][d] or NULL: row j of mode r holds H e_j.
 * Outputs may be host or device memory (copied with cudaMemcpyDefault); cov_out
 * needs a temporary device buffer of count*d*d floats (CHISAO_ERR_OOM without
 * it).  *count receives the number of modes; CHISAO_ERR_CAPACITY (nothing
 * written) when cap < count.  Synchronizes the stream. */
chisao_status chisao_widths(chisao_ctx *c, int32_t prob, float *w_out, float *cov_out,
                            int64_t cap, int64_t *count);

/* Counters of problem `prob` (synchronizes the stream).  When a kernel of the
 * problem gave up a bounded wait (the tensor-core objective's barrier waits have a
 * budget of about a second; kernels never trap), the counters are filled, the
 * device flag is cleared and CHISAO_ERR_TIMEOUT is returned. */
chisao_status chisao_get_counters(chisao_ctx *c, int32_t prob, chisao_counters *out);

/* The same counters under their short name (identical behaviour and errors):
 * evaluations, line-search trials, the stuck count and K_lost of Algorithm 1's
 * Phases 2-3, the reseeding strategy of Phase 4 (Sec. 3.2.4) and the step
 * sizes of Phases 5-6. */
chisao_status chisao_stats(chisao_ctx *c, int32_t prob, chisao_counters *out);

/* Test hook for that failure path: one kernel waits, with the library's bounded
 * wait, on a shared-memory barrier nothing arrives on; after budget_ns (1 .. 10^10)
 * it raises problem `prob`'s device error flag and returns.  Asynchronous. */
chisao_status chisao_selftest_wait(chisao_ctx *c, int32_t prob, int64_t budget_ns);

/* Evaluate problem `prob`'s objective at n device points x_dev[n][d]:
 * f_dev[n] (may be NULL) and, when g_dev[n][d] is not NULL, the gradient by
 * `grad_mode`.  This is the device objective the step uses, exposed for
 * autograd wrappers and tests.  Asynchronous on the context's stream. */
chisao_status chisao_eval(chisao_ctx *c, int32_t prob, const float *x_dev, int64_t n,
                          float *f_dev, float *g_dev, int32_t grad_mode);

/* Message of the last failed call on this context ("" if none). */
const char *chisao_last_error(const chisao_ctx *c);

/* Free the context and everything it allocated (not a caller arena). */
void chisao_destroy(chisao_ctx *c);

/* ---------------------------------------------------------------------------
 * Test hooks: per-phase entry points and raw state access, used by the parity
 * tests to run one phase from a state both sides share.  They act on one
 * problem, asynchronously on the context's stream unless stated.
 * ------------------------------------------------------------------------- */

typedef enum {
  CHISAO_FIELD_X = 0,        /* float [n][dp]   positions (dp = padded d)     */
  CHISAO_FIELD_G = 1,        /* float [n][dp]   gradient of f                  */
  CHISAO_FIELD_F = 2,        /* float [n]       f                              */
  CHISAO_FIELD_HS = 3,       /* float [n][m_max][dp]  s pairs, slot 0 newest    */
  CHISAO_FIELD_HY = 4,       /* float [n][m_max][dp]  y pairs of F = -f          */
  CHISAO_FIELD_HRHO = 5,     /* float [n][m_max]      1 / s^T y                  */
  CHISAO_FIELD_HLEN = 6,     /* int32 [n]       stored pairs                    */
  CHISAO_FIELD_STUCK = 7,    /* uint32 [ceil(n/32)] stuck bit mask               */
  CHISAO_FIELD_REMOVED = 8   /* uint32 [ceil(n/32)] removed-by-dedup bit mask     */
} chisao_field;

typedef enum {
  CHISAO_PHASE_LBFGS = 1,     /* arg iterations of Phase 1 (arg<0: -arg, no fresh gradient) */
  CHISAO_PHASE_FREEZE = 2,    /* Phase 2 on the current f, g                 */
  CHISAO_PHASE_DEDUP = 3,     /* Phase 3 on the stuck mask (compacts it first) */
  CHISAO_PHASE_RESEED = 4,    /* Phase 4 for cycle number arg                 */
  CHISAO_PHASE_HLC = 5,       /* Phase 5 for cycle number arg                 */
  CHISAO_PHASE_ANTI = 6,      /* Phase 6                                       */
  CHISAO_PHASE_DIRECTION = 7, /* write the L-BFGS direction p into G         */
  CHISAO_PHASE_LISTS = 8,     /* stuck &= ~removed, then the free / unfrozen /
                                 survivor lists from the two masks            */
  CHISAO_PHASE_REFINE = 9     /* arg FP32 L-BFGS steps (exact objective) on the
                                 survivor list                                */
} chisao_phase;

/* Padded row length dp and m_max used by the raw fields of problem prob. */
chisao_status chisao_layout(chisao_ctx *c, int32_t prob, int32_t *dp, int32_t *m_max);
/* Copy a raw field to / from host memory (synchronous; bytes must match). */
chisao_status chisao_state_get(chisao_ctx *c, int32_t prob, int32_t field, void *host, size_t bytes);
chisao_status chisao_state_set(chisao_ctx *c, int32_t prob, int32_t field, const void *host, size_t bytes);
/* Run one phase of problem prob (see chisao_phase); asynchronous on the
 * context's stream (state_get synchronizes). */
chisao_status chisao_run_phase(chisao_ctx *c, int32_t prob, int32_t phase, int32_t arg);
/* Set the Golden Rooster bookkeeping (enabled, idle generations, survivor
 * count at the previous generation, -1 for none). */
chisao_status chisao_set_gr_state(chisao_ctx *c, int32_t prob, int32_t enabled,
                                  int32_t noprog, int32_t prev_surv);
/* Set the tile shape chisao_autotune chooses for the grouped diagonal-mixture kernels
 * of padded dimension dp: ck = 2, 4 or 8 components per step (the results do not
 * depend on it).  CHISAO_ERR_ARG when ck is another value or the context has no such
 * group.  Synchronizes the stream; the next step recaptures its graph. */
chisao_status chisao_set_tile(chisao_ctx *c, int32_t dp, int32_t ck);

/* ---------------------------------------------------------------------------
 * Allocation-free deduplication.
 *
 * The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory and so cannot create a context: a host
 * application whose own memory pool has reserved the whole device and forbids
 * side allocations, a plug-in that is handed only its input and output
 * buffers, or a latency-critical loop in which a cudaMalloc/cudaFree pair
 * would synchronize the device.  It runs the Phase 3 decision (a stuck x_j is
 * removed when another stuck x_i ranks above it, f descending then index
 * ascending, and every |x_ik - x_jk| < eps_dup, compared in binary32) on
 * caller buffers only, and calls no cudaMalloc, cudaFree or other allocating
 * routine.
 *
 *   x_dev       device float [n][d], row-major, d in 1..CHISAO_MAX_DIM
 *   f_dev       device float [n]
 *   stuck_dev   device uint32 [ceil(n/32)] bit mask (bit i%32 of word i/32)
 *   removed_dev device uint32 [ceil(n/32)] output mask (cleared by the call)
 *   k_lost_dev  device int32 [1] output count, or NULL
 *   cuda_stream the cudaStream_t the kernels are queued on (NULL: default)
 *
 * Its scratch (the stuck list, CHISAO_DEDUP_NOALLOC_MAX_N ints plus 64
 * counters, about 1 MiB) is one file-scope device array per GPU, held by every
 * GPU that loads the library until the process exits.  n above
 * CHISAO_DEDUP_NOALLOC_MAX_N returns CHISAO_ERR_CAPACITY without launching
 * anything; bad pointers or sizes return CHISAO_ERR_ARG.
 *
 * Cost: unlike the context's spatial-hash dedup, each of the S stuck samples
 * scans the whole stuck list (S warps x S candidates, O(S^2 d)): about 1e10
 * candidate tests at S = 10^5 and 7e10 at the limit, seconds of GPU time.
 * Use it for stuck sets of a few ten thousand at most; larger sets belong to
 * the context path.
 *
 * Set-up: the first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the life
 * of the process; make that first call before any stream capture.  A device
 * reset (cudaDeviceReset) invalidates the kept address: do not call this
 * entry point again in a process that has reset the device.  All calls on a
 * device share the one array and each call starts by clearing the counters
 * it needs, so calls whose kernels overlap on the GPU (different streams, or
 * different host threads) race and must be serialized by the caller.
 * Asynchronous on cuda_stream. */
#define CHISAO_DEDUP_NOALLOC_MAX_N (1 << 18)
chisao_status chisao_dedup_noalloc(const float *x_dev, int32_t d, int64_t n,
                                   const float *f_dev, const uint32_t *stuck_dev,
                                   double eps_dup, uint32_t *removed_dev,
                                   int32_t *k_lost_dev, void *cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* CHISAO_H */
