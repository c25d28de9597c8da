/*
 * lra.h — C ABI of a GB300 (sm_103a) library for rank-k approximation by
 * shift-and-invert block power iteration with SVRG linear solves.
 *
 * Method: Gonen & Shalev-Shwartz, "Faster Low-rank Approximation using Adaptive
 * Gap-based Preconditioning" (arXiv 1607.02925), the q = k branch of
 * Algorithm 6 with s = 1:
 *   Algorithm 3 (k = 1) estimates lambda_1 of A = X X^T; Algorithm 7 tunes the
 *   shift lambda; Algorithm 1 (subspace iteration) runs on D = (lambda I - A)^-1
 *   with p > k columns, every product D S being a linear solve by SVRG
 *   (Sec. 2.3, Theorem 3); Algorithm 2 (Rayleigh-Ritz) with C = A returns U.
 *
 * Conventions for every entry point
 *  - X is d x n, column i is data point x_i (Sec. 1).  Dense X is given
 *    column-major with leading dimension ld >= d (equivalently an n x ld
 *    row-major array of data points).
 *  - "d x p blocks" are FP32, column-major, leading dimension d, unless stated.
 *  - A pointer argument documented "device" must be device memory of the
 *    context's GPU; "host or device" pointers are classified with
 *    cudaPointerGetAttributes.  The library never frees caller memory.
 *  - Entry points return lra_status.  Argument errors return LRA_EINVAL before
 *    any side effect.  A CUDA error returns LRA_ECUDA (lra_last_error() gives the
 *    message); the object stays valid only if the error was not sticky.
 *  - Calls on one lra_ctx (and objects created from it) are serialised by the
 *    context's lock; distinct contexts are independent.  Step entry points run
 *    on the context's stream and return after it has completed the work.
 *  - Nothing here traps or aborts; device-side waits are bounded.
 */
#ifndef LRA_H
#define LRA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lra_ctx lra_ctx;
typedef struct lra_mat lra_mat;
typedef uint64_t lra_job;

typedef enum {
    LRA_OK = 0,
    LRA_EINVAL = 1,       /* invalid argument; nothing was changed */
    LRA_ENOMEM = 2,       /* device or host allocation failed, or HBM budget exceeded */
    LRA_ECUDA = 3,        /* a CUDA runtime call failed */
    LRA_ENOTCONV = 4,     /* an iteration cap was reached; outputs are still written */
    LRA_EDIVERGED = 5,    /* SVRG residual grew > 10x, became non-finite, or lambda <= lambda_1 */
    LRA_ENUMERIC = 6,     /* Cholesky of a Gram matrix failed (not positive definite) */
    LRA_ETIMEOUT = 7,     /* lra_poll: the job did not finish within timeout_ms */
    LRA_EAGAIN = 8,       /* lra_poll with timeout 0: job still queued or running */
    LRA_EBUSY = 9,        /* the object is in use by a running job */
    LRA_ECANCELLED = 10,  /* the job was cancelled */
    LRA_EUNSUPPORTED = 11 /* valid request the library does not implement (e.g. p > 112) */
} lra_status;

typedef enum { LRA_F32 = 0, LRA_BF16 = 1, LRA_F16 = 2, LRA_F64 = 3 } lra_dtype;

/* Shift policies.  PAPER = Algorithm 7 (needs the gap budget Delta, Sec. 3);
 * FAR = lambda = 2 lambda1_up with lambda1_up = lambda_hat_1 / (1 - 1/4);
 * FIXED = options.lambda. */
enum { LRA_SHIFT_PAPER = 0, LRA_SHIFT_FAR = 1, LRA_SHIFT_FIXED = 2 };
/* SVRG column sampling: q_i ~ ||x_i||^2 (importance) or q_i = 1/n. */
enum { LRA_SAMPLE_IMPORTANCE = 0, LRA_SAMPLE_UNIFORM = 1 };

/* Counter-stream identifiers (the randomness of the method; see lra_stream_key). */
enum { LRA_STREAM_INIT = 1, LRA_STREAM_POWER_A = 2, LRA_STREAM_POWER_D = 3,
       LRA_STREAM_SVRG = 4, LRA_STREAM_DELTA = 5,
       LRA_STREAM_PART = 6,    /* stage seeds of Algorithm 6: stream_key(seed, PART, t, 0) */
       LRA_STREAM_BLOCK = 7 }; /* Gaussian starts of Algorithm 3 (a = 0 on A, 2 on D) and of
                                  Algorithm 1 on A (a = 1) within a stage */

/* Largest oversampling p supported (the p x p eigenproblem runs in one CTA). */
#define LRA_MAX_P 112

typedef struct lra_options {
    size_t struct_size;     /* sizeof(lra_options); set by lra_options_default */
    int shift_policy;       /* LRA_SHIFT_*; default PAPER */
    double lambda;          /* shift for FIXED; must exceed lambda_hat_1 / (1 - 1/4) */
    double delta;           /* gap budget Delta <= lambda_k - lambda_{p+1} <= 2 Delta (Sec. 3); 0 = estimate */
    double theta_eta;       /* step size eta = theta_eta mu / (lambda^2 + kappa lambda1_up); default 0.25 */
    double theta_m;         /* epoch length m = ceil(theta_m / (eta mu)); default 2 */
    double tau;             /* SVRG stop: ||M||_F <= tau ||B||_F; 0 = 1e-5 (FP32 X), 1e-4 (FP16 X), 1e-3 (BF16 X) */
    int max_epochs;         /* anchors per solve; default 60 */
    int64_t m_max;          /* cap on m; 0 = 50 n */
    int min_outer;          /* outer iterations before the stop rule may fire; default 3 */
    int max_outer;          /* default 2000 */
    int fixed_epochs;       /* > 0: every solve runs exactly this many anchors (no residual stop) */
    int sampling;           /* LRA_SAMPLE_*; default importance */
    int warm_start;         /* 1: W0 = S (lambda I - H)^-1 (Galerkin); 0: W0 = 0.  Default 1 */
    int max_shift_rounds;   /* Algorithm 7 rounds; default 30 */
    double lambda1_hat;     /* > 0: skip the lambda_1 estimate and use this value */
    double *trace_E;        /* optional host array: E_l = ||X||_F^2 - sum_{j<=k} rho_j per outer iteration */
    int trace_cap;          /* length of trace_E */
    int profile;            /* 1: time the X-streaming and inner-loop kernels with CUDA events
                               on the launching stream (fills the *_ms / *_launches fields) */
    int batch;              /* samples per SVRG inner step, 1..16 (default 1 = the step of
                               Sec. 2.3).  b > 1 averages the stochastic term over b samples
                               drawn at the same W (a minibatch, beyond the paper); the step
                               size becomes theta_eta mu/(lambda^2 + kappa lambda1_up / b) and
                               an epoch m = ceil(theta_m/(eta mu)) steps of b samples (at most
                               m_max samples).  Must be a power of two. */
    int acc;                /* 1: accelerated solves (AccSVRGsolve, Sec. 1 and Cor. mainCond;
                               the paper takes the acceleration of Frostig et al. 2015 without
                               printing it).  Read as accelerated proximal point around SVRG:
                               subproblem s solves ((lambda + gamma) I - X X^T) W = B + gamma Z_s
                               by SVRG from W_s, then Z_{s+1} = W_{s+1} + beta (W_{s+1} - W_s),
                               beta = (1 - sqrt q)/(1 + sqrt q), q = mu/(mu + gamma).  gamma is
                               the smallest >= 0 at which an epoch draws at most acc_target
                               samples (0 when plain SVRG already does: the plain solve runs).
                               A subproblem stops at ||M|| <= max(tau ||B||, acc_theta sqrt(q)
                               ||r_s||), r_s the original residual at W_s, read off its first
                               anchor; the solve ends when ||r_s|| <= tau ||B||.  Default 0. */
    double acc_theta;       /* subproblem accuracy factor in (0, 1]; default 0.5 */
    int acc_max_outer;      /* subproblems per accelerated solve; default 200 (then LRA_ENOTCONV
                               in lra_solve_info.status, the iterate is kept) */
    int64_t acc_target;     /* samples per epoch the proximal weight aims for; 0 = n */
    int partition;          /* 1: Algorithm 6 in full (Sec. 3): adaptive partitioning of {1..k}
                               with deflation.  Stage t at index s works on X_{-(s-1)} =
                               (I - U U^T) X applied on the fly (projected X passes, sampling
                               by ||x_i||^2 - ||U^T x_i||^2, inner steps on x_i - U U^T x_i; no
                               copy of X), runs Algorithm 3 on A_{-(s-1)} (eps' = 1/(9 p^2)) and
                               Algorithm 4; a multiplicative gap gives Algorithm 1 on A with
                               q - s + 1 columns, otherwise Algorithm 7, Algorithm 3 on
                               D_{-(s-1)} (eps' = 1/(9p)), Algorithm 5 and Algorithm 1 on D
                               with q - s + 1 columns (q < k) or p - (s - 1) (q = k).  Stage
                               randomness is keyed by stream_key(seed, PART, t, 0).  Needs
                               Delta (or p + 1 <= LRA_MAX_P to estimate it); shift_policy is
                               not used.  Default 0 (the q = k branch at s = 1). */
    int part_max_iters;     /* cap on Algorithm 3's ceil(eps'^-1 ln(d/eps')) iterations; default 2000 */
    int64_t wait_cycles;    /* lra_solve: a pipeline wait of the tensor-core X passes that has not
                               completed after this many SM cycles gives up; the kernel unwinds
                               (waiting, with the default limit, for its own copies and MMAs in
                               flight) and the solve returns LRA_ETIMEOUT.  0 = 4e9 cycles
                               (about 2 s).  Not from the paper: a failure-handling knob. */
} lra_options;

typedef struct lra_report {
    size_t struct_size;     /* caller sets sizeof(lra_report) */
    int status;
    int outer_iters;        /* subspace iterations (solves of the outer loop) */
    int shift_rounds;       /* Algorithm 7 rounds */
    int64_t solves;         /* SVRG solves (shift tuning + outer loop) */
    int64_t epochs;         /* anchor passes inside solves */
    int64_t inner_steps;    /* variance-reduced steps */
    int64_t x_passes;       /* full reads of X by the anchor / Ritz / power kernels */
    int64_t kernel_launches;/* CUDA kernels launched by this call */
    double lambda;          /* final shift */
    double lambda1_hat;     /* Algorithm 3 estimate of lambda_1 */
    double delta;           /* gap budget used (PAPER policy) */
    double mu_lb;           /* lower bound on lambda - lambda_1 used for eta and m */
    double eta;             /* step size of the outer-loop solves */
    int64_t m;              /* epoch length of the outer-loop solves */
    double fro2;            /* ||X||_F^2 (FP64) */
    double err_est;         /* final E = ||X||_F^2 - sum_{j<=k} rho_j (Frobenius error of U, FP64) */
    double last_residual;   /* ||M||_F / ||B||_F of the last anchor */
    double ms_setup, ms_shift, ms_outer, ms_final, ms_total;  /* host wall times */
    /* with options.profile = 1: summed device time and launch count of the
     * X^T W kernel, the X Y kernel and the SVRG inner-loop kernel */
    double xtw_ms, xy_ms, inner_ms;
    int64_t xtw_launches, xy_launches, inner_launches;
    int64_t xtw_cols;       /* total columns (p) processed by the X^T W launches */
    int64_t xy_cols;        /* total columns (p) processed by the X Y launches */
    /* with options.profile = 1: device time per phase of the solve, ms:
     * [0] X^T W, [1] X Y, [2] inner loop (as above), [3] Rayleigh-Ritz Gram
     * matrices and their correction, [4] eigensolver, [5] CholeskyQR2,
     * [6] basis rotation and warm start, [7] anchor epilogue and sampling */
    double phase_ms[8];
    /* options.partition = 1: stages of Algorithm 6, the last index q each found
     * and how (1 = Algorithm 4's multiplicative gap and Algorithm 1 on A,
     * 2 = shift-and-invert: Algorithms 7, 5 and 1 on D) */
    int part_stages;
    int part_q[LRA_MAX_P];
    int part_kind[LRA_MAX_P];
} lra_report;

/* ---------------------------------------------------------------------------
 * Context, matrices, the solve (problem statement: Sec. 1; method: Alg. 6)
 * ------------------------------------------------------------------------- */

/* Default options (struct_size filled in). */
void lra_options_default(lra_options *opt);

/* Create a context on CUDA device `device`.  hbm_budget_bytes caps the device
 * memory this context allocates (0 = no cap).  *out is owned by the caller and
 * released with lra_finalize. */
lra_status lra_init(int device, size_t hbm_budget_bytes, lra_ctx **out);

/* The CUDA stream (cudaStream_t) on which the context launches its kernels. */
void *lra_ctx_stream(lra_ctx *ctx);

/* Release a context.  Matrices created from it must be destroyed first
 * (LRA_EBUSY otherwise); pending serving jobs are cancelled. */
lra_status lra_finalize(lra_ctx *ctx);

/* Copy a dense X (d x n, column-major, leading dimension ld >= d) of type `src`
 * from host or device memory (src_on_device = 0/1) into library-owned device
 * storage of type `storage`, the element type the X passes of Sec. 2.3 stream
 * (conversions round to nearest even):
 *   LRA_F32  - FP32; the tensor-core passes stream it as a BF16 hi/lo pair;
 *   LRA_BF16 - BF16 (2 bytes per entry streamed);
 *   LRA_F16  - FP16 (2 bytes per entry streamed, 3 more significand bits than
 *              BF16): X is stored as fp16(s x) with s the power of two that
 *              puts max |x| in [2^14, 2^15), so entries far below FP16's
 *              normal range keep their precision; every pass divides s out
 *              again (exactly), so all entry points see X itself.
 * A BF16- or FP16-stored matrix also keeps an FP32 copy for the final
 * Rayleigh-Ritz step.  The caller may free X on return.  Requires 1 <= d,
 * 2 <= n. */
lra_status lra_create_dense(lra_ctx *ctx, int64_t d, int64_t n, lra_dtype src, const void *X,
                            int64_t ld, int src_on_device, lra_dtype storage, lra_mat **out);

/* Copy a sparse X (d x n, FP32 values) given as CSR of its d rows from host
 * or device memory (src_on_device = 0/1): rowptr[d+1] int64 with rowptr[0] = 0
 * and rowptr[d] = nnz, colidx[nnz] int32 in [0, n) strictly increasing within
 * each row (no duplicates), val[nnz] finite.  The library keeps its own copy
 * plus the compressed columns x_i (the sampled columns of the SVRG steps and
 * the operand of X^T W, Sec. 2.3 whose cost is O(nnz(X)) per anchor), so the
 * caller may free the arrays on return.  Every solve on a sparse X runs in
 * FP32 on the CUDA cores (the paper's nnz(X) regime, Theorem 3).  Requires
 * 1 <= d, 2 <= n, d and n < 2^31; invalid arrays give LRA_EINVAL (no matrix
 * is created; lra_last_error() names the violated rule). */
lra_status lra_create_csr(lra_ctx *ctx, int64_t d, int64_t n, int64_t nnz, const int64_t *rowptr,
                          const int32_t *colidx, const float *val, int src_on_device, lra_mat **out);

/* Release a matrix and its device memory (LRA_EBUSY while a job uses it). */
lra_status lra_mat_destroy(lra_mat *mat);

/* Shape, storage and ||X||_F^2 of a matrix (any output pointer may be NULL). */
lra_status lra_mat_info(const lra_mat *mat, int64_t *d, int64_t *n, lra_dtype *storage, double *fro2);

/* Rank-k approximation (Alg. 6, q = k branch): writes U (d x k, column-major,
 * leading dimension d, FP32, host or device, caller-owned) with orthonormal
 * columns spanning the approximate top-k left singular subspace, and
 * ritz[k] (FP64, host or device) = the Ritz values rho_1 >= ... >= rho_k of
 * X X^T on span(U).  Requires 1 <= k < p < d (Sec. 1), p <= n,
 * p <= LRA_MAX_P and 0 < eps < 1.  opt may be NULL (defaults); rep may be NULL.
 * Returns LRA_ENOTCONV (outputs written) when max_outer is reached,
 * LRA_EDIVERGED, LRA_ENUMERIC, LRA_ENOMEM, LRA_ECUDA on failure. */
lra_status lra_solve(lra_mat *mat, int k, int p, double eps, uint64_t seed, const lra_options *opt,
                     float *U, double *ritz, lra_report *rep);

/* ---------------------------------------------------------------------------
 * Request loop (continuous batching of many solves on one GPU)
 * ------------------------------------------------------------------------- */

/* Queue a solve; returns at once with a job id.  Jobs are admitted when their
 * device-memory footprint fits the context's budget; admitted jobs run
 * concurrently on their own streams.  The matrix must stay alive until the job
 * is polled or cancelled. */
lra_status lra_submit(lra_ctx *ctx, lra_mat *mat, int k, int p, double eps, uint64_t seed,
                      const lra_options *opt, lra_job *out);
/* (options.partition = 1 gives LRA_EUNSUPPORTED here: its stages allocate
 * per-stage buffers (U^T X, deflated sampling tables, the inner loop's deflated
 * columns) that a fixed admission footprint does not cover.) */

/* Wait up to timeout_ms (0 = do not wait, < 0 = forever) for a job.  On
 * completion copies U/ritz/report (each may be NULL) as lra_solve would, frees
 * the job and returns its status; returns LRA_EAGAIN (timeout 0) or
 * LRA_ETIMEOUT while it is still queued or running. */
lra_status lra_poll(lra_ctx *ctx, lra_job job, int timeout_ms, float *U, double *ritz, lra_report *rep);

/* Cancel a queued or running job (it stops at its next epoch boundary). */
lra_status lra_cancel(lra_ctx *ctx, lra_job job);

/* Human-readable status name; last error message of the calling thread. */
const char *lra_status_str(lra_status s);
const char *lra_last_error(void);

/* ---------------------------------------------------------------------------
 * Step entry points: one step of the path each, on device buffers.
 * They exist so each step can be checked on its own; lra_solve chains them.
 * ------------------------------------------------------------------------- */

/* Key of the counter stream (seed, stream, a, b): SplitMix64 (Steele, Lea and
 * Flood 2014) applied three times, h <- mix64(h + gamma (w + 1)) for
 * w = stream, a, b, starting from h = seed; the t-th random word of the stream
 * is mix64(key + gamma (t + 1)).  Host function. */
uint64_t lra_stream_key(uint64_t seed, uint64_t stream, uint64_t a, uint64_t b);

/* Setup (a0): norm2[i] = ||x_i||^2 (device, n doubles) and *fro2 = ||X||_F^2
 * (host), FP64 accumulation of the stored values.  Sec. 1 eq. (2) sr(X). */
lra_status lra_colnorms(lra_mat *mat, double *norm2, double *fro2);

/* Sampling distribution (a0; Theorem 3's sr(X) dependence): integer weights
 * w_i = max(1, floor(norm2_i * (2^32 / max_j norm2_j))) for norm2_i > 0 and 0
 * otherwise (uniform: w_i = 1), cum[i] = w_0 + ... + w_i (device, n uint64),
 * c[i] = (float)(total / w_i) (device, n floats, 0 where w_i = 0),
 * *total = sum w (host), *kappa = max_i (total / w_i) norm2_i (host, FP64).
 * norm2 is a device array of n doubles. */
lra_status lra_sampling_table(lra_ctx *ctx, int64_t n, const double *norm2, int mode,
                              uint64_t *cum, float *c, uint64_t *total, double *kappa);

/* Largest n accepted by lra_sampling_table_noalloc. */
#define LRA_NOALLOC_MAX_N (1ll << 24)

/* The same table as lra_sampling_table, built without allocating any memory.
 * The paper has no counterpart: this entry point exists for callers that cannot
 * call cudaMalloc / cudaFree when they build the table (for instance an
 * application whose framework reserves the GPU memory for its own pool, or one
 * that cannot afford the device-wide synchronisation of cudaFree mid-stream).
 * Inputs and outputs are the caller's, as for lra_sampling_table; the scratch
 * (about 0.5 MB) is a fixed device array of the library that stays resident on
 * every GPU that loads the library, until exit.  Requires 1 <= n <=
 * LRA_NOALLOC_MAX_N (LRA_EINVAL otherwise).  Calls no cudaMalloc, cudaFree or
 * allocating library routine.  All calls share the array: calls whose GPU work
 * overlaps (other streams or threads) race on it and must be serialised by the
 * caller.  The first call on a device looks the array's address up with that
 * device current; make it before any stream capture. */
lra_status lra_sampling_table_noalloc(lra_ctx *ctx, int64_t n, const double *norm2, int mode,
                                      uint64_t *cum, float *c, uint64_t *total, double *kappa);

/* Sampler (a7): idx[t] (device, m int32) = the first i with cum[i] > r_t,
 * r_t = floor(u_t * total / 2^64), u_t the t-th word of stream `key`. */
lra_status lra_sample(lra_ctx *ctx, int64_t n, const uint64_t *cum, uint64_t total, uint64_t key,
                      int64_t m, int32_t *idx);

/* Gaussian block (a3; Algorithm 1's S0 ~ N(0,1)^{d x p}): out (device, d x p)
 * element e = row + d col from Box-Muller on words 2(e/2), 2(e/2)+1 of stream
 * (seed, stream, a, 0): U1 = ((u >> 11) + 1) 2^-53, U2 = (u' >> 11) 2^-53,
 * sqrt(-2 ln U1) cos(2 pi U2) for even e and sin(2 pi U2) for odd e. */
lra_status lra_gaussian_block(lra_ctx *ctx, uint64_t seed, uint64_t stream, uint64_t a, int64_t d,
                              int p, float *out);

/* Anchor pass (a6; SVRGsolve's full gradient): M = lambda Wt - X (X^T Wt) - B
 * for d x p blocks Wt, B, M (device).  Optional *normM2, *normB2 (host) get
 * ||M||_F^2 and ||B||_F^2 (FP64 accumulation).  X is read once per product
 * (two passes). */
lra_status lra_anchor(lra_mat *mat, int p, const float *Wt, const float *B, double lambda, float *M,
                      double *normM2, double *normB2);

/* Products with X (a4/a6): Y = X^T W (n x p column-major, leading dim n) and
 * G = X Y (d x p) for device buffers.  use_f32_copy = 1 reads the FP32 copy of
 * a BF16-stored matrix. */
lra_status lra_xt_mul(lra_mat *mat, int p, const float *W, float *Y, int use_f32_copy);
lra_status lra_x_mul(lra_mat *mat, int p, const float *Y, float *G, int use_f32_copy);

/* SVRG inner loop (a7): m variance-reduced steps on the d x p block W (device,
 * in/out) from anchor Wt with anchor gradient M: for t < m, i = idx[t],
 * r = x_i^T (W - Wt), W <- W - eta [lambda (W - Wt) - c[i] x_i r + M].
 * The p columns are independent chains sharing the index sequence. */
lra_status lra_svrg_inner(lra_mat *mat, int p, float *W, const float *Wt, const float *M,
                          const int32_t *idx, int64_t m, const float *c, double eta, double lambda);

/* The same with a batch of `batch` samples per step (a power of two <= 16; the
 * minibatch reading of lra_options.batch): idx holds m * batch entries, step t
 * uses idx[t batch .. t batch + batch - 1], every r_u = x_{i_u}^T (W - Wt) is
 * taken at the same W and W <- W - eta [lambda (W - Wt) - (1/batch) sum_u
 * c[i_u] x_{i_u} r_u + M].  batch = 1 is lra_svrg_inner.  LRA_EUNSUPPORTED when
 * the batch does not fit the dense kernel's shared-memory ring for this d. */
lra_status lra_svrg_inner_batched(lra_mat *mat, int p, float *W, const float *Wt, const float *M,
                                  const int32_t *idx, int64_t m, int batch, const float *c, double eta,
                                  double lambda);

typedef struct lra_solve_info {
    int epochs;            /* anchors computed */
    int64_t inner_steps;
    int64_t m;             /* epoch length used */
    double eta;            /* step size used */
    double residual;       /* ||M||_F / ||B||_F at the last anchor (accelerated: the original
                              system's ||(lambda I - A) W - B||_F / ||B||_F at the last
                              subproblem's first anchor) */
    int status;            /* LRA_OK, LRA_ENOTCONV (cap), LRA_EDIVERGED */
    int outer;             /* accelerated solve: subproblems solved (solve ids solve_id ..
                              solve_id + outer - 1); 0 for the plain solve */
    double gamma;          /* accelerated solve: proximal weight (0 = plain solve ran) */
} lra_solve_info;

/* SVRGsolve (Sec. 2.3): W (device d x p, in: W0, out: solution) approximately
 * solves (lambda I - X X^T) W = B.  eta = theta_eta mu / (lambda^2 + kappa
 * lambda1_up), m = ceil(theta_m / (eta mu)), epochs keyed (seed, SVRG,
 * solve_id, epoch).  Stops at ||M|| <= tau ||B|| (tau from opt), on a stall
 * (after the 4th anchor, a residual above 0.9 x the previous one), or at the
 * epoch cap.  With opt->acc = 1 it is the accelerated solve (see
 * lra_options.acc), subproblem s keyed as solve solve_id + s. */
lra_status lra_svrg_solve(lra_mat *mat, int p, const float *B, float *W, double lambda, double mu,
                          double lambda1_up, uint64_t seed, int64_t solve_id,
                          const lra_options *opt, lra_solve_info *info);

/* Gram (a4/a8): G (device, p x p FP64, column-major) = A^T A for a device
 * rows x p block A (column-major, leading dimension lda >= rows). */
lra_status lra_gram(lra_ctx *ctx, int64_t rows, int p, const float *A, int64_t lda, double *G);

/* CholeskyQR2 (a8; Algorithm 1's QR step): W (device d x p) is replaced by Q of
 * W = Q R with diag(R) > 0, computed as G = W^T W (FP64), R = chol(G),
 * W <- W R^-1, twice.  LRA_ENUMERIC if a Gram is not positive definite. */
lra_status lra_cholqr2(lra_ctx *ctx, int64_t d, int p, float *W);

/* Symmetric eigendecomposition (a4; Algorithm 2): H (device p x p FP64,
 * column-major, symmetric) -> evals (device, p, descending) and evecs (device
 * p x p FP64 column-major), each eigenvector signed so that its largest-
 * magnitude entry is positive.  Eigenvectors by cyclic Jacobi, eigenvalues as
 * FP64 Rayleigh quotients. */
lra_status lra_sym_eig(lra_ctx *ctx, int p, const double *H, double *evals, double *evecs);

/* Rayleigh-Ritz (a4/a9; Algorithm 2 with C = X X^T): for an orthonormal
 * S (device d x p): H = (X^T S)^T (X^T S) (device p x p FP64, may be NULL),
 * evals (device, p, descending), evecs (device p x p).  use_f32_copy as in
 * lra_x_mul. */
lra_status lra_ritz(lra_mat *mat, int p, const float *S, int use_f32_copy, double *H, double *evals,
                    double *evecs);

/* lambda_1 estimate (a1; Algorithm 3 with C = X X^T, k = 1, eps = 1/4):
 * L = ceil(4 ln(4 d)) power steps from the Gaussian start of stream
 * (seed, POWER_A, 0), then lambda_hat = z^T C z. */
lra_status lra_lambda1_estimate(lra_mat *mat, uint64_t seed, double *lambda1_hat);

/* Shift tuning (a2; Algorithm 7): starting from lambda = 1.5 lambda1_hat, each
 * round estimates 1/lambda_1(D) by Algorithm 3 on D (k = 1, eps' = 1/9, start
 * vector of stream (seed, POWER_D, round)); stops when the estimate lies in
 * [delta/27, delta/5], else lambda <- lambda - (1 - 1/9)/2 * estimate.
 * Outputs (host): *lambda, *inv_est, *mu_lb, *rounds; history (host, may be
 * NULL) receives (lambda, estimate) pairs for up to max_shift_rounds rounds.
 * Solves are numbered from *solve_count (in/out). */
lra_status lra_shift_tune(lra_mat *mat, uint64_t seed, double lambda1_hat, double delta,
                          const lra_options *opt, int64_t *solve_count, double *lambda,
                          double *inv_est, double *mu_lb, int *rounds, double *history);

/* Gap budget (Sec. 3, no procedure given): Algorithm 3 on A with p+1 vectors,
 * eps' = 1/(9 p^2), L = min(200, ceil(ln(d / eps') / eps')), then
 * delta = (rho_k - rho_{p+1}) / 1.5. */
lra_status lra_delta_estimate(lra_mat *mat, int k, int p, uint64_t seed, double *delta);

#ifdef __cplusplus
}
#endif

#endif /* LRA_H */
