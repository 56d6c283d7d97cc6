/*
 * godec.h - C ABI of the GB300 (sm_103a) GoDec-BRP library.
 *
 * GoDec (Zhou & Tao, arXiv:1309.0302) splits a dense m x n matrix X into a
 * rank-r part L, a part S with at most k nonzeros and noise G (Sec. 2, eq.
 * GoDecMODEL), minimising ||X - L - S||_F^2 (eq. ls_app) by alternating an
 * L-step and an S-step (eq. raw_ls).  This library runs Algorithm 1 ("GoDec
 * by BRP"): the L-step is the bilateral random projection with power scheme
 * (Sec. 3.1, eqs. lr_app and mlr_app), the S-step is the entry-wise hard
 * threshold keeping the k largest |X - L| (eq. raw_lss).
 *
 * Forms: the plain float32 form (godec_init / iterate / solve); the precision form
 * (godec_params.precision = GODEC_PREC_BF16_REFINE: a float16 power chain and one
 * float32 correction per iteration); the batched form (godec_batch_*: many problems of
 * uneven m, n, r in one CUDA graph per batch iteration); the differentiated form
 * (godec_backward: the gradient with respect to X of a loss of T unrolled q = 0
 * iterations); godec_run_host (host buffers in and out).
 *
 * Conventions for every entry point:
 *  - Matrices are row-major.  "Device" pointers are CUDA global memory on the
 *    device that is current when godec_init is called; "host" pointers are
 *    ordinary (preferably pinned) host memory.
 *  - Every call returns a godec_status and never throws.  After an error the
 *    context stays usable unless the status is GODEC_ERR_STATE or
 *    GODEC_ERR_CUDA; godec_last_error() gives a one-line reason.
 *  - Calls on one context are not thread-safe; separate contexts are
 *    independent.  All GPU work of a context runs on the stream passed to
 *    godec_init (a cudaStream_t passed as void*; NULL = legacy default).
 *  - L is never formed densely: it is returned as U diag(sigma) V^T with
 *    U (m x r_eff) and V (n x r_eff) having orthonormal columns.
 *  - S is returned as COO: int64 linear indices i*n + j in ascending order
 *    and float32 values.
 */
#ifndef GODEC_H
#define GODEC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum godec_status {
  GODEC_OK = 0,
  GODEC_ERR_ARG = 1,         /* invalid argument (sizes, pointers, alignment) */
  GODEC_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  GODEC_ERR_OOM = 3,         /* device or host allocation failed */
  GODEC_ERR_NONFINITE = 4,   /* X or an intermediate holds NaN/Inf */
  GODEC_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
  GODEC_ERR_STATE = 6,       /* call not valid in the context's state */
  GODEC_ERR_UNSUPPORTED = 7  /* valid request outside the built limits */
} godec_status;

/* Arithmetic of the X-streaming products. */
enum {
  GODEC_PREC_FP32 = 0,        /* float32 X, float32 accumulation */
  GODEC_PREC_BF16_REFINE = 1  /* precision form (r <= 32): the power chain streams a
                                 16-bit (float16, scaled by the power of two s_Z) copy of
                                 X - S with float32 accumulation; then one float32 visit
                                 of X - S computes Z V and Z^T U and the tangent-space
                                 correction of the factors, re-truncated to rank r */
};

/* Maximum target rank handled by the kernels. */
#define GODEC_MAX_RANK 64

typedef struct godec_params {
  int64_t m, n;      /* X is m x n (m, n >= 1, m*n < 2^32: the S-step's histograms
                        count entries in 32 bits) */
  int64_t ldx;       /* row stride of X in elements, >= n */
  int32_t r;         /* target rank, 1 <= r <= min(m, n, GODEC_MAX_RANK) */
  int32_t q;         /* power-scheme exponent of eq. mlr_app, 0 <= q <= 8 */
  int64_t k;         /* cardinality bound of S, 0 <= k <= m*n */
  double tol;        /* epsilon of the stop test ||X-L-S||^2/||X||^2 <= tol */
  int32_t max_iter;  /* iteration cap of godec_solve, >= 1 */
  int32_t precision; /* GODEC_PREC_* */
  double rank_tol;   /* relative singular-value tolerance of the rank test of
                        Algorithm 1; <= 0 selects 1e-4 */
  int32_t flags;     /* GODEC_FLAG_* */
  int32_t reserved;  /* must be 0 */
} godec_params;

/* Reserved; ignored.  godec_backward needs no tape: it recomputes the per-iteration
   factors from X, A1 and the supports. */
#define GODEC_FLAG_TAPE 1
/* Precision form only: skip the float32 correction (diagnostic: the float16 chain's own
   accuracy). */
#define GODEC_FLAG_NO_REFINE 2
/* Factor the Gram of every critical-path orthonormalisation (the power-step products of
   the exact path, the CholeskyQR2 of Q1 and Q2, the precision form's correction) in
   float64 instead of float32.  GB300's float64 rate makes each such factorisation about
   3.5 times slower (about 110 us against 31 us at r = 50); the factor is applied in
   float32 either way. */
#define GODEC_FLAG_FP64_FACTOR 4
/* The chain's first projection (X - S) A1 (Algorithm 1's L-step; A1 is fixed for the run)
   is formed either by streaming X - S like the other products (the default,
   GODEC_FLAG_DENSE_FIRST), or, with GODEC_FLAG_SPARSE_FIRST, as X A1 - S A1 with X A1
   computed once per godec_init / godec_reset and S A1 summed over the k entries of S.
   The second reads S at random positions: on GB300 its kernel is faster only for sparse
   S (k below about m n / 200), and over whole iterations its rounding made the lagged
   normalisers' alarm trip more often on the inputs measured.  Both flags set:
   GODEC_ERR_ARG.  Plain form only: the precision form, GreBsmo, naive GoDec, LinGoDec and
   MSE training always stream. */
#define GODEC_FLAG_SPARSE_FIRST 8
#define GODEC_FLAG_DENSE_FIRST 16

typedef struct godec_ctx godec_ctx;

/*
 * Create a context for Algorithm 1 on X.
 *   X  : device, m x ldx float32, BORROWED: it must stay valid and unchanged
 *        until godec_destroy.  ldx*4 must be a multiple of 16 bytes.
 *   A1 : device, n x r float32 (row-major), the random test matrix of
 *        Algorithm 1 (the first factor of the power chain); copied.  Reading of the
 *        paper: A1 is drawn once
 *        by the caller (e.g. standard Gaussian) and kept for all iterations.
 *   stream : cudaStream_t (as void*) on which all work of the context runs.
 * The context owns its workspace (about 4*m*n bytes for the working copy of
 * X - S, plus O((m+n)*64 + k) bytes).  S starts at 0 and t at 0.
 * Errors: GODEC_ERR_ARG for invalid params or pointers, GODEC_ERR_OOM,
 * GODEC_ERR_CUDA.  On error *ctx is set to NULL.
 */
godec_status godec_init(godec_ctx** ctx, const godec_params* params,
                        const float* X, const float* A1, void* stream);

/* Restart from S = 0, t = 0 and the initial rank; X and A1 are kept. */
godec_status godec_reset(godec_ctx* ctx);

/*
 * Run exactly n_iter iterations of Algorithm 1, ignoring the
 * stop test.  Each iteration: Z = X - S_{t-1}; L_t from the BRP power chain
 * with the rank test; S_t = P_Omega(X - L_t) with Omega the nonzero subset of
 * the k largest |X - L_t| (ties by ascending linear index).
 * rel_err (host, nullable) receives ||X - L_t - S_t||_F^2 / ||X||_F^2 of the
 * last iteration.  Synchronises the stream before returning.
 * Errors: GODEC_ERR_NONFINITE if X - L holds NaN/Inf (state then reset),
 * GODEC_ERR_CUDA.
 */
godec_status godec_iterate(godec_ctx* ctx, int32_t n_iter, double* rel_err);

/*
 * Algorithm 1 with its stop test: iterate until
 * ||X - L_t - S_t||^2 / ||X||^2 <= tol or t = max_iter (a do-while: at least
 * one iteration).  iters and rel_err (host, nullable) receive t and the last
 * relative error.
 */
godec_status godec_solve(godec_ctx* ctx, int32_t* iters, double* rel_err);

/*
 * Copy the factors of L_t = U diag(sigma) V^T.
 *   U : device, m x r_eff float32 (row stride r_eff), nullable
 *   sigma : device, r_eff float32, descending, nullable
 *   V : device, n x r_eff float32 (row stride r_eff), nullable
 *   r_eff : host, receives the current rank (< r after a rank drop)
 * Buffers must hold at least params.r columns.  GODEC_ERR_STATE before the
 * first iteration.
 */
godec_status godec_get_L(godec_ctx* ctx, float* U, float* sigma, float* V, int32_t* r_eff);

/*
 * L_t as a dense matrix, L = U diag(sigma) V^T (eq. mlr_app: L = Q1 M^{1/(2q+1)} Q2^T,
 * with the factors godec_get_L returns), written by the library's own kernel in float32
 * (each entry a sum of r_eff products).  For callers that need L itself (a dense loss, the
 * differentiated form's output); the iteration never forms it.
 *   L : device, m x ldl float32 (ldl >= n), caller-owned, overwritten.
 * GODEC_ERR_STATE before the first iteration.  Synchronises the stream.
 */
godec_status godec_get_L_dense(godec_ctx* ctx, float* L, int64_t ldl);

/*
 * Copy S_t as COO sorted by ascending linear index i*n + j.
 *   idx : device int64[cap], val : device float32[cap] (both nullable when
 *   cap = 0), nnz : host, receives |Omega| (<= k).
 * GODEC_ERR_ARG if cap < nnz (nnz is still written).
 */
godec_status godec_get_S(godec_ctx* ctx, int64_t* idx, float* val, int64_t cap, int64_t* nnz);

/*
 * Dense residual R = X - L_t of the current state (the matrix the S-step of
 * Algorithm 1 thresholds, eq. raw_lss), computed by the same tensor-core kernel and
 * arithmetic as the S-step's residual pass.
 *   R : device, m x ldr float32, ldr >= n.
 * GODEC_ERR_STATE before the first iteration.  Synchronises the stream.
 */
godec_status godec_residual(godec_ctx* ctx, float* R, int64_t ldr);

/* State after the last committed iteration t: its objective
   ||X - L_t - S_t||_F^2 (E_t^2 of Appendix I), |Omega| and bookkeeping. */
typedef struct godec_info {
  int32_t iter;
  int32_t r_eff;
  double rel_err;
  double obj;          /* ||X - L_t - S_t||_F^2 */
  double normX2;       /* ||X||_F^2 */
  int64_t nnz;
  int32_t select_passes;   /* residual passes used by the last S-step (1-3) */
  int32_t rank_drops;      /* times the rank test lowered r */
  int32_t launches_per_iter;  /* nodes of one captured fast-path iteration */
  int32_t exact_iters;        /* iterations run on the exact (Cholesky on the critical
                                 path) power chain; the others used lagged normalisers */
  int32_t svd_sweeps;         /* Jacobi sweeps of the last core SVD */
  int32_t chol_shifts;        /* Cholesky factorisations that needed a diagonal shift */
  int32_t alarms;             /* fast-path iterations abandoned because a lagged normaliser no
                                 longer conditioned the chain (each redone on the exact path) */
} godec_info;
godec_status godec_get_info(godec_ctx* ctx, godec_info* info);

/* Release the context and its workspace (NULL is ignored). */
void godec_destroy(godec_ctx* ctx);

/* One-line description of the context's last error ("" if none; a static
   string for ctx == NULL). */
const char* godec_last_error(const godec_ctx* ctx);
const char* godec_status_string(godec_status s);

/*
 * Whole run from HOST buffers: copy X (m x n, row stride n) and A1 (n x r)
 * to the device, run n_iter iterations of Algorithm 1 (n_iter <= 0 means:
 * godec_solve with params->tol and params->max_iter), copy the results back
 * and release everything.
 *   U (m x r), sigma (r), V (n x r): host, nullable; r_eff host.
 *   S_idx, S_val: host arrays of S_cap entries (sorted COO), nullable.
 *   nnz, iters, rel_err: host, nullable.
 * All device memory is allocated and freed inside the call on `stream`.
 */
godec_status godec_run_host(const godec_params* params, const float* X_host,
                            const float* A1_host, int32_t n_iter, void* stream,
                            float* U, float* sigma, float* V, int32_t* r_eff,
                            int64_t* S_idx, float* S_val, int64_t S_cap, int64_t* nnz,
                            int32_t* iters, double* rel_err);

/*
 * Streaming tall-skinny products (the "(X - S) A" contractions of Sec. 3.1,
 * the power chain of Algorithm 1), exposed for testing and benchmarking.
 *   godec_mul_ZB : Y = Z B,    Z m x n (row stride ldz), B n x r, Y m x r
 *   godec_mul_ZtC: W = Z^T C,  Z m x n (row stride ldz), C m x r, W n x r
 * All pointers are device float32, row-major with row stride r for B, C, Y,
 * W.  1 <= r <= GODEC_MAX_RANK, ldz >= n, ldz*4 a multiple of 16 bytes, Z
 * 16-byte aligned.  Computed on the tensor cores with the two-term float16
 * split of both operands (float32-level accuracy, about 1e-7 relative); one
 * extra read of Z finds the power-of-two scale that keeps it in float16 range.
 * The call allocates its scratch on `stream` and frees it before returning
 * (stream-ordered), and does not synchronise.
 */
godec_status godec_mul_ZB(const float* Z, int64_t m, int64_t n, int64_t ldz,
                          const float* B, int32_t r, float* Y, void* stream);
godec_status godec_mul_ZtC(const float* Z, int64_t m, int64_t n, int64_t ldz,
                           const float* C, int32_t r, float* W, void* stream);

/*
 * Kernel-level timing: run n_iter real iterations (they advance the state like
 * godec_iterate) launching each kernel directly on the context stream with a
 * CUDA event before and after it, and accumulate per kernel class:
 *   ms[c]       : total device time in milliseconds (host arrays of
 *   launches[c] : number of launches               GODEC_PROF_CLASSES entries)
 * Classes: 0 streaming product (with its fused split-K reduction, normaliser
 * and Gram partials), 1 Gram sums, 2 r x r Cholesky (critical path), 3 tall x
 * r x r products, 4 lagged-normaliser updates (side stream), 5 rank test (side
 * stream), 6 core SVD and root, 7 residual pass (S-step), 8 selection control,
 * radix-select rounds and S emit, 9 sparse update of X - S and its transpose,
 * 10 the precision form's float32 correction apart from its two streaming
 * products (which count in class 0), 11 the chain's first projection from the
 * cached X A1 (X A1 - S A1 over the support of S, in place of the first
 * streaming product).
 * bytes_product (host, nullable) receives the algorithmic bytes of one
 * streaming product at the current rank: 4*m*n (X - S) + 4*(m + n)*r.
 */
#define GODEC_PROF_CLASSES 12
godec_status godec_profile(godec_ctx* ctx, int32_t n_iter, double* ms, int64_t* launches,
                           double* bytes_product);

/*
 * Self-test of the timeout path.  Every wait of the device pipelines (TMA, tensor-core
 * and epilogue hand-offs, see GODEC_ERR_TIMEOUT) is bounded: a wait that gives up flags
 * the context, the kernel drains what it has in flight and returns, and the host call
 * reports GODEC_ERR_TIMEOUT with the context still usable.  This call runs one such
 * wait that nothing completes, with `polls` polls of at most ~2 us each (1 .. 1 << 20),
 * on the context's stream, and reports it through the same path: it returns
 * GODEC_ERR_TIMEOUT (godec_last_error says which wait), the iteration count and the
 * factors are unchanged, and the next godec_iterate runs normally.  GODEC_ERR_ARG for
 * polls out of range.
 */
godec_status godec_check_timeout(godec_ctx* ctx, uint32_t polls);

/*
 * The launches of the last iteration that godec_profile ran, in enqueue order:
 * for each (up to cap) its class, whether it ran on the side stream, and its
 * start and end events in milliseconds after the iteration's first event
 * (host arrays of cap entries, each nullable).  count (host) receives the
 * number of launches recorded; 0 before any godec_profile call.
 */
godec_status godec_profile_trace(godec_ctx* ctx, int32_t cap, int32_t* cls, int32_t* side, float* t0, float* t1,
                                 int32_t* count);

/*
 * Differentiated form (q = 0): the gradient with respect to X of a loss of L_T after T
 * unrolled iterations of Algorithm 1 at q = 0 (L_t = Y1 (A2^T Y1)^{-1} Y2^T, eq. lr_app;
 * S_t = P_Omega_t(X - L_t), eq. raw_lss) with the supports Omega_1 .. Omega_{T-1} held
 * fixed (the selection is piecewise constant in X), starting from S_0 = 0.
 *   X        : device, m x ldx float32 (ldx*4 a multiple of 16 bytes)
 *   A1       : device, n x r float32 row-major (the same A1 as the forward run), r <= 64
 *   T        : number of iterations, >= 1
 *   supports : host array of T-1 device pointers; supports[t-1] holds the int64 linear
 *              indices (i*n + j, no duplicates, any order) of Omega_t
 *   support_nnz : host array of the T-1 sizes
 *   dLoss/dL_T, one of: gU (device m x g) and gV (device n x g) row-major, g <= 64,
 *              meaning gU gV^T; or gL (device, m x ldg float32, ldg*4 a multiple of
 *              16 bytes).  The unused pointers are null.
 *   dX       : device, m x lddx float32, overwritten with the gradient
 *   flags    : 0 or GODEC_BACKWARD_REBUILD
 * The per-iteration factors are recomputed in a forward sweep (checkpointed for the
 * backward sweep), so only the supports are needed from the forward run.  The iterates
 * Z_t and Z_t^T of the forward sweep are kept for the backward sweep when all T of them
 * fit in a quarter of the free device memory (2 T m n floats); with
 * GODEC_BACKWARD_REBUILD, or when they do not fit, one copy is kept and rebuilt from X
 * and the checkpoints in the backward sweep (slower, 2 m n floats).  Scratch is
 * allocated and freed on `stream` (stream-ordered); the call does not synchronise.
 * Float32 arithmetic with the float32-accurate tensor-core products; the sparse products
 * accumulate with float atomics (results may differ in the last bits between runs).
 * GODEC_ERR_ARG on invalid arguments, GODEC_ERR_OOM when scratch cannot be allocated.
 */
godec_status godec_backward(const float* X, int64_t m, int64_t n, int64_t ldx, const float* A1, int32_t r,
                            int32_t T, const int64_t* const* supports, const int64_t* support_nnz,
                            const float* gU, const float* gV, int32_t g_rank, const float* gL, int64_t ldg,
                            float* dX, int64_t lddx, int32_t flags, void* stream);
#define GODEC_BACKWARD_REBUILD 1

/*
 * Entry-wise hard threshold of a dense matrix (eq. raw_lss, the S-step of
 * Algorithm 1 with L = 0): the nonzero subset of the k largest |R|, ties by
 * ascending linear index, runs the same kernels as the S-step.
 *   R : device, m x ldr float32 (ldr*4 a multiple of 16 bytes, 16-byte aligned)
 *   idx, val : device int64[cap] / float32[cap], receive the COO sorted by
 *              linear index; nnz (host) receives min(k, #nonzeros of R).
 * Scratch is allocated and freed inside the call (stream-ordered); the call
 * synchronises the stream.  GODEC_ERR_ARG if cap < the result size or m*n >= 2^32.
 */
godec_status godec_hard_threshold(const float* R, int64_t m, int64_t n, int64_t ldr, int64_t k,
                                  int64_t* idx, float* val, int64_t cap, int64_t* nnz,
                                  void* stream);

/*
 * godec_mul_ZB_noalloc: Y = Z B like godec_mul_ZB, for callers that must not
 * allocate device memory while they run (an application that reserves all GPU
 * memory at start-up and forbids later allocations, or a latency-critical loop
 * that cannot afford an allocation's synchronisation).  The paper has no
 * counterpart; this is a library convenience.
 *   Same arguments and layout as godec_mul_ZB; computed with float32 FMAs on
 *   the CUDA cores (results agree with godec_mul_ZB to float32 rounding).
 *   Scratch: a fixed 32 MiB array in the library's device code.  A GPU holds it
 *   from the time that code is loaded there (with CUDA's default lazy loading, at
 *   the first use of the library on that device) until the process exits; no
 *   allocation or free happens in the call.  Problems whose scratch (padded B,
 *   split-K partials, padded Y) exceeds 32 MiB are rejected with
 *   GODEC_ERR_UNSUPPORTED and a message in godec_last_error(NULL).  Each call
 *   outside stream capture looks up the array's device address; a call made
 *   while `stream` is capturing reuses the address found by an earlier call on
 *   the same device, so make one call on each device before any capture (a
 *   first call under capture returns GODEC_ERR_STATE).
 *   All calls on a device share the array and leave its contents behind:
 *   calls that overlap on the GPU (different streams, threads or processes
 *   without ordering) race and corrupt each other's results.
 */
godec_status godec_mul_ZB_noalloc(const float* Z, int64_t m, int64_t n, int64_t ldz,
                                  const float* B, int32_t r, float* Y, void* stream);

/*
 * Naive GoDec (Sec. 2.1, eq. raw_lss): the L-step is the rank-r truncated SVD of
 * Z = X - S itself instead of BRP; the S-step is the same exact top-k as Algorithm 1's.
 * The truncated SVD runs as a block subspace iteration over p = godec_naive_columns(m, n,
 * r) columns (r plus up to 8 oversampling columns): from the basis B the previous
 * iteration ended with (orth(Omega) in the first), q times B = orth(Z^T orth(Z B)), then
 * the Rayleigh-Ritz step (Z B = Q R, SVD of the p x p R in float64, the leading r
 * triplets).  It converges to the exact truncated SVD at the rate
 * (sigma_{p+1} / sigma_r)^(2q) per iteration and, being warm-started, keeps converging
 * across iterations; the cold start gets 6 more power steps on X when the context is
 * created or reset.
 *   params : as godec_init, with q = power steps per L-step (1..8) and precision
 *            GODEC_PREC_FP32; there is no rank test (r stays fixed)
 *   Omega  : device, n x p float32 row-major, the first test matrix (copied)
 * The context runs with godec_iterate / godec_solve and the getters as a GoDec context
 * (godec_profile returns GODEC_ERR_STATE).  Errors as godec_init.
 */
int godec_naive_columns(int64_t m, int64_t n, int32_t r);
godec_status godec_naive_init(godec_ctx** ctx, const godec_params* params, const float* X, const float* Omega,
                              void* stream);

/*
 * GreBsmo, greedy bilateral smoothing (Sec. 3.2.1, Algorithm 2): X = U V + S + G with U
 * orthonormal (m x r), V (r x n) and S from the element-wise soft threshold (eq. softt).
 * Each inner step (eq. GreBsmoA), with Z = X - S:
 *   U = Q of QR(Z V^T) (CholeskyQR2),  V = U^T Z,  S = S_lambda(X - U V);
 * after K inner steps the relative error ||X - U V - S||^2 / ||X||^2 is tested against
 * tau; if it is above tau and r < r_max, dr rows are appended to V: the dr top right
 * singular vectors of X - U V - S (eq. GreBsmoD), here by the random-projection variant
 * the paper allows (a randomized subspace iteration: B = orth(Omega_s), q_inc times
 * B = orth(D^T orth(D B)), then the dr top right singular vectors of D B mapped back by
 * B).  The first V comes the same way from X (the greedy direction from U = 0, S = 0).
 * The products stream X - S through the same tensor-core kernel as GoDec; the soft
 * threshold runs in the residual pass (candidates |R| > lambda, S = R - lambda sgn R).
 */
typedef struct godec_grebsmo_params {
  int64_t m, n;        /* X is m x n, m n < 2^32 */
  int64_t ldx;         /* row stride of X in elements, >= n, ldx*4 a multiple of 16 */
  double lambda;       /* soft threshold of eq. softt, > 0 (exactly representable in
                          float32 keeps the GPU's support test |R| > lambda exact) */
  double tau;          /* stop when ||X - U V - S||^2 / ||X||^2 <= tau */
  int64_t s_cap;       /* initial capacity of S (entries); grown when the support is larger */
  int32_t dr;          /* rank increment, >= 1 */
  int32_t K;           /* inner steps per rank stage, >= 1 */
  int32_t r_max;       /* rank cap, dr <= r_max <= min(m, n, GODEC_MAX_RANK) */
  int32_t oversample;  /* extra columns of the random projection: p = dr + oversample <=
                          min(m, n, GODEC_MAX_RANK) */
  int32_t q_inc;       /* power steps of the increment's subspace iteration, 0..16 */
  int32_t flags;       /* GODEC_FLAG_FP64_FACTOR or 0 */
} godec_grebsmo_params;

/*
 * Create a GreBsmo context on X.
 *   X     : device, m x ldx float32, BORROWED (unchanged until godec_destroy)
 *   Omega : device, the random test matrices of the increments, BORROWED: stage s
 *           (s = 0 for the first V, then one per increment; at most
 *           1 + ceil((r_max - dr) / dr) stages) is the n x p row-major block at
 *           Omega + s n p, p = dr + oversample.
 * The context is a godec_ctx: after godec_grebsmo_run use godec_get_L (L = U diag(sigma)
 * V^T in the same orthonormal factored form as GoDec's), godec_get_L_dense, godec_get_S
 * (the support of S and its values), godec_residual, godec_get_info (iter = inner steps
 * run, rel_err of the last one) and godec_destroy.  godec_iterate, godec_solve and
 * godec_profile return GODEC_ERR_STATE on it.  Errors as godec_init.
 */
godec_status godec_grebsmo_init(godec_ctx** ctx, const godec_grebsmo_params* params, const float* X,
                                const float* Omega, void* stream);

/*
 * Run GreBsmo from U = 0, S = 0 to its stop (error <= tau or rank r_max).
 *   r_out     : host, receives the final rank
 *   stage_err : host array of cap entries (nullable): the relative error after each
 *               rank stage, in order; n_stages (host, nullable) receives their number
 * Synchronises the stream (the host tests the error after every stage).
 */
godec_status godec_grebsmo_run(godec_ctx* ctx, int32_t* r_out, double* stage_err, int32_t cap,
                               int32_t* n_stages);

/*
 * LinGoDec, linear functional GoDec (Sec. 4.3, eqs. LinGoDec and NLinGoDec): X (m users x
 * n items) = W F^T + S + G with the item features F (n x d) given, rank(W) <= r and S from
 * the soft threshold, by alternating exact minimisation of
 *   1/2 ||X - W F^T - S||_F^2 + lambda ||vec S||_1:
 * W = the rank-constrained least squares fit of X - S (with F = Qf Rf: W Rf^T is the rank-r
 * truncation of (X - S) Qf, eqs. NLinGoDec), then S = S_lambda(X - W F^T) (eq. softt).
 * (X - S) Qf streams through the tensor-core product; the truncation is a float64 SVD of
 * the d x d factor of its CholeskyQR2; the soft threshold runs in the residual pass.
 *   params : m, n, ldx, r (1 <= r <= d), k (initial capacity of S, grown as needed),
 *            precision GODEC_PREC_FP32, flags; tol and max_iter are not used
 *   lambda : the soft threshold, > 0 (exact in float32 keeps |R| > lambda exact)
 *   X      : device m x ldx float32, BORROWED;  F : device n x d float32 row-major, copied
 * The getters of a GoDec context apply (godec_get_L gives L = W F^T in factored form,
 * godec_get_S, godec_get_info with rel_err = ||X - W F^T - S||^2 / ||X||^2); godec_iterate,
 * godec_solve and godec_profile return GODEC_ERR_STATE.
 */
godec_status godec_lingodec_init(godec_ctx** ctx, const godec_params* params, double lambda, const float* X,
                                 const float* F, int32_t d, void* stream);
/* n_iter alternations (W-step, S-step) from the current state; rel_err (host, nullable) of
   the last.  Synchronises the stream after every iteration. */
godec_status godec_lingodec_iterate(godec_ctx* ctx, int32_t n_iter, double* rel_err);
/* W (device, m x d float32 row-major) of the last iteration.  Synchronises the stream. */
godec_status godec_lingodec_get_W(godec_ctx* ctx, float* W);

/*
 * MSE training, the multi-label subspace ensemble (Sec. 4.2.1, eqs. ms, mssub, msinitial,
 * Algorithm 4): X (n samples x p features) = sum_i L^i + S, L^i nonzero only on the rows
 * Omega_i of the samples that carry label i, rank(L^i) <= r_i, card(S) <= K.  Block
 * coordinate descent from L^i = (D^{-1} X) restricted to Omega_i (D = labels per sample),
 * S = 0: for each label in turn, L^i = the q = 0 bilateral random projection of
 * (X - sum_{j != i} L^j - S) on Omega_i with the Gaussian test matrix of that step (on the
 * GPU through a q = 0 GoDec context over the gathered rows); then S = the K largest
 * entries of X - sum L^i (the S-step of Algorithm 1).
 *   X       : device n x ldx float32 (ldx*4 a multiple of 16), read only
 *   labels  : host n x k int32, row-major, nonzero = the sample carries the label
 *   ranks   : host k int32, 1 <= r_i <= min(|Omega_i|, p, r_stride)
 *   K       : cardinality of S;  iters : outer iterations (>= 1)
 *   A1s     : device float32, iters x k blocks of p x r_stride (row-major): the test
 *             matrix of label i in iteration t is the first r_i columns of block t k + i
 *   C       : device k x r_stride x p float32 (nullable): rows 0 .. r_i - 1 of block i are an
 *             orthonormal basis of label i's subspace (the row space of L^i), the rest 0
 *   Lsum    : device n x ldl float32 (nullable): sum_i L^i
 *   S_idx, S_val : device, S_cap entries (nullable): S as COO sorted by linear index;
 *             nnz (host, nullable) receives its size
 *   history : host, iters entries (nullable): ||X - sum L^i - S||_F^2 after each iteration
 * All device memory is allocated and freed inside the call; the call synchronises the
 * stream.  GODEC_ERR_ARG on invalid arguments or S_cap < nnz (results written otherwise).
 */
godec_status godec_mse_train(const float* X, int64_t n, int64_t p, int64_t ldx, const int32_t* labels, int32_t k,
                             const int32_t* ranks, int64_t K, int32_t iters, const float* A1s, int32_t r_stride,
                             float* C, float* Lsum, int64_t ldl, int64_t* S_idx, float* S_val, int64_t S_cap,
                             int64_t* nnz, double* history, void* stream);

/*
 * Batched form: count independent GoDec-BRP problems (Algorithm 1 on each) of uneven
 * m, n and r, advanced together.  One batch iteration is one launch of one CUDA graph
 * that holds an iteration of every problem as a parallel branch, all on the exact-
 * normaliser path of the chain (the graph is captured once, and again after a rank
 * drop).  Each branch's kernels are sized for a share of the SMs (its budget: the
 * stream-K grid of the products and the S-step's grids), so branches run side by side.
 * An autotuner picks the budgets by timing the batch graph of each candidate policy on
 * the problems themselves (two warm-up and three batch iterations each, then every
 * problem is reset):
 *   policy 0: every problem gets all SMs;
 *   policy k = 1..4: problem i gets max(4, min(#SMs, ceil(2^(k-1) #SMs m_i n_i / sum m n))).
 * Each problem's results equal those of a godec_init context run on its own, up to
 * float32 rounding (grid sizes change the order of the stream-K partial sums).
 *   count  : 1 <= count <= GODEC_BATCH_MAX
 *   params : host array of count godec_params (precision GODEC_PREC_FP32)
 *   X, A1  : host arrays of count device pointers, each as in godec_init (borrowed)
 *   flags  : GODEC_BATCH_NO_TUNE gives every problem all SMs without timing
 *   stream : the CUDA stream of every call on the batch (nullable)
 * Device memory: that of count godec_init contexts.  Errors: as godec_init, with the
 * failing problem's index in the message; on failure *out is NULL and nothing leaks.
 */
typedef struct godec_batch godec_batch;
#define GODEC_BATCH_MAX 4096
#define GODEC_BATCH_NO_TUNE 1
#define GODEC_BATCH_POLICIES 5
godec_status godec_batch_init(godec_batch** out, int32_t count, const godec_params* params,
                              const float* const* X, const float* const* A1, int32_t flags, void* stream);

/*
 * n_iter more iterations of every problem: n_iter launches of the batch graph, then a
 * problem whose iteration aborted in the graph (rank drop, candidate buffer growth,
 * rescale of X - S) is handled as godec_iterate would and finishes its iterations on
 * its own graphs.  A problem that converged or failed earlier sits out.  The stop
 * test is off (each problem's tol is not used here).  Synchronises the stream.
 */
godec_status godec_batch_iterate(godec_batch* b, int32_t n_iter);

/* Back to S = 0 for every problem (godec_reset on each). */
godec_status godec_batch_reset(godec_batch* b);

/*
 * The context of problem i (0 <= i < count), owned by the batch: use it with
 * godec_get_L, godec_get_S, godec_get_info, godec_residual and godec_iterate; never
 * pass it to godec_destroy.  NULL if i is out of range.
 */
godec_ctx* godec_batch_problem(godec_batch* b, int32_t i);

/*
 * The tuner's result: sm (host, count entries, nullable) the budget of each problem;
 * policy_ms (host, GODEC_BATCH_POLICIES entries, nullable) milliseconds per batch
 * iteration of each timed policy (0 when not timed); policy (host, nullable) the one
 * in use; recaptures (host, nullable) batch graphs captured since init, tuning included.
 */
godec_status godec_batch_tuning(godec_batch* b, int32_t* sm, double* policy_ms, int32_t* policy,
                                int32_t* recaptures);

void godec_batch_destroy(godec_batch* b);

/* Message of the last failed call on b (b NULL: of the last failed godec_batch_init). */
const char* godec_batch_last_error(godec_batch* b);

/*
 * The tuner's budget rule, host logic only (no device work): sm[i] (host, count entries)
 * receives the SMs policy gives problem i of shape m[i] x n[i] (host arrays) on a device
 * of nsm SMs: policy 0 -> nsm; policy k = 1..4 -> max(min(4, nsm), min(nsm,
 * ceil(2^(k-1) nsm m_i n_i / sum m n))).  GODEC_ERR_ARG on a bad argument.
 */
godec_status godec_batch_budgets(int32_t count, const int64_t* m, const int64_t* n, int32_t nsm, int32_t policy,
                                 int32_t* sm);

/*
 * Stream-K geometry of the tensor-core product over a rows x K operand on nsm SMs, host
 * logic only (no device work).  out (host, 6 entries) receives: row tiles of 128,
 * K-stages of 64 per tile, stages S = tiles x stages, CTAs G (all SMs, or four fewer
 * above 16, at most S; CTA c owns stages [c S / G, (c+1) S / G)), the most CTAs that
 * share one tile (partial slots per tile), and the most tiles one CTA's range touches
 * (completions it may owe).  GODEC_ERR_ARG on a bad argument.
 */
godec_status godec_tc_geometry(int64_t rows, int64_t K, int32_t nsm, int64_t* out);

#ifdef __cplusplus
}
#endif

#endif /* GODEC_H */
