/*
 * rpcholqr.h -- C ABI of the GB300 (sm_103a) implementation of rpCholesky-QR
 * (J. E. Garrison and I. C. F. Ipsen, "A randomized preconditioned Cholesky-QR algorithm",
 * arXiv 2406.11751).
 *
 * The library computes the thin QR factorisation A = Q R of a tall-skinny A (m x n, m >> n,
 * rank n; the problem statement of Section 1 and Section 2.1) with Algorithm alg_2
 * ("rpCholesky-QR", Section 4):
 *
 *   sample        A_s = S A            s rows of A drawn uniformly, independently and with
 *                                      replacement, scaled by sqrt(m/s) (Remark r_exp, Section 5;
 *                                      the smoothing transform F is not applied)
 *   factor        A_s = Q_s R_s        Householder QR of the s x n sample, R_s kept
 *   precondition  A_1 = A R_s^{-1}     m independent row solves (row-wise view of Section 2.1)
 *   Gram          G_1 = A_1^T A_1      fused with the preconditioning pass
 *   Cholesky      G_1 = R_1^T R_1      (the paper's R_2)
 *   solve         Q   = A_1 R_1^{-1}   second streaming pass, in place over A_1
 *   recover       R   = R_1 R_s
 *
 * Conventions shared by every entry point
 *   - Matrices are ROW-MAJOR FP64 (double) with a leading dimension (elements between the starts of
 *     consecutive rows) >= the number of columns.  n x n triangular factors are dense row-major n x n
 *     arrays with leading dimension n; the strictly lower part is written as 0.
 *   - "device" pointers must be CUDA device (or managed) memory of the plan's device; "host" pointers
 *     are ordinary host memory.  The caller owns every buffer it passes; the library never frees them.
 *   - Calls are asynchronous on `stream` (a cudaStream_t passed as void*, NULL = legacy default
 *     stream) unless stated otherwise.  The return value reports argument and launch errors only.
 *     Numerical outcomes are written to a device int32 pair info[2] = {status, pivot}: status is an
 *     rpcholqr_status, pivot the failing Cholesky pivot (0-based) for RPCHOLQR_ERR_NOT_SPD, else -1.
 *     Once a step writes a non-zero status, every later step of the same call returns at once and
 *     leaves its outputs unwritten.
 *   - Sampling is deterministic: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) keyed by
 *     (seed, stream_id), counter block k = (k, 0, 0, 0); sample j takes word j mod 4 of block j/4 and
 *     maps it to the row floor(word * m / 2^64).  Results are bit-reproducible for a fixed plan, shape
 *     and seed on one GPU model.
 *   - No entry point falls back to the host: every arithmetic step runs in this library's kernels.
 */
#ifndef RPCHOLQR_H
#define RPCHOLQR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RPCHOLQR_OK = 0,
    RPCHOLQR_ERR_ARG = 1,             /* invalid argument (shape, pointer, leading dimension)     */
    RPCHOLQR_ERR_NONFINITE = 2,       /* A holds a NaN or an infinity                             */
    RPCHOLQR_ERR_SINGULAR_SKETCH = 3, /* a diagonal of R_s is 0, subnormal or non-finite: the
                                         sample has rank < n (Lemma l_31 and Theorem t_prob need
                                         rank(A_s) = n)                                           */
    RPCHOLQR_ERR_NOT_SPD = 4,         /* Cholesky of G_1 met a pivot that is not > 0 (Theorem
                                         t_perturb2 assumes kappa(A_1)^2 gamma_2 < 1)             */
    RPCHOLQR_ERR_TIMEOUT = 5,         /* a bounded device-side wait gave up                       */
    RPCHOLQR_ERR_CUDA = 6,            /* a CUDA runtime call failed                               */
    RPCHOLQR_ERR_NOMEM = 7,           /* workspace allocation failed                              */
    RPCHOLQR_ERR_UNSUPPORTED = 8      /* the requested mode or shape is not built                 */
} rpcholqr_status;

typedef enum {
    RPCHOLQR_FP64 = 0,   /* every step in FP64 (FP64 tensor-core mma.sync m16n8k16 + DFMA)        */
    RPCHOLQR_SPLIT64 = 1, /* FP64-accurate split precision: sketch QR, Cholesky and the diagonal
                            blocks of the row solves in FP64; the Gram matrix, the off-diagonal
                            block update of the row solve (n > 64) and Q = A1 R1^{-1} (explicit
                            inverse of the well-conditioned R1) as Ozaki-split BF16 tensor-core
                            (tcgen05) products with exact FP32 group sums and int64 combination.
                            Q = A1 R1^{-1} takes that path only while ||R1||_F ||R1^{-1}||_F / n <= 2
                            (A1 well conditioned, as for incoherent or smoothed A); otherwise an FP64
                            row-wise substitution keeps the residual at the FP64 level (decided on
                            the device, see rpcholqr_plan_split_pass2_fp64).
                            Needs an extra max_m x n FP64 plan buffer for A1.                      */
    RPCHOLQR_FP32 = 2    /* single precision for FP32 data (A, Q, R float; rpcholqr_factor_f32 only):
                            the sample is widened to FP64, R_s (Householder) and R1 (Cholesky of
                            the Gram matrix, summed in FP64 from FP32 partials) are FP64; both
                            m-row passes run in FP32 on the FMA pipe.  Accuracy is that of FP32
                            (||Q^T Q - I|| of order 1e-6 for well-sampled A up to kappa ~ 1e5). */
} rpcholqr_mode;

/* Largest n a plan accepts (FP32 plans: 512).  Up to 128 columns the row passes keep a whole row panel
 * in shared memory; above, both modes run left-looking blocked solves over 64-column blocks. */
#define RPCHOLQR_MAX_N 2048

typedef struct rpcholqr_plan_s* rpcholqr_plan;

/* Create a plan for matrices up to max_m x max_n sampled with up to max_s rows, on `device`.
 * The plan owns its device workspace (sample, R_s, fragment tables, per-CTA Gram partials),
 * allocated here with cudaMalloc; *plan receives the handle.  autotune_json (nullable): a tuning table
 * written by rpcholqr_autotune -- its JSON text (starting with '{') or the path of its file; every call
 * on the plan then takes the launch parameters of the table entry of its mode and padded n nearest in
 * log2 m (no entry: the built-in rules).  A table that cannot be read or parsed is RPCHOLQR_ERR_ARG.
 * Requires 1 <= max_n <= RPCHOLQR_MAX_N (512 for RPCHOLQR_FP32), max_s >= max_n, max_m >= max_s.
 * Errors: RPCHOLQR_ERR_ARG, RPCHOLQR_ERR_UNSUPPORTED (mode), RPCHOLQR_ERR_NOMEM, RPCHOLQR_ERR_CUDA. */
rpcholqr_status rpcholqr_plan_create(rpcholqr_plan* plan, int device, rpcholqr_mode mode,
                                     int64_t max_m, int32_t max_n, int32_t max_s, const char* autotune_json);

/* Autotuner (no counterpart in the paper: launch parameters of this implementation).  For each shape
 * class c (host arrays m[c], n[c], s[c] within the plan's limits) it fills a synthetic m x n matrix
 * (uniform entries; any full-rank matrix serves), times rpcholqr_factor on it -- one warm-up and `reps`
 * timed calls, CUDA events -- for every candidate set of launch parameters, and keeps the fastest in the
 * plan's table under (mode, padded n, ceil(log2 m)):
 *   SPLIT64: the width of the first pass's FP64 diagonal-block solves (16 or 32 columns; the rest of
 *            the solve is split tensor-core updates) x the row ranges (split-K factor) of the Gram
 *            matrix (the built-in rule, one per SM over the output tiles, twice that);
 *   FP64, n > 128: the row ranges (split-K factor) of the wide Gram matrix (x1, x4 of one wave).
 * Other shapes are timed with the built-in rules and recorded as such.  out_json (nullable): file the
 * whole table is written to (the format rpcholqr_plan_create reads).  Synchronous; allocates and frees
 * the test matrices (cudaMalloc); the results of the timed calls are discarded.  Parameters change
 * rounding only (every candidate passes the same accuracy gates).  FP32 plans: ERR_UNSUPPORTED. */
rpcholqr_status rpcholqr_autotune(rpcholqr_plan plan, int32_t nclasses, const int64_t* m, const int32_t* n,
                                  const int32_t* s, int32_t reps, const char* out_json);

/* The plan's tuning table as JSON text (host): *length = its length in bytes (without the terminating
 * 0); with out != NULL, up to capacity - 1 bytes are copied to out and 0-terminated. */
rpcholqr_status rpcholqr_autotune_table(rpcholqr_plan plan, char* out, size_t capacity, size_t* length);

/* Host-only check of a tuning table (JSON text starting with '{', or a file path): *entries = the number
 * of entries; RPCHOLQR_ERR_ARG when it cannot be read or parsed. */
rpcholqr_status rpcholqr_autotune_parse(const char* json_or_path, int32_t* entries);

/* Plan options (rpcholqr_plan_set_option / rpcholqr_plan_get_option); each holds until changed. */
typedef enum {
    RPCHOLQR_OPT_SPIN_LIMIT = 0,    /* polls a device-side pipeline wait makes before it gives up and the
                                       call reports RPCHOLQR_ERR_TIMEOUT (default 2^24, 1 <= value <=
                                       2^40).  A kernel's final wait for its own tensor-core work, before
                                       it releases its tensor memory, always uses the default. */
    RPCHOLQR_OPT_SCALE_SAMPLE = 1,  /* 1 (default): the sample is scaled by sqrt(m/s) (Remark r_exp);
                                       0: unscaled.  R is the same in exact arithmetic either way. */
    RPCHOLQR_OPT_DETERMINISTIC = 2, /* 1 (default, the only value built): every reduction is a
                                       fixed-order sum, so results are bit-reproducible for a fixed plan
                                       shape and seed; 0 returns RPCHOLQR_ERR_UNSUPPORTED. */
    RPCHOLQR_OPT_BATCH_CAPACITY = 3, /* matrices rpcholqr_factor_batched can take without allocating:
                                       setting it allocates (cudaMalloc) the batched kernel's workspace
                                       now -- about (max_s + 5 np) np + 2 (np/8) 64 doubles per matrix,
                                       np = max_n rounded up to 16, plus its work list; 0 frees it.
                                       Default 0: the first batched call allocates for its count. */
    RPCHOLQR_OPT_IMAGE_ROWS = 4     /* SPLIT64 plans above 128 columns: rows of the stage images (the
                                       BF16 slices the wide passes stream, 16 bytes a value) kept at a
                                       time; the first pass and the Gram run chunk by chunk of that
                                       many rows, the second pass by chunks of at most 8 GiB of images.
                                       0 (default): every row when their images take at most a quarter
                                       of the device memory, else 8 GiB-sized chunks.  value > 0: that many
                                       rows (rounded up to 128).  Results differ only in rounding.
                                       Setting it synchronizes the device and reallocates the images
                                       (the new buffer before the old one is freed: RPCHOLQR_ERR_NOMEM
                                       leaves the plan as it was); get returns the rows in use.
                                       RPCHOLQR_ERR_UNSUPPORTED for other plans. */
} rpcholqr_option;

/* Set option `option` of the plan to `value` (host call; affects later calls).
 * Errors: RPCHOLQR_ERR_ARG (unknown option or value out of range), RPCHOLQR_ERR_UNSUPPORTED. */
rpcholqr_status rpcholqr_plan_set_option(rpcholqr_plan plan, int32_t option, int64_t value);

/* Read option `option` of the plan into *value (host). */
rpcholqr_status rpcholqr_plan_get_option(rpcholqr_plan plan, int32_t option, int64_t* value);

/* Free the plan and its workspace (synchronises the plan's device first).  NULL is accepted. */
rpcholqr_status rpcholqr_plan_destroy(rpcholqr_plan plan);

/* Bytes of device workspace a plan with these limits allocates at creation (host-only query): a plan of
 * `plan`'s mode on its device, or, with plan = NULL, an RPCHOLQR_FP64 plan on a 152-SM GPU.  Not
 * counted: the staging of rpcholqr_factor_host, smoothing buffers and the batch workspace, which are
 * allocated when first needed. */
rpcholqr_status rpcholqr_workspace_size(rpcholqr_plan plan, int64_t max_m, int32_t max_n, int32_t max_s,
                                        size_t* bytes);

/* rpCholesky-QR of A (Algorithm alg_2, Section 4).
 *   A    device, m x n row-major, lda >= n; read only.
 *   s    number of sampled rows, n <= s <= m (the paper's c; s = 3n is its recommendation).
 *   seed Philox key word 0 (key word 1 = stream_id = 0).
 *   Q    device, m x n row-major, ldq >= n; must not overlap A.  Holds A_1 between the passes.
 *   R    device, n x n row-major upper triangular (strict lower part set to 0).
 *   info device int32[2], see above; written by every call.
 * Requires 1 <= n <= plan max_n, s <= plan max_s, m <= plan max_m, m >= s >= n, and an FP64 or
 * SPLIT64 plan (ERR_ARG for an FP32 plan).
 * On a non-zero info status the contents of Q and R are unspecified. */
rpcholqr_status rpcholqr_factor(rpcholqr_plan plan, const double* A, int64_t m, int32_t n,
                                int64_t lda, int32_t s, uint64_t seed, double* Q, int64_t ldq,
                                double* R, int32_t* info, void* stream);

/* Batched rpCholesky-QR: Algorithm alg_2 for `count` independent matrices in ONE persistent kernel launch
 * (plus a one-CTA setup launch), the workload of block-Krylov / LOBPCG solvers that orthogonalise many
 * tall-skinny blocks of uneven size (Section 1).  Every per-matrix array is DEVICE-resident, of length
 * count: A[i] (device pointer, m[i] x n[i], lda[i]), s[i], seed[i] (Philox key word 0, stream_id 0),
 * Q[i] (device, m[i] x n[i], ldq[i]; holds A1 between the passes), R[i] (device, n[i] x n[i], ld n[i]);
 * info: device int32[2 count], {status, pivot} per matrix as for rpcholqr_factor.  A matrix whose shape
 * does not fit the plan (n[i] <= max_n, n[i] <= s[i] <= max_s, s[i] <= m[i] <= max_m, lda[i], ldq[i] >=
 * n[i], non-NULL pointers) gets RPCHOLQR_ERR_ARG in its info and is skipped; the others are factored.
 * Each matrix's Q, R and status are bit-identical to rpcholqr_factor on an FP64 plan with the same
 * limits, whatever else is in the batch.  The kernel's CTAs (one per SM) take work items -- per matrix:
 * sample + Householder R_s; pass-1 parts (row solve + Gram partial); Cholesky + R; pass-2 parts -- from
 * a device work list in order and wait (bounded by RPCHOLQR_OPT_SPIN_LIMIT polls, sleeping between
 * polls) for the items of the same matrix before them; a wait that gives up sets RPCHOLQR_ERR_TIMEOUT
 * in that matrix's info.  The call is asynchronous on `stream` and can be captured in a CUDA graph once
 * the plan's batch capacity covers count (RPCHOLQR_OPT_BATCH_CAPACITY; otherwise this call allocates).
 * Requires an RPCHOLQR_FP64 plan with max_n <= 128 and no smoothing (RPCHOLQR_ERR_UNSUPPORTED
 * otherwise); 1 <= count <= 65536.  Errors: ERR_ARG, ERR_UNSUPPORTED, ERR_NOMEM, ERR_CUDA. */
rpcholqr_status rpcholqr_factor_batched(rpcholqr_plan plan, int32_t count, const double* const* A, const int64_t* m,
                                        const int32_t* n, const int64_t* lda, const int32_t* s, const uint64_t* seed,
                                        double* const* Q, const int64_t* ldq, double* const* R, int32_t* info,
                                        void* stream);

/* FP32 factorisation (the FP32 mode; no counterpart in the paper, which works in double precision):
 * the same steps as rpcholqr_factor with A (m x n, lda), Q (m x n, ldq) and R (n x n, dense
 * row-major, ld n) as device float arrays.  The plan must be an RPCHOLQR_FP32 plan (ERR_ARG
 * otherwise).  Q receives A1 = A R_s^{-1} during the call and Q at its end.  info as in
 * rpcholqr_factor; an R_s or R1 diagonal that is not a normal float sets SINGULAR_SKETCH or NOT_SPD
 * with the pivot. */
rpcholqr_status rpcholqr_factor_f32(rpcholqr_plan plan, const float* A, int64_t m, int32_t n, int64_t lda,
                                    int32_t s, uint64_t seed, float* Q, int64_t ldq, float* R, int32_t* info,
                                    void* stream);

/* End-to-end variant of rpcholqr_factor on HOST buffers: copies A (host, m x n, lda) to a device
 * staging buffer the plan allocates on first use, factors it, copies Q (host, ldq) and R (host)
 * back, and returns only after the copies completed.  info_host (int32[2], host) receives the
 * numerical status.  Staging buffers are kept for later calls and freed with the plan.  With a
 * SPLIT64 plan, n <= 128, lda = ldq = n, no smoothing and m >= 512 the copies overlap the work: A
 * goes over in four row blocks on a second stream (created with the plan's first such call, with
 * pinned host buffers for the sample) while the sample, gathered on the host from the device-drawn
 * indices, is factored and pass 1 solves the blocks that have arrived; Q comes back block by block
 * behind pass 2.  The results equal rpcholqr_factor's.  A, Q should be pinned (page-locked) for the
 * copies to overlap. */
rpcholqr_status rpcholqr_factor_host(rpcholqr_plan plan, const double* A, int64_t m, int32_t n,
                                     int64_t lda, int32_t s, uint64_t seed, double* Q, int64_t ldq,
                                     double* R, int32_t* info_host, void* stream);

/* ---- individual steps (the same kernels rpcholqr_factor launches), for testing and composition ---- */

/* Sampling matrix S of Section 4: idx[j] (device int64[s]) = 0-based row of sample j. */
rpcholqr_status rpcholqr_sample_indices(uint64_t seed, uint64_t stream_id, int64_t m, int32_t s,
                                        int64_t* idx, void* stream);

/* Sample + Householder QR (steps 'sample' and 'factor'): Rs (device, n x n) receives R_s with a
 * positive diagonal (rows negated where Householder produced a negative diagonal).  info as above
 * (RPCHOLQR_ERR_NONFINITE for a non-finite sampled entry, RPCHOLQR_ERR_SINGULAR_SKETCH). */
rpcholqr_status rpcholqr_sketch_r(rpcholqr_plan plan, const double* A, int64_t m, int32_t n,
                                  int64_t lda, int32_t s, uint64_t seed, double* Rs, int32_t* info,
                                  void* stream);

/* Fused preconditioning pass (steps 'precondition' and 'Gram'): A1 = A Rs^{-1} (device, m x n,
 * ld1; may not overlap A) and G = A1^T A1 (device, n x n, full symmetric).  Rs: device n x n upper
 * triangular with a non-zero diagonal.  Sets RPCHOLQR_ERR_NONFINITE if A holds a NaN/Inf. */
rpcholqr_status rpcholqr_precondition_gram(rpcholqr_plan plan, const double* A, int64_t m,
                                           int32_t n, int64_t lda, const double* Rs, double* A1,
                                           int64_t ld1, double* G, int32_t* info, void* stream);

/* Cholesky (step 'Cholesky'): G = R1^T R1 for device n x n symmetric G; R1 device n x n upper.
 * RPCHOLQR_ERR_NOT_SPD with the pivot index when a pivot is not > 0. */
rpcholqr_status rpcholqr_cholesky(rpcholqr_plan plan, const double* G, int32_t n, double* R1,
                                  int32_t* info, void* stream);

/* Row-wise triangular solve (step 'solve'): Y = X T^{-1}, T device n x n upper triangular with a
 * non-zero diagonal, X and Y device m x n (ldx, ldy); X == Y (same ld) solves in place, any other
 * overlap is an error of the caller.  m <= plan max_m, n <= plan max_n. */
rpcholqr_status rpcholqr_solve_rows(rpcholqr_plan plan, const double* X, int64_t m, int32_t n,
                                    int64_t ldx, const double* T, double* Y, int64_t ldy,
                                    int32_t* info, void* stream);

/* R = R1 Rs for device n x n upper-triangular R1, Rs (step 'recover'); R device n x n. */
rpcholqr_status rpcholqr_triu_mul(const double* R1, const double* Rs, int32_t n, double* R,
                                  void* stream);

/* Split-precision FP64 product C = X Y on the BF16 tensor cores (the kernel SPLIT64 uses):
 * X device m x K (ldx), Y device K x N (ldy), C device m x N (ldc; must not overlap X), K, N <= plan
 * max_n; each entry carries an absolute error below ~2^-53 * 2^(Ex+Ey) (Ex, Ey: power-of-two bounds
 * of row i of X and column j of Y).  The plan must be a SPLIT64 plan.  info as above (RPCHOLQR_ERR_TIMEOUT if a bounded
 * tensor-core wait gave up). */
rpcholqr_status rpcholqr_ozaki_gemm(rpcholqr_plan plan, const double* X, int64_t m, int32_t K, int64_t ldx,
                                    const double* Y, int32_t N, int64_t ldy, double* C, int64_t ldc,
                                    int32_t* info, void* stream);

/* Split-precision update C = B - X Y (the off-diagonal block update of the blocked row solve,
 * Section 4's A1 = A Rs^{-1} by column blocks): the product as rpcholqr_ozaki_gemm, subtracted from B
 * in FP64 (B device m x N, ldb; C device m x N, ldc; C may equal B, must not overlap X).  K <= 32 runs
 * the update kernel of SPLIT64's first pass, larger K the windowed product in subtract form.  Same
 * error bound per entry as rpcholqr_ozaki_gemm plus the rounding of the subtraction.  SPLIT64 plan. */
rpcholqr_status rpcholqr_ozaki_update(rpcholqr_plan plan, const double* X, int64_t m, int32_t K, int64_t ldx,
                                      const double* Y, int32_t N, int64_t ldy, const double* B, int64_t ldb,
                                      double* C, int64_t ldc, int32_t* info, void* stream);

/* Split-precision Gram matrix G = X^T X (device n x n, full) of X (device m x n, ldx), the kernel
 * SPLIT64 uses for G1; error per entry below ~2^-53 * 2^(Ep+Eq) * rows (Ep: power-of-two bound of
 * column p).  SPLIT64 plan, m <= plan max_m. */
rpcholqr_status rpcholqr_ozaki_gram(rpcholqr_plan plan, const double* X, int64_t m, int32_t n, int64_t ldx,
                                    double* G, int32_t* info, void* stream);

/* Basic Cholesky-QR (Algorithm alg_0, Section 2.1): G = A^T A, G = R^T R, Q = A R^{-1}, all in FP64
 * with the same kernels as rpcholqr_factor (preconditioner = identity).  Arguments as for
 * rpcholqr_factor without s/seed.  Breaks down (RPCHOLQR_ERR_NOT_SPD) when kappa(A)^2 u >~ 1. */
rpcholqr_status rpcholqr_cholqr(rpcholqr_plan plan, const double* A, int64_t m, int32_t n, int64_t lda,
                                double* Q, int64_t ldq, double* R, int32_t* info, void* stream);

/* Cholesky-QR2 (Yamamoto et al., the comparison method of Section 5.3): Cholesky-QR of A, then of the
 * first Q; R = R_b R_a.  The breakdown reference for numerically singular inputs. */
rpcholqr_status rpcholqr_cholqr2(rpcholqr_plan plan, const double* A, int64_t m, int32_t n, int64_t lda,
                                 double* Q, int64_t ldq, double* R, int32_t* info, void* stream);

/* FP64 tensor-pipe throughput probe: runs `iters` chains of dependent m16n8k16 FP64 mma on every
 * SM and writes the sustained FLOP/s to *flops_per_s (host).  Synchronous.  Used to report the
 * FP64 roofline denominator measured on the running GPU. */
rpcholqr_status rpcholqr_probe_fp64_mma(int device, int32_t iters, double* flops_per_s);

/* Allocation-free variant of rpcholqr_precondition_gram (same arguments without the plan, same
 * results on the same GPU).  The paper has no counterpart: this exists for callers that may not
 * allocate device memory once running -- code living inside a framework whose allocator owns the
 * device memory, or services that reserve memory at start-up and forbid cudaMalloc/cudaFree later
 * (both synchronise the device and can fail under pressure).  Such callers cannot create a plan.
 * Scratch comes from one fixed __device__ array of about 5.3 MB inside the library, which every
 * GPU that loads the library holds until the process exits; it fits n <= 64 (larger n returns
 * RPCHOLQR_ERR_UNSUPPORTED; any m is accepted).  The call allocates nothing and calls no
 * allocating library routine.  Runs on the current device; `stream` must belong to it
 * (RPCHOLQR_ERR_ARG otherwise).  The first call on each device looks up
 * the array's device address (cudaGetSymbolAddress) with that device current, so make that first
 * call before any stream capture.  Every call shares the array and leaves its contents behind:
 * calls whose kernels overlap on the GPU (other streams, other threads) race on it and must be
 * serialised by the caller. */
rpcholqr_status rpcholqr_precondition_gram_noalloc(const double* A, int64_t m, int32_t n, int64_t lda,
                                                   const double* Rs, double* A1, int64_t ld1,
                                                   double* G, int32_t* info, void* stream);

/* Shifted Cholesky-QR3 (Fukaya, Kannan, Nakatsukasa, Yamamoto, Yanagisawa 2020; the remedy for
 * Cholesky-QR2's breakdown cited in Section 1): G = A^T A + sigma I, sigma = 11 (m n + n (n + 1)) u
 * trace(A^T A) (u = 2^-53), R_1 = chol(G), Q_1 = A R_1^{-1}, then Cholesky-QR2 of Q_1; R = R_3 R_2 R_1.
 * FP64 kernels; arguments and errors as rpcholqr_cholqr2.  Works while sqrt(sigma) kappa(A) stays
 * below ~u^-1/2 (about kappa(A) < 1e13 at m = 3000, n = 40); beyond, NOT_SPD. */
rpcholqr_status rpcholqr_scholqr3(rpcholqr_plan plan, const double* A, int64_t m, int32_t n, int64_t lda,
                                  double* Q, int64_t ldq, double* R, int32_t* info, void* stream);

/* SPLIT64 plans: *used_fp64 = 1 when the last factorisation on this plan computed Q = A1 R1^{-1}
 * by FP64 substitution (A1 judged ill conditioned), 0 when by the split tensor-core product.
 * Synchronises with the device. */
rpcholqr_status rpcholqr_plan_split_pass2_fp64(rpcholqr_plan plan, int32_t* used_fp64);

/* ---- smoothing F = F_T D before sampling ----
 * Algorithm alg_2 samples rows of F A, F = F_T D (the Blendenpik remark of Section 4; Remark r_exp).
 * kind 0 (the default): F = I, rows of A are sampled directly.  kind 1: F_T is the orthogonal
 * Walsh-Hadamard transform of order m' = 2^ceil(log2 m) (natural order); kind 2: the orthonormal
 * DCT-II of order m' (MATLAB's dct, which Remark r_exp uses).  Both act on A padded with zero rows;
 * D_ii = -1 when bit 63 of Philox word (i mod 4) of block i/4 under key (seed, 1) is set; the s sampled
 * rows are drawn from [0, m') and scaled by sqrt(m'/s).  Needed for coherent A (rows of A carrying
 * most of its column space, e.g. [R_A; 0]), whose unsmoothed sample is singular.  The Walsh-Hadamard
 * rows restricted to the first n columns repeat with period 2^ceil(log2 n), so on such inputs it needs
 * s >~ n ln n samples; the cosine rows are all distinct.  Costs two extra passes over an m' x n buffer
 * the plan allocates here (8 m' pad8(max_n) bytes for m' of max_m, twice that for the cosine);
 * m' <= 2^25.  Applies to rpcholqr_factor, rpcholqr_factor_f32, rpcholqr_factor_host and
 * rpcholqr_sketch_r on this plan.  Errors: ARG (kind), UNSUPPORTED (max_m > 2^25), NOMEM. */
rpcholqr_status rpcholqr_plan_set_smoothing(rpcholqr_plan plan, int32_t kind);

/* The smoothed sample alone (the plan's kind): As (device, s x n row-major, ld ld_as) =
 * sqrt(m'/s) (F A)(idx, :).
 * The plan must have smoothing enabled (ERR_ARG otherwise).  info as in rpcholqr_factor
 * (NONFINITE for any non-finite entry of A: every row enters the sample). */
rpcholqr_status rpcholqr_smoothed_sample(rpcholqr_plan plan, const double* A, int64_t m, int32_t n, int64_t lda,
                                         int32_t s, uint64_t seed, double* As, int64_t ld_as, int32_t* info,
                                         void* stream);

/* ---- row-sharded factorisation (A split by contiguous row blocks over processes) ----
 * Algorithm alg_2 with A partitioned by rows: both passes and the Gram partials are row-local, and
 * the processes exchange only the s x n sample (before the sketch QR) and the n x n Gram partials
 * (before the Cholesky factorisation).  The exchanges themselves belong to the caller's
 * communication layer; these calls are the non-local steps around them.  The local passes are
 * rpcholqr_precondition_gram, rpcholqr_cholesky, rpcholqr_solve_rows and rpcholqr_triu_mul. */

/* The rows of the global sample owned by this block: As (device, s x n row-major, ld ld_as) row j =
 * sqrt(m/s) A[idx_j - row_offset, :] when row_offset <= idx_j < row_offset + m_local (idx_j from
 * the Philox stream of the whole m x n matrix, stream_id 0), else zeros.  Summing the blocks'
 * As over all processes gives exactly the sample rpcholqr_factor draws.  A_local: device, m_local x n
 * (lda), may be NULL when m_local = 0.  info: device int32[2] (NONFINITE for a non-finite owned
 * sample entry). */
rpcholqr_status rpcholqr_gather_owned_rows(const double* A_local, int64_t m_local, int32_t n, int64_t lda,
                                           int64_t row_offset, int64_t m, int32_t s, uint64_t seed, double* As,
                                           int64_t ld_as, int32_t* info, void* stream);

/* R_s of a given s x n sample (device, row-major, ld ld_as): the Householder step of
 * rpcholqr_sketch_r on an already gathered and scaled sample.  Rs: device n x n. */
rpcholqr_status rpcholqr_sketch_r_from_sample(rpcholqr_plan plan, const double* As, int32_t s, int32_t n,
                                              int64_t ld_as, double* Rs, int32_t* info, void* stream);

/* G (device, n x n) = sum of parts[k] (device, nparts x n x n, contiguous) in the order k = 0, 1, ...
 * (the same bits for the same parts on every process). */
rpcholqr_status rpcholqr_sum_partials(const double* parts, int32_t nparts, int32_t n, double* G, void* stream);

/* ---- batches of independent matrices ----
 * A batch object owns `slots` independent plans (each with its own workspace and CUDA stream).  The
 * matrices of a batch call are dealt round-robin to the slots, so small matrices -- whose row passes
 * fill only part of the GPU -- run concurrently; the caller's stream forks to the slot streams and
 * joins them again (the call stays asynchronous on `stream`).  The sequence can be captured once into
 * a CUDA graph and replayed as one launch (the workload of block-Krylov / LOBPCG solvers, which
 * orthogonalise many tall-skinny blocks).  All per-matrix arrays below are HOST arrays of length count;
 * the pointed-to matrices are device memory; info is a DEVICE int32 array of 2*count entries
 * ({status, pivot} per matrix, see rpcholqr_factor).  Every matrix must fit the batch limits. */
typedef struct rpcholqr_batch_s* rpcholqr_batch;

rpcholqr_status rpcholqr_batch_create(rpcholqr_batch* batch, int device, rpcholqr_mode mode, int64_t max_m,
                                      int32_t max_n, int32_t max_s, int32_t slots);
rpcholqr_status rpcholqr_batch_destroy(rpcholqr_batch batch);

/* Factor count matrices (rpcholqr_factor semantics each, Philox stream_id = 0, key = seed[i]). */
rpcholqr_status rpcholqr_batch_factor(rpcholqr_batch batch, int32_t count, const double* const* A,
                                        const int64_t* m, const int32_t* n, const int64_t* lda,
                                        const int32_t* s, const uint64_t* seed, double* const* Q,
                                        const int64_t* ldq, double* const* R, int32_t* info, void* stream);

/* Capture the same work as rpcholqr_batch_factor into a CUDA graph held by the batch (replacing a
 * previous one); nothing runs until rpcholqr_batch_replay.  The buffers must stay valid while the
 * graph is replayed.  Uses the slot count the batch currently has. */
rpcholqr_status rpcholqr_batch_capture(rpcholqr_batch batch, int32_t count, const double* const* A,
                                       const int64_t* m, const int32_t* n, const int64_t* lda,
                                       const int32_t* s, const uint64_t* seed, double* const* Q,
                                       const int64_t* ldq, double* const* R, int32_t* info, void* stream);

/* Launch the captured graph on `stream` (RPCHOLQR_ERR_ARG if none was captured). */
rpcholqr_status rpcholqr_batch_replay(rpcholqr_batch batch, void* stream);

/* Autotuner: times rpcholqr_batch_factor on these matrices with 1, 2, 4, ... up to the batch's slot
 * count of concurrent slots (one warm-up and `reps` timed runs each, synchronous), keeps the fastest
 * as the batch's active slot count and returns it in *best_slots (host) and the per-run time in
 * *best_ms (host). */
rpcholqr_status rpcholqr_batch_autotune(rpcholqr_batch batch, int32_t count, const double* const* A,
                                        const int64_t* m, const int32_t* n, const int64_t* lda,
                                        const int32_t* s, const uint64_t* seed, double* const* Q,
                                        const int64_t* ldq, double* const* R, int32_t* info, int32_t reps,
                                        int32_t* best_slots, float* best_ms, void* stream);

/* ---- per-phase timing (CUDA events on the call's stream) ----
 * Phases of one rpcholqr_factor call, in launch order. */
enum {
    RPCHOLQR_PHASE_SAMPLE = 0,    /* Philox indices + gather/scale of the s rows           */
    RPCHOLQR_PHASE_SKETCH_QR,     /* Householder QR of the sample                           */
    RPCHOLQR_PHASE_PREP_RS,       /* fragment tables of R_s                                 */
    RPCHOLQR_PHASE_PASS1,         /* FP64: fused A1 = A R_s^{-1} + Gram partials;
                                     SPLIT64: row solve of the first (<= 64-column) block       */
    RPCHOLQR_PHASE_PASS1_UPDATE,  /* SPLIT64, n > 64: tensor-core off-diagonal block update     */
    RPCHOLQR_PHASE_PASS1_SOLVE2,  /* SPLIT64, n > 64: row solve of the second block            */
    RPCHOLQR_PHASE_GRAM_REDUCE,   /* FP64: fixed-order sum of the Gram partials;
                                     SPLIT64: tensor-core Gram matrix and its sum              */
    RPCHOLQR_PHASE_CHOLESKY,      /* G1 = R1^T R1                                           */
    RPCHOLQR_PHASE_PREP_R1,       /* FP64: fragment tables of R1; SPLIT64: R1^{-1}          */
    RPCHOLQR_PHASE_PASS2,         /* Q = A1 R1^{-1} (FP64: in place; SPLIT64: tensor cores) */
    RPCHOLQR_PHASE_RECOVER_R,     /* R = R1 R_s                                             */
    RPCHOLQR_NUM_PHASES
};

/* Kernel classes of rpcholqr_plan_collect_kernel_timing. */
enum {
    RPCHOLQR_KERNEL_ROWPASS = 0,     /* FP64 row passes: fused pass 1, pass 2, diagonal-block solves       */
    RPCHOLQR_KERNEL_SPLIT_UPDATE,    /* split C = B - X Y with K <= 32 (k_ozaki_update)                    */
    RPCHOLQR_KERNEL_SPLIT_GEMM_SUB,  /* split C = B - X Y, K > 32 (wide pass-1 block updates)              */
    RPCHOLQR_KERNEL_SPLIT_GEMM,      /* split C = X Y (pass 2, Q = A1 R1^{-1})                              */
    RPCHOLQR_KERNEL_SPLIT_GRAM,      /* split Gram matrix                                                   */
    RPCHOLQR_KERNEL_FP64_GEMM,       /* FP64 block updates of the wide solves                               */
    RPCHOLQR_KERNEL_FP64_SYRK,       /* FP64 Gram matrix of wide panels                                     */
    RPCHOLQR_KERNEL_SKETCH_QR,       /* Householder QR of the sample                                        */
    RPCHOLQR_KERNEL_CHOLESKY,        /* Cholesky factorisation of G1                                        */
    RPCHOLQR_NUM_KERNEL_CLASSES
};

/* Enable (max_calls > 0, at most 4096) or disable (0) event timing of the next rpcholqr_factor calls
 * on this plan: events are recorded on the call's stream around every phase, and around every launch
 * of the kernel classes above, for up to max_calls calls (later calls are not timed).  Creating the
 * events happens here, not in rpcholqr_factor. */
rpcholqr_status rpcholqr_plan_enable_timing(rpcholqr_plan plan, int32_t max_calls);

/* Wait for the recorded events and report, summed over the timed calls since the last collect:
 * ms_per_phase[RPCHOLQR_NUM_PHASES] (host), *calls (host) = number of timed calls, and *launches
 * (host) = kernels this plan launched since the last collect (timed or not).  Resets the counts. */
rpcholqr_status rpcholqr_plan_collect_timing(rpcholqr_plan plan, float* ms_per_phase, int32_t* calls,
                                             int64_t* launches);

/* Per kernel class, summed over the timed calls since the last rpcholqr_plan_collect_timing (call this
 * one first: that call resets the count): ms_per_class[RPCHOLQR_NUM_KERNEL_CLASSES] (host) = the classes'
 * launch durations (CUDA events around each launch, on the call's stream), launches_per_class (host)
 * and flops_per_class (host) = the launches' algorithmic FP64 flops (row solve of b columns: m b^2,
 * fused with the Gram: 2 m n^2; product: 2 m K N, with an upper-triangular right factor
 * m sum_j 2 min(j + 1, K); Gram: m n^2; Householder: 2 s n^2 - 2 n^3 / 3; Cholesky: n^3 / 3).  Any
 * pointer may be NULL.  Synchronises with the recorded events. */
rpcholqr_status rpcholqr_plan_collect_kernel_timing(rpcholqr_plan plan, float* ms_per_class,
                                                    int64_t* launches_per_class, double* flops_per_class);

/* Human-readable name of a status code (static string). */
const char* rpcholqr_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* RPCHOLQR_H */
