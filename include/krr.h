/*
 * krr.h -- C ABI of the GB300 kernel ridge regression library (libkrr.so).
 *
 * The library runs the three phases of the paper's KRR driver (Alg. 1) on one
 * GPU:  Build (Alg. 2 with the Gaussian kernel of Alg. 5), Associate (Alg. 3:
 * factorise K + lambda I, solve for the weights) and Predict (Alg. 4).
 *
 * Conventions for every call:
 *  - Every call returns a krr_status; nothing throws across this boundary.
 *    On failure krr_last_error() returns a message for the context.
 *  - Matrices are row-major with an explicit leading dimension (elements).
 *    Sizes and leading dimensions are int64_t.
 *  - Pointer arguments may point to device memory or to host memory (pageable
 *    or pinned); the library tells them apart with cudaPointerGetAttributes
 *    and stages host buffers through its own device buffers.  Caller buffers
 *    are only borrowed for the duration of the call.
 *  - The context owns every internal buffer (packed genotypes, norms, kernel
 *    tiles, factor tiles, precision map) and frees them in krr_destroy().
 *  - Work is issued on the stream given to krr_create().  A call that returns
 *    host-visible results (info structs, host output buffers) synchronises
 *    that stream before it returns.  krr_factor() with options.lookahead also
 *    uses a second stream of the context's own (made on first use); every
 *    piece of work on it is joined back into the context's stream by an
 *    event before the call returns, so ordering on the caller's stream is
 *    unchanged.
 *  - A context is not thread safe; use one context per host thread.
 *
 * Notation: N training patients, M SNPs, P phenotypes, N_t held-out patients,
 * b tile edge, NT = ceil(N / b) tiles per side.
 */
#ifndef KRR_H
#define KRR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum krr_status {
    KRR_OK = 0,
    KRR_EINVAL = 1,   /* bad argument: shape, leading dimension, gamma <= 0, NaN lambda */
    KRR_ENOMEM = 2,   /* a device or pinned-host allocation failed */
    KRR_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
    KRR_ENOTPD = 4,   /* a pivot of the Cholesky factorisation was not positive */
    KRR_ENOCONV = 5,  /* iterative refinement did not reach the requested residual */
    KRR_ETIMEOUT = 6, /* a bounded device-side wait ran out (see krr_set_wait_budget) */
    KRR_ESTATE = 7    /* calls out of order (e.g. solve before factor) */
} krr_status;

typedef enum krr_mode {
    /* Tensor-core path: exact distances on FP8 (E4M3) operands with FP32
     * accumulation, adaptive per-tile precision of the factor (FP32 / FP16 /
     * E4M3), FP16 tensor-core trailing updates, refinement to FP32 accuracy. */
    KRR_MODE_MIXED = 0,
    /* Plain FP32 on CUDA cores for every step: the comparison path. */
    KRR_MODE_FP32 = 1
} krr_mode;

/* Tile precisions reported by krr_get_precision_map(). */
enum { KRR_PREC_FP64 = 0, KRR_PREC_FP32 = 1, KRR_PREC_FP16 = 2, KRR_PREC_E4M3 = 3 };

/* Adaptive-precision rules (krr_options.prec_rule) for an off-diagonal factor
 * tile (i, k), stored at the lowest unit roundoff u of {E4M3 2^-4, FP16
 * 2^-11} the rule admits, else at FP32 accuracy:
 *   KRR_RULE_LAMBDA: u max|L_ik| max|L_kk| <= eps * lambda -- the rounding of
 *     L_ik perturbs L L^T by about u |L_ik| |L_kk|, which stays below the
 *     smallest eigenvalue K + lambda I can have (default);
 *   KRR_RULE_KNORM: u ||K_ik||_F <= eps ||K||_F / NT -- the Frobenius-norm
 *     rule on the tiles of K of the adaptive-precision Cholesky the paper
 *     cites (Sec. IV-C, "Precision Heatmaps"), with ||K_ik||_F from the
 *     build. */
enum { KRR_RULE_LAMBDA = 0, KRR_RULE_KNORM = 1 };

/* Kernel functions of Alg. 5 (krr_options.kernel):
 *   KRR_KERNEL_GAUSSIAN: K_ij = exp(-gamma ||g_i - g_j||^2) (default);
 *   KRR_KERNEL_IBS: identity by state, K_ij = (g_i ~ g_j) / M with
 *     (g_i ~ g_j) = sum_k (2 - |g_ik - g_jk|) the number of alleles the two
 *     patients share at the M loci (K_ii = 2; gamma is not used).  It is
 *     computed on the same integer-exact tensor-core Gram machinery: each
 *     genotype becomes the two indicators [g >= 1], [g >= 2], whose squared
 *     Euclidean distance is the L1 distance |g_i - g_j|_1, and
 *     (g_i ~ g_j) = 2M - |g_i - g_j|_1.  krr_get_distances() then returns the
 *     L1 distances.  m <= 2^21. */
enum { KRR_KERNEL_GAUSSIAN = 0, KRR_KERNEL_IBS = 1 };

typedef struct krr_options {
    int64_t tile;            /* b: tile edge, a power of two in [256, 4096] (default 1024) */
    int32_t mode;            /* krr_mode (default KRR_MODE_MIXED) */
    int32_t allow_fp8;       /* 1: E4M3 allowed for factor tiles (default 1) */
    double eps;              /* adaptive-precision threshold of prec_rule (default 6e-4) */
    double ir_tol;           /* refinement stops at ||R||_F / ||Y||_F <= ir_tol (default 1e-7) */
    int32_t ir_max;          /* maximum refinement iterations (default 30; 0 = none) */
    int32_t diag_fp64;       /* 1: diagonal-tile Cholesky in FP64, 0: FP32 (default 0) */
    int64_t wait_budget_ns;  /* limit of every bounded device wait (default 2e9) */
    int32_t prec_rule;       /* KRR_RULE_LAMBDA (default) or KRR_RULE_KNORM; eps is the
                                threshold of either rule */
    int32_t kernel;          /* KRR_KERNEL_GAUSSIAN (default) or KRR_KERNEL_IBS */
    int32_t lookahead;       /* 1: the diagonal step of column k + 1 overlaps the trailing
                                update of step k on a second stream (mixed mode, FP32
                                diagonal step; default 1), 0: strictly in sequence */
    int32_t reserved;        /* must be 0 */
} krr_options;

/* Per-call reports; valid when the call returns. */
typedef struct krr_factor_info {
    int64_t nt;              /* tiles per side */
    int64_t tiles_fp32;      /* off-diagonal factor tiles stored FP32 */
    int64_t tiles_fp16;      /* ... stored FP16 */
    int64_t tiles_e4m3;      /* ... stored E4M3 */
    int64_t factor_bytes;    /* bytes of the stored off-diagonal factor tiles */
    int64_t bad_tile;        /* KRR_ENOTPD: diagonal tile of the first bad pivot, else -1 */
    int64_t bad_column;      /* KRR_ENOTPD: global column of the first bad pivot, else -1 */
    double min_pivot;        /* smallest diagonal entry of L */
} krr_factor_info;

typedef struct krr_solve_info {
    int32_t iterations;      /* refinement iterations taken */
    int32_t converged;       /* 1: ||R||_F / ||Y||_F <= ir_tol; 2: refinement stopped at the
                                attainable floor (a step that did not halve the residual);
                                0: no refinement or not converged */
    double rel_residual;     /* final ||Y - (K + lambda I) A||_F / ||Y||_F */
    double history[32];      /* relative residual after the first solve and each iteration */
} krr_solve_info;

typedef struct krr_ctx krr_ctx;

/* Fills *opt with the defaults listed above. */
void krr_default_options(krr_options *opt);

/*
 * Creates a context bound to the current CUDA device and to `stream`
 * (a cudaStream_t; NULL = the legacy default stream).  opt may be NULL for
 * the defaults.  Returns KRR_EINVAL for a tile edge that is not a power of
 * two in [256, 4096] or an unknown mode.
 */
krr_status krr_create(krr_ctx **out, const krr_options *opt, void *stream);

/*
 * Phase 1, Build (Alg. 2 with the Gaussian kernel of Alg. 5, distance form of
 * Sec. IV-B): K_ij = exp(-gamma * ||g_i - g_j||^2) over the lower-triangle
 * tiles of K (i >= j tile-wise; diagonal tiles in full).
 *   G     : n x m int8 genotypes, row-major with leading dimension ldg >= m,
 *           values in {0, 1, 2} (other values give undefined results), host
 *           or device.  Copied and packed; the caller may free it afterwards.
 *   gamma : kernel bandwidth, > 0 and finite.
 * Squared distances are exact integers (m <= 2^22).  Rows past n up to the
 * tile multiple are padding with K = identity.
 * Errors: KRR_EINVAL (n < 1, m < 1, m > 2^22, ldg < m, bad gamma), KRR_ENOMEM,
 * KRR_ECUDA.  Invalidates any earlier factor.
 */
krr_status krr_build_kernel(krr_ctx *ctx, const int8_t *G, int64_t n, int64_t m, int64_t ldg,
                            double gamma);

/*
 * Build with confounders (Sec. IV-B, distance section: squared distances of
 * the real-valued confounder columns -- age, sex, principal components, ...
 * -- are accumulated in floating point and added to the integer genotype
 * distances before the exponential of the Gaussian kernel):
 *   K_ij = exp(-gamma (||g_i - g_j||^2 + ||c_i - c_j||^2)).
 *   C  : n x nc FP32 confounders, leading dimension ldc >= nc, host or device;
 *        0 <= nc <= 16 (nc = 0 is krr_build_kernel).
 * The confounder distance is summed term by term in FP32 in the same
 * epilogue that forms the genotype distance (no N x N buffer).  Predict on
 * such a context needs the held-out rows' confounders: krr_predict_conf().
 * Gaussian kernel only; krr_grad_hyper() and krr_predict_noalloc() reject
 * a context with confounders.
 * Errors: as krr_build_kernel, and KRR_EINVAL for a bad nc, ldc or kernel.
 */
krr_status krr_build_kernel_conf(krr_ctx *ctx, const int8_t *G, int64_t n, int64_t m, int64_t ldg,
                                 const float *C, int64_t nc, int64_t ldc, double gamma);

/*
 * Phase 2a (Alg. 3, Factorize): tile Cholesky L L^T = K + lambda I.
 * Diagonal tiles are factorised in FP32 or FP64 (options.diag_fp64); each
 * off-diagonal factor tile is stored in the lowest precision the adaptive
 * rule allows (mixed mode) or in FP32 (fp32 mode).  K itself is kept for the
 * refinement residual.
 *   lambda : regularisation, finite (lambda >= 0).
 *   info   : optional report (may be NULL).
 * Errors: KRR_ESTATE (no kernel built), KRR_EINVAL, KRR_ENOTPD (info gives
 * the tile and column), KRR_ECUDA.
 */
krr_status krr_factor(krr_ctx *ctx, double lambda, krr_factor_info *info);

/*
 * Phase 2b (Alg. 3, Solve): A = (K + lambda I)^-1 Y for p right-hand sides by
 * forward and backward substitution with the factor, followed by iterative
 * refinement (residual accumulated in FP64 against the FP32 kernel) in mixed
 * mode.  The factor is reused across calls, so many phenotype sets can be
 * solved against one factorisation.
 *   Y : n x p FP32, leading dimension ldy >= p, host or device (read only).
 *   A : n x p FP32 output, leading dimension lda >= p, host or device.
 * Refinement stops when ||R||_F / ||Y||_F <= ir_tol, when a step fails to
 * halve it, or when a step makes it worse (that step is undone): the floor set
 * by FP32 storage of K and A.  A holds the best iterate.
 * Errors: KRR_ESTATE (no factor), KRR_EINVAL, KRR_ENOCONV (non-finite
 * residual, or ir_max iterations without reaching the tolerance or the
 * floor), KRR_ECUDA.
 */
krr_status krr_solve(krr_ctx *ctx, const float *Y, int64_t p, int64_t ldy, float *A, int64_t lda,
                     krr_solve_info *info);

/*
 * Phase 3 (Alg. 4, Predict): Yt = K_test A with K_test = Build(gamma, T, G),
 * the n_test x n test-by-training kernel, never stored: each distance tile is
 * exponentiated and multiplied by the matching rows of A in one pass, and
 * the per-tile partial products are summed in a fixed order.
 *   T  : n_test x m int8 genotypes, leading dimension ldt >= m, host or device.
 *   A  : n x p FP32 weights (from krr_solve), leading dimension lda >= p.
 *   Yt : n_test x p FP32 output, leading dimension ldyt >= p.
 * Errors: KRR_ESTATE (no kernel built), KRR_EINVAL, KRR_ENOMEM, KRR_ECUDA.
 */
krr_status krr_predict(krr_ctx *ctx, const int8_t *T, int64_t n_test, int64_t ldt, const float *A,
                       int64_t lda, int64_t p, float *Yt, int64_t ldyt);

/*
 * Predict (Alg. 4) on a kernel built with confounders: K_test from the
 * held-out genotypes T and their confounders Ct (n_test x nc FP32, leading
 * dimension ldct >= nc, host or device) against the training rows' genotypes
 * and confounders.  Other arguments and errors as krr_predict(); KRR_EINVAL
 * when the kernel has no confounders.
 */
krr_status krr_predict_conf(krr_ctx *ctx, const int8_t *T, int64_t n_test, int64_t ldt, const float *Ct,
                            int64_t ldct, const float *A, int64_t lda, int64_t p, float *Yt, int64_t ldyt);

/*
 * Ridge regression (Sec. IV-A, Eq. 2): beta = (X^T X + lambda I)^-1 X^T Y with
 * X = [G C], G the n x m genotypes and C the n x nc real confounders of the
 * training patients.  Three calls around the same factor and solve:
 *   1. krr_rr_build: the context's matrix becomes the Gram matrix X^T X of
 *      order m + nc (genotype columns first), by the paper's mixed-precision
 *      SYRK: G^T G on the tensor cores from exact E4M3 operands with FP32
 *      accumulation (entries below 4n, so exact: n <= 2^22), the columns with
 *      confounders in FP32 products summed in FP64;
 *   2. krr_rr_rhs: B = X^T Y (m + nc rows, p columns), FP32 products summed in
 *      FP64 over patient chunks;
 *   3. krr_factor(ctx, lambda, ...) and krr_solve(ctx, B, ...) -> beta, the
 *      same adaptive-precision Cholesky, substitution and refinement as KRR;
 *   4. krr_rr_predict: Yt = T beta_g + Ct beta_c for held-out patients.
 *   X  : n x m int8 genotypes {0, 1, 2}, leading dimension ldx >= m, host or
 *        device; C: n x nc FP32 (ldc >= nc), 0 <= nc <= 16 (C may be NULL
 *        when nc = 0).
 *   Y  : n x p FP32 phenotypes (ldy >= p); B: (m + nc) x p FP32 output
 *        (ldb >= p); T: n_test x m int8 (ldt >= m); Ct: n_test x nc FP32
 *        (ldct >= nc); beta: (m + nc) x p FP32 (ldbeta >= p); Yt: n_test x p
 *        FP32 output (ldyt >= p).  Any of them host or device.
 * krr_build_kernel / krr_build_kernel_conf replace the Gram matrix with a KRR
 * kernel again; krr_predict, krr_predict_conf, krr_grad_hyper and
 * krr_predict_noalloc reject a context that holds a Gram matrix.
 * Errors: KRR_EINVAL (shapes), KRR_ESTATE (rhs / predict before build),
 * KRR_ENOMEM, KRR_ECUDA.
 */
krr_status krr_rr_build(krr_ctx *ctx, const int8_t *X, int64_t n, int64_t m, int64_t ldx, const float *C,
                        int64_t nc, int64_t ldc);
krr_status krr_rr_rhs(krr_ctx *ctx, const float *Y, int64_t p, int64_t ldy, float *B, int64_t ldb);
krr_status krr_rr_predict(krr_ctx *ctx, const int8_t *T, int64_t n_test, int64_t ldt, const float *Ct,
                          int64_t ldct, const float *beta, int64_t ldbeta, int64_t p, float *Yt, int64_t ldyt);

/*
 * Copies the per-tile precision map of the current factor (the "mosaic" of
 * the paper's adaptive-precision Cholesky) to host memory: map[i * nt + j]
 * for tile row i >= tile column j holds a KRR_PREC_* value (diagonal tiles
 * report their factorisation precision); entries above the diagonal are 255.
 * map may be NULL to query nt only.  Errors: KRR_ESTATE (no factor),
 * KRR_EINVAL (map_capacity < nt * nt).
 */
krr_status krr_get_precision_map(krr_ctx *ctx, uint8_t *map, int64_t map_capacity, int64_t *nt);

/*
 * Copies the squared distances of the lower-triangle tiles to a caller
 * buffer for testing: D is n x n uint32 row-major (leading dimension ldd),
 * entries (i, j) with j > i tile-wise are left untouched.  Needs a context
 * created with keep_distances set through krr_set_keep_distances() before
 * krr_build_kernel().  Host or device buffer.
 */
krr_status krr_set_keep_distances(krr_ctx *ctx, int32_t keep);
krr_status krr_get_distances(krr_ctx *ctx, uint32_t *D, int64_t ldd);

/*
 * Copies the FP32 kernel matrix K (without lambda) for tile row i >= tile
 * column j to a caller buffer: K is n x n FP32 row-major (leading dimension
 * ldk); the strictly-upper tiles are left untouched.  Host or device buffer.
 */
krr_status krr_get_kernel(krr_ctx *ctx, float *K, int64_t ldk);

/*
 * Copies the stored factor to a caller buffer for testing: L is n x n FP32
 * row-major (leading dimension ldl), lower triangular; every tile is read in
 * its storage precision and de-scaled, so L L^T shows the backward error of
 * the mixed-precision factorisation.  Entries above the diagonal are 0 for a
 * host buffer and left untouched for a device buffer.  Errors: KRR_ESTATE.
 */
krr_status krr_get_factor(krr_ctx *ctx, float *L, int64_t ldl);

/*
 * Predict without allocating.  The paper has no counterpart: this entry point
 * exists for callers that must not allocate device memory at call time --
 * processes whose device memory is owned up front by another allocator (a
 * pool or arena that has to account for every byte), or latency-critical
 * callers that must not enter the driver's allocator, whose calls can block
 * and synchronise the device.  It computes the same Yt = K_test A as
 * krr_predict() with the same kernels, but every working buffer lives in one
 * file-scope device array of fixed size (about 16.8 MB, present on every GPU
 * that loads the library until the process exits), so it calls no
 * cudaMalloc / cudaFree.
 *   T, A, Yt : device pointers only (host pointers give KRR_EINVAL).
 *   Limits   : 1 <= n_test <= 256, 1 <= p <= 8, padded N <= 131072, padded
 *              M <= 16384, context in KRR_MODE_MIXED; otherwise KRR_EINVAL.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  All calls share the array: calls whose work
 * overlaps on the GPU (different streams or contexts) race on it.
 * Errors: KRR_ESTATE (no kernel built), KRR_EINVAL, KRR_ECUDA.
 */
krr_status krr_predict_noalloc(krr_ctx *ctx, const int8_t *T, int64_t n_test, int64_t ldt,
                               const float *A, int64_t lda, int64_t p, float *Yt, int64_t ldyt);

/*
 * Gradient of the held-out loss with respect to the hyperparameters (the
 * paper picks gamma and alpha by cross-validation, Sec. III; the gradient
 * itself is not in the paper).  With M = K + lambda I, A = M^-1 Y (the
 * caller's current solution), Yhat = K_test A and
 *     loss = ||Yhat - Yt||_F^2 / (n_test p):
 *   G_p = 2 (Yhat - Yt) / (n_test p);  B = K_test^T G_p;  Z = M^-1 B (the
 *   stored factor with refinement);
 *   d loss / d log lambda = -lambda <Z, A>;
 *   d loss / d log gamma  = gamma ( sum_ij D_ij K_ij (Z A^T)_ij
 *                                  - sum_tj D_tj K_tj (G_p A^T)_tj ),
 * with D the exact squared distances, recomputed on the tensor cores.
 *   T  : n_test x m int8 held-out genotypes (ldt >= m), host or device.
 *   Yt : n_test x p FP32 held-out phenotypes (ldy >= p), host or device.
 *   A  : n x p FP32 weights from krr_solve (lda >= p), host or device.
 *   out: host double[3] = {loss, d loss / d log gamma, d loss / d log lambda}.
 * Needs a factorisation in KRR_MODE_MIXED; 1 <= p <= 16.
 * Errors: KRR_ESTATE, KRR_EINVAL, KRR_ENOMEM, KRR_ECUDA.
 */
krr_status krr_grad_hyper(krr_ctx *ctx, const int8_t *T, int64_t n_test, int64_t ldt, const float *Yt,
                          int64_t ldy, const float *A, int64_t lda, int64_t p, double *out);

/*
 * Batched problems: many (cohort, cross-validation fold, lambda) problems of
 * uneven size -- the paper picks gamma and alpha by cross-validation (Sec.
 * III), i.e. by solving many such problems.  krr_batch_create() gives every
 * problem its own context and stream, picks each problem's tile edge with an
 * autotuner, runs every pipeline once to allocate, and captures Build ->
 * Factor -> Solve (with
 * options->ir_max refinement steps, no host decisions) -> Predict of all
 * problems into one CUDA graph with a fork/join over the problem streams.
 * krr_batch_run() launches that graph once and reports per-problem status,
 * tile and final relative residual.  The graph is captured on a stream of
 * the batch's own and launched on `stream` (which may be the legacy default
 * stream).  All pointers are device pointers and are read at every run
 * (update the data in place between runs).  krr_batch_last_error(NULL) gives
 * the message of the calling thread's last failed krr_batch_create().
 *   autotune : 0 = every problem at options->tile; 1 = timed trial runs of
 *              the smallest, median and largest problem with tile edges
 *              256 / 512 / 1024, each problem taking the edge of the measured
 *              problem nearest to it in log N; 2 = that choice and every
 *              uniform edge, each captured and timed as the whole batch (a
 *              few graph runs per candidate), the fastest kept.
 * Errors: KRR_EINVAL, KRR_ENOMEM, KRR_ECUDA, and the first per-problem error.
 */
typedef struct krr_batch_problem {
    const int8_t *G;    /* n x m training genotypes, leading dimension ldg */
    int64_t n, ldg;
    double gamma, lambda;
    const float *Y;     /* n x p phenotypes, leading dimension ldy */
    int64_t ldy;
    float *A;           /* n x p weights (output), leading dimension lda */
    int64_t lda;
    const int8_t *T;    /* n_test x m held-out genotypes (ldt), or NULL */
    int64_t n_test, ldt;
    float *Yt;          /* n_test x p predictions (output), leading dimension ldyt */
    int64_t ldyt;
} krr_batch_problem;

typedef struct krr_batch_result {
    int32_t status;         /* KRR_OK or the problem's device-side error */
    int32_t tile;           /* tile edge the autotuner picked */
    double rel_residual;    /* final ||Y - (K + lambda I) A||_F / ||Y||_F */
} krr_batch_result;

typedef struct krr_batch krr_batch;

krr_status krr_batch_create(krr_batch **out, const krr_options *opt, void *stream, int64_t m, int64_t p,
                            const krr_batch_problem *problems, int32_t count, int32_t autotune);
krr_status krr_batch_run(krr_batch *bt, krr_batch_result *results);
const char *krr_batch_last_error(const krr_batch *bt);
void krr_batch_destroy(krr_batch *bt);

/* Kernel classes timed by the optional profiler. */
enum {
    KRR_PROF_PACK = 0,     /* genotype packing and norms */
    KRR_PROF_BUILD = 1,    /* distance GEMM + exp epilogue (Build) */
    KRR_PROF_DIAG = 2,     /* diagonal-tile Cholesky + inverse */
    KRR_PROF_TRSM = 3,     /* panel solve of a tile column */
    KRR_PROF_CAST = 4,     /* adaptive-precision cast of a column */
    KRR_PROF_UPDATE = 5,   /* trailing update */
    KRR_PROF_SOLVE = 6,    /* forward + backward substitution */
    KRR_PROF_RESIDUAL = 7, /* refinement residual */
    KRR_PROF_PREDICT = 8,  /* predict (distance GEMM + exp + weights) */
    KRR_PROF_UPDATE_SHARED = 9, /* trailing-update launches of the lookahead: the diagonal
                                   target alone, and the targets that share the GPU with
                                   the diagonal step of the next column */
    KRR_PROF_CLASSES = 10
};

/*
 * Measurement report: CUDA events recorded on the context's stream around
 * every region of a class while profiling is on.  flops / bytes are the
 * algorithmic operation counts and compulsory HBM bytes of the timed
 * regions (for the trailing update 2 b^3 per off-diagonal target tile and
 * b^3 per diagonal target; for the build 2 M per lower-triangle entry), not
 * counter values.
 * launches counts the kernels this library launched (all contexts) since the
 * last reset.
 */
typedef struct krr_profile {
    int64_t launches;
    int64_t count[KRR_PROF_CLASSES];
    double ms[KRR_PROF_CLASSES];
    double flops[KRR_PROF_CLASSES];
    double bytes[KRR_PROF_CLASSES];
} krr_profile;

/* Turns event timing of the kernel classes on (1) or off (0). */
krr_status krr_set_profiling(krr_ctx *ctx, int32_t on);

/* Synchronises the stream and sums the timed regions into *out; reset = 1
 * clears the records and the launch counter afterwards. */
krr_status krr_get_profile(krr_ctx *ctx, krr_profile *out, int32_t reset);

/*
 * Changes the limit of every bounded device wait of the context's later
 * launches (krr_options.wait_budget_ns; ns >= 1).  A wait that runs out ends
 * its kernel early, after the kernel's own copies and MMAs in flight have
 * finished, and the call that launched it returns KRR_ETIMEOUT (krr_factor,
 * krr_solve); the context stays usable, and a later call with a sufficient
 * budget recomputes what was cut short.  Errors: KRR_EINVAL.
 */
krr_status krr_set_wait_budget(krr_ctx *ctx, int64_t ns);

/* Waits for all work issued by the context. */
krr_status krr_sync(krr_ctx *ctx);

/* Message of the last failed call on ctx (or of the last failed krr_create
 * when ctx is NULL).  Owned by the library. */
const char *krr_last_error(const krr_ctx *ctx);

/* Frees every buffer of the context.  ctx may be NULL. */
void krr_destroy(krr_ctx *ctx);

#ifdef __cplusplus
}
#endif

#endif /* KRR_H */
