// Internal declarations of the KRR engine: context layout, tile indexing,
// kernel launchers.  Not part of the C ABI.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/krr.h"

namespace krr {

// ---------------------------------------------------------------------------
// Tile indexing.  K (and its factor) is kept as the lower triangle of an
// NT x NT grid of b x b tiles, every tile row-major and contiguous.
//   lower-triangle tile (i, j), i >= j :  tri_index = i (i + 1) / 2 + j
//   strictly-lower tile (i, j), i > j  :  off_index = i (i - 1) / 2 + j
// ---------------------------------------------------------------------------
__host__ __device__ inline int64_t tri_index(int64_t i, int64_t j) { return i * (i + 1) / 2 + j; }
__host__ __device__ inline int64_t off_index(int64_t i, int64_t j) { return i * (i - 1) / 2 + j; }

// Inverse of the triangular numbering: t -> (i, j) with j <= i.
__host__ __device__ inline void tri_decode(int64_t t, int64_t *i, int64_t *j) {
    // single-precision estimate, corrected exactly by the loops below
    int64_t r = (int64_t)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
    while (r * (r + 1) / 2 > t) --r;
    while ((r + 1) * (r + 2) / 2 <= t) ++r;
    *i = r;
    *j = t - r * (r + 1) / 2;
}

// Kernel function of Alg. 5 applied to the exact integer distance d of the
// encoded rows: Gaussian exp(-gamma d) on the squared Euclidean distance, or
// IBS (2M - d) / M on the L1 distance (the encoded rows' squared distance),
// one correctly rounded division of exact integers.
// dc: the squared distance of the two rows' confounders (FP32; 0 without
// confounders), added to the exact genotype distance before the exponential.
// gram = 1 (ridge regression): the kernel is the Gram product S itself.
struct KernelFn {
    int ibs, gram;
    float two_m, m;
    __device__ __forceinline__ float value(float gamma, int32_t d, float dc = 0.f) const {
        return ibs ? __fdiv_rn(two_m - (float)d, m) : expf(-gamma * ((float)d + dc));
    }
};

// Confounders (real-valued covariates) per row: at most CONF_MAX, stored
// n_pad x CONF_MAX FP32 with zero padding.
constexpr int CONF_MAX = 16;

// Squared distance of two confounder rows, term by term in FP32 (no
// cancellation): ci in registers, cj in memory, nc <= CONF_MAX.
__device__ __forceinline__ float conf_dist(const float (&ci)[CONF_MAX], const float *cj, int nc) {
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < CONF_MAX; ++q) {
        if (q < nc) {
            const float t = ci[q] - cj[q];
            s = fmaf(t, t, s);
        }
    }
    return s;
}

// Limit of the waits that drain a kernel's own copies and MMAs in flight
// after another wait ran out: those complete in microseconds, so the limit
// only bounds the wait; it is never shorter than 20 ms, whatever the
// context's wait budget, so that no CTA leaves with a copy into its shared
// memory or an MMA into its tensor memory still pending.
__host__ __device__ inline uint64_t drain_limit(uint64_t wait_ns) {
    return wait_ns > 20000000ull ? wait_ns : 20000000ull;
}

// Slots of the small FP64 reduction buffer Ctx::red.
constexpr int RED_RNORM = 0;     // [0] ||R||_F^2, [1] ||Y||_F^2 of the last residual
constexpr int RED_KNORM2 = 2;    // ||K||_F^2
constexpr int RED_KSUM = 3;      // sum of the entries of K
constexpr int RED_KSHIFT = 4;    // mean off-diagonal entry of K (residual shift)
constexpr int RED_KBOUND = 5;    // max_i K_ii: bounds every |K_ij| (K is positive semidefinite)
constexpr int RED_MINPIV = 64;   // nt * (b / 64) block minimum pivots, then nt max|L_kk| bounds

// Storage precision of an off-diagonal factor tile (values of the
// KRR_PREC_* enum of krr.h).
// Mixed mode: FP16 and E4M3 tiles hold scale * L; an FP32-class tile holds
// scale * L as an exact pair of FP16 planes (hi = fp16(x), lo = fp16(x - hi),
// about 22 significant bits), hi plane first.  An E4M3 tile also has an FP16
// copy in its trailing slot W(i, k), which is spent once the column is
// factored.  fp32 mode: every tile is plain FP32 with scale 1.
struct TileDesc {
    int64_t offset;   // byte offset of the tile in the factor pool
    float scale;      // stored value = scale * L (power of two)
    int32_t prec;     // KRR_PREC_FP32 / KRR_PREC_FP16 / KRR_PREC_E4M3
};

// Device error record written by kernels that detect a failure.  Each field
// is written with atomics so the first failure wins.
struct DevErrors {
    int32_t code;         // 0 = none, else a krr_status value
    int32_t pad;
    int64_t bad_tile;     // ENOTPD: diagonal tile index
    int64_t bad_column;   // ENOTPD: global column
    double bad_value;
    int64_t fp8_tiles, fp16_tiles, fp32_tiles, pool_cursor;
    double min_pivot;
};

struct Ctx {
    // configuration
    krr_options opt;
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    std::string last_error;

    // problem
    int64_t n = 0, m = 0, m_pad = 0, b = 0, nt = 0, n_pad = 0;
    double gamma = 0.0, lambda = 0.0;
    bool built = false, factored = false;
    int keep_distances = 0;

    // build products
    uint8_t *g8 = nullptr;     // E4M3 genotypes, n_pad x m_pad (mixed mode)
    float *gf = nullptr;       // FP32 genotypes, n_pad x m_pad (fp32 mode)
    int32_t *norms = nullptr;  // squared row norms, n_pad
    float *Kd = nullptr;       // FP32 kernel tiles, lower triangle incl. diagonal
    uint32_t *Dd = nullptr;    // exact squared distances (only with keep_distances)
    double *knorm2 = nullptr;  // per lower-triangle tile sum of K^2
    size_t g_bytes = 0, kd_bytes = 0, dd_bytes = 0;

    // factor state
    void *W = nullptr;         // strictly-lower trailing tiles: FP16 (mixed) / FP32 (fp32)
    float *Wd = nullptr;       // diagonal working tiles, FP32, overwritten by L_kk
    float *Linv = nullptr;     // inverse of every diagonal factor tile, FP32
    float *LinvT = nullptr;    // and its transpose (row-oriented backward sweep)
    __half *Linv_hi = nullptr, *Linv_lo = nullptr;  // FP16 split of Linv (mixed)
    double *diag64 = nullptr;  // FP64 scratch diagonal tile (diag_fp64); FP32 scratch otherwise
    int *diag_ctr = nullptr;   // progress counters of the diagonal-step kernel
    double *diag64_inv = nullptr;
    uint8_t *pool = nullptr;   // off-diagonal factor tiles, each in its precision
    size_t pool_bytes = 0;
    TileDesc *ltab = nullptr;  // per strictly-lower tile: where/how L is stored
    float *colbuf = nullptr;   // FP32 TRSM output of one tile column
    __half *pan_hi = nullptr, *pan_lo = nullptr;  // FP16 operand copies of one column
    float *colmax = nullptr;     // per block of the column's tiles: max |L| (panel-solve epilogue)
    uint8_t *precmap = nullptr;  // device copy of the precision map (nt x nt)
    DevErrors *derr = nullptr;
    DevErrors *herr = nullptr;   // pinned host mirror
    size_t w_bytes = 0;

    // solve / predict scratch
    float *ybuf = nullptr, *zbuf = nullptr;  // n_pad x p work vectors
    double *rbuf = nullptr;                  // n_pad x p residual (FP64)
    float *abuf = nullptr;                   // n_pad x p current solution
    float *dabuf = nullptr;                  // n_pad x p correction
    double *red = nullptr;                   // reductions (norms), small; slots RED_*
    double *colsum = nullptr;                // column sums of the current iterate (FP64)
    int64_t colsum_cap = 0;
    double *hred = nullptr;                  // pinned host mirror of red
    int64_t vec_cap = 0;                     // capacity in elements of the n_pad x p buffers
    float *pred_part = nullptr;              // predict partial products
    size_t pred_part_cap = 0;
    int *sw_flags = nullptr;                 // sweep item counter, abort flag, progress counters
    int64_t sw_flags_cap = 0;
    __half *ts_v0 = nullptr, *ts_v1 = nullptr;  // tensor-core sweep: FP16 pairs of vector blocks
    size_t ts_vcap = 0;
    void *ts_aux = nullptr;                  // tensor-core sweep: block scales, slab maxima, counters
    size_t ts_aux_cap = 0;
    float *ts_xt = nullptr;                  // tensor-core sweep: column-major copy of the right-hand sides
    size_t ts_xcap = 0;
    float *pred_out = nullptr;               // reduced predictions, rows_pad x p
    size_t pred_out_cap = 0;
    // hyperparameter gradient buffers (krr_grad_hyper)
    float *g_yt = nullptr, *g_gp = nullptr, *g_aw = nullptr, *g_part = nullptr;
    double *g_sq = nullptr, *g_tpart = nullptr, *g_kpart = nullptr, *g_scal = nullptr;
    size_t g_rows_cap = 0, g_aw_cap = 0, g_part_cap = 0, g_tpart_cap = 0, g_kpart_cap = 0;
    // confounders of the training rows (krr_build_kernel_conf), n_pad x
    // CONF_MAX, and of the held-out rows of the current predict
    float *conf = nullptr, *tconf = nullptr;
    size_t conf_cap = 0, tconf_cap = 0;
    int64_t nconf = 0;
    uint8_t *t8 = nullptr;                   // packed test genotypes (E4M3 / FP32 bytes)
    size_t t_cap = 0;
    int32_t *tnorms = nullptr;
    size_t tnorm_cap = 0;
    void *stage = nullptr;                   // device staging for host arguments
    size_t stage_cap = 0;

    // tensor-core launch plumbing (opaque, owned by tc_gemm.cu)
    void *tc = nullptr;

    // profiler (opaque, owned by krr_api.cu)
    void *prof = nullptr;
    int prof_on = 0;

    // ridge regression (ridge.cu): the context's matrix is the Gram matrix
    // X^T X of order n = rr_m genotype columns + rr_nc confounder columns;
    // m is then the number of patients (the contraction length)
    int rr = 0;
    int64_t rr_m = 0, rr_nc = 0;
    void *rr_state = nullptr;
    // build products read from another context (adopt_build), not owned
    int build_borrowed = 0;
    // at most this many CTAs per launch (0: one per SM), in general and per
    // kernel class (GL_*; 0: the general cap); the batch runner sets them so
    // that the kernels of concurrent problems share the GPU
    int cta_cap = 0;
    int cta_caps[6] = {0, 0, 0, 0, 0, 0};

    // lookahead of the factorisation: the diagonal step of column k + 1 runs
    // on this second stream while the trailing update of step k continues
    // (created on the first factorisation that uses it)
    cudaStream_t la_stream = nullptr;
    cudaEvent_t la_ev[2] = {nullptr, nullptr};

    // graph mode: no host synchronisation or readback inside build / factor /
    // solve / predict, fixed refinement count (used by the batch runner)
    int graph_mode = 0;
    size_t red_cap = 0;
};

inline bool is_ibs(const Ctx *c) { return c->opt.kernel == KRR_KERNEL_IBS; }
// Kernel classes with a CTA cap of their own: the diagonal step (a dependency
// chain: most of its CTAs wait), the substitution sweeps, the refinement
// residual, the CTA-pair kernels (panel solve, trailing update) and the other
// tensor-core kernels (build, predict, gradient).
enum GridClass { GL_DEFAULT = 0, GL_DIAG = 1, GL_SWEEP = 2, GL_RESIDUAL = 3, GL_PAIR = 4, GL_SINGLE = 5 };
// CTAs a persistent launch of this class may use.
inline int64_t grid_limit(const Ctx *c, int cls = GL_DEFAULT) {
    const int cap = c->cta_caps[cls] > 0 ? c->cta_caps[cls] : c->cta_cap;
    return (cap > 0 && cap < c->num_sms) ? cap : c->num_sms;
}
inline KernelFn kernel_fn(const Ctx *c) {
    KernelFn f;
    f.ibs = is_ibs(c) ? 1 : 0;
    f.gram = c->rr;
    f.two_m = (float)(2 * c->m);
    f.m = (float)c->m;
    return f;
}
// Rows whose kernel entries are real (the rest is padding with K = I): the
// training rows, or the genotype columns of a ridge-regression Gram matrix
// (its confounder rows are written afterwards).
inline int64_t real_rows(const Ctx *c) { return c->rr ? c->rr_m : c->n; }
// Ridge regression buffers (ridge.cu), released with the context.
void rr_free(Ctx *c);

// Width of the packed operand rows before padding: M, or 2M for IBS.
inline int64_t encoded_width(const Ctx *c, int64_t m) { return is_ibs(c) ? 2 * m : m; }

// One-time set-up per device: cudaFuncSetAttribute and the occupancy queries
// act on the current device only, so a process that drives several GPUs
// repeats them on each.  Objects of this type live in static storage (zero
// initialised); two threads racing on the same device only repeat an
// idempotent set-up call.  Devices past MAX_DEVICES are set up on every call.
constexpr int MAX_DEVICES = 64;
struct PerDevice {
    std::atomic<int> done[MAX_DEVICES];
    std::atomic<int> value[MAX_DEVICES];
    bool has(int dev) const {
        return dev >= 0 && dev < MAX_DEVICES && done[dev].load(std::memory_order_acquire) != 0;
    }
    int get(int dev) const { return value[dev].load(std::memory_order_relaxed); }
    void put(int dev, int v = 1) {
        if (dev < 0 || dev >= MAX_DEVICES) return;
        value[dev].store(v, std::memory_order_relaxed);
        done[dev].store(1, std::memory_order_release);
    }
};

// Device buffers owned by a context: (re)allocation with the failure message
// recorded in the context (KRR_ENOMEM), and release.
template <typename T>
krr_status dev_alloc(Ctx *c, T **p, size_t count, const char *what) {
    if (*p) {
        cudaFree(*p);
        *p = nullptr;
    }
    if (count == 0) return KRR_OK;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        c->last_error = std::string("cudaMalloc failed for ") + what + " (" +
                        std::to_string(count * sizeof(T)) + " bytes): " + cudaGetErrorString(e);
        return KRR_ENOMEM;
    }
    return KRR_OK;
}

template <typename T>
void dev_free(T **p) {
    if (*p) cudaFree(*p);
    *p = nullptr;
}

// Host-side helpers of the driver (krr_api.cu), shared by the entry points of
// the other translation units.
bool is_device_ptr(const void *p);
const void *pinned_host_alias(const void *p);
// Makes the context's device staging buffer for host arguments at least `bytes`.
krr_status stage(Ctx *c, size_t bytes);
// KRR_ECUDA with the message of the last launch error, if any.
krr_status check_launch(Ctx *c, const char *where);
// n x cols caller matrix (host or device, leading dimension ld) -> dense device
// matrix of rows_pad rows (zero padded).
krr_status load_rows_f32(Ctx *c, const float *src, int64_t n, int64_t cols, int64_t ld, int64_t rows_pad,
                         float *dst);
// First n rows of a dense device matrix -> caller matrix (host or device).
krr_status store_rows_f32(Ctx *c, const float *src, int64_t n, int64_t cols, float *dst, int64_t ld);
// Confounders (n x nc) -> dense rows_pad x CONF_MAX device layout.
krr_status load_conf(Ctx *c, const float *src, int64_t n, int64_t nc, int64_t ld, int64_t rows_pad, float *dst);
void free_factor(Ctx *c);
void free_build(Ctx *c);
// Shares src's build (genotypes, norms, kernel tiles, kernel statistics) with
// dst, read-only, for several factorisations of one kernel matrix.
krr_status adopt_build(Ctx *dst, const Ctx *src);
// Buffers and shape fields of a build over n rows, packed operand rows of
// m_pad columns (keep_d: keep the exact distances as well).
krr_status prepare_build(Ctx *c, int64_t n, int64_t m_pad, int keep_d);
bool mixed(const Ctx *c);

// Kernel launch counter of the whole library (reported by krr_get_profile).
void count_launch();

// Error helpers --------------------------------------------------------------
#define KRR_CUDA_TRY(ctx, expr)                                                  \
    do {                                                                         \
        cudaError_t _e = (expr);                                                 \
        if (_e != cudaSuccess) {                                                 \
            (ctx)->last_error = std::string(#expr) + ": " + cudaGetErrorString(_e); \
            return KRR_ECUDA;                                                    \
        }                                                                        \
    } while (0)

#define KRR_TRY(expr)                  \
    do {                               \
        krr_status _s = (expr);        \
        if (_s != KRR_OK) return _s;   \
    } while (0)

// ---------------------------------------------------------------------------
// SIMT kernels (simt_kernels.cu)
// ---------------------------------------------------------------------------
// Pack int8 genotypes: E4M3 bytes (mixed) or FP32 (fp32) with zero padding to
// n_pad x m_pad, plus exact squared row norms.
// thermo = 1: the IBS encoding (two indicators per genotype, m_pad >= 2m;
// norms = row sums of g).
void launch_pack_genotypes(const int8_t *g, int64_t n, int64_t m, int64_t ldg, int64_t n_pad,
                           int64_t m_pad, uint8_t *out_e4m3, float *out_f32, int32_t *norms,
                           cudaStream_t s, int thermo = 0);

// Generic FP32/FP64 tiled GEMM on CUDA cores: C = alpha * op(A) op(B)^T + beta * Cin,
// with A (M x K, row-major) and B either N x K row-major (b_trans = 0) or
// K x N row-major (b_trans = 1).  'lower' skips 128 x 128 blocks strictly above
// the diagonal of C.  Batched over `batch` problems with fixed strides.
template <typename T>
void launch_gemm_simt(int M, int N, int K, T alpha, const T *A, int64_t lda, int64_t strideA,
                      const T *B, int64_t ldb, int64_t strideB, int b_trans, T beta,
                      const T *Cin, int64_t ldcin, int64_t strideCin, T *C, int64_t ldc,
                      int64_t strideC, int batch, int lower, cudaStream_t s);

// FP32 Build on CUDA cores over lower-triangle tiles (fp32 mode).
void launch_build_simt(Ctx *c);
// FP32 trailing update of step k on CUDA cores (fp32 mode).
void launch_update_simt(Ctx *c, int64_t k);
// FP32 panel TRSM of column k on CUDA cores (fp32 mode): L_ik = W_ik Linv_kk^T.
void launch_trsm_simt(Ctx *c, int64_t k);
// FP32 predict partial products on CUDA cores (fp32 mode).  rows_pad is the
// number of packed test rows (a multiple of 128); part is
// (n_pad / 128) x rows_pad x p.
void launch_predict_simt(Ctx *c, const float *tf, const int32_t *tn, int64_t n_test,
                         int64_t rows_pad, const float *A, int64_t p, float *part,
                         const float *tconf = nullptr);

// Diagonal-step dataflow kernel (diag.cu): FP32 factor of tile W, inverse X,
// its transpose XT and FP16 split hi/lo (optional); ctr holds
// diag_counter_count(b) ints, minpiv b / 64 doubles.
int64_t diag_counter_count(int64_t b);
krr_status launch_diag_dataflow(Ctx *c, int64_t k, float *W, float *X, float *XT, __half *hi, __half *lo,
                                float *tmp, int *ctr, double *minpiv, cudaStream_t s, int64_t cta_cap);

// Diagonal step: in-place Cholesky of Wd tile k and its inverse into Linv.
// Factor and inverse of diagonal tile k, on stream s (nullptr: the context's
// stream) with at most cta_cap CTAs for the dataflow kernel (0: class limit).
krr_status diag_step(Ctx *c, int64_t k, cudaStream_t s = nullptr, int64_t cta_cap = 0);

// Number of max |L_ik| partials per panel tile written by the tensor-core
// panel solve (one per 128 x 256 output block).
inline int64_t tile_max_partials(int64_t b) { return (b / 128) * (b / 256); }
// Casts the FP32 TRSM output of column k into the factor pool with the
// precision chosen by the adaptive rule, plus the operand panels (mixed mode).
// The tile maxima come from the panel solve (c->colmax).
// ||K||_F^2 is read from c->red[2] (written by the build).
void launch_column_cast(Ctx *c, int64_t k);

// Triangular solves with the stored factor: X <- (L L^T)^-1 X, n_pad x p
// (row-major, leading dimension p); tmp is n_pad x p scratch.
krr_status solve_inplace(Ctx *c, float *x, float *tmp, int64_t p);

// Persistent dataflow sweeps (sweep.cu): the two substitutions of a solve
// on CUDA cores (fp32 mode), and the residual r = y - (K + lambda I) a given
// the column sums of a in c->colsum.
krr_status sweep_solve(Ctx *c, float *x, float *tmp, int64_t p);
// The two substitutions on the tensor cores (tcsweep.cu, mixed mode).
krr_status tc_sweep_solve(Ctx *c, float *x, float *tmp, int64_t p);
// The refinement residual on the tensor cores (tcsweep.cu, mixed mode).
krr_status tc_residual(Ctx *c, const float *y, const float *a, double *r, int64_t p);
krr_status sweep_residual(Ctx *c, const float *y, const float *a, double *r, int64_t p);

// r = y - (K + lambda I) a (FP64 accumulation), norms into c->red.
krr_status launch_residual(Ctx *c, const float *y, const float *a, double *r, int64_t p);

// Resets the device error record and the precision map, and (fp32 mode)
// fills the tile table: every factor tile FP32 at a fixed slot.
void launch_factor_init(Ctx *c);

// Small helpers.
void launch_fill_zero(void *p, size_t bytes, cudaStream_t s);
// part: norm_partial_count() doubles of scratch (the context's reduction buffer
// keeps them after its other slots, see red_norm_part()).
constexpr int64_t norm_partial_count() { return 2 * 256; }
void launch_reduce_norms(const double *r, const float *y, int64_t n, int64_t p, double *out, double *part,
                         cudaStream_t s);
void launch_axpy_r(const double *r, float *dst, int64_t count, cudaStream_t s);
void launch_add_scaled(float *a, const float *da, float alpha, int64_t count, cudaStream_t s);
// Yt = sum of the per-block partials; when shift is given the partials are of
// (K - c) A and c (1^T A) is added (c = *shift rounded to FP32, colsum = 1^T A).
void launch_predict_reduce(const float *part, int64_t nblk, int64_t rows_pad, int64_t n_test,
                           int64_t p, float *out, int64_t ldo, cudaStream_t s, const double *shift = nullptr,
                           const double *colsum = nullptr);
// out[q] = sum of column q of a (n x p, row-major), FP64.
void launch_colsum(const float *a, int64_t n, int64_t p, double *out, cudaStream_t s);
void launch_copy_rows(const float *src, int64_t lds, float *dst, int64_t ldd, int64_t rows,
                      int64_t cols, int64_t rows_pad, cudaStream_t s);
// out[0] = ||K||_F^2, out[1] = sum of K, out[2] = mean off-diagonal entry.
void launch_kernel_sumsq(Ctx *c, double *out);
// Dense lower-triangular copy of the stored factor into dst (n x n, device).
void launch_factor_to_dense(Ctx *c, float *dst, int64_t ld);

// Gradient helpers: G_p and squared errors, FP64 sums and dot products.
void launch_grad_prep(const float *yhat, const float *yt, int64_t n_test, int64_t p, int64_t rows,
                      float *gp, double *sq, cudaStream_t s);
void launch_sum_f64(const double *x, int64_t n, double *out, cudaStream_t s);
void launch_dot_f32(const float *a, const float *b, int64_t n, double *out, cudaStream_t s);

// ---------------------------------------------------------------------------
// Tensor-core kernels (tc_gemm.cu)
// ---------------------------------------------------------------------------
krr_status tc_init(Ctx *c);
void tc_free(Ctx *c);
krr_status tc_build(Ctx *c);                 // distance GEMM + exp epilogue (E4M3)
// (Re)makes the tensor map of the packed training genotypes (c->g8), which
// Predict and the gradient read; tc_build does it itself.
krr_status tc_bind_genotypes(Ctx *c);
krr_status tc_trsm(Ctx *c, int64_t k);       // panel TRSM of column k (FP16 split)
// Trailing update of step k over target tiles [tile0, tile0 + tiles) of the
// step's order (tile 0 is the diagonal target (k + 1, k + 1); tiles < 0: to
// the end), on at most cta_cap CTAs (0: the class limit).
krr_status tc_update(Ctx *c, int64_t k, int64_t tile0 = 0, int64_t tiles = -1, int64_t cta_cap = 0);
// Second stream and events of the factorisation lookahead (made once; in
// graph mode it must be made before the capture).
krr_status ensure_lookahead_stream(Ctx *c);
// Algorithmic flops of those target tiles: 2 b^3 per off-diagonal target,
// b^3 per diagonal target.
double update_flops(const Ctx *c, int64_t k, int64_t tile0, int64_t tiles);
// Predict partial products for weight columns A[:, 0:p] (p <= 32, leading
// dimension lda): part is (n_pad / 128) x rows_pad x p.
// With kshift the partials are of (K - c) A, c = *kshift (the reduction adds
// c (1^T A) back).
// With confounders (c->nconf > 0) tconf holds the held-out rows' and p <= 16.
krr_status tc_predict(Ctx *c, const uint8_t *t8, const int32_t *tn, int64_t n_test,
                      int64_t rows_pad, const float *A, int64_t lda, int64_t p, float *part,
                      const double *kshift = nullptr, const float *tconf = nullptr);
// B = K_test^T G_p (roles swapped): part is (2 * test_rows256 / 256) x n_pad x p.
krr_status tc_predict_t(Ctx *c, const uint8_t *t8, const int32_t *tn, int64_t n_test,
                        int64_t test_rows256, const float *gp, int64_t ldgp, int64_t p, float *part);
// d K-weighted gradient contractions, one partial per block (p <= 16).
krr_status tc_grad_terms(Ctx *c, const uint8_t *t8, const int32_t *tn, int64_t n_test,
                         int64_t test_rows, const float *aw, const float *zw, const float *gp,
                         int64_t ld, int64_t p, double *part_t, double *part_k, int64_t *items_t,
                         int64_t *items_k);
// Forget the cached factor tensor maps (the factor buffers were reallocated).
void tc_invalidate_factor_maps(Ctx *c);

}  // namespace krr
