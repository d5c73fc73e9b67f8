// C ABI of the KRR engine (include/krr.h) and the host-side orchestration of
// the three phases of the paper's driver (Alg. 1): Build (Alg. 2), Associate
// (Alg. 3: tile Cholesky + solves + refinement) and Predict (Alg. 4).
#include <cuda_runtime.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <new>
#include <string>
#include <vector>

#include "krr_internal.h"

using namespace krr;

struct krr_ctx : public Ctx {};

static thread_local std::string g_create_error;

namespace krr {
static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace krr

namespace {

// Event-timed regions per kernel class (krr_get_profile).
struct ProfRec {
    int cls;
    cudaEvent_t a, b;
    double flops, bytes;
};
struct ProfState {
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    cudaEvent_t take() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};

// Opens a timed region of class cls on stream s (nullptr: the context's
// stream); returns its index or -1 when off.
int prof_begin(Ctx *c, int cls, cudaStream_t s = nullptr) {
    if (!c->prof_on || !c->prof) return -1;
    ProfState *ps = (ProfState *)c->prof;
    ProfRec r;
    r.cls = cls;
    r.a = ps->take();
    r.b = ps->take();
    r.flops = r.bytes = 0.0;
    cudaEventRecord(r.a, s ? s : c->stream);
    ps->recs.push_back(r);
    return (int)ps->recs.size() - 1;
}

void prof_end(Ctx *c, int idx, double flops, double bytes, cudaStream_t s = nullptr) {
    if (idx < 0 || !c->prof) return;
    ProfState *ps = (ProfState *)c->prof;
    ProfRec &r = ps->recs[idx];
    r.flops = flops;
    r.bytes = bytes;
    cudaEventRecord(r.b, s ? s : c->stream);
}

}  // namespace

namespace krr {

// Device address of page-locked host memory (the GPU reads it over the host
// link, no staging copy), or nullptr for anything else.
const void *pinned_host_alias(const void *p) {
    if (!p) return nullptr;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return (a.type == cudaMemoryTypeHost) ? a.devicePointer : nullptr;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

krr_status stage(Ctx *c, size_t bytes) {
    if (bytes <= c->stage_cap) return KRR_OK;
    void *p = nullptr;
    if (c->stage) cudaFree(c->stage);
    c->stage = nullptr;
    c->stage_cap = 0;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        c->last_error = "cudaMalloc failed for the host-argument staging buffer";
        return KRR_ENOMEM;
    }
    c->stage = p;
    c->stage_cap = bytes;
    return KRR_OK;
}

krr_status check_launch(Ctx *c, const char *where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->last_error = std::string(where) + ": " + cudaGetErrorString(e);
        return KRR_ECUDA;
    }
    return KRR_OK;
}

// Copies an n x cols row-major caller matrix (host or device, leading
// dimension ld) into a dense device matrix with rows_pad rows (zero padded).
krr_status load_rows_f32(Ctx *c, const float *src, int64_t n, int64_t cols, int64_t ld,
                         int64_t rows_pad, float *dst) {
    const float *dsrc = src;
    if (!is_device_ptr(src)) {
        KRR_TRY(stage(c, (size_t)n * ld * sizeof(float)));
        KRR_CUDA_TRY(c, cudaMemcpyAsync(c->stage, src, (size_t)n * ld * sizeof(float),
                                        cudaMemcpyHostToDevice, c->stream));
        dsrc = (const float *)c->stage;
    }
    launch_copy_rows(dsrc, ld, dst, cols, n, cols, rows_pad, c->stream);
    return check_launch(c, "copy rows");
}

// Confounders (n x nc, leading dimension ld, host or device) into the
// context's dense n_pad x CONF_MAX layout with zero padding.
krr_status load_conf(Ctx *c, const float *src, int64_t n, int64_t nc, int64_t ld, int64_t rows_pad, float *dst) {
    const float *dsrc = src;
    KRR_CUDA_TRY(c, cudaMemsetAsync(dst, 0, (size_t)rows_pad * CONF_MAX * sizeof(float), c->stream));
    if (!is_device_ptr(src)) {
        KRR_TRY(stage(c, (size_t)n * ld * sizeof(float)));
        KRR_CUDA_TRY(c, cudaMemcpyAsync(c->stage, src, (size_t)n * ld * sizeof(float), cudaMemcpyHostToDevice,
                                        c->stream));
        dsrc = (const float *)c->stage;
    }
    launch_copy_rows(dsrc, ld, dst, CONF_MAX, n, nc, n, c->stream);
    return check_launch(c, "copy confounders");
}

// Copies the first n rows of a dense device matrix to a caller matrix.
krr_status store_rows_f32(Ctx *c, const float *src, int64_t n, int64_t cols, float *dst,
                          int64_t ld) {
    if (is_device_ptr(dst)) {
        launch_copy_rows(src, cols, dst, ld, n, cols, n, c->stream);
        return check_launch(c, "copy rows");
    }
    if (ld == cols) {  // contiguous rows: one linear copy
        KRR_CUDA_TRY(c, cudaMemcpyAsync(dst, src, (size_t)n * cols * sizeof(float), cudaMemcpyDeviceToHost,
                                        c->stream));
    } else {
        KRR_CUDA_TRY(c, cudaMemcpy2DAsync(dst, ld * sizeof(float), src, cols * sizeof(float),
                                          cols * sizeof(float), n, cudaMemcpyDeviceToHost, c->stream));
    }
    KRR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return KRR_OK;
}

// Packs n x m int8 genotypes (host or device) into the context's padded
// operand layout.
krr_status pack(Ctx *c, const int8_t *g, int64_t n, int64_t m, int64_t ldg, int64_t rows_pad,
                uint8_t *out8, float *outf, int32_t *norms) {
    const int8_t *dg = g;
    const void *alias = is_device_ptr(g) ? nullptr : pinned_host_alias(g);
    if (alias) {
        dg = (const int8_t *)alias;  // page-locked: the pack kernel reads it in place
    } else if (!is_device_ptr(g)) {
        KRR_TRY(stage(c, (size_t)n * m));
        // one linear copy when the rows are contiguous (a pitched copy of short
        // rows runs far below the host link's rate)
        if (ldg == m) {
            KRR_CUDA_TRY(c, cudaMemcpyAsync(c->stage, g, (size_t)n * m, cudaMemcpyHostToDevice, c->stream));
        } else {
            KRR_CUDA_TRY(c, cudaMemcpy2DAsync(c->stage, m, g, ldg, m, n, cudaMemcpyHostToDevice, c->stream));
        }
        dg = (const int8_t *)c->stage;
        ldg = m;
    }
    launch_pack_genotypes(dg, n, m, ldg, rows_pad, c->m_pad, out8, outf, norms, c->stream, is_ibs(c) ? 1 : 0);
    return check_launch(c, "pack genotypes");
}

void free_factor(Ctx *c) {
    tc_invalidate_factor_maps(c);
    dev_free(&c->W);
    dev_free(&c->Wd);
    dev_free(&c->Linv);
    dev_free(&c->LinvT);
    dev_free(&c->Linv_hi);
    dev_free(&c->Linv_lo);
    dev_free(&c->diag64);
    dev_free(&c->diag64_inv);
    dev_free(&c->diag_ctr);
    dev_free(&c->pool);
    dev_free(&c->ltab);
    dev_free(&c->colbuf);
    dev_free(&c->pan_hi);
    dev_free(&c->pan_lo);
    dev_free(&c->colmax);
    dev_free(&c->precmap);
    c->pool_bytes = 0;
    c->w_bytes = 0;
    c->factored = false;
}

void free_build(Ctx *c) {
    if (c->build_borrowed) {  // another context owns these buffers
        c->g8 = nullptr;
        c->gf = nullptr;
        c->norms = nullptr;
        c->Kd = nullptr;
        c->Dd = nullptr;
        c->knorm2 = nullptr;
        c->build_borrowed = 0;
    }
    dev_free(&c->g8);
    dev_free(&c->gf);
    dev_free(&c->norms);
    dev_free(&c->Kd);
    dev_free(&c->Dd);
    dev_free(&c->knorm2);
    c->g_bytes = c->kd_bytes = c->dd_bytes = 0;
    c->built = false;
}

// dst reads the build products of src (same device, same tile edge): the
// packed genotypes, norms and kernel tiles are shared read-only -- nothing
// after the build writes them -- and the kernel statistics (||K||, the
// shift, the bound on |K|) are copied on dst's stream, after work that
// dst's stream already waits for.  src must outlive dst's use of them.
krr_status adopt_build(Ctx *dst, const Ctx *src) {
    if (!src->built || src->opt.tile != dst->opt.tile || src->opt.mode != dst->opt.mode ||
        src->opt.kernel != dst->opt.kernel || src->rr) {
        dst->last_error = "adopt_build: incompatible source context";
        return KRR_EINVAL;
    }
    if (dst->nt != src->nt || dst->b != src->b) free_factor(dst);
    free_build(dst);
    dst->g8 = src->g8;
    dst->gf = src->gf;
    dst->norms = src->norms;
    dst->Kd = src->Kd;
    dst->knorm2 = src->knorm2;
    dst->Dd = nullptr;
    dst->build_borrowed = 1;
    dst->g_bytes = src->g_bytes;
    dst->kd_bytes = src->kd_bytes;
    dst->dd_bytes = 0;
    dst->n = src->n;
    dst->m = src->m;
    dst->m_pad = src->m_pad;
    dst->b = src->b;
    dst->nt = src->nt;
    dst->n_pad = src->n_pad;
    dst->gamma = src->gamma;
    dst->nconf = 0;
    dst->rr = 0;
    const size_t red_count = src->red_cap;
    if (dst->red_cap < red_count) {
        KRR_TRY(dev_alloc(dst, &dst->red, red_count, "reduction buffer"));
        dst->red_cap = red_count;
    }
    if (!dst->hred && cudaMallocHost((void **)&dst->hred, 64 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        dst->hred = nullptr;
        dst->last_error = "pinned allocation failed";
        return KRR_ENOMEM;
    }
    KRR_CUDA_TRY(dst, cudaMemcpyAsync(dst->red + RED_KNORM2, src->red + RED_KNORM2,
                                      (RED_KBOUND - RED_KNORM2 + 1) * sizeof(double), cudaMemcpyDeviceToDevice,
                                      dst->stream));
    // the tensor map of the shared genotypes, which this context's Predict reads
    if (mixed(dst)) KRR_TRY(tc_bind_genotypes(dst));
    dst->built = true;
    dst->factored = false;
    return KRR_OK;
}

bool mixed(const Ctx *c) { return c->opt.mode == KRR_MODE_MIXED; }

}  // namespace krr

namespace {
// Scratch of the residual-norm reduction: the last norm_partial_count()
// doubles of the reduction buffer.
double *red_norm_part(Ctx *c) { return c->red + c->red_cap - norm_partial_count(); }

// Allocates (or keeps) the n_pad x p work vectors of the solve.
krr_status ensure_vectors(Ctx *c, int64_t p) {
    const int64_t cnt = c->n_pad * p;
    if (c->vec_cap < cnt) {
        KRR_TRY(dev_alloc(c, &c->ybuf, (size_t)cnt, "solve vectors"));
        KRR_TRY(dev_alloc(c, &c->zbuf, (size_t)cnt, "solve vectors"));
        KRR_TRY(dev_alloc(c, &c->abuf, (size_t)cnt, "solve vectors"));
        KRR_TRY(dev_alloc(c, &c->dabuf, (size_t)cnt, "solve vectors"));
        KRR_TRY(dev_alloc(c, &c->rbuf, (size_t)cnt, "residual"));
        c->vec_cap = cnt;
    }
    if (c->colsum_cap < p) {
        KRR_TRY(dev_alloc(c, &c->colsum, (size_t)p, "column sums"));
        c->colsum_cap = p;
    }
    return KRR_OK;
}

// A = (K + lambda I)^-1 ybuf into abuf with the stored factor, then
// refinement (mixed mode) or one residual for the report (info != NULL).
krr_status solve_device(Ctx *c, int64_t p, krr_solve_info *info) {
    cudaStream_t s = c->stream;
    const int64_t cnt = c->n_pad * p;
    KRR_CUDA_TRY(c, cudaMemcpyAsync(c->abuf, c->ybuf, cnt * sizeof(float), cudaMemcpyDeviceToDevice, s));
    // compulsory bytes of one pair of sweeps: the stored factor read twice
    // (diagonal inverses in FP32 plus the off-diagonal pool) and the vectors
    const double pool_used = mixed(c) ? (double)c->herr->pool_cursor
                                      : (double)c->nt * (c->nt - 1) / 2 * c->b * c->b * 4.0;
    const double factor_bytes_all = pool_used + (double)c->nt * c->b * c->b * 4.0;
    const double sweep_bytes = 2.0 * factor_bytes_all + 4.0 * (double)cnt * 4.0;
    const double sweep_flops = 2.0 * 2.0 * (double)c->n_pad * c->n_pad * p;
    int pr = prof_begin(c, KRR_PROF_SOLVE);
    KRR_TRY(solve_inplace(c, c->abuf, c->zbuf, p));
    prof_end(c, pr, sweep_flops, sweep_bytes);
    KRR_TRY(check_launch(c, "solve"));
    krr_solve_info si;
    memset(&si, 0, sizeof(si));
    krr_status st = KRR_OK;
    if (c->graph_mode) {
        // fixed number of refinement steps without host decisions; the final
        // relative residual is left in red[RED_RNORM..+1] for the caller
        const int iters = mixed(c) ? c->opt.ir_max : 0;
        for (int it = 0; it < iters; ++it) {
            KRR_TRY(launch_residual(c, c->ybuf, c->abuf, c->rbuf, p));
            launch_axpy_r(c->rbuf, c->dabuf, cnt, s);
            KRR_TRY(solve_inplace(c, c->dabuf, c->zbuf, p));
            launch_add_scaled(c->abuf, c->dabuf, 1.0f, cnt, s);
        }
        KRR_TRY(launch_residual(c, c->ybuf, c->abuf, c->rbuf, p));
        launch_reduce_norms(c->rbuf, c->ybuf, c->n_pad, p, c->red + RED_RNORM, red_norm_part(c), s);
        KRR_TRY(check_launch(c, "refinement (graph mode)"));
        if (info) *info = si;
        return KRR_OK;
    }
    const bool refine = mixed(c) && c->opt.ir_max > 0;
    if (refine || info) {
        double best = INFINITY;
        for (int it = 0;; ++it) {
            int rr = prof_begin(c, KRR_PROF_RESIDUAL);
            KRR_TRY(launch_residual(c, c->ybuf, c->abuf, c->rbuf, p));
            launch_reduce_norms(c->rbuf, c->ybuf, c->n_pad, p, c->red + RED_RNORM, red_norm_part(c), s);
            // the lower-triangle K tiles are read once by the row pass and
            // once by the column pass
            prof_end(c, rr, 2.0 * (double)c->n_pad * c->n_pad * p, 2.0 * (double)c->kd_bytes);
            KRR_TRY(check_launch(c, "residual"));
            KRR_CUDA_TRY(c, cudaMemcpyAsync(c->hred, c->red, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
            KRR_CUDA_TRY(c, cudaStreamSynchronize(s));
            const double ynorm = sqrt(c->hred[1]);
            const double rel = ynorm > 0 ? sqrt(c->hred[0]) / ynorm : sqrt(c->hred[0]);
            if (it < 32) si.history[it] = rel;
            si.rel_residual = rel;
            si.iterations = it;
            if (it == 0) best = rel;
            if (!(rel == rel) || rel > 1e300) {  // NaN or overflow
                st = KRR_ENOCONV;
                break;
            }
            if (it > 0 && rel > best) {
                // the last correction made things worse: the floor set by FP32
                // storage of K and A is reached -- undo it and keep the best
                launch_add_scaled(c->abuf, c->dabuf, -1.0f, cnt, s);
                si.rel_residual = best;
                si.converged = best <= c->opt.ir_tol ? 1 : 2;
                break;
            }
            if (rel <= c->opt.ir_tol) {
                si.converged = 1;
                break;
            }
            if (!refine) break;
            if (it >= c->opt.ir_max) {
                st = KRR_ENOCONV;
                break;
            }
            // stagnation: a step that did not halve the residual shows the
            // floor set by FP32 storage of K and A; a further step would only
            // move along it
            if (it > 0 && rel > 0.5 * best) {
                si.converged = 2;
                break;
            }
            best = std::min(best, rel);
            launch_axpy_r(c->rbuf, c->dabuf, cnt, s);
            int sr = prof_begin(c, KRR_PROF_SOLVE);
            KRR_TRY(solve_inplace(c, c->dabuf, c->zbuf, p));
            prof_end(c, sr, sweep_flops, sweep_bytes);
            launch_add_scaled(c->abuf, c->dabuf, 1.0f, cnt, s);
            KRR_TRY(check_launch(c, "refinement step"));
        }
    }
    if (info) *info = si;
    if (st == KRR_ENOCONV)
        c->last_error = "krr_solve: refinement stopped at relative residual " + std::to_string(si.rel_residual);
    return st;
}
}  // namespace

namespace krr {
// Buffers of a build over an n x n lower-triangle tile grid (tile edge from
// the options) with packed operand rows of m_pad columns; sets the shape
// fields of the context.
krr_status prepare_build(Ctx *c, int64_t n, int64_t m_pad, int keep_d) {
    const int64_t b = c->opt.tile;
    const int64_t nt = (n + b - 1) / b;
    if (nt != c->nt || b != c->b) free_factor(c);  // factor buffers depend on the tile grid
    const int64_t n_pad = nt * b;
    const size_t g_bytes = (size_t)n_pad * m_pad * (mixed(c) ? 1 : 4);
    const int64_t ntri = nt * (nt + 1) / 2;
    const size_t kd_bytes = (size_t)ntri * b * b * sizeof(float);
    if (c->g_bytes != g_bytes || c->kd_bytes != kd_bytes || c->b != b || c->nt != nt || c->build_borrowed) {
        free_build(c);
        if (mixed(c)) KRR_TRY(dev_alloc(c, &c->g8, g_bytes, "packed genotypes"));
        else KRR_TRY(dev_alloc(c, &c->gf, g_bytes / 4, "FP32 genotypes"));
        KRR_TRY(dev_alloc(c, &c->norms, (size_t)n_pad, "row norms"));
        KRR_TRY(dev_alloc(c, &c->Kd, (size_t)ntri * b * b, "kernel tiles"));
        // per-tile partial sums of K^2: one per 128 x 256 (tensor-core) or
        // 128 x 128 (CUDA-core) block
        const size_t per_tile = mixed(c) ? (size_t)(b / 128) * (b / 256) : (size_t)(b / 128) * (b / 128);
        KRR_TRY(dev_alloc(c, &c->knorm2, (size_t)2 * ntri * per_tile, "tile norms"));
        c->g_bytes = g_bytes;
        c->kd_bytes = kd_bytes;
    }
    const size_t dd_bytes = keep_d ? (size_t)ntri * b * b * sizeof(uint32_t) : 0;
    if (dd_bytes != c->dd_bytes) {
        KRR_TRY(dev_alloc(c, &c->Dd, dd_bytes / sizeof(uint32_t), "distance tiles"));
        c->dd_bytes = dd_bytes;
    }
    c->n = n;
    c->m_pad = m_pad;
    c->b = b;
    c->nt = nt;
    c->n_pad = n_pad;
    const size_t red_count = RED_MINPIV + (size_t)nt * (b / 64) + (size_t)nt + 16 + (size_t)norm_partial_count();
    if (c->red_cap < red_count) {
        KRR_TRY(dev_alloc(c, &c->red, red_count, "reduction buffer"));
        c->red_cap = red_count;
    }
    if (!c->hred && cudaMallocHost((void **)&c->hred, 64 * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->hred = nullptr;
        c->last_error = "pinned allocation failed";
        return KRR_ENOMEM;
    }
    return KRR_OK;
}
krr_status ensure_lookahead_stream(Ctx *c) {
    if (c->la_stream) return KRR_OK;
    if (c->graph_mode) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        KRR_CUDA_TRY(c, cudaStreamIsCapturing(c->stream, &cs));
        if (cs != cudaStreamCaptureStatusNone) return KRR_OK;  // made before the capture, or not at all
    }
    int lo = 0, hi = 0;
    KRR_CUDA_TRY(c, cudaDeviceGetStreamPriorityRange(&lo, &hi));
    KRR_CUDA_TRY(c, cudaStreamCreateWithPriority(&c->la_stream, cudaStreamNonBlocking, hi));
    for (cudaEvent_t &e : c->la_ev) KRR_CUDA_TRY(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return KRR_OK;
}

}  // namespace krr

extern "C" {

void krr_default_options(krr_options *opt) {
    if (!opt) return;
    opt->tile = 1024;
    opt->mode = KRR_MODE_MIXED;
    opt->allow_fp8 = 1;
    opt->eps = 6e-4;
    opt->ir_tol = 1e-7;
    opt->ir_max = 30;
    opt->diag_fp64 = 0;
    opt->wait_budget_ns = 2000000000LL;
    opt->prec_rule = KRR_RULE_LAMBDA;
    opt->kernel = KRR_KERNEL_GAUSSIAN;
    opt->lookahead = 1;
    opt->reserved = 0;
}

krr_status krr_create(krr_ctx **out, const krr_options *opt, void *stream) {
    if (!out) {
        g_create_error = "out is NULL";
        return KRR_EINVAL;
    }
    *out = nullptr;
    krr_options o;
    krr_default_options(&o);
    if (opt) o = *opt;
    // a power of two: the diagonal step inverts the factor by recursive
    // doubling over 64-wide blocks
    if (o.tile < 256 || o.tile > 4096 || (o.tile & (o.tile - 1)) != 0) {
        g_create_error = "tile must be a power of two in [256, 4096]";
        return KRR_EINVAL;
    }
    if (o.mode != KRR_MODE_MIXED && o.mode != KRR_MODE_FP32) {
        g_create_error = "unknown mode";
        return KRR_EINVAL;
    }
    if (!(o.eps > 0.0) || !(o.ir_tol > 0.0) || o.ir_max < 0 || o.ir_max > 1000) {
        g_create_error = "eps and ir_tol must be positive, ir_max in [0, 1000]";
        return KRR_EINVAL;
    }
    if (o.prec_rule != KRR_RULE_LAMBDA && o.prec_rule != KRR_RULE_KNORM) {
        g_create_error = "unknown precision rule";
        return KRR_EINVAL;
    }
    if (o.kernel != KRR_KERNEL_GAUSSIAN && o.kernel != KRR_KERNEL_IBS) {
        g_create_error = "unknown kernel function";
        return KRR_EINVAL;
    }
    if ((o.lookahead != 0 && o.lookahead != 1) || o.reserved != 0) {
        g_create_error = "lookahead must be 0 or 1 and reserved 0";
        return KRR_EINVAL;
    }
    krr_ctx *c = new (std::nothrow) krr_ctx();
    if (!c) {
        g_create_error = "out of host memory";
        return KRR_ENOMEM;
    }
    c->opt = o;
    c->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
        cudaGetLastError();
        g_create_error = "no usable CUDA device";
        delete c;
        return KRR_ECUDA;
    }
    if (cudaMalloc((void **)&c->derr, sizeof(DevErrors)) != cudaSuccess ||
        cudaMallocHost((void **)&c->herr, sizeof(DevErrors)) != cudaSuccess) {
        cudaGetLastError();
        g_create_error = "allocation of the error record failed";
        krr_destroy(c);
        return KRR_ENOMEM;
    }
    if (mixed(c)) {
        krr_status s = tc_init(c);
        if (s != KRR_OK) {
            g_create_error = c->last_error;
            krr_destroy(c);
            return s;
        }
    }
    *out = c;
    return KRR_OK;
}

void krr_destroy(krr_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    free_factor(c);
    free_build(c);
    dev_free(&c->derr);
    if (c->herr) cudaFreeHost(c->herr);
    if (c->hred) cudaFreeHost(c->hred);
    dev_free(&c->red);
    dev_free(&c->ybuf);
    dev_free(&c->zbuf);
    dev_free(&c->rbuf);
    dev_free(&c->abuf);
    dev_free(&c->dabuf);
    dev_free(&c->pred_part);
    dev_free(&c->pred_out);
    dev_free(&c->colsum);
    dev_free(&c->sw_flags);
    dev_free(&c->ts_v0);
    dev_free(&c->ts_xt);
    dev_free(&c->ts_v1);
    if (c->ts_aux) cudaFree(c->ts_aux);
    c->ts_aux = nullptr;
    dev_free(&c->g_yt);
    dev_free(&c->g_gp);
    dev_free(&c->g_aw);
    dev_free(&c->g_part);
    dev_free(&c->g_sq);
    dev_free(&c->g_tpart);
    dev_free(&c->g_kpart);
    dev_free(&c->g_scal);
    dev_free(&c->t8);
    dev_free(&c->tnorms);
    dev_free(&c->conf);
    dev_free(&c->tconf);
    if (c->stage) cudaFree(c->stage);
    if (c->la_stream) {
        cudaStreamSynchronize(c->la_stream);
        cudaStreamDestroy(c->la_stream);
    }
    for (cudaEvent_t &e : c->la_ev)
        if (e) cudaEventDestroy(e);
    tc_free(c);
    rr_free(c);
    if (c->prof) {
        ProfState *ps = (ProfState *)c->prof;
        for (const ProfRec &r : ps->recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        for (cudaEvent_t e : ps->pool) cudaEventDestroy(e);
        delete ps;
    }
    delete c;
}

const char *krr_last_error(const krr_ctx *c) {
    if (!c) return g_create_error.c_str();
    return c->last_error.c_str();
}

krr_status krr_sync(krr_ctx *c) {
    if (!c) return KRR_EINVAL;
    KRR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return KRR_OK;
}

krr_status krr_set_keep_distances(krr_ctx *c, int32_t keep) {
    if (!c) return KRR_EINVAL;
    c->keep_distances = keep ? 1 : 0;
    return KRR_OK;
}

static krr_status build_common(krr_ctx *c, const int8_t *G, int64_t n, int64_t m, int64_t ldg, const float *C,
                        int64_t nc, int64_t ldc, double gamma) {
    if (!c) return KRR_EINVAL;
    if (nc < 0 || nc > CONF_MAX || (nc > 0 && (!C || ldc < nc || is_ibs(c)))) {
        c->last_error = "krr_build_kernel_conf: need 0 <= nc <= 16, C != NULL and ldc >= nc when nc > 0, "
                        "and the Gaussian kernel";
        return KRR_EINVAL;
    }
    if (!G || n < 1 || m < 1 || m > (int64_t(1) << (is_ibs(c) ? 21 : 22)) || ldg < m ||
        (!is_ibs(c) && (!(gamma > 0.0) || !isfinite(gamma)))) {
        c->last_error = "krr_build_kernel: need G != NULL, n >= 1, 1 <= m <= 2^22 (IBS: 2^21), ldg >= m, "
                        "0 < gamma < inf (Gaussian kernel)";
        return KRR_EINVAL;
    }
    c->built = false;
    c->factored = false;
    c->rr = 0;
    c->rr_m = c->rr_nc = 0;
    const int64_t b = c->opt.tile;
    const int64_t nt = (n + b - 1) / b;
    const int64_t n_pad = nt * b;
    const int64_t m_pad = (encoded_width(c, m) + 127) / 128 * 128;
    const size_t g_bytes = (size_t)n_pad * m_pad * (mixed(c) ? 1 : 4);
    c->m = m;  // set before packing: the IBS encoding and kernel function read it
    c->gamma = gamma;
    KRR_TRY(prepare_build(c, n, m_pad, c->keep_distances));
    int pr = prof_begin(c, KRR_PROF_PACK);
    KRR_TRY(pack(c, G, n, m, ldg, n_pad, c->g8, c->gf, c->norms));
    prof_end(c, pr, 0.0, (double)n * m + (double)g_bytes);
    c->nconf = 0;
    if (nc > 0) {
        const size_t cnt = (size_t)n_pad * CONF_MAX;
        if (c->conf_cap < cnt) {
            KRR_TRY(dev_alloc(c, &c->conf, cnt, "confounders"));
            c->conf_cap = cnt;
        }
        KRR_TRY(load_conf(c, C, n, nc, ldc, n_pad, c->conf));
        c->nconf = nc;
    }
    pr = prof_begin(c, KRR_PROF_BUILD);
    if (mixed(c)) {
        KRR_TRY(tc_build(c));
    } else {
        launch_build_simt(c);
    }
    // algorithmic work: 2 M multiply-adds per entry of the lower-triangle
    // tiles (2 x 2M for the IBS encoding); compulsory bytes: the K tiles
    // written once (FP32)
    const double ntri = (double)nt * (nt + 1) / 2;
    prof_end(c, pr, 2.0 * ntri * b * b * (double)encoded_width(c, m), (double)c->kd_bytes);
    KRR_TRY(check_launch(c, "build"));
    launch_kernel_sumsq(c, c->red + RED_KNORM2);
    KRR_TRY(check_launch(c, "kernel norm"));
    c->built = true;
    return KRR_OK;
}

krr_status krr_build_kernel(krr_ctx *c, const int8_t *G, int64_t n, int64_t m, int64_t ldg, double gamma) {
    return build_common(c, G, n, m, ldg, nullptr, 0, 0, gamma);
}

krr_status krr_build_kernel_conf(krr_ctx *c, const int8_t *G, int64_t n, int64_t m, int64_t ldg, const float *C,
                                 int64_t nc, int64_t ldc, double gamma) {
    return build_common(c, G, n, m, ldg, C, nc, ldc, gamma);
}

namespace {

// Lookahead of the factorisation (mixed mode, outside graph capture, FP32
// diagonal step).  Per step, the diagonal step of the next column runs on
// `ctas` CTAs beside the first `tiles` target tiles of the update (after its
// diagonal target) on the other SMs.  The choice comes from a model of the
// two kernels measured on GB300 (152 SMs) while they share the GPU:
//   diagonal step on R CTAs: T(R) = a + c / R, a chain of b / 64 block
//     factorisations (a = 600 us at b = 1024, proportional to b) plus work
//     spread over the CTAs (c = 13 CTA-ms at b = 1024, proportional to b^3);
//     on 16 / 24 / 32 / 48 CTAs it took 1.42 / 1.11 / 0.95 / 0.81 ms, on 136
//     alone 0.59 ms;
//   trailing update: about 8.3 TF/s per SM (2 b^3 per off-diagonal target).
// The plan minimises the step's time: T(R) while the update fits beside the
// diagonal step, else T(R) plus the rest of the update on every SM; the
// launch of the diagonal target alone adds about 25 us.  When the update is
// small (the last steps, small problems) the plain sequence is faster: the
// diagonal step alone on 136 CTAs, 0.59 ms at b = 1024, then the update.  The
// update part beside it is sized 30 % above T(R): if it ended first, the
// other SMs would idle until the diagonal step ends, while if it ends last
// only the diagonal step's R SMs wait.  At N = 131072 the factorisation
// takes 660 ms this way and 697 ms in sequence; fixed R = 24 and R = 48 gave
// the same 658-662 ms, R = 8 690 ms.
//
// A context of a batch (graph mode) shares the GPU with the other problems
// and its kernels are capped per class: there the diagonal step keeps its
// class cap and the whole rest of the update runs beside it (on the
// cross-validation workload, 64 problems: 170.4-171.8 ms per run against
// 172.9-175.4 ms in sequence).
struct LookaheadPlan {
    bool on = false;
    int64_t ctas = 0, tiles = 0;  // 0 CTAs: the class limit
    int64_t upd_ctas = 0;         // CTAs of the update launch beside it (0: class limit)
};

bool lookahead_enabled(const Ctx *c) {
    // in graph mode the second stream must exist before the capture began
    if (c->graph_mode && !c->la_stream) return false;
    return c->opt.lookahead && mixed(c) && !c->opt.diag_fp64 && c->nt >= 3 && c->num_sms >= 32;
}

LookaheadPlan lookahead_plan(const Ctx *c, int64_t k) {
    LookaheadPlan pl;
    const int64_t u = c->nt - k - 1;
    const int64_t tiles = u * (u + 1) / 2;
    if (tiles < 2) return pl;
    if (c->graph_mode) {
        pl.on = true;
        pl.tiles = tiles - 1;
        return pl;
    }
    const double bd = (double)c->b, rel = bd / 1024.0;
    const double a_us = 600.0 * rel, c_us = 13000.0 * rel * rel * rel;
    const double tile_sm_us = 2.0 * bd * bd * bd / 8.3e12 * 1e6;  // SM-microseconds per target tile
    const double work = (double)(tiles - 1) * tile_sm_us;
    const int64_t sms = c->num_sms;
    // in sequence: the diagonal step alone on 136 CTAs (0.59 ms at b = 1024),
    // then the whole update on every SM
    double best = 590.0 * rel + (work + tile_sm_us) / (double)sms;
    static const int64_t cand[] = {16, 20, 24, 32, 48, 64, 96, 128};
    for (int64_t r : cand) {
        if (r + 16 > sms) break;
        const double td = a_us + c_us / (double)r;
        const double beside = (double)(sms - r) * td;  // SM-us of update beside the diagonal step
        // plus the launch of the diagonal target alone (about 25 us)
        const double t = 25.0 + ((work <= beside) ? td : td + (work - beside) / (double)sms);
        if (t < best) {
            best = t;
            pl.ctas = r;
            pl.upd_ctas = sms - r;
            pl.tiles = std::min<int64_t>(tiles - 1, (int64_t)std::ceil(1.3 * beside / tile_sm_us));
        }
    }
    pl.on = pl.ctas > 0 && pl.tiles > 0;
    return pl;
}

}  // namespace

krr_status krr_factor(krr_ctx *c, double lambda, krr_factor_info *info) {
    if (!c) return KRR_EINVAL;
    if (!c->built) {
        c->last_error = "krr_factor: no kernel built";
        return KRR_ESTATE;
    }
    if (!isfinite(lambda)) {
        c->last_error = "krr_factor: lambda must be finite";
        return KRR_EINVAL;
    }
    c->factored = false;
    c->lambda = lambda;
    const int64_t b = c->b, nt = c->nt, bb = b * b;
    const int64_t noff = nt * (nt - 1) / 2;
    const bool mx = mixed(c);
    cudaStream_t s = c->stream;
    // buffers (kept across factorisations of the same shape)
    const size_t w_bytes = (size_t)noff * bb * (mx ? 2 : 4);
    if (!c->Wd || c->w_bytes != w_bytes) {
        free_factor(c);
        if (noff > 0) {
            if (mx) {
                KRR_TRY(dev_alloc(c, (__half **)&c->W, (size_t)noff * bb, "trailing tiles"));
            } else {
                KRR_TRY(dev_alloc(c, (float **)&c->W, (size_t)noff * bb, "trailing tiles"));
            }
        }
        c->w_bytes = w_bytes;
        KRR_TRY(dev_alloc(c, &c->Wd, (size_t)nt * bb, "diagonal tiles"));
        KRR_TRY(dev_alloc(c, &c->Linv, (size_t)nt * bb, "diagonal inverses"));
        KRR_TRY(dev_alloc(c, &c->LinvT, (size_t)nt * bb, "transposed diagonal inverses"));
        KRR_TRY(dev_alloc(c, &c->diag64, (size_t)bb, "FP64 diagonal scratch"));
        KRR_TRY(dev_alloc(c, &c->diag64_inv, (size_t)2 * bb, "FP64 inverse scratch"));
        KRR_TRY(dev_alloc(c, &c->diag_ctr, (size_t)diag_counter_count(b), "diagonal-step counters"));
        const size_t pool_bytes = (size_t)std::max<int64_t>(noff, 1) * bb * 4;
        KRR_TRY(dev_alloc(c, &c->pool, pool_bytes, "factor pool"));
        c->pool_bytes = pool_bytes;
        KRR_TRY(dev_alloc(c, &c->ltab, (size_t)std::max<int64_t>(noff, 1), "tile table"));
        KRR_TRY(dev_alloc(c, &c->precmap, (size_t)nt * nt, "precision map"));
        if (mx) {
            KRR_TRY(dev_alloc(c, &c->Linv_hi, (size_t)nt * bb, "inverse split"));
            KRR_TRY(dev_alloc(c, &c->Linv_lo, (size_t)nt * bb, "inverse split"));
            const size_t colt = (size_t)std::max<int64_t>(nt - 1, 1);
            KRR_TRY(dev_alloc(c, &c->colbuf, colt * bb, "column buffer"));
            KRR_TRY(dev_alloc(c, &c->pan_hi, colt * bb, "operand panel"));
            KRR_TRY(dev_alloc(c, &c->pan_lo, colt * bb, "operand panel"));
            KRR_TRY(dev_alloc(c, &c->colmax, colt * (size_t)tile_max_partials(b), "column maxima"));
        }
    }
    // reset the error record, the precision map and (fp32 mode) the tile
    // table on the device: no host data, so the sequence can be captured
    launch_factor_init(c);
    KRR_TRY(check_launch(c, "factor init"));
    const double bd = (double)b;
    // Lookahead: the diagonal step of column k + 1 needs only the diagonal
    // target of step k's trailing update.  That tile is updated first; the
    // diagonal step then runs on a second stream on la_ctas CTAs while the
    // update goes on with the other SMs, and the rest of the update takes
    // every SM again once the diagonal step is done.
    const bool la_on = mx && lookahead_enabled(c);
    if (la_on) KRR_TRY(ensure_lookahead_stream(c));
    bool diag_ahead = false;  // diagonal step k already issued by step k - 1
    for (int64_t k = 0; k < nt; ++k) {
        if (!diag_ahead) {
            int pr = prof_begin(c, KRR_PROF_DIAG);
            KRR_TRY(diag_step(c, k));
            prof_end(c, pr, 2.0 * bd * bd * bd / 3.0, 0.0);
            KRR_TRY(check_launch(c, "diagonal step"));
        }
        diag_ahead = false;
        if (k + 1 >= nt) break;
        const double u = (double)(nt - k - 1);
        // algorithmic work: triangular solve b^3 per panel tile; update 2 b^3
        // per off-diagonal target and b^3 per diagonal target
        const double trsm_flops = u * bd * bd * bd;
        const double upd_flops = (u * (u - 1) / 2.0) * 2.0 * bd * bd * bd + u * bd * bd * bd;
        if (mx) {
            int pr = prof_begin(c, KRR_PROF_TRSM);
            KRR_TRY(tc_trsm(c, k));
            prof_end(c, pr, trsm_flops, 0.0);
            pr = prof_begin(c, KRR_PROF_CAST);
            launch_column_cast(c, k);
            prof_end(c, pr, 0.0, u * bd * bd * (4.0 + 2.0));
            KRR_TRY(check_launch(c, "column cast"));
            const int64_t tiles = (nt - k - 1) * (nt - k) / 2;
            const LookaheadPlan la = la_on ? lookahead_plan(c, k) : LookaheadPlan();
            if (la.on) {
                // the diagonal target (k + 1, k + 1), b^3 flops
                pr = prof_begin(c, KRR_PROF_UPDATE_SHARED);
                KRR_TRY(tc_update(c, k, 0, 1, 0));
                prof_end(c, pr, bd * bd * bd, 0.0);
                KRR_CUDA_TRY(c, cudaEventRecord(c->la_ev[0], s));
                KRR_CUDA_TRY(c, cudaStreamWaitEvent(c->la_stream, c->la_ev[0], 0));
                pr = prof_begin(c, KRR_PROF_DIAG, c->la_stream);
                KRR_TRY(diag_step(c, k + 1, c->la_stream, la.ctas));
                prof_end(c, pr, 2.0 * bd * bd * bd / 3.0, 0.0, c->la_stream);
                KRR_TRY(check_launch(c, "diagonal step"));
                KRR_CUDA_TRY(c, cudaEventRecord(c->la_ev[1], c->la_stream));
                // the targets that run beside the diagonal step, then the
                // rest on every SM (each launch timed on its own: the wait
                // for the diagonal step lies between them)
                const int64_t side = std::min<int64_t>(tiles - 1, la.tiles);
                pr = prof_begin(c, KRR_PROF_UPDATE_SHARED);
                KRR_TRY(tc_update(c, k, 1, side, la.upd_ctas));
                prof_end(c, pr, update_flops(c, k, 1, side), 0.0);
                KRR_CUDA_TRY(c, cudaStreamWaitEvent(s, c->la_ev[1], 0));
                if (1 + side < tiles) {
                    pr = prof_begin(c, KRR_PROF_UPDATE);
                    KRR_TRY(tc_update(c, k, 1 + side, tiles - 1 - side, 0));
                    prof_end(c, pr, update_flops(c, k, 1 + side, tiles - 1 - side), 0.0);
                }
                diag_ahead = true;
            } else {
                pr = prof_begin(c, KRR_PROF_UPDATE);
                KRR_TRY(tc_update(c, k));
                prof_end(c, pr, upd_flops, 0.0);
            }
        } else {
            int pr = prof_begin(c, KRR_PROF_TRSM);
            launch_trsm_simt(c, k);
            prof_end(c, pr, trsm_flops, 0.0);
            KRR_TRY(check_launch(c, "trsm"));
            pr = prof_begin(c, KRR_PROF_UPDATE);
            launch_update_simt(c, k);
            prof_end(c, pr, upd_flops, 0.0);
            KRR_TRY(check_launch(c, "update"));
        }
    }
    if (c->graph_mode) {  // results are read after the captured sequence ran
        c->factored = true;
        if (info) memset(info, 0, sizeof(*info));
        return KRR_OK;
    }
    KRR_CUDA_TRY(c, cudaMemcpyAsync(c->herr, c->derr, sizeof(DevErrors), cudaMemcpyDeviceToHost, s));
    KRR_CUDA_TRY(c, cudaStreamSynchronize(s));
    const DevErrors &he = *c->herr;
    if (info) {
        info->nt = nt;
        info->tiles_fp32 = mx ? he.fp32_tiles : noff;
        info->tiles_fp16 = mx ? he.fp16_tiles : 0;
        info->tiles_e4m3 = mx ? he.fp8_tiles : 0;
        info->factor_bytes = mx ? he.pool_cursor : noff * bb * 4;
        info->bad_tile = he.bad_tile;
        info->bad_column = he.bad_column;
        info->min_pivot = he.min_pivot;
    }
    if (he.code == KRR_ENOTPD) {
        c->last_error = "krr_factor: matrix not positive definite (pivot <= 0 at column " +
                        std::to_string(he.bad_column) + ")";
        return KRR_ENOTPD;
    }
    if (he.code != 0) {
        c->last_error = "krr_factor: device error " + std::to_string(he.code);
        return (krr_status)he.code;
    }
    c->factored = true;
    return KRR_OK;
}

krr_status krr_solve(krr_ctx *c, const float *Y, int64_t p, int64_t ldy, float *A, int64_t lda,
                     krr_solve_info *info) {
    if (!c) return KRR_EINVAL;
    if (!c->factored) {
        c->last_error = "krr_solve: no factorisation";
        return KRR_ESTATE;
    }
    if (!Y || !A || p < 1 || ldy < p || lda < p) {
        c->last_error = "krr_solve: need Y, A != NULL, p >= 1, ldy >= p, lda >= p";
        return KRR_EINVAL;
    }
    KRR_TRY(ensure_vectors(c, p));
    // the sweep and residual kernels record an expired wait in the error
    // record (the factor stays valid: they do not write it)
    KRR_CUDA_TRY(c, cudaMemsetAsync(&c->derr->code, 0, sizeof(int32_t), c->stream));
    KRR_TRY(load_rows_f32(c, Y, c->n, p, ldy, c->n_pad, c->ybuf));
    krr_status st = solve_device(c, p, info);
    if (st != KRR_OK && st != KRR_ENOCONV) return st;
    KRR_TRY(store_rows_f32(c, c->abuf, c->n, p, A, lda));
    if (!c->graph_mode) {
        KRR_CUDA_TRY(c, cudaMemcpyAsync(&c->herr->code, &c->derr->code, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                        c->stream));
        KRR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        const int32_t code = c->herr->code;
        if (code != 0) {
            c->last_error = "krr_solve: device error " + std::to_string(code) +
                            (code == KRR_ETIMEOUT ? " (a bounded device wait ran out)" : "");
            return (krr_status)code;
        }
    }
    return st;
}

krr_status krr_set_wait_budget(krr_ctx *c, int64_t ns) {
    if (!c) return KRR_EINVAL;
    if (ns < 1) {
        c->last_error = "krr_set_wait_budget: the budget must be positive";
        return KRR_EINVAL;
    }
    c->opt.wait_budget_ns = ns;
    return KRR_OK;
}

static krr_status predict_common(krr_ctx *c, const int8_t *T, int64_t n_test, int64_t ldt, const float *Ct, int64_t ldct,
                          const float *A, int64_t lda, int64_t p, float *Yt, int64_t ldyt) {
    if (!c) return KRR_EINVAL;
    if (!c->built) {
        c->last_error = "krr_predict: no kernel built";
        return KRR_ESTATE;
    }
    if (!T || !A || !Yt || n_test < 1 || ldt < c->m || p < 1 || p > 256 || lda < p || ldyt < p) {
        c->last_error = "krr_predict: bad arguments (need 1 <= p <= 256, ldt >= m, lda, ldyt >= p)";
        return KRR_EINVAL;
    }
    if (c->rr) {
        c->last_error = "krr_predict: the context holds a ridge-regression Gram matrix: use krr_rr_predict";
        return KRR_EINVAL;
    }
    if ((c->nconf > 0) != (Ct != nullptr) || (Ct && ldct < c->nconf)) {
        c->last_error = c->nconf > 0 ? "krr_predict: the kernel has confounders: use krr_predict_conf with the "
                                       "held-out rows' confounders (ldct >= nc)"
                                     : "krr_predict_conf: the kernel was built without confounders";
        return KRR_EINVAL;
    }
    const bool mx = mixed(c);
    const int64_t rows_pad = (n_test + 127) / 128 * 128;
    const size_t tbytes = (size_t)rows_pad * c->m_pad * (mx ? 1 : 4);
    if (c->t_cap < tbytes) {
        KRR_TRY(dev_alloc(c, &c->t8, tbytes, "test genotypes"));
        c->t_cap = tbytes;
    }
    if (c->tnorm_cap < (size_t)rows_pad) {
        KRR_TRY(dev_alloc(c, &c->tnorms, (size_t)rows_pad, "test norms"));
        c->tnorm_cap = rows_pad;
    }
    const int64_t cnt = c->n_pad * p;
    if (c->vec_cap < cnt) {
        KRR_TRY(dev_alloc(c, &c->ybuf, (size_t)cnt, "solve vectors"));
        KRR_TRY(dev_alloc(c, &c->zbuf, (size_t)cnt, "solve vectors"));
        KRR_TRY(dev_alloc(c, &c->abuf, (size_t)cnt, "solve vectors"));
        KRR_TRY(dev_alloc(c, &c->dabuf, (size_t)cnt, "solve vectors"));
        KRR_TRY(dev_alloc(c, &c->rbuf, (size_t)cnt, "residual"));
        c->vec_cap = cnt;
    }
    const int64_t nblk = c->n_pad / 128;  // partial products per 128 training rows
    const size_t part = (size_t)nblk * rows_pad * p;
    if (c->pred_part_cap < part) {
        KRR_TRY(dev_alloc(c, &c->pred_part, part, "predict partials"));
        c->pred_part_cap = part;
    }
    if (c->pred_out_cap < (size_t)rows_pad * p) {
        KRR_TRY(dev_alloc(c, &c->pred_out, (size_t)rows_pad * p, "predictions"));
        c->pred_out_cap = (size_t)rows_pad * p;
    }
    KRR_TRY(pack(c, T, n_test, c->m, ldt, rows_pad, mx ? c->t8 : nullptr,
                 mx ? nullptr : (float *)c->t8, c->tnorms));
    float *aw = c->dabuf;  // padded copy of the weights
    KRR_TRY(load_rows_f32(c, A, c->n, p, lda, c->n_pad, aw));
    const float *tconf = nullptr;
    if (c->nconf > 0) {
        const size_t cnt = (size_t)rows_pad * CONF_MAX;
        if (c->tconf_cap < cnt) {
            KRR_TRY(dev_alloc(c, &c->tconf, cnt, "held-out confounders"));
            c->tconf_cap = cnt;
        }
        KRR_TRY(load_conf(c, Ct, n_test, c->nconf, ldct, rows_pad, c->tconf));
        tconf = c->tconf;
    }
    float *out = c->pred_out;
    if (mx && c->colsum_cap < p) {
        KRR_TRY(dev_alloc(c, &c->colsum, (size_t)p, "column sums"));
        c->colsum_cap = p;
    }
    int pr = prof_begin(c, KRR_PROF_PREDICT);
    if (mx) {
        // products of the shifted kernel K - c, then + c (1^T A) in FP64
        const double *shift = c->red + RED_KSHIFT;
        launch_colsum(aw, c->n_pad, p, c->colsum, c->stream);
        // the tensor-core epilogue holds at most 32 weight columns (16 with
        // confounders, which take the other 16 slots of a staged row): chunk p
        const int64_t chunk = c->nconf ? 16 : 32;
        for (int64_t q0 = 0; q0 < p; q0 += chunk) {
            const int64_t pc = std::min<int64_t>(chunk, p - q0);
            KRR_TRY(tc_predict(c, c->t8, c->tnorms, n_test, rows_pad, aw + q0, p, pc, c->pred_part, shift, tconf));
            launch_predict_reduce(c->pred_part, nblk, rows_pad, n_test, pc, out + q0, p, c->stream, shift,
                                  c->colsum + q0);
        }
    } else {
        launch_predict_simt(c, (const float *)c->t8, c->tnorms, n_test, rows_pad, aw, p,
                            c->pred_part, tconf);
        launch_predict_reduce(c->pred_part, nblk, rows_pad, n_test, p, out, p, c->stream);
    }
    prof_end(c, pr, 2.0 * (double)n_test * c->n * encoded_width(c, c->m) + 2.0 * (double)n_test * c->n * p, 0.0);
    KRR_TRY(check_launch(c, "predict"));
    return store_rows_f32(c, out, n_test, p, Yt, ldyt);
}

krr_status krr_predict(krr_ctx *c, const int8_t *T, int64_t n_test, int64_t ldt, const float *A, int64_t lda,
                       int64_t p, float *Yt, int64_t ldyt) {
    return predict_common(c, T, n_test, ldt, nullptr, 0, A, lda, p, Yt, ldyt);
}

krr_status krr_predict_conf(krr_ctx *c, const int8_t *T, int64_t n_test, int64_t ldt, const float *Ct,
                            int64_t ldct, const float *A, int64_t lda, int64_t p, float *Yt, int64_t ldyt) {
    if (!c) return KRR_EINVAL;
    if (!Ct) {
        c->last_error = "krr_predict_conf: Ct is NULL";
        return KRR_EINVAL;
    }
    return predict_common(c, T, n_test, ldt, Ct, ldct, A, lda, p, Yt, ldyt);
}

krr_status krr_get_precision_map(krr_ctx *c, uint8_t *map, int64_t cap, int64_t *nt) {
    if (!c) return KRR_EINVAL;
    if (!c->factored) {
        c->last_error = "krr_get_precision_map: no factorisation";
        return KRR_ESTATE;
    }
    if (nt) *nt = c->nt;
    if (!map) return KRR_OK;
    if (cap < c->nt * c->nt) {
        c->last_error = "krr_get_precision_map: map_capacity < nt * nt";
        return KRR_EINVAL;
    }
    KRR_CUDA_TRY(c, cudaMemcpyAsync(map, c->precmap, (size_t)c->nt * c->nt,
                                    is_device_ptr(map) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                    c->stream));
    KRR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return KRR_OK;
}

}  // extern "C"

// Tile-to-dense copies for tests --------------------------------------------
namespace {
template <typename T>
__global__ void tiles_to_dense_kernel(const T *tiles, int64_t b, int64_t n, T *dst, int64_t ld) {
    const int64_t t = blockIdx.y;
    int64_t ti, tj;
    tri_decode(t, &ti, &tj);
    const T *src = tiles + t * b * b;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < b * b;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = ti * b + e / b, q = tj * b + e % b;
        if (r < n && q < n) dst[r * ld + q] = src[e];
    }
}

template <typename T>
krr_status tiles_to_dense(Ctx *c, const T *tiles, T *dst, int64_t ld) {
    const int64_t ntri = c->nt * (c->nt + 1) / 2;
    T *ddst = dst;
    const bool dev = is_device_ptr(dst);
    if (!dev) {
        KRR_TRY(stage(c, (size_t)c->n * ld * sizeof(T)));
        ddst = (T *)c->stage;
        KRR_CUDA_TRY(c, cudaMemcpyAsync(ddst, dst, (size_t)c->n * ld * sizeof(T),
                                        cudaMemcpyHostToDevice, c->stream));
    }
    count_launch(), tiles_to_dense_kernel<T><<<dim3(64, (unsigned)ntri), 256, 0, c->stream>>>(tiles, c->b, c->n, ddst, ld);
    KRR_TRY(check_launch(c, "tiles to dense"));
    if (!dev)
        KRR_CUDA_TRY(c, cudaMemcpyAsync(dst, ddst, (size_t)c->n * ld * sizeof(T),
                                        cudaMemcpyDeviceToHost, c->stream));
    KRR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return KRR_OK;
}
}  // namespace

extern "C" krr_status krr_get_distances(krr_ctx *c, uint32_t *D, int64_t ldd) {
    if (!c) return KRR_EINVAL;
    if (!c->built || !c->Dd) {
        c->last_error = "krr_get_distances: build with krr_set_keep_distances(ctx, 1) first";
        return KRR_ESTATE;
    }
    if (!D || ldd < c->n) return KRR_EINVAL;
    return tiles_to_dense<uint32_t>(c, c->Dd, D, ldd);
}

extern "C" krr_status krr_get_kernel(krr_ctx *c, float *K, int64_t ldk) {
    if (!c) return KRR_EINVAL;
    if (!c->built) {
        c->last_error = "krr_get_kernel: no kernel built";
        return KRR_ESTATE;
    }
    if (!K || ldk < c->n) return KRR_EINVAL;
    return tiles_to_dense<float>(c, c->Kd, K, ldk);
}

extern "C" krr_status krr_set_profiling(krr_ctx *c, int32_t on) {
    if (!c) return KRR_EINVAL;
    if (on && !c->prof) {
        c->prof = new (std::nothrow) ProfState();
        if (!c->prof) return KRR_ENOMEM;
    }
    c->prof_on = on ? 1 : 0;
    return KRR_OK;
}

extern "C" krr_status krr_get_profile(krr_ctx *c, krr_profile *out, int32_t reset) {
    if (!c || !out) return KRR_EINVAL;
    memset(out, 0, sizeof(*out));
    KRR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (c->la_stream) KRR_CUDA_TRY(c, cudaStreamSynchronize(c->la_stream));
    out->launches = (int64_t)g_launches.load();
    if (c->prof) {
        ProfState *ps = (ProfState *)c->prof;
        for (const ProfRec &r : ps->recs) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            out->count[r.cls] += 1;
            out->ms[r.cls] += ms;
            out->flops[r.cls] += r.flops;
            out->bytes[r.cls] += r.bytes;
        }
        if (reset) {
            for (const ProfRec &r : ps->recs) {
                ps->pool.push_back(r.a);
                ps->pool.push_back(r.b);
            }
            ps->recs.clear();
        }
    }
    if (reset) g_launches.store(0);
    return KRR_OK;
}

extern "C" krr_status krr_get_factor(krr_ctx *c, float *L, int64_t ldl) {
    if (!c) return KRR_EINVAL;
    if (!c->factored) {
        c->last_error = "krr_get_factor: no factorisation";
        return KRR_ESTATE;
    }
    if (!L || ldl < c->n) return KRR_EINVAL;
    const bool dev = is_device_ptr(L);
    float *dst = L;
    const size_t bytes = (size_t)c->n * ldl * sizeof(float);
    if (!dev) {
        KRR_TRY(stage(c, bytes));
        dst = (float *)c->stage;
        KRR_CUDA_TRY(c, cudaMemsetAsync(dst, 0, bytes, c->stream));
    }
    launch_factor_to_dense(c, dst, ldl);
    KRR_TRY(check_launch(c, "factor to dense"));
    if (!dev) KRR_CUDA_TRY(c, cudaMemcpyAsync(L, dst, bytes, cudaMemcpyDeviceToHost, c->stream));
    KRR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return KRR_OK;
}

extern "C" krr_status krr_grad_hyper(krr_ctx *c, const int8_t *T, int64_t n_test, int64_t ldt,
                                     const float *Yt, int64_t ldy, const float *A, int64_t lda,
                                     int64_t p, double *out) {
    if (!c) return KRR_EINVAL;
    if (!c->factored) {
        c->last_error = "krr_grad_hyper: no factorisation";
        return KRR_ESTATE;
    }
    if (!mixed(c) || !c->tc || is_ibs(c) || c->nconf > 0 || c->rr) {
        c->last_error = "krr_grad_hyper: needs a context in KRR_MODE_MIXED with the Gaussian kernel and no "
                        "confounders";
        return KRR_EINVAL;
    }
    if (!T || !Yt || !A || !out || n_test < 1 || ldt < c->m || p < 1 || p > 16 || ldy < p || lda < p) {
        c->last_error = "krr_grad_hyper: bad arguments (need 1 <= p <= 16, ldt >= m, ldy, lda >= p)";
        return KRR_EINVAL;
    }
    cudaStream_t s = c->stream;
    const int64_t rows = (n_test + 255) / 256 * 256;
    const int64_t npad = c->n_pad;
    // buffers
    const size_t tbytes = (size_t)rows * c->m_pad;
    if (c->t_cap < tbytes) {
        KRR_TRY(dev_alloc(c, &c->t8, tbytes, "test genotypes"));
        c->t_cap = tbytes;
    }
    if (c->tnorm_cap < (size_t)rows) {
        KRR_TRY(dev_alloc(c, &c->tnorms, (size_t)rows, "test norms"));
        c->tnorm_cap = rows;
    }
    KRR_TRY(ensure_vectors(c, p));
    if (c->g_rows_cap < (size_t)rows * p) {
        KRR_TRY(dev_alloc(c, &c->g_yt, (size_t)rows * p, "gradient buffers"));
        KRR_TRY(dev_alloc(c, &c->g_gp, (size_t)rows * p, "gradient buffers"));
        KRR_TRY(dev_alloc(c, &c->g_sq, (size_t)rows * p, "gradient buffers"));
        KRR_TRY(dev_alloc(c, &c->pred_out, (size_t)rows * p, "predictions"));
        c->pred_out_cap = (size_t)rows * p;
        c->g_rows_cap = (size_t)rows * p;
    }
    if (c->g_aw_cap < (size_t)npad * p) {
        KRR_TRY(dev_alloc(c, &c->g_aw, (size_t)npad * p, "gradient buffers"));
        c->g_aw_cap = (size_t)npad * p;
    }
    const size_t part_pred = (size_t)(npad / 128) * rows * p;      // Yhat partials
    const size_t part_t = (size_t)(2 * rows / 256) * npad * p;     // K_t^T G_p partials
    const size_t part = std::max(part_pred, part_t);
    if (c->g_part_cap < part) {
        KRR_TRY(dev_alloc(c, &c->g_part, part, "gradient partials"));
        c->g_part_cap = part;
    }
    const size_t it = (size_t)(rows / 128) * (npad / 256);
    const size_t ik = (size_t)c->nt * (c->nt + 1) / 2 * (c->b / 128) * (c->b / 256);
    if (c->g_tpart_cap < it) {
        KRR_TRY(dev_alloc(c, &c->g_tpart, it, "gradient partials"));
        c->g_tpart_cap = it;
    }
    if (c->g_kpart_cap < ik) {
        KRR_TRY(dev_alloc(c, &c->g_kpart, ik, "gradient partials"));
        c->g_kpart_cap = ik;
    }
    if (!c->g_scal) KRR_TRY(dev_alloc(c, &c->g_scal, (size_t)8, "gradient scalars"));

    // 1. inputs: packed test genotypes, padded weights and held-out phenotypes
    KRR_TRY(pack(c, T, n_test, c->m, ldt, rows, c->t8, nullptr, c->tnorms));
    KRR_TRY(load_rows_f32(c, A, c->n, p, lda, npad, c->g_aw));
    KRR_TRY(load_rows_f32(c, Yt, n_test, p, ldy, rows, c->g_yt));
    // 2. Yhat = K_t A (Alg. 4), as in krr_predict: (K - c) A + c (1^T A)
    if (c->colsum_cap < p) {
        KRR_TRY(dev_alloc(c, &c->colsum, (size_t)p, "column sums"));
        c->colsum_cap = p;
    }
    launch_colsum(c->g_aw, npad, p, c->colsum, s);
    KRR_TRY(tc_predict(c, c->t8, c->tnorms, n_test, rows, c->g_aw, p, p, c->g_part, c->red + RED_KSHIFT));
    launch_predict_reduce(c->g_part, npad / 128, rows, n_test, p, c->pred_out, p, s, c->red + RED_KSHIFT,
                          c->colsum);
    // 3. G_p = d loss / d Yhat and the loss
    launch_grad_prep(c->pred_out, c->g_yt, n_test, p, rows, c->g_gp, c->g_sq, s);
    launch_sum_f64(c->g_sq, rows * p, c->g_scal + 0, s);
    // 4. B = K_t^T G_p into the solve's right-hand side, then Z = (K + lambda I)^-1 B
    KRR_TRY(tc_predict_t(c, c->t8, c->tnorms, n_test, rows, c->g_gp, p, p, c->g_part));
    launch_predict_reduce(c->g_part, 2 * rows / 256, npad, npad, p, c->ybuf, p, s);
    KRR_TRY(check_launch(c, "gradient adjoint right-hand side"));
    krr_solve_info si;
    krr_status st = solve_device(c, p, &si);
    if (st != KRR_OK && st != KRR_ENOCONV) return st;
    // 5. <Z, A> and the two d K-weighted contractions
    launch_dot_f32(c->abuf, c->g_aw, npad * p, c->g_scal + 1, s);
    int64_t nit = 0, nik = 0;
    KRR_TRY(tc_grad_terms(c, c->t8, c->tnorms, n_test, rows, c->g_aw, c->abuf, c->g_gp, p, p,
                          c->g_tpart, c->g_kpart, &nit, &nik));
    launch_sum_f64(c->g_tpart, nit, c->g_scal + 2, s);
    launch_sum_f64(c->g_kpart, nik, c->g_scal + 3, s);
    KRR_TRY(check_launch(c, "gradient sums"));
    KRR_CUDA_TRY(c, cudaMemcpyAsync(c->hred, c->g_scal, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    KRR_CUDA_TRY(c, cudaStreamSynchronize(s));
    const double loss = c->hred[0] / (double)(n_test * p);
    out[0] = loss;
    out[1] = c->gamma * (c->hred[3] - c->hred[2]);
    out[2] = -c->lambda * c->hred[1];
    return KRR_OK;
}
