// Ridge regression (Sec. IV-A, "Ridge Regression with Precision-Adaptive
// Computations"): beta = (X^T X + lambda I)^-1 X^T Y with X = [G C] the N x M
// genotype columns and the nc real confounder columns of the patients.
//
// The context's matrix becomes the Gram matrix X^T X of order M + nc, stored
// in the same lower-triangle tiles as the KRR kernel, so krr_factor() and
// krr_solve() run the same mixed-precision Cholesky, substitution and
// refinement on it.  The Gram product is the paper's mixed-precision SYRK:
//   - G^T G (integer entries below 4N) on the tensor cores from E4M3
//     operands with FP32 accumulation -- exact -- or on CUDA cores in FP32
//     (fp32 mode; also exact below 2^24);
//   - the columns that involve confounders (G^T C, C^T C) in FP32 on CUDA
//     cores, summed over patients in chunks and the chunks in FP64.
// X^T Y and the predictions T beta + Ct beta_c are FP32 products on CUDA
// cores (Y has few columns, as the paper notes), with FP64 sums of chunks.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "krr_internal.h"

namespace krr {

namespace {

inline unsigned cdivu(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// ---------------------------------------------------------------------------
// Transposed packing: X (n patients x m genotypes, int8, leading dimension ldx)
// -> packed operand rows = genotype columns (rows_pad x cols_pad, patients
// along the row), E4M3 codes of {0, 1, 2} (mixed) or FP32 (fp32 mode); the
// padding is written as zeros.  32 x 32 tiles through shared memory.
// ---------------------------------------------------------------------------
__global__ void rr_pack_t_kernel(const int8_t *__restrict__ x, int64_t n, int64_t m, int64_t ldx, int64_t rows_pad,
                                 int64_t cols_pad, uint8_t *__restrict__ out8, float *__restrict__ outf) {
    __shared__ int t[32][33];
    const int64_t p0 = (int64_t)blockIdx.x * 32, f0 = (int64_t)blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t p = p0 + r, f = f0 + threadIdx.x;
        t[r][threadIdx.x] = (p < n && f < m) ? (int)x[p * ldx + f] : 0;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t f = f0 + r, p = p0 + threadIdx.x;
        if (f < rows_pad && p < cols_pad) {
            const int v = t[threadIdx.x][r];
            if (out8) out8[f * cols_pad + p] = (uint8_t)(v == 0 ? 0x00 : (v == 1 ? 0x38 : (v == 2 ? 0x40 : 0x48)));
            if (outf) outf[f * cols_pad + p] = (float)v;
        }
    }
}

// Confounders transposed: ct[q][p] = cpad[p][q] (cpad rows_pad x CONF_MAX).
__global__ void rr_conf_t_kernel(const float *cpad, int64_t rows, int nc, float *ct) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * nc) return;
    const int64_t q = e / rows, p = e % rows;
    ct[q * rows + p] = cpad[p * CONF_MAX + q];
}

// ---------------------------------------------------------------------------
// Row-block products with few output columns, split over the contraction:
//   part[chunk][r][q] = sum_{k in chunk} a(r, k) B[k][q],  r < rows, q < nq <= 32,
// a from row r of A: int8 values (KIND 0), E4M3 codes of {0, 1, 2} (KIND 1)
// or FP32 (KIND 2).  One CTA per 64 rows and chunk; 128-wide slabs of A and B
// through shared memory; thread (r, g) accumulates columns [8 g, 8 g + 8) of
// row r in FP32.  The chunks are summed in FP64 by rr_reduce_kernel.
// ---------------------------------------------------------------------------
constexpr int RG_R = 64, RG_K = 128;

template <int KIND>
__device__ __forceinline__ float rg_load(const void *A, int64_t idx) {
    if (KIND == 0) return (float)reinterpret_cast<const int8_t *>(A)[idx];
    if (KIND == 1) {
        const uint8_t v = reinterpret_cast<const uint8_t *>(A)[idx];
        return v == 0x38 ? 1.f : (v == 0x40 ? 2.f : (v == 0x48 ? 3.f : 0.f));
    }
    return reinterpret_cast<const float *>(A)[idx];
}

template <int KIND>
__global__ void __launch_bounds__(256) rr_rowgemm_kernel(const void *A, int64_t lda, int64_t rows, int64_t K,
                                                         int64_t kchunk, const float *B, int64_t ldb, int nq,
                                                         float *part) {
    __shared__ float As[RG_R][RG_K + 1];
    __shared__ float Bs[RG_K][32];
    const int64_t r0 = (int64_t)blockIdx.x * RG_R;
    const int64_t kbeg = (int64_t)blockIdx.y * kchunk;
    const int64_t kend = min(K, kbeg + kchunk);
    const int tr = threadIdx.x >> 2, qg = threadIdx.x & 3;
    float acc[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) acc[e] = 0.f;
    for (int64_t k0 = kbeg; k0 < kend; k0 += RG_K) {
        for (int e = threadIdx.x; e < RG_R * RG_K; e += 256) {
            const int rr = e / RG_K, kk = e % RG_K;
            const int64_t r = r0 + rr, k = k0 + kk;
            As[rr][kk] = (r < rows && k < kend) ? rg_load<KIND>(A, r * lda + k) : 0.f;
        }
        for (int e = threadIdx.x; e < RG_K * 32; e += 256) {
            const int kk = e / 32, q = e % 32;
            const int64_t k = k0 + kk;
            Bs[kk][q] = (k < kend && q < nq) ? B[k * ldb + q] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < RG_K; ++kk) {
            const float a = As[tr][kk];
#pragma unroll
            for (int e = 0; e < 8; ++e) acc[e] = fmaf(a, Bs[kk][qg * 8 + e], acc[e]);
        }
        __syncthreads();
    }
    const int64_t r = r0 + tr;
    if (r < rows) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int q = qg * 8 + e;
            if (q < nq) part[((int64_t)blockIdx.y * rows + r) * nq + q] = acc[e];
        }
    }
}

// out[e] = sum over chunks c of part[c][e] in FP64, e < count (fixed order).
__global__ void rr_reduce_kernel(const float *part, int64_t nchunk, int64_t count, double *out) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= count) return;
    double s = 0.0;
    for (int64_t c = 0; c < nchunk; ++c) s += (double)part[c * count + e];
    out[e] = s;
}

// Confounder rows of the Gram matrix: g[j][q] = X[:, j]^T X[:, M + q] (FP64)
// becomes entry (M + q, j) for j <= M + q of the lower-triangle tiles, and
// also its mirror (j, M + q) when both lie in one diagonal tile (diagonal
// tiles are stored in full).
__global__ void rr_scatter_kernel(const double *g, int64_t F, int64_t M, int nc, int64_t b, float *Kd) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= F * nc) return;
    const int64_t q = e / F, j = e % F, r = M + q;
    if (j > r) return;
    const float v = (float)g[j * nc + q];
    const int64_t ti = r / b, tj = j / b, rr = r % b, cc = j % b;
    Kd[tri_index(ti, tj) * b * b + rr * b + cc] = v;
    if (ti == tj) Kd[tri_index(ti, ti) * b * b + cc * b + rr] = v;
}

// Block sums of K^2 and K of the tiles in tile rows [ti0, ti0 + gridDim.y)
// (recomputed after the confounder rows were written): one CTA per 128 x bn
// block, the layout of the build epilogues' partials (slot = tile * per_tile
// + block; K^2 first, then K after ntri * per_tile entries).
__global__ void rr_tile_sums_kernel(const float *Kd, int64_t b, int64_t bn, int64_t ti0, int64_t ntri,
                                    double *part) {
    const int64_t ti = ti0 + blockIdx.y;
    const int64_t per_tile = (b / 128) * (b / bn);
    const int64_t tj = blockIdx.x / per_tile, blk = blockIdx.x % per_tile;
    if (tj > ti) return;
    const int64_t sm = blk / (b / bn), sn = blk % (b / bn);
    const float *base = Kd + tri_index(ti, tj) * b * b + sm * 128 * b + sn * bn;
    double s2 = 0.0, s1 = 0.0;
    for (int64_t e = threadIdx.x; e < 128 * bn; e += blockDim.x) {
        const double v = (double)base[(e / bn) * b + e % bn];
        s2 += v * v;
        s1 += v;
    }
    __shared__ double r2[256], r1[256];
    r2[threadIdx.x] = s2;
    r1[threadIdx.x] = s1;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            r2[threadIdx.x] += r2[threadIdx.x + o];
            r1[threadIdx.x] += r1[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int64_t slot = tri_index(ti, tj) * per_tile + blk;
        part[slot] = r2[0];
        part[ntri * per_tile + slot] = r1[0];
    }
}

// dst[r * ldd + q0 + q] = src[r * pc + q] (FP64 -> FP32), r < rows, q < pc.
__global__ void rr_store_cols_kernel(const double *src, int64_t rows, int pc, float *dst, int64_t ldd, int64_t q0) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * pc) return;
    dst[(e / pc) * ldd + q0 + e % pc] = (float)src[e];
}

// Buffers of the ridge-regression entry points, owned by the context.
struct RRState {
    float *cpad = nullptr;    // patients_pad x CONF_MAX confounders of the build
    float *ct = nullptr;      // nc x patients_pad, the same transposed
    float *part = nullptr;    // chunk partials of the row-block products
    double *out = nullptr;    // their FP64 sums
    float *fout = nullptr;    // FP32 results before the copy to the caller
    int8_t *t = nullptr;      // held-out genotypes
    float *tc = nullptr;      // held-out confounders
    float *beta = nullptr;    // weights
    float *y = nullptr;       // phenotypes
    size_t cpad_cap = 0, ct_cap = 0, part_cap = 0, out_cap = 0, fout_cap = 0, t_cap = 0, tc_cap = 0,
           beta_cap = 0, y_cap = 0;
    int64_t npat = 0;         // patients of the build
};

RRState *state(Ctx *c) {
    if (!c->rr_state) c->rr_state = new (std::nothrow) RRState();
    return (RRState *)c->rr_state;
}

template <typename T>
krr_status grow(Ctx *c, T **p, size_t *cap, size_t count, const char *what) {
    if (*cap >= count) return KRR_OK;
    KRR_TRY(dev_alloc(c, p, count, what));
    *cap = count;
    return KRR_OK;
}

// rows x row_bytes of a caller matrix (host or device, ld_bytes apart) into a
// dense device buffer.
krr_status copy_in(Ctx *c, void *dst, const void *src, int64_t rows, size_t row_bytes, size_t ld_bytes) {
    KRR_CUDA_TRY(c, cudaMemcpy2DAsync(dst, row_bytes, src, ld_bytes, row_bytes, (size_t)rows, cudaMemcpyDefault,
                                      c->stream));
    return KRR_OK;
}

// Split of a contraction of length K for `rows` output rows: enough CTAs to
// fill the GPU twice over, and at most RG_KMAX terms summed in FP32 per chunk.
constexpr int64_t RG_KMAX = 2048;
void split(const Ctx *c, int64_t rows, int64_t K, int64_t *nchunk, int64_t *kchunk) {
    const int64_t rb = (rows + RG_R - 1) / RG_R;
    int64_t want = std::max<int64_t>(1, (4 * (int64_t)c->num_sms + rb - 1) / rb);
    want = std::min<int64_t>(want, std::max<int64_t>(1, (K + RG_K - 1) / RG_K));
    int64_t kc = (K + want - 1) / want;
    kc = (kc + RG_K - 1) / RG_K * RG_K;
    *kchunk = std::min<int64_t>(std::max<int64_t>(kc, RG_K), RG_KMAX);
    *nchunk = (K + *kchunk - 1) / *kchunk;
}

template <int KIND>
void rowgemm(Ctx *c, const void *A, int64_t lda, int64_t rows, int64_t K, const float *B, int64_t ldb, int nq,
             float *part, int64_t nchunk, int64_t kchunk) {
    count_launch(), rr_rowgemm_kernel<KIND><<<dim3(cdivu(rows, RG_R), (unsigned)nchunk), 256, 0, c->stream>>>(
        A, lda, rows, K, kchunk, B, ldb, nq, part);
}

}  // namespace

void rr_free(Ctx *c) {
    RRState *st = (RRState *)c->rr_state;
    if (!st) return;
    dev_free(&st->cpad);
    dev_free(&st->ct);
    dev_free(&st->part);
    dev_free(&st->out);
    dev_free(&st->fout);
    dev_free(&st->t);
    dev_free(&st->tc);
    dev_free(&st->beta);
    dev_free(&st->y);
    delete st;
    c->rr_state = nullptr;
}

}  // namespace krr

using namespace krr;

namespace {

// FP64 sums of the partial products of a chunked launch into st->out.
void reduce_parts(Ctx *c, const float *part, int64_t nchunk, int64_t count, double *out) {
    count_launch(), rr_reduce_kernel<<<cdivu(count, 256), 256, 0, c->stream>>>(part, nchunk, count, out);
}

// Rows [0, m) of the packed genotype operand times B (patients x nq, ldb) and,
// with confounders, the nc confounder rows: FP64 results out[(m + nc) x nq].
krr_status xt_times(Ctx *c, RRState *st, const float *B, int64_t ldb, int nq, double *out) {
    const int64_t m = c->rr_m, nc = c->rr_nc, K = st->npat;
    int64_t n1, k1, n2 = 0, k2 = 0;
    split(c, m, K, &n1, &k1);
    if (nc > 0) split(c, nc, K, &n2, &k2);
    const size_t need = (size_t)(n1 * m + n2 * nc) * nq;
    KRR_TRY(grow(c, &st->part, &st->part_cap, need, "ridge partial products"));
    if (mixed(c))
        rowgemm<1>(c, c->g8, c->m_pad, m, K, B, ldb, nq, st->part, n1, k1);
    else
        rowgemm<2>(c, c->gf, c->m_pad, m, K, B, ldb, nq, st->part, n1, k1);
    reduce_parts(c, st->part, n1, m * nq, out);
    if (nc > 0) {
        float *p2 = st->part + (size_t)n1 * m * nq;
        rowgemm<2>(c, st->ct, c->m_pad, nc, K, B, ldb, nq, p2, n2, k2);
        reduce_parts(c, p2, n2, nc * nq, out + m * nq);
    }
    return check_launch(c, "ridge X^T B");
}

}  // namespace

extern "C" krr_status krr_rr_build(krr_ctx *ctx, const int8_t *X, int64_t n, int64_t m, int64_t ldx, const float *C,
                                   int64_t nc, int64_t ldc) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return KRR_EINVAL;
    if (!X || n < 1 || m < 1 || ldx < m || n > (int64_t(1) << 22) || nc < 0 || nc > CONF_MAX ||
        (nc > 0 && (!C || ldc < nc))) {
        c->last_error = "krr_rr_build: need X != NULL, 1 <= n <= 2^22, m >= 1, ldx >= m, 0 <= nc <= 16 and "
                        "C != NULL with ldc >= nc when nc > 0";
        return KRR_EINVAL;
    }
    RRState *st = state(c);
    if (!st) {
        c->last_error = "out of host memory";
        return KRR_ENOMEM;
    }
    c->built = c->factored = false;
    c->rr = 0;
    const int64_t F = m + nc;
    const int64_t m_pad = (n + 127) / 128 * 128;  // patients: the contraction of the Gram product
    KRR_TRY(prepare_build(c, F, m_pad, 0));
    c->m = n;
    c->gamma = 0.0;
    c->nconf = 0;
    c->rr = 1;
    c->rr_m = m;
    c->rr_nc = nc;
    st->npat = n;
    // genotype columns as operand rows (patients along the row)
    const int8_t *dx = X;
    if (!is_device_ptr(X)) {
        const void *alias = pinned_host_alias(X);
        if (alias) {
            dx = (const int8_t *)alias;
        } else {
            KRR_TRY(stage(c, (size_t)n * m));
            KRR_CUDA_TRY(c, cudaMemcpy2DAsync(c->stage, m, X, ldx, m, n, cudaMemcpyHostToDevice, c->stream));
            dx = (const int8_t *)c->stage;
            ldx = m;
        }
    }
    count_launch(), rr_pack_t_kernel<<<dim3((unsigned)(m_pad / 32), (unsigned)(c->n_pad / 32)), dim3(32, 8), 0,
                                       c->stream>>>(dx, n, m, ldx, c->n_pad, m_pad, mixed(c) ? c->g8 : nullptr,
                                                    mixed(c) ? nullptr : c->gf);
    KRR_CUDA_TRY(c, cudaMemsetAsync(c->norms, 0, (size_t)c->n_pad * sizeof(int32_t), c->stream));
    KRR_TRY(check_launch(c, "ridge packing"));
    if (nc > 0) {
        KRR_TRY(grow(c, &st->cpad, &st->cpad_cap, (size_t)m_pad * CONF_MAX, "ridge confounders"));
        KRR_TRY(load_conf(c, C, n, nc, ldc, m_pad, st->cpad));
        KRR_TRY(grow(c, &st->ct, &st->ct_cap, (size_t)nc * m_pad, "ridge confounders"));
        count_launch(), rr_conf_t_kernel<<<cdivu(m_pad * nc, 256), 256, 0, c->stream>>>(st->cpad, m_pad, (int)nc,
                                                                                         st->ct);
    }
    // G^T G: the integer-exact Gram product over the genotype columns
    if (mixed(c)) {
        KRR_TRY(tc_build(c));
    } else {
        launch_build_simt(c);
    }
    KRR_TRY(check_launch(c, "ridge Gram product"));
    if (nc > 0) {
        // X^T C: the Gram columns of the confounders, in FP32 products summed in FP64
        KRR_TRY(grow(c, &st->out, &st->out_cap, (size_t)F * nc, "ridge products"));
        KRR_TRY(xt_times(c, st, st->cpad, CONF_MAX, (int)nc, st->out));
        count_launch(), rr_scatter_kernel<<<cdivu(F * nc, 256), 256, 0, c->stream>>>(st->out, F, m, (int)nc, c->b,
                                                                                     c->Kd);
        const int64_t ti0 = m / c->b, ti1 = (F - 1) / c->b;
        const int64_t bn = mixed(c) ? 256 : 128;
        const int64_t per_tile = (c->b / 128) * (c->b / bn);
        const int64_t ntri = c->nt * (c->nt + 1) / 2;
        count_launch(), rr_tile_sums_kernel<<<dim3((unsigned)((ti1 + 1) * per_tile), (unsigned)(ti1 - ti0 + 1)), 256,
                                              0, c->stream>>>(c->Kd, c->b, bn, ti0, ntri, c->knorm2);
        KRR_TRY(check_launch(c, "ridge confounder columns"));
    }
    launch_kernel_sumsq(c, c->red + RED_KNORM2);
    KRR_TRY(check_launch(c, "ridge Gram norms"));
    c->built = true;
    return KRR_OK;
}

extern "C" krr_status krr_rr_rhs(krr_ctx *ctx, const float *Y, int64_t p, int64_t ldy, float *B, int64_t ldb) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return KRR_EINVAL;
    if (!c->built || !c->rr) {
        c->last_error = "krr_rr_rhs: no ridge-regression Gram matrix built";
        return KRR_ESTATE;
    }
    if (!Y || !B || p < 1 || ldy < p || ldb < p) {
        c->last_error = "krr_rr_rhs: need Y, B != NULL, p >= 1, ldy >= p, ldb >= p";
        return KRR_EINVAL;
    }
    RRState *st = state(c);
    const int64_t F = c->n, n = st->npat;
    KRR_TRY(grow(c, &st->y, &st->y_cap, (size_t)n * p, "ridge phenotypes"));
    KRR_TRY(copy_in(c, st->y, Y, n, (size_t)p * sizeof(float), (size_t)ldy * sizeof(float)));
    KRR_TRY(grow(c, &st->out, &st->out_cap, (size_t)F * std::min<int64_t>(p, 32), "ridge products"));
    KRR_TRY(grow(c, &st->fout, &st->fout_cap, (size_t)F * p, "ridge products"));
    for (int64_t q0 = 0; q0 < p; q0 += 32) {
        const int pc = (int)std::min<int64_t>(32, p - q0);
        KRR_TRY(xt_times(c, st, st->y + q0, p, pc, st->out));
        count_launch(), rr_store_cols_kernel<<<cdivu(F * pc, 256), 256, 0, c->stream>>>(st->out, F, pc, st->fout, p,
                                                                                         q0);
    }
    KRR_TRY(check_launch(c, "ridge X^T Y"));
    KRR_CUDA_TRY(c, cudaMemcpy2DAsync(B, (size_t)ldb * sizeof(float), st->fout, (size_t)p * sizeof(float),
                                      (size_t)p * sizeof(float), (size_t)F, cudaMemcpyDefault, c->stream));
    KRR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return KRR_OK;
}

extern "C" krr_status krr_rr_predict(krr_ctx *ctx, const int8_t *T, int64_t n_test, int64_t ldt, const float *Ct,
                                     int64_t ldct, const float *beta, int64_t ldbeta, int64_t p, float *Yt,
                                     int64_t ldyt) {
    Ctx *c = reinterpret_cast<Ctx *>(ctx);
    if (!c) return KRR_EINVAL;
    if (!c->built || !c->rr) {
        c->last_error = "krr_rr_predict: no ridge-regression Gram matrix built";
        return KRR_ESTATE;
    }
    const int64_t m = c->rr_m, nc = c->rr_nc, F = c->n;
    if (!T || !beta || !Yt || n_test < 1 || ldt < m || p < 1 || ldbeta < p || ldyt < p ||
        (nc > 0 && (!Ct || ldct < nc))) {
        c->last_error = "krr_rr_predict: need T, beta, Yt != NULL, n_test >= 1, ldt >= m, p >= 1, ldbeta, ldyt >= p "
                        "and Ct (ldct >= nc) when the model has confounders";
        return KRR_EINVAL;
    }
    RRState *st = state(c);
    KRR_TRY(grow(c, &st->t, &st->t_cap, (size_t)n_test * m, "held-out genotypes"));
    KRR_TRY(copy_in(c, st->t, T, n_test, (size_t)m, (size_t)ldt));
    KRR_TRY(grow(c, &st->beta, &st->beta_cap, (size_t)F * p, "ridge weights"));
    KRR_TRY(copy_in(c, st->beta, beta, F, (size_t)p * sizeof(float), (size_t)ldbeta * sizeof(float)));
    if (nc > 0) {
        KRR_TRY(grow(c, &st->tc, &st->tc_cap, (size_t)n_test * nc, "held-out confounders"));
        KRR_TRY(copy_in(c, st->tc, Ct, n_test, (size_t)nc * sizeof(float), (size_t)ldct * sizeof(float)));
    }
    int64_t n1, k1;
    split(c, n_test, m, &n1, &k1);
    const int64_t pc_max = std::min<int64_t>(p, 32);
    KRR_TRY(grow(c, &st->part, &st->part_cap, (size_t)(n1 + 1) * n_test * pc_max, "ridge partial products"));
    KRR_TRY(grow(c, &st->out, &st->out_cap, (size_t)n_test * pc_max, "ridge products"));
    KRR_TRY(grow(c, &st->fout, &st->fout_cap, (size_t)n_test * p, "ridge products"));
    for (int64_t q0 = 0; q0 < p; q0 += 32) {
        const int pc = (int)std::min<int64_t>(32, p - q0);
        // genotype part T beta_g (chunks over the SNPs), then the confounder
        // part Ct beta_c as one more chunk; FP64 sum over all of them
        rowgemm<0>(c, st->t, m, n_test, m, st->beta + q0, p, pc, st->part, n1, k1);
        int64_t chunks = n1;
        if (nc > 0) {
            rowgemm<2>(c, st->tc, nc, n_test, nc, st->beta + m * p + q0, p, pc,
                       st->part + (size_t)n1 * n_test * pc, 1, (nc + RG_K - 1) / RG_K * RG_K);
            chunks += 1;
        }
        reduce_parts(c, st->part, chunks, n_test * pc, st->out);
        count_launch(), rr_store_cols_kernel<<<cdivu(n_test * pc, 256), 256, 0, c->stream>>>(st->out, n_test, pc,
                                                                                              st->fout, p, q0);
    }
    KRR_TRY(check_launch(c, "ridge predict"));
    KRR_CUDA_TRY(c, cudaMemcpy2DAsync(Yt, (size_t)ldyt * sizeof(float), st->fout, (size_t)p * sizeof(float),
                                      (size_t)p * sizeof(float), (size_t)n_test, cudaMemcpyDefault, c->stream));
    KRR_CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return KRR_OK;
}
