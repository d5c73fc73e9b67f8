// CUDA-core kernels of the KRR engine:
//  - genotype packing and squared row norms (the folded norm vector of the
//    paper's distance section, Sec. IV-B);
//  - a register-blocked FP32/FP64 GEMM used by the plain-FP32 path and by the
//    diagonal-tile Cholesky / inverse;
//  - the diagonal-tile Cholesky (Alg. 3, Factorize) and triangular inverse;
//  - the adaptive-precision cast of each factor column;
//  - forward/backward substitution (Alg. 3, Solve) with the stored factor;
//  - the refinement residual and the predict reduction (Alg. 4).
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <math.h>

#include <algorithm>

#include "krr_internal.h"

namespace krr {

static inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// ----------------------------------------------------------------------------
// Genotype packing.  One block per padded row.  E4M3 encodings of 0, 1, 2 are
// 0x00, 0x38, 0x40 (exact).  Norm n_i = sum_k g_ik^2 (exact int32).
// ----------------------------------------------------------------------------
__global__ void pack_genotypes_kernel(const int8_t *__restrict__ g, int64_t n, int64_t m,
                                      int64_t ldg, int64_t m_pad, uint8_t *__restrict__ out8,
                                      float *__restrict__ outf, int32_t *__restrict__ norms) {
    int64_t row = blockIdx.x;
    int32_t s = 0;
    for (int64_t k = threadIdx.x; k < m_pad; k += blockDim.x) {
        int v = 0;
        if (row < n && k < m) v = g[row * ldg + k];
        s += v * v;
        if (out8) out8[row * m_pad + k] = v == 0 ? 0x00 : (v == 1 ? 0x38 : (v == 2 ? 0x40 : 0x48));
        if (outf) outf[row * m_pad + k] = (float)v;
    }
    __shared__ int32_t red[32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) norms[row] = s;
    }
}

void launch_pack_genotypes(const int8_t *g, int64_t n, int64_t m, int64_t ldg, int64_t n_pad,
                           int64_t m_pad, uint8_t *out8, float *outf, int32_t *norms,
                           cudaStream_t s) {
    count_launch(), pack_genotypes_kernel<<<(unsigned)n_pad, 256, 0, s>>>(g, n, m, ldg, m_pad, out8, outf, norms);
}

// ----------------------------------------------------------------------------
// Register-blocked CUDA-core GEMM microkernel: a 128 x 128 block of
// C = A B^T (b_trans = 0, B is N x K) or C = A B (b_trans = 1, B is K x N),
// 256 threads, 8 x 8 outputs per thread, BK = 8, double-buffered shared memory
// with a register prefetch of the next slab.  Requires K % 8 == 0, leading
// dimensions that are multiples of 4 and 16-byte aligned operands.
// Thread (tx, ty) owns rows {ty*4 + i, 64 + ty*4 + i} and columns
// {tx*4 + j, 64 + tx*4 + j}, i, j < 4.
// ----------------------------------------------------------------------------
constexpr int SG_BM = 128, SG_BN = 128, SG_BK = 8;

template <typename T>
struct Vec4;
template <>
struct Vec4<float> {
    float v[4];
    __device__ void load(const float *p) {
        float4 t = *reinterpret_cast<const float4 *>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
};
template <>
struct Vec4<double> {
    double v[4];
    __device__ void load(const double *p) {
        double2 a = reinterpret_cast<const double2 *>(p)[0];
        double2 b = reinterpret_cast<const double2 *>(p)[1];
        v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
    }
};

template <typename T, int BTRANS>
__device__ __forceinline__ void sg_load(const T *__restrict__ A, int64_t lda, const T *__restrict__ B,
                                        int64_t ldb, int k0, int mvalid, int nvalid, Vec4<T> &ra,
                                        Vec4<T> &rb) {
    const int tid = threadIdx.x;
    {
        int r = tid >> 1, kc = (tid & 1) * 4;
        if (r < mvalid) ra.load(A + (int64_t)r * lda + k0 + kc);
        else ra.v[0] = ra.v[1] = ra.v[2] = ra.v[3] = T(0);
    }
    if (!BTRANS) {
        int r = tid >> 1, kc = (tid & 1) * 4;
        if (r < nvalid) rb.load(B + (int64_t)r * ldb + k0 + kc);
        else rb.v[0] = rb.v[1] = rb.v[2] = rb.v[3] = T(0);
    } else {
        int kr = tid >> 5, nc = (tid & 31) * 4;
        if (nc + 3 < nvalid) {
            rb.load(B + (int64_t)(k0 + kr) * ldb + nc);
        } else {
            for (int e = 0; e < 4; ++e)
                rb.v[e] = (nc + e < nvalid) ? B[(int64_t)(k0 + kr) * ldb + nc + e] : T(0);
        }
    }
}

template <typename T, int BTRANS>
__device__ __forceinline__ void sg_store(T (*As)[SG_BM], T (*Bs)[SG_BN], const Vec4<T> &ra,
                                         const Vec4<T> &rb) {
    const int tid = threadIdx.x;
    {
        int r = tid >> 1, kc = (tid & 1) * 4;
        for (int e = 0; e < 4; ++e) As[kc + e][r] = ra.v[e];
    }
    if (!BTRANS) {
        int r = tid >> 1, kc = (tid & 1) * 4;
        for (int e = 0; e < 4; ++e) Bs[kc + e][r] = rb.v[e];
    } else {
        int kr = tid >> 5, nc = (tid & 31) * 4;
        for (int e = 0; e < 4; ++e) Bs[kr][nc + e] = rb.v[e];
    }
}

template <typename T, int BTRANS>
__device__ __forceinline__ void sg_mainloop(const T *__restrict__ A, int64_t lda,
                                            const T *__restrict__ B, int64_t ldb, int K, int mvalid,
                                            int nvalid, T (&acc)[8][8]) {
    __shared__ __align__(16) T As[2][SG_BK][SG_BM];
    __shared__ __align__(16) T Bs[2][SG_BK][SG_BN];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = T(0);
    if (K <= 0) return;
    Vec4<T> ra, rb;
    sg_load<T, BTRANS>(A, lda, B, ldb, 0, mvalid, nvalid, ra, rb);
    sg_store<T, BTRANS>(As[0], Bs[0], ra, rb);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < K; k0 += SG_BK) {
        const bool more = k0 + SG_BK < K;
        if (more) sg_load<T, BTRANS>(A, lda, B, ldb, k0 + SG_BK, mvalid, nvalid, ra, rb);
#pragma unroll
        for (int kk = 0; kk < SG_BK; ++kk) {
            T a[8], bv[8];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                a[i] = As[buf][kk][ty * 4 + i];
                a[4 + i] = As[buf][kk][64 + ty * 4 + i];
                bv[i] = Bs[buf][kk][tx * 4 + i];
                bv[4 + i] = Bs[buf][kk][64 + tx * 4 + i];
            }
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
        }
        if (more) {
            sg_store<T, BTRANS>(As[buf ^ 1], Bs[buf ^ 1], ra, rb);
            __syncthreads();
            buf ^= 1;
        }
    }
}

__device__ __forceinline__ int sg_row(int i) { return (i < 4) ? ((threadIdx.x >> 4) * 4 + i) : (64 + (threadIdx.x >> 4) * 4 + i - 4); }
__device__ __forceinline__ int sg_col(int j) { return (j < 4) ? ((threadIdx.x & 15) * 4 + j) : (64 + (threadIdx.x & 15) * 4 + j - 4); }

// Generic batched GEMM ------------------------------------------------------
template <typename T, int BTRANS>
__global__ void __launch_bounds__(256) gemm_simt_kernel(int M, int N, int K, T alpha,
                                                        const T *A, int64_t lda, int64_t sA,
                                                        const T *B, int64_t ldb, int64_t sB, T beta,
                                                        const T *Cin, int64_t ldcin, int64_t sCin,
                                                        T *C, int64_t ldc, int64_t sC, int lower) {
    const int bm = blockIdx.x, bn = blockIdx.y, z = blockIdx.z;
    if (lower && bn > bm) return;
    const int m0 = bm * SG_BM, n0 = bn * SG_BN;
    A += z * sA + (int64_t)m0 * lda;
    B += z * sB + (BTRANS ? (int64_t)n0 : (int64_t)n0 * ldb);
    C += z * sC;
    if (Cin) Cin += z * sCin;
    T acc[8][8];
    sg_mainloop<T, BTRANS>(A, lda, B, ldb, K, M - m0, N - n0, acc);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        int r = m0 + sg_row(i);
        if (r >= M) continue;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            int cidx = n0 + sg_col(j);
            if (cidx >= N) continue;
            T v = alpha * acc[i][j];
            if (Cin) v += beta * Cin[(int64_t)r * ldcin + cidx];
            C[(int64_t)r * ldc + cidx] = v;
        }
    }
}

template <typename T>
void launch_gemm_simt(int M, int N, int K, T alpha, const T *A, int64_t lda, int64_t sA, const T *B,
                      int64_t ldb, int64_t sB, int b_trans, T beta, const T *Cin, int64_t ldcin,
                      int64_t sCin, T *C, int64_t ldc, int64_t sC, int batch, int lower,
                      cudaStream_t s) {
    if (M <= 0 || N <= 0 || batch <= 0) return;
    dim3 grid(cdiv(M, SG_BM), cdiv(N, SG_BN), batch);
    if (b_trans)
        count_launch(), gemm_simt_kernel<T, 1><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta,
                                                    Cin, ldcin, sCin, C, ldc, sC, lower);
    else
        count_launch(), gemm_simt_kernel<T, 0><<<grid, 256, 0, s>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta,
                                                    Cin, ldcin, sCin, C, ldc, sC, lower);
}
template void launch_gemm_simt<float>(int, int, int, float, const float *, int64_t, int64_t,
                                      const float *, int64_t, int64_t, int, float, const float *,
                                      int64_t, int64_t, float *, int64_t, int64_t, int, int,
                                      cudaStream_t);
template void launch_gemm_simt<double>(int, int, int, double, const double *, int64_t, int64_t,
                                       const double *, int64_t, int64_t, int, double,
                                       const double *, int64_t, int64_t, double *, int64_t,
                                       int64_t, int, int, cudaStream_t);

// ----------------------------------------------------------------------------
// FP32 Build on CUDA cores (fp32 mode).  One CTA per 128 x 128 block of a
// lower-triangle tile.  d = n_i + n_j - 2 s with s the FP32 dot product of
// integer genotypes (exact below 2^24), K = exp(-gamma d); padded rows give
// the identity.  Per-CTA partial sums of K^2 go to knorm_part.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) build_simt_kernel(const float *gf, const int32_t *norms,
                                                         int64_t m_pad, int64_t n, int64_t b,
                                                         float gamma, float *Kd, uint32_t *Dd,
                                                         double *knorm_part) {
    const int64_t sub_side = b / SG_BM, sub_per_tile = sub_side * sub_side;
    const int64_t t = blockIdx.x / sub_per_tile, sub = blockIdx.x % sub_per_tile;
    int64_t ti, tj;
    tri_decode(t, &ti, &tj);
    const int64_t sm = sub / sub_side, sn = sub % sub_side;
    const int64_t r0 = ti * b + sm * SG_BM, c0 = tj * b + sn * SG_BN;
    float acc[8][8];
    sg_mainloop<float, 0>(gf + r0 * m_pad, m_pad, gf + c0 * m_pad, m_pad, (int)m_pad, SG_BM, SG_BN,
                          acc);
    float *kt = Kd + tri_index(ti, tj) * b * b;
    uint32_t *dt = Dd ? Dd + tri_index(ti, tj) * b * b : nullptr;
    double ss = 0.0, s1 = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t lr = sm * SG_BM + sg_row(i), gi = ti * b + lr;
        const int32_t ni = norms[gi];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t lc = sn * SG_BN + sg_col(j), gj = tj * b + lc;
            int32_t d = ni + norms[gj] - 2 * (int32_t)acc[i][j];
            float kv;
            if (gi < n && gj < n) kv = expf(-gamma * (float)d);
            else kv = (gi == gj) ? 1.0f : 0.0f;
            kt[lr * b + lc] = kv;
            if (dt) dt[lr * b + lc] = (gi < n && gj < n) ? (uint32_t)d : 0u;
            ss += (double)kv * (double)kv;
            s1 += (double)kv;
        }
    }
    __shared__ double red[16];
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_down_sync(0xffffffffu, ss, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = ss;
        red[8 + (threadIdx.x >> 5)] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b1 = 0;
        for (int w = 0; w < 8; ++w) {
            a += red[w];
            b1 += red[8 + w];
        }
        knorm_part[blockIdx.x] = a;
        knorm_part[gridDim.x + blockIdx.x] = b1;
    }
}

void launch_build_simt(Ctx *c) {
    const int64_t ntri = c->nt * (c->nt + 1) / 2;
    const int64_t sub = (c->b / SG_BM) * (c->b / SG_BM);
    count_launch(), build_simt_kernel<<<(unsigned)(ntri * sub), 256, 0, c->stream>>>(
        c->gf, c->norms, c->m_pad, c->n, c->b, (float)c->gamma, c->Kd, c->Dd, c->knorm2);
}

// Deterministic sums of the per-block partials: out[0] = ||K||_F^2 and
// out[1] = sum of all entries of K (off-diagonal tiles counted twice), and
// out[2] = the mean off-diagonal entry c used to shift the refinement
// residual.  part holds ntri * per_tile sums of K^2 then as many sums of K.
__global__ void kernel_sumsq_kernel(const double *part, int64_t ntri, int64_t per_tile,
                                    int64_t n_pad, double *out) {
    __shared__ double red[64];
    double s = 0.0, s1 = 0.0;
    const double *part1 = part + ntri * per_tile;
    for (int64_t t = threadIdx.x; t < ntri; t += blockDim.x) {
        int64_t i, j;
        tri_decode(t, &i, &j);
        double ts = 0.0, ts1 = 0.0;
        for (int64_t q = 0; q < per_tile; ++q) {
            ts += part[t * per_tile + q];
            ts1 += part1[t * per_tile + q];
        }
        s += (i == j) ? ts : 2.0 * ts;
        s1 += (i == j) ? ts1 : 2.0 * ts1;
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_down_sync(0xffffffffu, s, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = s;
        red[32 + (threadIdx.x >> 5)] = s1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0.0, tot1 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            tot += red[w];
            tot1 += red[32 + w];
        }
        out[0] = tot;
        out[1] = tot1;
        const double nn = (double)n_pad;
        out[2] = nn > 1 ? (tot1 - nn) / (nn * nn - nn) : 0.0;
    }
}

// ----------------------------------------------------------------------------
// FP32 trailing update of step k (fp32 mode): for k < j <= i < NT,
// W_ij <- W_ij - L_ik L_jk^T.  At k = 0 the input is K (+ lambda on the
// diagonal of diagonal tiles); diagonal targets go to Wd.  Blocks strictly
// above the diagonal of a diagonal target are skipped.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) update_simt_kernel(int64_t k, int64_t nt, int64_t b,
                                                          float lambda, const float *Kd,
                                                          float *W, float *Wd, const uint8_t *pool,
                                                          const TileDesc *ltab) {
    const int64_t sub_side = b / SG_BM, sub_per_tile = sub_side * sub_side;
    const int64_t t = blockIdx.x / sub_per_tile, sub = blockIdx.x % sub_per_tile;
    int64_t ii, jj;
    tri_decode(t, &ii, &jj);
    const int64_t i = k + 1 + ii, j = k + 1 + jj;
    const int64_t sm = sub / sub_side, sn = sub % sub_side;
    if (i == j && sn > sm) return;
    const float *Li = (const float *)(pool + ltab[off_index(i, k)].offset);
    const float *Lj = (const float *)(pool + ltab[off_index(j, k)].offset);
    float acc[8][8];
    sg_mainloop<float, 0>(Li + sm * SG_BM * b, b, Lj + sn * SG_BN * b, b, (int)b, SG_BM, SG_BN, acc);
    const float *cin;
    float *cout;
    if (i == j) {
        cout = Wd + i * b * b;
        cin = (k == 0) ? Kd + tri_index(i, i) * b * b : cout;
    } else {
        cout = W + off_index(i, j) * b * b;
        cin = (k == 0) ? Kd + tri_index(i, j) * b * b : cout;
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int64_t lr = sm * SG_BM + sg_row(r);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t lc = sn * SG_BN + sg_col(q);
            float v = cin[lr * b + lc];
            if (k == 0 && i == j && lr == lc) v += lambda;
            cout[lr * b + lc] = v - acc[r][q];
        }
    }
}

void launch_update_simt(Ctx *c, int64_t k) {
    const int64_t u = c->nt - k - 1;
    if (u <= 0) return;
    const int64_t tiles = u * (u + 1) / 2, sub = (c->b / SG_BM) * (c->b / SG_BM);
    count_launch(), update_simt_kernel<<<(unsigned)(tiles * sub), 256, 0, c->stream>>>(
        k, c->nt, c->b, (float)c->lambda, c->Kd, (float *)c->W, c->Wd, c->pool, c->ltab);
}

// ----------------------------------------------------------------------------
// FP32 panel TRSM of column k (fp32 mode): L_ik = W_ik Linv_kk^T, written to
// the tile's FP32 slot of the pool.  Linv is lower triangular, so output
// columns [n0, n0 + 128) only need K-range [0, n0 + 128).
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) trsm_simt_kernel(int64_t k, int64_t b, const float *Kd,
                                                        const float *W, const float *Linv,
                                                        uint8_t *pool, const TileDesc *ltab) {
    const int64_t sub_side = b / SG_BM, sub_per_tile = sub_side * sub_side;
    const int64_t i = k + 1 + blockIdx.x / sub_per_tile, sub = blockIdx.x % sub_per_tile;
    const int64_t sm = sub / sub_side, sn = sub % sub_side;
    const float *a = (k == 0) ? Kd + tri_index(i, 0) * b * b : W + off_index(i, k) * b * b;
    const float *li = Linv + k * b * b;
    const int kext = (int)(b < (sn + 1) * SG_BN ? b : (sn + 1) * SG_BN);
    float acc[8][8];
    sg_mainloop<float, 0>(a + sm * SG_BM * b, b, li + sn * SG_BN * b, b, kext, SG_BM, SG_BN, acc);
    float *out = (float *)(pool + ltab[off_index(i, k)].offset);
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        const int64_t lr = sm * SG_BM + sg_row(r);
#pragma unroll
        for (int q = 0; q < 8; ++q) out[lr * b + sn * SG_BN + sg_col(q)] = acc[r][q];
    }
}

void launch_trsm_simt(Ctx *c, int64_t k) {
    const int64_t u = c->nt - k - 1;
    if (u <= 0) return;
    const int64_t sub = (c->b / SG_BM) * (c->b / SG_BM);
    count_launch(), trsm_simt_kernel<<<(unsigned)(u * sub), 256, 0, c->stream>>>(k, c->b, c->Kd, (const float *)c->W,
                                                                c->Linv, c->pool, c->ltab);
}

// ----------------------------------------------------------------------------
// FP32 predict on CUDA cores (fp32 mode).  One CTA per 128 x 128 block of
// test-row tile x training-row tile: K_test block -> shared memory -> times
// the 128 matching rows of A -> partial (128 x p) written to
// part[colblock][row][p]; colblock = training column / 128.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) predict_simt_kernel(const float *tf, const int32_t *tn,
                                                           int64_t n_test, const float *gf,
                                                           const int32_t *gn, int64_t n,
                                                           int64_t m_pad, int64_t ncolblk,
                                                           float gamma, const float *A, int64_t p,
                                                           int64_t ntest_pad, float *part) {
    extern __shared__ float sh[];
    float *Ks = sh;                    // 128 x 129
    float *As = sh + 128 * 129;        // 128 x p
    const int64_t rb = blockIdx.x / ncolblk, cb = blockIdx.x % ncolblk;
    const int64_t r0 = rb * SG_BM, c0 = cb * SG_BN;
    float acc[8][8];
    sg_mainloop<float, 0>(tf + r0 * m_pad, m_pad, gf + c0 * m_pad, m_pad, (int)m_pad, SG_BM, SG_BN,
                          acc);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t gi = r0 + sg_row(i);
        const int32_t ni = tn[gi];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t gj = c0 + sg_col(j);
            int32_t d = ni + gn[gj] - 2 * (int32_t)acc[i][j];
            Ks[sg_row(i) * 129 + sg_col(j)] = (gi < n_test && gj < n) ? expf(-gamma * (float)d) : 0.f;
        }
    }
    for (int64_t e = threadIdx.x; e < 128 * p; e += blockDim.x) {
        int64_t r = e / p, q = e % p;
        As[e] = (c0 + r < n) ? A[(c0 + r) * p + q] : 0.f;
    }
    __syncthreads();
    for (int64_t e = threadIdx.x; e < 128 * p; e += blockDim.x) {
        int64_t r = e / p, q = e % p;
        float s = 0.f;
        for (int cc = 0; cc < 128; ++cc) s = fmaf(Ks[r * 129 + cc], As[cc * p + q], s);
        part[(cb * ntest_pad + r0 + r) * p + q] = s;
    }
}

void launch_predict_simt(Ctx *c, const float *tf, const int32_t *tn, int64_t n_test,
                         int64_t rows_pad, const float *A, int64_t p, float *part) {
    const int64_t nrb = rows_pad / SG_BM, ncb = c->n_pad / SG_BN;
    size_t sh = (128 * 129 + 128 * p) * sizeof(float);
    if (sh > 48 * 1024)
        cudaFuncSetAttribute(predict_simt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    count_launch(), predict_simt_kernel<<<(unsigned)(nrb * ncb), 256, sh, c->stream>>>(
        tf, tn, n_test, c->gf, c->norms, c->n, c->m_pad, ncb, (float)c->gamma, A, p, rows_pad, part);
}

// Sum of partial products over column blocks in a fixed order.
__global__ void predict_reduce_kernel(const float *part, int64_t nblk, int64_t rows_pad,
                                      int64_t n_test, int64_t p, float *out, int64_t ldo) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_test * p) return;
    int64_t r = e / p, q = e % p;
    double s = 0.0;
    for (int64_t c = 0; c < nblk; ++c) s += (double)part[(c * rows_pad + r) * p + q];
    out[r * ldo + q] = (float)s;
}

void launch_predict_reduce(const float *part, int64_t nblk, int64_t rows_pad, int64_t n_test,
                           int64_t p, float *out, int64_t ldo, cudaStream_t s) {
    count_launch(), predict_reduce_kernel<<<cdiv(n_test * p, 256), 256, 0, s>>>(part, nblk, rows_pad, n_test, p,
                                                               out, ldo);
}

// ----------------------------------------------------------------------------
// Diagonal-tile Cholesky, blocked by NB = 64 inside the b x b tile.
// potrf_block_kernel factorises the NB x NB block (q, q) in shared memory
// (right-looking, one column per step), writes L_qq back (zero above the
// diagonal) and writes inv(L_qq) into the same block of the inverse tile.
// A pivot that is not positive is recorded in the error record (first one
// wins) and replaced by 1 so the rest of the factorisation stays finite.
// ----------------------------------------------------------------------------
constexpr int DNB = 64;

template <typename T>
__global__ void __launch_bounds__(256) potrf_block_kernel(T *W, T *Winv, int64_t b, int q,
                                                          int64_t tile_k, DevErrors *err,
                                                          double *minpiv) {
    __shared__ T a[DNB][DNB + 1];
    __shared__ int bad;
    T *blk = W + (int64_t)q * DNB * b + q * DNB;
    for (int e = threadIdx.x; e < DNB * DNB; e += blockDim.x) a[e / DNB][e % DNB] = blk[(e / DNB) * b + e % DNB];
    if (threadIdx.x == 0) bad = -1;
    __syncthreads();
    double mp = 1e300;
    for (int c = 0; c < DNB; ++c) {
        if (threadIdx.x == 0) {
            T d = a[c][c];
            if (!(d > T(0))) {
                if (bad < 0) bad = c;
                d = T(1);
            }
            a[c][c] = sqrt(d);
        }
        __syncthreads();
        const T piv = a[c][c];
        if (threadIdx.x == 0 && (double)piv < mp) mp = (double)piv;
        for (int r = c + 1 + threadIdx.x; r < DNB; r += blockDim.x) a[r][c] /= piv;
        __syncthreads();
        for (int e = threadIdx.x; e < (DNB - c - 1) * (DNB - c - 1); e += blockDim.x) {
            int r = c + 1 + e / (DNB - c - 1), s = c + 1 + e % (DNB - c - 1);
            if (s <= r) a[r][s] -= a[r][c] * a[s][c];
        }
        __syncthreads();
    }
    // inverse by forward substitution: thread t < DNB owns column t of inv(L)
    // and reads back only the entries it wrote itself.
    T *iblk = Winv + (int64_t)q * DNB * b + q * DNB;
    if (threadIdx.x < DNB) {
        const int col = threadIdx.x;
        for (int r = 0; r < DNB; ++r) {
            T v = T(0);
            if (r >= col) {
                T s = (r == col) ? T(1) : T(0);
                for (int kk = col; kk < r; ++kk) s -= a[r][kk] * iblk[(int64_t)kk * b + col];
                v = s / a[r][r];
            }
            iblk[(int64_t)r * b + col] = v;
        }
    }
    for (int e = threadIdx.x; e < DNB * DNB; e += blockDim.x) {
        int r = e / DNB, s = e % DNB;
        blk[r * b + s] = (s <= r) ? a[r][s] : T(0);
    }
    if (threadIdx.x == 0) {
        minpiv[q] = mp;
        if (bad >= 0 && atomicCAS(&err->code, 0, (int)KRR_ENOTPD) == 0) {
            err->bad_tile = tile_k;
            err->bad_column = tile_k * b + (int64_t)q * DNB + bad;
        }
    }
}

__global__ void f32_to_f64_kernel(const float *src, double *dst, int64_t count, double diag_add,
                                  int64_t b) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= count) return;
    double v = src[e];
    if (diag_add != 0.0 && (e / b) == (e % b)) v += diag_add;
    dst[e] = v;
}

__global__ void copy_add_diag_kernel(const float *src, float *dst, int64_t count, float diag_add,
                                     int64_t b) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= count) return;
    float v = src[e];
    if ((e / b) == (e % b)) v += diag_add;
    dst[e] = v;
}

// FP64 inverse -> FP32 Linv (+ FP16 split); FP32 inverse -> FP16 split only.
__global__ void finish_inverse_kernel(const double *inv64, float *inv32, __half *hi, __half *lo,
                                      int64_t count) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= count) return;
    float v = inv64 ? (float)inv64[e] : inv32[e];
    if (inv64) inv32[e] = v;
    if (hi) {
        __half h = __float2half_rn(v);
        hi[e] = h;
        lo[e] = __float2half_rn(v - __half2float(h));
    }
}

template <typename T>
static void diag_factor_tile(Ctx *c, T *W, T *Winv, T *tmp, int64_t k, double *minpiv) {
    const int64_t b = c->b;
    const int nq = (int)(b / DNB);
    cudaStream_t s = c->stream;
    cudaMemsetAsync(Winv, 0, sizeof(T) * b * b, s);
    for (int q = 0; q < nq; ++q) {
        count_launch(), potrf_block_kernel<T><<<1, 256, 0, s>>>(W, Winv, b, q, k, c->derr, minpiv + k * nq);
        const int rest = (int)(b - (int64_t)(q + 1) * DNB);
        if (rest <= 0) break;
        T *panel = W + (int64_t)(q + 1) * DNB * b + q * DNB;
        // panel <- panel * inv(L_qq)^T  (in place: each CTA owns its rows)
        launch_gemm_simt<T>(rest, DNB, DNB, T(1), panel, b, 0, Winv + (int64_t)q * DNB * b + q * DNB,
                            b, 0, 0, T(0), nullptr, 0, 0, panel, b, 0, 1, 0, s);
        // trailing lower part <- trailing - panel panel^T
        T *trail = W + (int64_t)(q + 1) * DNB * b + (q + 1) * DNB;
        launch_gemm_simt<T>(rest, rest, DNB, T(-1), panel, b, 0, panel, b, 0, 0, T(1), trail, b, 0,
                            trail, b, 0, 1, 1, s);
    }
    // Triangular inverse by block diagonals: X_ij = -X_ii sum_{l=j}^{i-1} L_il X_lj.
    for (int d = 1; d < nq; ++d) {
        const int cnt = nq - d;
        const int64_t diag_stride = (int64_t)DNB * b + DNB;
        // tmp_j = L[i-block, j..i-1 blocks] * X[j..i-1 blocks, j-block]   (i = j + d)
        launch_gemm_simt<T>(DNB, DNB, DNB * d, T(1), W + (int64_t)d * DNB * b, b, diag_stride, Winv,
                            b, diag_stride, 1, T(0), nullptr, 0, 0, tmp, DNB, DNB * DNB, cnt, 0, s);
        // X_ij = -X_ii tmp_j
        launch_gemm_simt<T>(DNB, DNB, DNB, T(-1), Winv + (int64_t)d * DNB * b + d * DNB, b,
                            diag_stride, tmp, DNB, DNB * DNB, 1, T(0), nullptr, 0, 0,
                            Winv + (int64_t)d * DNB * b, b, diag_stride, cnt, 0, s);
    }
}

// sqrt of the largest diagonal entry of W_kk: a bound on every |L_kk| entry
// (|L_rc| <= sqrt(W_rr) for a Cholesky factor).
__global__ void diag_max_kernel(const float *w, int64_t b, double *out) {
    __shared__ float red[32];
    float mx = 0.f;
    for (int64_t r = threadIdx.x; r < b; r += blockDim.x) mx = fmaxf(mx, w[r * b + r]);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) m = fmaxf(m, red[q]);
        *out = sqrt((double)fmaxf(m, 0.f));
    }
}

__global__ void f64_to_f32_kernel(const double *src, float *dst, int64_t count) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < count) dst[e] = (float)src[e];
}

__global__ void min_pivot_kernel(const double *mp, int n, DevErrors *err) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double m = err->min_pivot;
    for (int i = 0; i < n; ++i) m = fmin(m, mp[i]);
    err->min_pivot = m;
}

krr_status diag_step(Ctx *c, int64_t k) {
    const int64_t b = c->b, bb = b * b;
    cudaStream_t s = c->stream;
    float *wd = c->Wd + k * bb;
    float *linv = c->Linv + k * bb;
    const int nq = (int)(b / DNB);
    double *minpiv = c->red + RED_MINPIV;
    double *lkk = c->red + RED_MINPIV + c->nt * nq;
    unsigned g = cdiv(bb, 256);
    if (k == 0) count_launch(), copy_add_diag_kernel<<<g, 256, 0, s>>>(c->Kd, wd, bb, (float)c->lambda, b);
    count_launch(), diag_max_kernel<<<1, 256, 0, s>>>(wd, b, lkk + k);
    if (c->opt.diag_fp64) {
        count_launch(), f32_to_f64_kernel<<<g, 256, 0, s>>>(wd, c->diag64, bb, 0.0, b);
        diag_factor_tile<double>(c, c->diag64, c->diag64_inv, c->diag64_inv + bb, k, minpiv);
        count_launch(), f64_to_f32_kernel<<<g, 256, 0, s>>>(c->diag64, wd, bb);
        count_launch(), finish_inverse_kernel<<<g, 256, 0, s>>>(c->diag64_inv, linv,
                                                c->Linv_hi ? c->Linv_hi + k * bb : nullptr,
                                                c->Linv_lo ? c->Linv_lo + k * bb : nullptr, bb);
    } else {
        diag_factor_tile<float>(c, wd, linv, (float *)c->diag64, k, minpiv);
        if (c->Linv_hi)
            count_launch(), finish_inverse_kernel<<<g, 256, 0, s>>>(nullptr, linv, c->Linv_hi + k * bb,
                                                    c->Linv_lo + k * bb, bb);
    }
    count_launch(), min_pivot_kernel<<<1, 1, 0, s>>>(minpiv + k * nq, nq, c->derr);
    return KRR_OK;
}

// ----------------------------------------------------------------------------
// Adaptive precision of one factor column (mixed mode).
// Tile (i, k), i > k, is stored at unit roundoff u_p when
//     u_p * max|L_ik| * max|L_kk| <= eps * lambda,
// the lowest allowed of E4M3 (u = 2^-4) and FP16 (u = 2^-11), else FP32.
// Rounding L_ik perturbs L L^T in block (i, k) by about u_p |L_ik| |L_kk|;
// the refinement converges while that stays well below lambda, the smallest
// possible eigenvalue of K + lambda I.  max|L_kk| is bounded by
// sqrt(max_r W_kk[r, r]) from the diagonal step.  FP16/E4M3 tiles carry a
// power-of-two scale so the largest entry sits near the top of the format.
// ----------------------------------------------------------------------------
__global__ void column_stats_kernel(const float *col, int64_t bb, int chunks, double *part_ss,
                                    float *part_max) {
    const int64_t tile = blockIdx.y, ch = blockIdx.x;
    const int64_t per = bb / chunks;
    const float4 *src = reinterpret_cast<const float4 *>(col + tile * bb + ch * per);
    double ss = 0.0;
    float mx = 0.f;
    for (int64_t e = threadIdx.x; e < per / 4; e += blockDim.x) {
        float4 v = src[e];
        ss += (double)v.x * v.x + (double)v.y * v.y + (double)v.z * v.z + (double)v.w * v.w;
        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    __shared__ double rs[32];
    __shared__ float rm[32];
    for (int o = 16; o > 0; o >>= 1) {
        ss += __shfl_down_sync(0xffffffffu, ss, o);
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) { rs[threadIdx.x >> 5] = ss; rm[threadIdx.x >> 5] = mx; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        float m = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { s += rs[w]; m = fmaxf(m, rm[w]); }
        part_ss[tile * chunks + ch] = s;
        part_max[tile * chunks + ch] = m;
    }
}

__device__ inline float pow2_scale(float mx, float top) {
    if (!(mx > 0.f)) return 1.f;
    int e = (int)floorf(log2f(top / mx));
    e = max(-100, min(100, e));
    float s = ldexpf(1.f, e);
    while (mx * s > top) s *= 0.5f;
    return s;
}

__global__ void column_decide_kernel(int64_t k, int64_t nt, int64_t bb, int chunks,
                                     const double *part_ss, const float *part_max, double thresh,
                                     const double *lkk_max, int allow_fp8, TileDesc *ltab,
                                     uint8_t *precmap, DevErrors *err) {
    const int64_t tile = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tile >= nt - k - 1) return;
    double ss = 0;
    float mx = 0;
    for (int q = 0; q < chunks; ++q) {
        ss += part_ss[tile * chunks + q];
        mx = fmaxf(mx, part_max[tile * chunks + q]);
    }
    const double w = (double)mx * lkk_max[k];
    int prec;
    if (allow_fp8 && 0.0625 * w <= thresh) prec = KRR_PREC_E4M3;
    else if (0x1p-11 * w <= thresh) prec = KRR_PREC_FP16;
    else prec = KRR_PREC_FP32;
    (void)ss;
    const int64_t i = k + 1 + tile;
    TileDesc d;
    d.prec = prec;
    d.scale = (prec == KRR_PREC_E4M3) ? pow2_scale(mx, 448.f) : pow2_scale(mx, 32768.f);
    const int64_t bytes = bb * (prec == KRR_PREC_FP32 ? 4 : (prec == KRR_PREC_FP16 ? 2 : 1));
    d.offset = (int64_t)atomicAdd((unsigned long long *)&err->pool_cursor, (unsigned long long)bytes);
    ltab[off_index(i, k)] = d;
    precmap[i * nt + k] = (uint8_t)prec;
    atomicAdd((unsigned long long *)(prec == KRR_PREC_E4M3 ? &err->fp8_tiles
                                     : prec == KRR_PREC_FP16 ? &err->fp16_tiles : &err->fp32_tiles),
              1ull);
}

__global__ void column_write_kernel(int64_t k, int64_t bb, const float *col, const TileDesc *ltab,
                                    uint8_t *pool, __half *pan_hi, __half *pan_lo,
                                    uint8_t *pan_f8) {
    const int64_t tile = blockIdx.y;
    const int64_t i = k + 1 + tile;
    const TileDesc d = ltab[off_index(i, k)];
    const float *src = col + tile * bb;
    __half *hi = pan_hi + tile * bb;
    __half *lo = pan_lo + tile * bb;
    uint8_t *f8 = pan_f8 + tile * bb;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < bb;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float v = src[e];
        const float sv = v * d.scale;
        if (d.prec == KRR_PREC_E4M3) {
            __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(sv, __NV_SATFINITE, __NV_E4M3);
            f8[e] = q;
            pool[d.offset + e] = q;
            __half_raw hr = __nv_cvt_fp8_to_halfraw(q, __NV_E4M3);
            hi[e] = __half(hr);
        } else if (d.prec == KRR_PREC_FP16) {
            __half h = __float2half_rn(sv);
            hi[e] = h;
            reinterpret_cast<__half *>(pool + d.offset)[e] = h;
        } else {
            reinterpret_cast<float *>(pool + d.offset)[e] = v;
            __half h = __float2half_rn(sv);
            hi[e] = h;
            lo[e] = __float2half_rn(sv - __half2float(h));
        }
    }
}

void launch_column_cast(Ctx *c, int64_t k) {
    const int64_t u = c->nt - k - 1;
    if (u <= 0) return;
    const int64_t bb = c->b * c->b;
    const int chunks = 16;
    double *part_ss = c->colnorm2;
    float *part_max = c->colmax;
    count_launch(), column_stats_kernel<<<dim3(chunks, (unsigned)u), 256, 0, c->stream>>>(c->colbuf, bb, chunks,
                                                                          part_ss, part_max);
    const double thresh = c->opt.eps * c->lambda;
    const double *lkk = c->red + RED_MINPIV + c->nt * (c->b / 64);
    count_launch(), column_decide_kernel<<<cdiv(u, 128), 128, 0, c->stream>>>(k, c->nt, bb, chunks, part_ss, part_max,
                                                               thresh, lkk, c->opt.allow_fp8,
                                                               c->ltab, c->precmap, c->derr);
    count_launch(), column_write_kernel<<<dim3(64, (unsigned)u), 256, 0, c->stream>>>(k, bb, c->colbuf, c->ltab,
                                                                      c->pool, c->pan_hi, c->pan_lo,
                                                                      c->pan_f8);
}

void launch_kernel_sumsq(Ctx *c, double *out) {
    const int64_t ntri = c->nt * (c->nt + 1) / 2;
    const int64_t per = (c->opt.mode == KRR_MODE_FP32) ? (c->b / SG_BM) * (c->b / SG_BM)
                                                       : (c->b / 128) * (c->b / 256);
    count_launch(), kernel_sumsq_kernel<<<1, 1024, 0, c->stream>>>(c->knorm2, ntri, per, c->n_pad, out);
}

// ----------------------------------------------------------------------------
// Triangular solves with the stored factor, p right-hand sides (columns
// processed in chunks of at most PC).  Forward: for k = 0..NT-1,
// Z_k = Linv_kk Y_k, then Y_i -= L_ik Z_k for i > k.  Backward: for
// k = NT-1..0, A_k = Linv_kk^T Z_k, then Z_j -= L_kj^T A_k for j < k.
// Every output element has one owner (no atomics): results are deterministic.
// ----------------------------------------------------------------------------
constexpr int PC = 32;

__device__ __forceinline__ float load_l(const uint8_t *base, int prec, int64_t e) {
    if (prec == KRR_PREC_FP32) return reinterpret_cast<const float *>(base)[e];
    if (prec == KRR_PREC_FP16) return __half2float(reinterpret_cast<const __half *>(base)[e]);
    __half_raw h = __nv_cvt_fp8_to_halfraw(base[e], __NV_E4M3);
    return __half2float(__half(h));
}

// Forward kernel: out rows (-)= M x_k, one warp per row, lanes over c.
// mode 0: M = Linv_kk (FP32, lower: c <= r); out = block k of `out`, stored.
// mode 1: M = L_ik for every i > k (grid.y); out = block i of `out`,
//         subtracted.  x_k is block k of `in`; `in` and the written blocks of
//         `out` never overlap.
__global__ void __launch_bounds__(256) solve_fwd_kernel(int mode, int64_t k, int64_t b,
                                                        const float *Linv, const uint8_t *pool,
                                                        const TileDesc *ltab, const float *in,
                                                        float *out, int64_t ldx, int q0, int pc) {
    extern __shared__ float zs[];  // b x pc
    const float *zsrc = in + k * b * ldx;
    for (int64_t e = threadIdx.x; e < b * pc; e += blockDim.x) zs[e] = zsrc[(e / pc) * ldx + q0 + e % pc];
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t tile = (mode == 0) ? k : (k + 1 + blockIdx.y);
    const int64_t rbase = blockIdx.x * 64;
    const uint8_t *base;
    int prec;
    float inv_scale;
    if (mode == 0) {
        base = reinterpret_cast<const uint8_t *>(Linv + k * b * b);
        prec = KRR_PREC_FP32;
        inv_scale = 1.f;
    } else {
        const TileDesc d = ltab[off_index(tile, k)];
        base = pool + d.offset;
        prec = d.prec;
        inv_scale = (prec == KRR_PREC_FP32) ? 1.f : 1.f / d.scale;
    }
    float *dst_blk = out + tile * b * ldx;
    for (int64_t r = rbase + warp; r < rbase + 64; r += 8) {
        float acc[PC];
#pragma unroll
        for (int q = 0; q < PC; ++q) acc[q] = 0.f;
        const int64_t cend = (mode == 0) ? r + 1 : b;
        for (int64_t cidx = lane; cidx < cend; cidx += 32) {
            const float l = load_l(base, prec, r * b + cidx);
            const float *zr = zs + cidx * pc;
#pragma unroll
            for (int q = 0; q < PC; ++q)
                if (q < pc) acc[q] = fmaf(l, zr[q], acc[q]);
        }
        float mine = 0.f;
#pragma unroll
        for (int q = 0; q < PC; ++q) {
            if (q >= pc) break;
            float v = acc[q];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == q) mine = v;
        }
        if (lane < pc) {
            float *dst = dst_blk + r * ldx + q0 + lane;
            if (mode == 0) *dst = mine * inv_scale;
            else *dst -= mine * inv_scale;
        }
    }
}

// Backward kernel: out cols (-)= M^T x_k, one thread per column c.
// mode 0: M = Linv_kk (lower: r >= c); out = block k of `out`, stored.
// mode 1: M = L_kj for every j < k (grid.y); out = block j of `out`,
//         subtracted.  x_k is block k of `in`.
__global__ void __launch_bounds__(128) solve_bwd_kernel(int mode, int64_t k, int64_t b,
                                                        const float *Linv, const uint8_t *pool,
                                                        const TileDesc *ltab, const float *in,
                                                        float *out, int64_t ldx, int q0, int pc) {
    extern __shared__ float as[];  // b x pc
    const float *asrc = in + k * b * ldx;
    for (int64_t e = threadIdx.x; e < b * pc; e += blockDim.x) as[e] = asrc[(e / pc) * ldx + q0 + e % pc];
    __syncthreads();
    const int64_t cidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t j = (mode == 0) ? k : blockIdx.y;
    const uint8_t *base;
    int prec;
    float inv_scale;
    if (mode == 0) {
        base = reinterpret_cast<const uint8_t *>(Linv + k * b * b);
        prec = KRR_PREC_FP32;
        inv_scale = 1.f;
    } else {
        const TileDesc d = ltab[off_index(k, j)];
        base = pool + d.offset;
        prec = d.prec;
        inv_scale = (prec == KRR_PREC_FP32) ? 1.f : 1.f / d.scale;
    }
    float acc[PC];
#pragma unroll
    for (int q = 0; q < PC; ++q) acc[q] = 0.f;
    const int64_t rstart = (mode == 0) ? cidx : 0;
    for (int64_t r = rstart; r < b; ++r) {
        const float l = load_l(base, prec, r * b + cidx);
        const float *ar = as + r * pc;
#pragma unroll
        for (int q = 0; q < PC; ++q)
            if (q < pc) acc[q] = fmaf(l, ar[q], acc[q]);
    }
    float *dst = out + (j * b + cidx) * ldx + q0;
#pragma unroll
    for (int q = 0; q < PC; ++q) {
        if (q >= pc) break;
        if (mode == 0) dst[q] = acc[q] * inv_scale;
        else dst[q] -= acc[q] * inv_scale;
    }
}

// x (n_pad x p) <- (L L^T)^-1 x.  tmp is n_pad x p scratch.  Forward:
// tmp_k = Linv_kk x_k, then x_i -= L_ik tmp_k (i > k); tmp ends as Z.
// Backward: x_k = Linv_kk^T tmp_k, then tmp_j -= L_kj^T x_k (j < k).
void solve_inplace(Ctx *c, float *x, float *tmp, int64_t p) {
    const int64_t b = c->b, nt = c->nt;
    cudaStream_t s = c->stream;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(solve_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(solve_bwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    const int pcmax = (int)std::max<int64_t>(1, std::min<int64_t>(PC, 32768 / b));
    for (int q0 = 0; q0 < p; q0 += pcmax) {
        const int pc = (int)std::min<int64_t>(pcmax, p - q0);
        const size_t sh = (size_t)b * pc * sizeof(float);
        for (int64_t k = 0; k < nt; ++k) {
            count_launch(), solve_fwd_kernel<<<dim3((unsigned)(b / 64), 1), 256, sh, s>>>(0, k, b, c->Linv, c->pool,
                                                                           c->ltab, x, tmp, p, q0, pc);
            if (k + 1 < nt)
                count_launch(), solve_fwd_kernel<<<dim3((unsigned)(b / 64), (unsigned)(nt - k - 1)), 256, sh, s>>>(
                    1, k, b, c->Linv, c->pool, c->ltab, tmp, x, p, q0, pc);
        }
        for (int64_t k = nt - 1; k >= 0; --k) {
            count_launch(), solve_bwd_kernel<<<dim3((unsigned)(b / 128), 1), 128, sh, s>>>(0, k, b, c->Linv, c->pool,
                                                                            c->ltab, tmp, x, p, q0, pc);
            if (k > 0)
                count_launch(), solve_bwd_kernel<<<dim3((unsigned)(b / 128), (unsigned)k), 128, sh, s>>>(
                    1, k, b, c->Linv, c->pool, c->ltab, x, tmp, p, q0, pc);
        }
    }
}

// ----------------------------------------------------------------------------
// Residual r = y - lambda a - K a with K read from the FP32 lower-triangle
// tiles (symmetric use).  Products in FP32, partial sums per tile row in
// FP32, tiles accumulated in FP64.  Two passes so that every output element
// has one owner: the N pass covers tiles (i, j <= i) row-wise, the T pass
// covers tiles (j > i, i) column-wise.
// ----------------------------------------------------------------------------
__global__ void __launch_bounds__(256) residual_n_kernel(int64_t nt, int64_t b, float lambda,
                                                         const float *Kd, const float *y,
                                                         const float *a, double *r, int64_t p,
                                                         int q0, int pc, const double *shift,
                                                         const double *colsum) {
    const float cs = (float)*shift;
    extern __shared__ float ash[];  // b x pc (block j of a)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t i = blockIdx.y;
    const int64_t rbase = blockIdx.x * 64;
    // each warp owns 8 rows: rbase + warp + 8 * t
    double rowacc[8];
    for (int t = 0; t < 8; ++t) rowacc[t] = 0.0;
    for (int64_t j = 0; j <= i; ++j) {
        __syncthreads();
        for (int64_t e = threadIdx.x; e < b * pc; e += blockDim.x)
            ash[e] = a[(j * b + e / pc) * p + q0 + e % pc];
        __syncthreads();
        const float *kt = Kd + tri_index(i, j) * b * b;
        for (int t = 0; t < 8; ++t) {
            const int64_t row = rbase + warp + 8 * t;
            float acc[PC];
#pragma unroll
            for (int q = 0; q < PC; ++q) acc[q] = 0.f;
            for (int64_t cidx = lane; cidx < b; cidx += 32) {
                const float kv = kt[row * b + cidx] - cs;
                const float *ar = ash + cidx * pc;
#pragma unroll
                for (int q = 0; q < PC; ++q)
                    if (q < pc) acc[q] = fmaf(kv, ar[q], acc[q]);
            }
#pragma unroll
            for (int q = 0; q < PC; ++q) {
                if (q >= pc) break;
                float v = acc[q];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                if (lane == q) rowacc[t] += (double)v;
            }
        }
    }
    for (int t = 0; t < 8; ++t) {
        const int64_t row = i * b + rbase + warp + 8 * t;
        if (lane < pc) {
            const int64_t e = row * p + q0 + lane;
            r[e] = (double)y[e] - (double)lambda * (double)a[e] - rowacc[t] -
                   (double)cs * colsum[q0 + lane];
        }
    }
}

__global__ void __launch_bounds__(128) residual_t_kernel(int64_t nt, int64_t b, const float *Kd,
                                                         const float *a, double *r, int64_t p,
                                                         int q0, int pc, const double *shift) {
    const float cs = (float)*shift;
    extern __shared__ float ash[];  // b x pc (block j of a)
    const int64_t i = blockIdx.y;
    const int64_t cidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double acc64[PC];
#pragma unroll
    for (int q = 0; q < PC; ++q) acc64[q] = 0.0;
    for (int64_t j = i + 1; j < nt; ++j) {
        __syncthreads();
        for (int64_t e = threadIdx.x; e < b * pc; e += blockDim.x)
            ash[e] = a[(j * b + e / pc) * p + q0 + e % pc];
        __syncthreads();
        const float *kt = Kd + tri_index(j, i) * b * b;
        float acc[PC];
#pragma unroll
        for (int q = 0; q < PC; ++q) acc[q] = 0.f;
        for (int64_t rr = 0; rr < b; ++rr) {
            const float kv = kt[rr * b + cidx] - cs;
            const float *ar = ash + rr * pc;
#pragma unroll
            for (int q = 0; q < PC; ++q)
                if (q < pc) acc[q] = fmaf(kv, ar[q], acc[q]);
        }
#pragma unroll
        for (int q = 0; q < PC; ++q) acc64[q] += (double)acc[q];
    }
    for (int q = 0; q < pc; ++q) r[(i * b + cidx) * p + q0 + q] -= acc64[q];
}

// Column sums of a (n x p) in FP64, one block per column.
__global__ void colsum_kernel(const float *a, int64_t n, int64_t p, double *out) {
    __shared__ double red[32];
    const int64_t q = blockIdx.x;
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) s += (double)a[r * p + q];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        out[q] = t;
    }
}

// K A = (K - c 1 1^T) A + c 1 (1^T A): the shifted products are small, so
// FP32 products and partial sums lose far less to cancellation; c 1^T A is
// formed in FP64.  c = the mean off-diagonal entry of K (red[RED_KSHIFT]).
void launch_residual(Ctx *c, const float *y, const float *a, double *r, int64_t p) {
    const int64_t b = c->b, nt = c->nt;
    const int pcmax = (int)std::max<int64_t>(1, std::min<int64_t>(PC, 32768 / b));
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(residual_n_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        cudaFuncSetAttribute(residual_t_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        attr_set = true;
    }
    const double *shift = c->red + RED_KSHIFT;
    count_launch(), colsum_kernel<<<(unsigned)p, 512, 0, c->stream>>>(a, c->n_pad, p, c->colsum);
    for (int q0 = 0; q0 < p; q0 += pcmax) {
        const int pc = (int)std::min<int64_t>(pcmax, p - q0);
        const size_t sh = (size_t)b * pc * sizeof(float);
        count_launch(), residual_n_kernel<<<dim3((unsigned)(b / 64), (unsigned)nt), 256, sh, c->stream>>>(
            nt, b, (float)c->lambda, c->Kd, y, a, r, p, q0, pc, shift, c->colsum);
        count_launch(), residual_t_kernel<<<dim3((unsigned)(b / 128), (unsigned)nt), 128, sh, c->stream>>>(
            nt, b, c->Kd, a, r, p, q0, pc, shift);
    }
}

// ||r||_F^2 and ||y||_F^2 into out[0], out[1] (deterministic single block).
__global__ void reduce_norms_kernel(const double *r, const float *y, int64_t count, double *out) {
    __shared__ double s1[32], s2[32];
    double a = 0, bsum = 0;
    for (int64_t e = threadIdx.x; e < count; e += blockDim.x) {
        a += r[e] * r[e];
        bsum += (double)y[e] * (double)y[e];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        bsum += __shfl_down_sync(0xffffffffu, bsum, o);
    }
    if ((threadIdx.x & 31) == 0) { s1[threadIdx.x >> 5] = a; s2[threadIdx.x >> 5] = bsum; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double x = 0, z = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { x += s1[w]; z += s2[w]; }
        out[0] = x;
        out[1] = z;
    }
}

void launch_reduce_norms(const double *r, const float *y, int64_t n, int64_t p, double *out,
                         cudaStream_t s) {
    count_launch(), reduce_norms_kernel<<<1, 1024, 0, s>>>(r, y, n * p, out);
}

__global__ void d2f_kernel(const double *r, float *dst, int64_t count) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < count) dst[e] = (float)r[e];
}
void launch_axpy_r(const double *r, float *dst, int64_t count, cudaStream_t s) {
    count_launch(), d2f_kernel<<<cdiv(count, 256), 256, 0, s>>>(r, dst, count);
}

__global__ void add_kernel(float *a, const float *da, float alpha, int64_t count) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < count) a[e] += alpha * da[e];
}
void launch_add_scaled(float *a, const float *da, float alpha, int64_t count, cudaStream_t s) {
    count_launch(), add_kernel<<<cdiv(count, 256), 256, 0, s>>>(a, da, alpha, count);
}

// dst (rows_pad x cols, dense) <- src rows (zero padding rows >= rows).
__global__ void copy_rows_kernel(const float *src, int64_t lds, float *dst, int64_t ldd,
                                 int64_t rows, int64_t cols, int64_t rows_pad) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows_pad * cols) return;
    int64_t r = e / cols, q = e % cols;
    dst[r * ldd + q] = (r < rows) ? src[r * lds + q] : 0.f;
}
void launch_copy_rows(const float *src, int64_t lds, float *dst, int64_t ldd, int64_t rows,
                      int64_t cols, int64_t rows_pad, cudaStream_t s) {
    count_launch(), copy_rows_kernel<<<cdiv(rows_pad * cols, 256), 256, 0, s>>>(src, lds, dst, ldd, rows, cols,
                                                                rows_pad);
}

void launch_fill_zero(void *p, size_t bytes, cudaStream_t s) { cudaMemsetAsync(p, 0, bytes, s); }

// Dense lower-triangular copy of the stored factor (diagonal tiles from Wd,
// off-diagonal tiles from the pool in their precision, de-scaled).
__global__ void factor_to_dense_kernel(const float *Wd, const uint8_t *pool, const TileDesc *ltab,
                                       int64_t b, int64_t n, float *dst, int64_t ld) {
    const int64_t t = blockIdx.y;
    int64_t ti, tj;
    tri_decode(t, &ti, &tj);
    const uint8_t *base;
    int prec;
    float inv_scale = 1.f;
    if (ti == tj) {
        base = reinterpret_cast<const uint8_t *>(Wd + ti * b * b);
        prec = KRR_PREC_FP32;
    } else {
        const TileDesc d = ltab[off_index(ti, tj)];
        base = pool + d.offset;
        prec = d.prec;
        if (prec != KRR_PREC_FP32) inv_scale = 1.f / d.scale;
    }
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < b * b;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lr = e / b, lc = e % b;
        const int64_t r = ti * b + lr, q = tj * b + lc;
        if (r >= n || q >= n) continue;
        float v = load_l(base, prec, e) * inv_scale;
        if (ti == tj && lc > lr) v = 0.f;
        dst[r * ld + q] = v;
    }
}

void launch_factor_to_dense(Ctx *c, float *dst, int64_t ld) {
    const int64_t ntri = c->nt * (c->nt + 1) / 2;
    count_launch(), factor_to_dense_kernel<<<dim3(64, (unsigned)ntri), 256, 0, c->stream>>>(
        c->Wd, c->pool, c->ltab, c->b, c->n, dst, ld);
}

}  // namespace krr
