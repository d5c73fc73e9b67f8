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

// The same with 16 genotypes per thread and step (16-byte loads and stores):
// rows 16-byte aligned, m a multiple of 16.
__global__ void pack_genotypes16_kernel(const int8_t *__restrict__ g, int64_t n, int64_t m, int64_t ldg,
                                        int64_t m_pad, uint8_t *__restrict__ out8, float *__restrict__ outf,
                                        int32_t *__restrict__ norms) {
    const int64_t row = blockIdx.x;
    int32_t s = 0;
    for (int64_t k = (int64_t)threadIdx.x * 16; k < m_pad; k += (int64_t)blockDim.x * 16) {
        uint4 in = make_uint4(0u, 0u, 0u, 0u);
        if (row < n && k < m) in = __ldcs(reinterpret_cast<const uint4 *>(g + row * ldg + k));
        const uint32_t w[4] = {in.x, in.y, in.z, in.w};
        uint32_t o[4];
        float f[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t acc = 0u;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int v = (int)(int8_t)((w[q] >> (8 * e)) & 0xffu);
                s += v * v;
                const uint32_t code = v == 0 ? 0x00u : (v == 1 ? 0x38u : (v == 2 ? 0x40u : 0x48u));
                acc |= code << (8 * e);
                f[4 * q + e] = (float)v;
            }
            o[q] = acc;
        }
        if (out8) *reinterpret_cast<uint4 *>(out8 + row * m_pad + k) = make_uint4(o[0], o[1], o[2], o[3]);
        if (outf) {
            float4 *dst = reinterpret_cast<float4 *>(outf + row * m_pad + k);
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[q] = make_float4(f[4 * q], f[4 * q + 1], f[4 * q + 2], f[4 * q + 3]);
        }
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

// IBS encoding (Alg. 5, second branch): genotype g becomes the two
// indicators [g >= 1], [g >= 2] (E4M3 0x38 = 1, 0x00 = 0).  The squared
// Euclidean distance of two encoded rows is then the L1 distance of the
// genotypes, and the encoded row's squared norm is n_i = sum_k g_ik.
// Encoded column k holds locus k / 2, level k % 2.
__global__ void pack_thermo_kernel(const int8_t *__restrict__ g, int64_t n, int64_t m, int64_t ldg, int64_t m_pad,
                                   uint8_t *__restrict__ out8, float *__restrict__ outf, int32_t *__restrict__ norms) {
    const int64_t row = blockIdx.x;
    int32_t s = 0;
    for (int64_t k = threadIdx.x; k < m_pad; k += blockDim.x) {
        const int64_t locus = k >> 1;
        int v = 0;
        if (row < n && locus < m) v = g[row * ldg + locus];
        const int f = (v >= 1 + (int)(k & 1)) ? 1 : 0;
        s += f;
        if (out8) out8[row * m_pad + k] = f ? 0x38 : 0x00;
        if (outf) outf[row * m_pad + k] = (float)f;
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
                           cudaStream_t s, int thermo) {
    if (thermo) {
        count_launch(), pack_thermo_kernel<<<(unsigned)n_pad, 256, 0, s>>>(g, n, m, ldg, m_pad, out8, outf, norms);
        return;
    }
    const bool wide = ((reinterpret_cast<uintptr_t>(g) | (uintptr_t)ldg | (uintptr_t)m) & 15u) == 0 &&
                      m_pad % 16 == 0;
    if (wide)
        count_launch(), pack_genotypes16_kernel<<<(unsigned)n_pad, 256, 0, s>>>(g, n, m, ldg, m_pad, out8, outf, norms);
    else
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
                                                         float gamma, KernelFn kf, const float *conf, int nc,
                                                         float *Kd, uint32_t *Dd, double *knorm_part) {
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
        float ci[CONF_MAX];
#pragma unroll
        for (int q = 0; q < CONF_MAX; ++q) ci[q] = (q < nc) ? conf[gi * CONF_MAX + q] : 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t lc = sn * SG_BN + sg_col(j), gj = tj * b + lc;
            int32_t d = ni + norms[gj] - 2 * (int32_t)acc[i][j];
            const float dc = nc ? conf_dist(ci, conf + gj * CONF_MAX, nc) : 0.f;
            float kv;
            if (gi < n && gj < n) kv = kf.gram ? acc[i][j] : kf.value(gamma, d, dc);
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
        c->gf, c->norms, c->m_pad, real_rows(c), c->b, (float)c->gamma, kernel_fn(c), c->conf, (int)c->nconf, c->Kd,
        c->Dd, c->knorm2);
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
                                                           float gamma, KernelFn kf, const float *tconf,
                                                           const float *gconf, int nc, const float *A, int64_t p,
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
        float ci[CONF_MAX];
#pragma unroll
        for (int q = 0; q < CONF_MAX; ++q) ci[q] = (q < nc) ? tconf[gi * CONF_MAX + q] : 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int64_t gj = c0 + sg_col(j);
            int32_t d = ni + gn[gj] - 2 * (int32_t)acc[i][j];
            const float dc = nc ? conf_dist(ci, gconf + gj * CONF_MAX, nc) : 0.f;
            Ks[sg_row(i) * 129 + sg_col(j)] = (gi < n_test && gj < n) ? kf.value(gamma, d, dc) : 0.f;
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
                         int64_t rows_pad, const float *A, int64_t p, float *part, const float *tconf) {
    const int64_t nrb = rows_pad / SG_BM, ncb = c->n_pad / SG_BN;
    size_t sh = (128 * 129 + 128 * p) * sizeof(float);
    if (sh > 48 * 1024)
        cudaFuncSetAttribute(predict_simt_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    count_launch(), predict_simt_kernel<<<(unsigned)(nrb * ncb), 256, sh, c->stream>>>(
        tf, tn, n_test, c->gf, c->norms, c->n, c->m_pad, ncb, (float)c->gamma, kernel_fn(c), tconf, c->conf,
        (int)c->nconf, A, p, rows_pad, part);
}

// Sum of partial products over column blocks in a fixed order; with a shift
// c (the partials hold (K - c) A), plus c (1^T A) from the FP64 column sums.
__global__ void predict_reduce_kernel(const float *part, int64_t nblk, int64_t rows_pad,
                                      int64_t n_test, int64_t p, float *out, int64_t ldo,
                                      const double *shift, const double *colsum) {
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_test * p) return;
    int64_t r = e / p, q = e % p;
    double s = 0.0;
    for (int64_t c = 0; c < nblk; ++c) s += (double)part[(c * rows_pad + r) * p + q];
    if (shift) s += (double)(float)*shift * colsum[q];
    out[r * ldo + q] = (float)s;
}

void launch_predict_reduce(const float *part, int64_t nblk, int64_t rows_pad, int64_t n_test,
                           int64_t p, float *out, int64_t ldo, cudaStream_t s, const double *shift,
                           const double *colsum) {
    count_launch(), predict_reduce_kernel<<<cdiv(n_test * p, 256), 256, 0, s>>>(part, nblk, rows_pad, n_test, p,
                                                               out, ldo, shift, colsum);
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

constexpr int PB_THREADS = 1024;

template <typename T>
__global__ void __launch_bounds__(PB_THREADS) potrf_block_kernel(T *W, T *Winv, int64_t b, int q,
                                                          int64_t tile_k, DevErrors *err,
                                                          double *minpiv) {
    // dynamic shared memory: a[DNB][DNB + 1] (the block, then L_qq) and
    // x[DNB][DNB + 1] (its inverse).  Thread (tx, ty) = (t % 64, t / 64)
    // owns column tx and rows ty, ty + 16, ... of the rank-1 updates.
    extern __shared__ __align__(16) unsigned char pb_smem[];
    T (*a)[DNB + 1] = reinterpret_cast<T (*)[DNB + 1]>(pb_smem);
    T (*x)[DNB + 1] = reinterpret_cast<T (*)[DNB + 1]>(pb_smem + sizeof(T) * DNB * (DNB + 1));
    __shared__ int bad;
    const int tx = threadIdx.x & (DNB - 1), ty = threadIdx.x / DNB;
    constexpr int RS = PB_THREADS / DNB;  // row stride of a thread
    T *blk = W + (int64_t)q * DNB * b + q * DNB;
    for (int r = ty; r < DNB; r += RS) {
        a[r][tx] = blk[(int64_t)r * b + tx];
        x[r][tx] = (r == tx) ? T(1) : T(0);
    }
    if (threadIdx.x == 0) bad = -1;
    __syncthreads();
    double mp = 1e300;
    // Cholesky, right-looking: pivot, scale the column, rank-1 update
    for (int c = 0; c < DNB; ++c) {
        if (threadIdx.x == 0) {
            T d = a[c][c];
            if (!(d > T(0))) {
                if (bad < 0) bad = c;
                d = T(1);
            }
            a[c][c] = sqrt(d);
            if ((double)a[c][c] < mp) mp = (double)a[c][c];
        }
        __syncthreads();
        if (ty == 0 && tx > c) a[tx][c] /= a[c][c];
        __syncthreads();
        if (tx > c) {
            const T lsc = a[tx][c];
#pragma unroll
            for (int r = ty; r < DNB; r += RS)
                if (r >= tx) a[r][tx] -= a[r][c] * lsc;
        }
        __syncthreads();
    }
    // inverse, right-looking forward substitution on the identity:
    // row c of X is final after the division; then rows r > c are updated
    for (int c = 0; c < DNB; ++c) {
        if (ty == 0 && tx <= c) x[c][tx] /= a[c][c];
        __syncthreads();
        if (tx <= c) {
            const T xc = x[c][tx];
#pragma unroll
            for (int r = ty; r < DNB; r += RS)
                if (r > c) x[r][tx] -= a[r][c] * xc;
        }
        __syncthreads();
    }
    T *iblk = Winv + (int64_t)q * DNB * b + q * DNB;
    for (int r = ty; r < DNB; r += RS) {
        blk[(int64_t)r * b + tx] = (tx <= r) ? a[r][tx] : T(0);
        iblk[(int64_t)r * b + tx] = (tx <= r) ? x[r][tx] : T(0);
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
    const size_t pb_smem = 2 * sizeof(T) * DNB * (DNB + 1);
    static PerDevice pb_attr;
    if (!pb_attr.has(c->device)) {
        if (cudaFuncSetAttribute(potrf_block_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pb_smem) ==
            cudaSuccess)
            pb_attr.put(c->device);
        else
            cudaGetLastError();  // the launch below reports the failure
    }
    for (int q = 0; q < nq; ++q) {
        count_launch(), potrf_block_kernel<T><<<1, PB_THREADS, pb_smem, s>>>(W, Winv, b, q, k, c->derr, minpiv + k * nq);
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
    // Triangular inverse by recursive doubling: with the 64-blocks X_qq already
    // inverted, for s = 64, 128, ..., b / 2 and every pair of diagonal
    // s-blocks, X_21 = -X_22 (L_21 X_11) (two batched GEMMs per level).
    for (int64_t sz = DNB; sz < b; sz *= 2) {
        const int pairs = (int)(b / (2 * sz));
        const int64_t pstride = 2 * sz * b + 2 * sz;
        // tmp_p = L_21 X_11
        launch_gemm_simt<T>((int)sz, (int)sz, (int)sz, T(1), W + sz * b, b, pstride, Winv, b, pstride, 1, T(0),
                            nullptr, 0, 0, tmp, sz, sz * sz, pairs, 0, s);
        // X_21 = -X_22 tmp_p
        launch_gemm_simt<T>((int)sz, (int)sz, (int)sz, T(-1), Winv + sz * b + sz, b, pstride, tmp, sz, sz * sz, 1,
                            T(0), nullptr, 0, 0, Winv + sz * b, b, pstride, pairs, 0, s);
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

// dst = src^T for one b x b tile (32 x 32 shared-memory tiles).
__global__ void transpose_kernel(const float *src, float *dst, int64_t b) {
    __shared__ float t[32][33];
    const int64_t bx = blockIdx.x * 32, by = blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) t[r][threadIdx.x] = src[(by + r) * b + bx + threadIdx.x];
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) dst[(bx + r) * b + by + threadIdx.x] = t[threadIdx.x][r];
}

__global__ void min_pivot_kernel(const double *mp, int n, DevErrors *err) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double m = err->min_pivot;
    for (int i = 0; i < n; ++i) m = fmin(m, mp[i]);
    err->min_pivot = m;
}

krr_status diag_step(Ctx *c, int64_t k, cudaStream_t s, int64_t cta_cap) {
    const int64_t b = c->b, bb = b * b;
    if (!s) s = c->stream;
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
        count_launch(), transpose_kernel<<<dim3((unsigned)(b / 32), (unsigned)(b / 32)), dim3(32, 8), 0, s>>>(
            linv, c->LinvT + k * bb, b);
    } else {
        // one dataflow launch: factor, inverse, transpose and FP16 split
        KRR_TRY(launch_diag_dataflow(c, k, wd, linv, c->LinvT + k * bb, c->Linv_hi ? c->Linv_hi + k * bb : nullptr,
                                     c->Linv_lo ? c->Linv_lo + k * bb : nullptr, (float *)c->diag64, c->diag_ctr,
                                     minpiv + k * nq, s, cta_cap));
    }
    count_launch(), min_pivot_kernel<<<1, 1, 0, s>>>(minpiv + k * nq, nq, c->derr);
    return KRR_OK;
}

// ----------------------------------------------------------------------------
// Adaptive precision of one factor column (mixed mode).
// Tile (i, k), i > k, is stored at the lowest unit roundoff u_p of E4M3
// (u = 2^-4) and FP16 (u = 2^-11) that the rule admits, else FP32:
//   lambda rule:  u_p * max|L_ik| * max|L_kk| <= eps * lambda.
//     Rounding L_ik perturbs L L^T in block (i, k) by about u_p |L_ik| |L_kk|;
//     the refinement converges while that stays well below lambda, the
//     smallest possible eigenvalue of K + lambda I.  max|L_kk| is bounded by
//     sqrt(max_r W_kk[r, r]) from the diagonal step.
//   K-norm rule (the Frobenius rule on the tiles of K of the adaptive-
//     precision Cholesky the paper cites, Sec. IV-C):
//     u_p * ||K_ik||_F <= eps * ||K||_F / NT, both norms from the build.
// FP16/E4M3 tiles carry a power-of-two scale so the largest entry sits near
// the top of the format.
// ----------------------------------------------------------------------------
__device__ inline float pow2_scale(float mx, float top) {
    if (!(mx > 0.f)) return 1.f;
    int e = (int)floorf(log2f(top / mx));
    e = max(-100, min(100, e));
    float s = ldexpf(1.f, e);
    while (mx * s > top) s *= 0.5f;
    return s;
}

__global__ void column_decide_kernel(int64_t k, int64_t nt, int64_t bb, int chunks,
                                     const float *part_max, double thresh,
                                     const double *lkk_max, int allow_fp8, int rule, double eps,
                                     const double *knorm_part, int64_t knorm_per_tile,
                                     const double *knorm2_total, TileDesc *ltab,
                                     uint8_t *precmap, DevErrors *err) {
    const int64_t tile = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tile >= nt - k - 1) return;
    const int64_t i = k + 1 + tile;
    float mx = 0;
    for (int q = 0; q < chunks; ++q) mx = fmaxf(mx, part_max[tile * chunks + q]);
    double w, thr;
    if (rule == KRR_RULE_KNORM) {
        const double *tp = knorm_part + tri_index(i, k) * knorm_per_tile;
        double s2 = 0.0;
        for (int64_t q = 0; q < knorm_per_tile; ++q) s2 += tp[q];
        w = sqrt(s2);
        thr = eps * sqrt(*knorm2_total) / (double)nt;
    } else {
        w = (double)mx * lkk_max[k];
        thr = thresh;
    }
    int prec;
    if (allow_fp8 && 0.0625 * w <= thr) prec = KRR_PREC_E4M3;
    else if (0x1p-11 * w <= thr) prec = KRR_PREC_FP16;
    else prec = KRR_PREC_FP32;
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

// Four consecutive elements per thread: vector loads and stores.
__global__ void column_write_kernel(int64_t k, int64_t bb, const float *col, const TileDesc *ltab,
                                    uint8_t *pool, __half *pan_hi, __half *pan_lo, __half *wsh) {
    const int64_t tile = blockIdx.y;
    const int64_t i = k + 1 + tile;
    const TileDesc d = ltab[off_index(i, k)];
    // E4M3 tiles: FP16 copy in the spent trailing slot W(i, k)
    __half2 *sh = reinterpret_cast<__half2 *>(wsh + off_index(i, k) * bb);
    const float4 *src = reinterpret_cast<const float4 *>(col + tile * bb);
    __half2 *hi = reinterpret_cast<__half2 *>(pan_hi + tile * bb);
    __half2 *lo = reinterpret_cast<__half2 *>(pan_lo + tile * bb);
    for (int64_t e4 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e4 < bb / 4;
         e4 += (int64_t)gridDim.x * blockDim.x) {
        const float4 v = src[e4];
        const float sv[4] = {v.x * d.scale, v.y * d.scale, v.z * d.scale, v.w * d.scale};
        if (d.prec == KRR_PREC_E4M3) {
            uint32_t packed = 0;
            __half h[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const __nv_fp8_storage_t qv = __nv_cvt_float_to_fp8(sv[t], __NV_SATFINITE, __NV_E4M3);
                packed |= (uint32_t)qv << (8 * t);
                h[t] = __half(__nv_cvt_fp8_to_halfraw(qv, __NV_E4M3));
            }
            reinterpret_cast<uint32_t *>(pool + d.offset)[e4] = packed;
            hi[2 * e4] = sh[2 * e4] = __halves2half2(h[0], h[1]);
            hi[2 * e4 + 1] = sh[2 * e4 + 1] = __halves2half2(h[2], h[3]);
        } else if (d.prec == KRR_PREC_FP16) {
            // the trailing update reads FP16 tiles from the pool itself
            const __half2 a = __floats2half2_rn(sv[0], sv[1]), b2 = __floats2half2_rn(sv[2], sv[3]);
            __half2 *pp = reinterpret_cast<__half2 *>(pool + d.offset);
            pp[2 * e4] = a;
            pp[2 * e4 + 1] = b2;
        } else {
            // FP32 class: the exact FP16 pair (hi plane, then lo plane)
            const __half2 a = __floats2half2_rn(sv[0], sv[1]), b2 = __floats2half2_rn(sv[2], sv[3]);
            const float2 fa = __half22float2(a), fb = __half22float2(b2);
            const __half2 la = __floats2half2_rn(sv[0] - fa.x, sv[1] - fa.y);
            const __half2 lb = __floats2half2_rn(sv[2] - fb.x, sv[3] - fb.y);
            __half2 *ph = reinterpret_cast<__half2 *>(pool + d.offset);
            __half2 *pl = ph + bb / 2;
            hi[2 * e4] = ph[2 * e4] = a;
            hi[2 * e4 + 1] = ph[2 * e4 + 1] = b2;
            lo[2 * e4] = pl[2 * e4] = la;
            lo[2 * e4 + 1] = pl[2 * e4 + 1] = lb;
        }
    }
}

void launch_column_cast(Ctx *c, int64_t k) {
    const int64_t u = c->nt - k - 1;
    if (u <= 0) return;
    const int64_t bb = c->b * c->b;
    // per-block max |L_ik| partials written by the panel-solve epilogue
    const int chunks = (int)tile_max_partials(c->b);
    const double thresh = c->opt.eps * c->lambda;
    const double *lkk = c->red + RED_MINPIV + c->nt * (c->b / 64);
    // K-norm rule: sums of K^2 per 128 x 256 block of every lower-triangle tile (build epilogue)
    const int64_t kper = (c->b / 128) * (c->b / 256);
    count_launch(), column_decide_kernel<<<cdiv(u, 128), 128, 0, c->stream>>>(
        k, c->nt, bb, chunks, c->colmax, thresh, lkk, c->opt.allow_fp8, c->opt.prec_rule, c->opt.eps, c->knorm2, kper,
        c->red + RED_KNORM2, c->ltab, c->precmap, c->derr);
    count_launch(), column_write_kernel<<<dim3(64, (unsigned)u), 256, 0, c->stream>>>(k, bb, c->colbuf, c->ltab,
                                                                      c->pool, c->pan_hi, c->pan_lo,
                                                                      (__half *)c->W);
}

// Largest diagonal entry of K over the diagonal tiles (padding included):
// K is positive semidefinite, so it bounds every |K_ij|.
__global__ void kernel_bound_kernel(const float *Kd, int64_t nt, int64_t b, double *out) {
    __shared__ float red[32];
    float mx = 0.f;
    for (int64_t e = threadIdx.x; e < nt * b; e += blockDim.x) {
        const int64_t t = e / b, r = e % b;
        mx = fmaxf(mx, fabsf(Kd[tri_index(t, t) * b * b + r * b + r]));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmaxf(mx, red[w]);
        *out = (double)mx;
    }
}

void launch_kernel_sumsq(Ctx *c, double *out) {
    const int64_t ntri = c->nt * (c->nt + 1) / 2;
    const int64_t per = (c->opt.mode == KRR_MODE_FP32) ? (c->b / SG_BM) * (c->b / SG_BM)
                                                       : (c->b / 128) * (c->b / 256);
    count_launch(), kernel_sumsq_kernel<<<1, 1024, 0, c->stream>>>(c->knorm2, ntri, per, c->n_pad, out);
    count_launch(), kernel_bound_kernel<<<1, 1024, 0, c->stream>>>(c->Kd, c->nt, c->b, c->red + RED_KBOUND);
}

// x (n_pad x p) <- (L L^T)^-1 x.  tmp is n_pad x p scratch (ends as Z).
krr_status solve_inplace(Ctx *c, float *x, float *tmp, int64_t p) {
    return c->opt.mode == KRR_MODE_MIXED ? tc_sweep_solve(c, x, tmp, p) : sweep_solve(c, x, tmp, p);
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

void launch_colsum(const float *a, int64_t n, int64_t p, double *out, cudaStream_t s) {
    count_launch(), colsum_kernel<<<(unsigned)p, 512, 0, s>>>(a, n, p, out);
}

krr_status launch_residual(Ctx *c, const float *y, const float *a, double *r, int64_t p) {
    count_launch(), colsum_kernel<<<(unsigned)p, 512, 0, c->stream>>>(a, c->n_pad, p, c->colsum);
    return c->opt.mode == KRR_MODE_MIXED ? tc_residual(c, y, a, r, p) : sweep_residual(c, y, a, r, p);
}

// ||r||_F^2 and ||y||_F^2 into out[0], out[1]: fixed per-block partial sums
// (NORM_BLOCKS blocks, grid-stride), then one block adds them in order, so
// the result is deterministic.
constexpr int NORM_BLOCKS = 256;

__global__ void norm_partial_kernel(const double *r, const float *y, int64_t count, double *part) {
    __shared__ double s1[32], s2[32];
    double a = 0, bsum = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
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
        part[blockIdx.x] = x;
        part[gridDim.x + blockIdx.x] = z;
    }
}

__global__ void norm_final_kernel(const double *part, int nb, double *out) {
    __shared__ double s1[32], s2[32];
    double a = 0, bsum = 0;
    for (int e = threadIdx.x; e < nb; e += blockDim.x) {
        a += part[e];
        bsum += part[nb + e];
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

void launch_reduce_norms(const double *r, const float *y, int64_t n, int64_t p, double *out, double *part,
                         cudaStream_t s) {
    count_launch(), norm_partial_kernel<<<NORM_BLOCKS, 256, 0, s>>>(r, y, n * p, part);
    count_launch(), norm_final_kernel<<<1, 256, 0, s>>>(part, NORM_BLOCKS, out);
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

// One stored factor element in its precision (not de-scaled).
__device__ __forceinline__ float load_l(const uint8_t *base, int prec, int64_t e) {
    if (prec == KRR_PREC_FP32) return reinterpret_cast<const float *>(base)[e];
    if (prec == KRR_PREC_FP16) return __half2float(reinterpret_cast<const __half *>(base)[e]);
    __half_raw h = __nv_cvt_fp8_to_halfraw(base[e], __NV_E4M3);
    return __half2float(__half(h));
}

// Dense lower-triangular copy of the stored factor (diagonal tiles from Wd,
// off-diagonal tiles from the pool in their precision, de-scaled).
__global__ void factor_to_dense_kernel(const float *Wd, const uint8_t *pool, const TileDesc *ltab,
                                       int64_t b, int64_t n, int mixed, float *dst, int64_t ld) {
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
        inv_scale = 1.f / d.scale;
    }
    // mixed mode: an FP32-class tile is an FP16 pair (hi plane, lo plane)
    const bool pair = mixed && ti != tj && prec == KRR_PREC_FP32;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < b * b;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lr = e / b, lc = e % b;
        const int64_t r = ti * b + lr, q = tj * b + lc;
        if (r >= n || q >= n) continue;
        float v;
        if (pair) {
            const __half *h = reinterpret_cast<const __half *>(base);
            v = (__half2float(h[e]) + __half2float(h[b * b + e])) * inv_scale;
        } else {
            v = load_l(base, prec, e) * inv_scale;
        }
        if (ti == tj && lc > lr) v = 0.f;
        dst[r * ld + q] = v;
    }
}

void launch_factor_to_dense(Ctx *c, float *dst, int64_t ld) {
    const int64_t ntri = c->nt * (c->nt + 1) / 2;
    count_launch(), factor_to_dense_kernel<<<dim3(64, (unsigned)ntri), 256, 0, c->stream>>>(
        c->Wd, c->pool, c->ltab, c->b, c->n, c->opt.mode == KRR_MODE_MIXED ? 1 : 0, dst, ld);
}

}  // namespace krr

namespace krr {
// ---------------------------------------------------------------------------
// Helpers of the hyperparameter gradient (deterministic single-block sums).
// ---------------------------------------------------------------------------
// gp[r][q] = 2 (yhat - yt) / (n_test p) for r < n_test, 0 for padding rows;
// sq[r * p + q] = (yhat - yt)^2 (r < n_test).
__global__ void grad_prep_kernel(const float *yhat, const float *yt, int64_t n_test, int64_t p,
                                 int64_t rows, float *gp, double *sq) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= rows * p) return;
    const int64_t r = e / p;
    if (r < n_test) {
        const double d = (double)yhat[e] - (double)yt[e];
        gp[e] = (float)(2.0 * d / (double)(n_test * p));
        sq[e] = d * d;
    } else {
        gp[e] = 0.f;
        sq[e] = 0.0;
    }
}

__global__ void sum_f64_kernel(const double *x, int64_t n, double *out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) s += x[e];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *out = t;
    }
}

__global__ void dot_f32_kernel(const float *a, const float *b, int64_t n, double *out) {
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t e = threadIdx.x; e < n; e += blockDim.x) s += (double)a[e] * (double)b[e];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        *out = t;
    }
}

void launch_grad_prep(const float *yhat, const float *yt, int64_t n_test, int64_t p, int64_t rows,
                      float *gp, double *sq, cudaStream_t s) {
    count_launch(), grad_prep_kernel<<<cdiv(rows * p, 256), 256, 0, s>>>(yhat, yt, n_test, p, rows, gp, sq);
}
void launch_sum_f64(const double *x, int64_t n, double *out, cudaStream_t s) {
    count_launch(), sum_f64_kernel<<<1, 1024, 0, s>>>(x, n, out);
}
void launch_dot_f32(const float *a, const float *b, int64_t n, double *out, cudaStream_t s) {
    count_launch(), dot_f32_kernel<<<1, 1024, 0, s>>>(a, b, n, out);
}
}  // namespace krr

namespace krr {
__global__ void factor_init_kernel(DevErrors *err, uint8_t *precmap, TileDesc *ltab, int64_t nt,
                                   int64_t bb, int diag_code, int fp32_mode) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e == 0) {
        err->code = 0;
        err->pad = 0;
        err->bad_tile = -1;
        err->bad_column = -1;
        err->bad_value = 0.0;
        err->fp8_tiles = err->fp16_tiles = err->fp32_tiles = err->pool_cursor = 0;
        err->min_pivot = INFINITY;
    }
    if (e < nt * nt) {
        const int64_t i = e / nt, j = e % nt;
        precmap[e] = (i == j) ? (uint8_t)diag_code : ((j < i && fp32_mode) ? (uint8_t)KRR_PREC_FP32 : (uint8_t)255);
    }
    if (fp32_mode && e < nt * (nt - 1) / 2) {
        TileDesc d;
        d.offset = e * bb * 4;
        d.scale = 1.f;
        d.prec = KRR_PREC_FP32;
        ltab[e] = d;
    }
}

void launch_factor_init(Ctx *c) {
    const int64_t nt = c->nt;
    const int64_t count = nt * nt > 1 ? nt * nt : 1;
    count_launch(), factor_init_kernel<<<cdiv(count, 256), 256, 0, c->stream>>>(
        c->derr, c->precmap, c->ltab, nt, c->b * c->b, c->opt.diag_fp64 ? KRR_PREC_FP64 : KRR_PREC_FP32,
        c->opt.mode == KRR_MODE_FP32 ? 1 : 0);
}
}  // namespace krr
