// Diagonal step of the tile Cholesky (Alg. 3, the POTRF of tile (k, k)) and
// the triangular inverse of the factor, as one persistent dataflow kernel over
// 64 x 64 blocks of the b x b tile (FP32).
//
// Items, claimed from a device counter in an order that respects their
// dependencies:
//   factor (NB = b / 64):
//     P(q)        for q >= 1 first L_q,q-1 = A_q,q-1 X_q-1,q-1^T (published at
//                 once) and A_qq -= L_q,q-1 L_q,q-1^T, then L_qq = chol(A_qq)
//                 and X_qq = inv(L_qq) in shared memory: the chain from one
//                 diagonal block to the next is a single item
//     T(i, q)     L_iq = A_iq X_qq^T                     (i > q + 1)
//     U(i, j, q)  A_ij -= L_iq L_jq^T                    (q < j <= i, i > q + 1)
//   listed as P(0), then for q = 0 .. NB-2: P(q + 1) and the T and U items of
//   column q;
//   inverse X = L^-1 by recursive doubling, for s = 64, 128, ..., b / 2 and
//   every pair of diagonal s-blocks:
//     step 1      T_p = L_21 X_11                        (one 64 x 64 output block per item)
//     step 2      X_21 = -X_22 T_p
//   finish        X^T (for the backward substitution) and the FP16 hi/lo
//                 split of X (operands of the tensor-core panel solve), per
//                 64 x 64 block, as soon as that block of X is final.
// Progress counters: upd[i][j] (updates applied to block (i, j)), pdone[q],
// tdone[i][q], and finished items of each inverse pair (step 1 and step 2
// separately).  Inverse items wait only for the blocks they read: a step-1
// item for its row of L_21 (T items) and for X_11 (the pair's first half),
// a step-2 item for X_22 and the pair's step-1 products, a finishing item for
// the pairs whose second half holds its rows; so the inverse of the leading
// blocks runs while the factorisation of the trailing ones goes on.  An item
// only waits for items claimed before it by running CTAs, so the kernel always
// progresses; every wait is bounded (%globaltimer) and ends the kernel with
// KRR_ETIMEOUT.  Blocks written by other CTAs are read through L2
// (ld.global.cg).
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "krr_internal.h"

namespace krr {

namespace {

constexpr int DB = 64;          // block edge
constexpr int DT = 256;         // threads per CTA
constexpr int DMAX_NB = 64;     // blocks per tile edge supported (b <= 4096)

struct DiagParams {
    float *W;          // tile, overwritten by L (lower part)
    float *X;          // inverse (zeroed before the launch)
    float *XT;         // transpose of the inverse
    __half *hi, *lo;   // FP16 split of the inverse (or null)
    float *tmp;        // b * b / 2 floats: products of the inverse steps, one region per level
    int64_t b;
    int NB, levels;
    int64_t tile_k;
    int64_t n_factor;  // number of factor items
    int64_t items;
    int *ctr;          // counters (layout in ctr_* below)
    double *minpiv;    // NB minimum pivots of this tile
    DevErrors *err;
    uint64_t wait_ns;
};

// counter layout: [0] item counter, [1] abort, then pdone[NB], tdone[NB * NB],
// upd[NB * NB], and per inverse pair (all levels, fewer than NB pairs) the
// finished step-1 items i1done[NB] and step-2 items i2done[NB]
__device__ __forceinline__ int *ctr_pdone(const DiagParams &p) { return p.ctr + 2; }
__device__ __forceinline__ int *ctr_tdone(const DiagParams &p) { return ctr_pdone(p) + p.NB; }
__device__ __forceinline__ int *ctr_upd(const DiagParams &p) { return ctr_tdone(p) + p.NB * p.NB; }
__device__ __forceinline__ int *ctr_i1done(const DiagParams &p) { return ctr_upd(p) + p.NB * p.NB; }
__device__ __forceinline__ int *ctr_i2done(const DiagParams &p) { return ctr_i1done(p) + p.NB; }

// Slot of pair `pr` of inverse level l (levels before it hold NB / 2,
// NB / 4, ... pairs).
__device__ __forceinline__ int pair_slot(const DiagParams &p, int l, int pr) {
    int base = 0;
    for (int q = 0; q < l; ++q) base += p.NB >> (q + 1);
    return base + pr;
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded wait (one thread) until *c >= target; false on expiry / abort.
// Polls back off exponentially (32 ns up to 256 ns) so that many waiting
// CTAs do not flood the L2 slice holding the counters.
__device__ bool wait_ge(const int *c, int target, const DiagParams &p) {
    if (ld_acquire(c) >= target) return true;
    const uint64_t t0 = globaltimer();
    uint32_t nap = 32;
    for (uint32_t it = 1;; ++it) {
        __nanosleep(nap);
        if (nap < 256) nap <<= 1;
        if (ld_acquire(c) >= target) return true;
        if ((it & 15) == 0) {
            if (*(volatile int *)&p.ctr[1]) return false;
            if (globaltimer() - t0 > p.wait_ns) {
                atomicExch(&p.ctr[1], 1);
                atomicCAS(&p.err->code, 0, (int)KRR_ETIMEOUT);
                return false;
            }
        }
    }
}

// Publishes the CTA's finished writes and increments a counter.
__device__ __forceinline__ void signal(int *c) {
    __threadfence();
    atomicAdd(c, 1);
}

// ---------------------------------------------------------------------------
// Item list.
// ---------------------------------------------------------------------------
enum DiagKind { K_P = 0, K_T = 1, K_U = 2, K_I1 = 3, K_I2 = 4, K_FIN = 5 };

struct DItem {
    int kind;
    int q, i, j;     // factor blocks
    int level, pair, a, c;  // inverse output block (a, c) of pair `pair` at `level`
    int phase;       // inverse step index 2 * level + (0 | 1)
};

// Items of factor group q (0 <= q <= NB - 2): P(q + 1), then for every row
// i = q + 2 .. NB - 1 the items T(i, q), U(i, q + 1 .. i, q).
__host__ __device__ inline int64_t factor_group_items(int NB, int q) {
    const int64_t m = NB - q - 1;  // rows below block q
    return m + m * (m + 1) / 2 - 1;
}

__host__ __device__ inline int64_t factor_items_for(int NB) {
    int64_t n = 1;  // P(0)
    for (int q = 0; q + 1 < NB; ++q) n += factor_group_items(NB, q);
    return n;
}

// Items of inverse step (level l, step s): pairs * (sz / 64)^2.
__host__ __device__ inline int64_t inv_step_items(int NB, int l) {
    const int64_t nb = (int64_t)1 << l;   // sz / 64
    const int64_t pairs = NB / (2 * nb);
    return pairs * nb * nb;
}

__device__ void decode_item(const DiagParams &p, int64_t t, DItem &it) {
    const int NB = p.NB;
    if (t < p.n_factor) {
        if (t == 0) {
            it.kind = K_P;
            it.q = 0;
            return;
        }
        // walk the q groups: P(q + 1), then rows i = q + 2.. with T(i, q) and U(i, j, q)
        int64_t r = t - 1;
        for (int q = 0; q + 1 < NB; ++q) {
            const int64_t g = factor_group_items(NB, q);
            if (r >= g) {
                r -= g;
                continue;
            }
            if (r == 0) {
                it.kind = K_P;
                it.q = q + 1;
                return;
            }
            it.q = q;
            --r;
            for (int i = q + 2; i < NB; ++i) {
                const int64_t row = 1 + (i - q);  // T + U(i, q+1..i)
                if (r < row) {
                    it.i = i;
                    if (r == 0) {
                        it.kind = K_T;
                    } else {
                        it.kind = K_U;
                        it.j = q + (int)r;
                    }
                    return;
                }
                r -= row;
            }
        }
    }
    int64_t r = t - p.n_factor;
    for (int l = 0; l < p.levels; ++l) {
        const int64_t per = inv_step_items(NB, l);
        for (int s = 0; s < 2; ++s) {
            if (r < per) {
                const int64_t nb = (int64_t)1 << l;
                it.kind = s == 0 ? K_I1 : K_I2;
                it.level = l;
                it.phase = 2 * l + s;
                it.pair = (int)(r / (nb * nb));
                it.a = (int)((r % (nb * nb)) / nb);
                it.c = (int)(r % nb);
                return;
            }
            r -= per;
        }
    }
    it.kind = K_FIN;
    it.i = (int)(r / NB);  // block (i, j) of the inverse
    it.j = (int)(r % NB);
}

// ---------------------------------------------------------------------------
// 64 x 64 block product on 256 threads: C = alpha * sum_k A_k op(B_k) + beta * C.
// Thread (tx, ty) = (t % 16, t / 16) owns rows ty + 16 u and columns tx + 16 v.
// ---------------------------------------------------------------------------
struct BlkSmem {
    float a[DB][DB + 1];
    float b[DB][DB + 1];
};

__device__ __forceinline__ void load_blk(float (*dst)[DB + 1], const float *src, int64_t ld, bool trans) {
    // 64 x 64 floats, 16 per thread as 4 float4 loads through L2
    for (int e = threadIdx.x; e < DB * DB / 4; e += DT) {
        const int r = e / (DB / 4), c4 = (e % (DB / 4)) * 4;
        const float4 v = __ldcg(reinterpret_cast<const float4 *>(src + r * ld + c4));
        if (trans) {
            dst[c4 + 0][r] = v.x; dst[c4 + 1][r] = v.y; dst[c4 + 2][r] = v.z; dst[c4 + 3][r] = v.w;
        } else {
            dst[r][c4 + 0] = v.x; dst[r][c4 + 1] = v.y; dst[r][c4 + 2] = v.z; dst[r][c4 + 3] = v.w;
        }
    }
}

// acc += A_blk (64 x 64) * Bs (64 x 64, [k][n] layout)
__device__ __forceinline__ void mac_blk(const BlkSmem &s, float (&acc)[4][4]) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll 8
    for (int k = 0; k < DB; ++k) {
        float av[4], bv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) av[u] = s.a[ty + 16 * u][k];
#pragma unroll
        for (int v = 0; v < 4; ++v) bv[v] = s.b[k][tx + 16 * v];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
    }
}

// C (ld) = alpha * acc + beta * C
__device__ __forceinline__ void store_blk(float *C, int64_t ld, const float (&acc)[4][4], float alpha, float beta) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            float *cp = C + (int64_t)(ty + 16 * u) * ld + tx + 16 * v;
            const float old = (beta != 0.f) ? __ldcg(cp) : 0.f;
            __stcg(cp, alpha * acc[u][v] + beta * old);
        }
}

// ---------------------------------------------------------------------------
// P(q): Cholesky and inverse of the 64 x 64 diagonal block in shared memory,
// blocked by 16 (a pivot that is not positive is recorded, first one wins,
// and replaced by 1 so the rest stays finite):
//   for each 16-block q of the diagonal:
//     warp 0 factors A_qq and inverts L_qq in registers (lane l owns row l;
//     columns and rows are broadcast by warp shuffles);
//     L_iq = A_iq X_qq^T for the 16-row blocks below (all threads);
//     A_ij -= L_iq L_jq^T on the trailing lower triangle (all threads, 16 x 16
//     thread grid, rows of L_iq / L_jq held in registers);
//   then X = L^-1 below the diagonal blocks, by block diagonals:
//     X_iq = -X_ii (sum_{k=q}^{i-1} L_ik X_kq).
// a holds A on entry and L on exit, x receives X; tmp is 3 x 16 x 17 floats.
// ---------------------------------------------------------------------------
__device__ void chol_inv_64(float (*a)[65], float (*x)[65], float (*tmp)[16][17], float *dinv,
                                            int &bad, float &mpiv) {
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const unsigned FULL = 0xffffffffu;
    for (int e = t; e < 64 * 64; e += 256) x[e >> 6][e & 63] = 0.f;
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
        const int o = 16 * q;
        if (warp == 0) {
            const int l = lane & 15;
            float v[16], xr[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = (j <= l) ? a[o + l][o + j] : 0.f;
#pragma unroll
            for (int k = 0; k < 16; ++k) xr[k] = (k == l) ? 1.f : 0.f;
            // column c of the factor, then column c of the inverse (it needs
            // only columns 0 .. c of L): one loop, so the inverse step of
            // column c fills the latency of column c + 1's pivot chain
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                float d = __shfl_sync(FULL, v[c], c);
                if (!(d > 0.f)) {
                    if (bad < 0) bad = o + c;
                    d = 1.f;
                }
                // 1 / sqrt(d): hardware estimate refined by one Newton-Raphson
                // step for the reciprocal square root, x <- x (3 - d x^2) / 2
                float inv = rsqrtf(d);
                inv = inv * fmaf(-0.5f * d * inv, inv, 1.5f);
                const float lcc = d * inv;
                mpiv = fminf(mpiv, lcc);
                if (l == c) {
                    v[c] = lcc;
                    if (lane == c) dinv[o + c] = inv;
                } else if (l > c) {
                    v[c] *= inv;
                }
                // constant loop bounds (j > c as a condition) keep v in registers
#pragma unroll
                for (int j = 1; j < 16; ++j) {
                    if (j > c) {
                        const float ljc = __shfl_sync(FULL, v[c], j);
                        if (l >= j) v[j] = fmaf(-v[c], ljc, v[j]);
                    }
                }
                // inverse: row c of X is final once scaled by 1 / L[c][c]
                if (l == c) {
#pragma unroll
                    for (int k = 0; k <= c; ++k) xr[k] *= inv;
                }
#pragma unroll
                for (int k = 0; k <= c; ++k) {
                    const float xck = __shfl_sync(FULL, xr[k], c);
                    if (l > c) xr[k] = fmaf(-v[c], xck, xr[k]);
                }
            }
            if (lane < 16) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (j <= l) {
                        a[o + l][o + j] = v[j];
                        x[o + l][o + j] = xr[j];
                    }
                }
            }
        }
        __syncthreads();
        const int rows = 64 - o - 16;
        if (rows > 0) {
            const int tc = t & 15, tr = t >> 4;
            float res[3];
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int rr = tr + 16 * u;
                if (rr < rows) {
                    const int i = o + 16 + rr, c = o + tc;
                    float acc = 0.f;
#pragma unroll
                    for (int k = 0; k < 16; ++k) acc = fmaf(a[i][o + k], x[c][o + k], acc);
                    res[u] = acc;
                }
            }
            __syncthreads();
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                const int rr = tr + 16 * u;
                if (rr < rows) a[o + 16 + rr][o + tc] = res[u];
            }
            __syncthreads();
            const int nb = rows / 16;
            float li[3][16], lj[3][16];
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                if (u < nb) {
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        li[u][k] = a[o + 16 + tr + 16 * u][o + k];
                        lj[u][k] = a[o + 16 + tc + 16 * u][o + k];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 3; ++u) {
#pragma unroll
                for (int w = 0; w < 3; ++w) {
                    if (u < nb && w <= u) {
                        const int i = o + 16 + tr + 16 * u, j = o + 16 + tc + 16 * w;
                        if (i >= j) {
                            float acc = 0.f;
#pragma unroll
                            for (int k = 0; k < 16; ++k) acc = fmaf(li[u][k], lj[w][k], acc);
                            a[i][j] -= acc;
                        }
                    }
                }
            }
        }
        __syncthreads();
    }
    // off-diagonal blocks of X = L^-1: X_iq = -X_ii sum_{k=q}^{i-1} L_ik X_kq
    const int tc = t & 15, tr = t >> 4;
    for (int dd = 1; dd < 4; ++dd) {
        const int npair = 4 - dd;
        for (int qq = 0; qq < npair; ++qq) {
            const int ib = qq + dd;
            float acc = 0.f;
            for (int kb = qq; kb < ib; ++kb) {
#pragma unroll
                for (int k = 0; k < 16; ++k) acc = fmaf(a[16 * ib + tr][16 * kb + k], x[16 * kb + k][16 * qq + tc], acc);
            }
            tmp[qq][tr][tc] = acc;
        }
        __syncthreads();
        for (int qq = 0; qq < npair; ++qq) {
            const int ib = qq + dd;
            float acc = 0.f;
#pragma unroll
            for (int k = 0; k < 16; ++k) acc = fmaf(x[16 * ib + tr][16 * ib + k], tmp[qq][k][tc], acc);
            x[16 * ib + tr][16 * qq + tc] = -acc;
        }
        __syncthreads();
    }
}

// sub (optional): a product to subtract from A_qq first, held as the 16 x 16
// thread grid of mac_blk holds it.
__device__ void potrf_inv_block(const DiagParams &p, int q, BlkSmem &s, const float (*sub)[4] = nullptr) {
    float (*a)[DB + 1] = s.a;
    float (*x)[DB + 1] = s.b;
    const int64_t b = p.b;
    float *blk = p.W + (int64_t)q * DB * b + q * DB;
    __shared__ float dinv[DB];
    __shared__ float tmp[3][16][17];
    const int tx = threadIdx.x & (DB - 1), ty = threadIdx.x / DB;  // 4 row groups
    constexpr int RS = DT / DB;
    for (int r = ty; r < DB; r += RS) a[r][tx] = __ldcg(blk + (int64_t)r * b + tx);
    __syncthreads();
    if (sub) {
        const int gx = threadIdx.x & 15, gy = threadIdx.x >> 4;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) a[gy + 16 * u][gx + 16 * v] -= sub[u][v];
        __syncthreads();
    }
    int bad = -1;
    float mpiv = 3.0e38f;
    chol_inv_64(a, x, tmp, dinv, bad, mpiv);
    float *iblk = p.X + (int64_t)q * DB * b + q * DB;
    for (int r = ty; r < DB; r += RS) {
        __stcg(blk + (int64_t)r * b + tx, (tx <= r) ? a[r][tx] : 0.f);
        __stcg(iblk + (int64_t)r * b + tx, (tx <= r) ? x[r][tx] : 0.f);
    }
    if (threadIdx.x == 0) {
        p.minpiv[q] = (double)mpiv;
        if (bad >= 0 && atomicCAS(&p.err->code, 0, (int)KRR_ENOTPD) == 0) {
            p.err->bad_tile = p.tile_k;
            p.err->bad_column = p.tile_k * b + (int64_t)q * DB + bad;
        }
    }
}

__global__ void __launch_bounds__(DT) diag_kernel(const DiagParams p) {
    __shared__ BlkSmem s;
    __shared__ int64_t item_s;
    __shared__ int ok_s;
    const int64_t b = p.b;
    const int NB = p.NB;
    while (true) {
        if (threadIdx.x == 0) item_s = atomicAdd(&p.ctr[0], 1);
        __syncthreads();
        const int64_t t = item_s;
        if (t >= p.items) break;
        DItem it;
        decode_item(p, t, it);
        // ---- wait for the inputs (one thread), then all threads proceed
        if (threadIdx.x == 0) {
            bool ok = true;
            int *upd = ctr_upd(p), *tdone = ctr_tdone(p), *pdone = ctr_pdone(p);
            if (it.kind == K_P) {
                // P(q), q >= 1: X_q-1,q-1, and blocks (q, q-1) and (q, q) with the
                // updates of columns 0 .. q-2
                // (the other two inputs are awaited in the item body, after the
                // first block is loaded)
                if (it.q > 0) ok = wait_ge(upd + it.q * NB + it.q - 1, it.q - 1, p);
            } else if (it.kind == K_T) {
                ok = wait_ge(pdone + it.q, 1, p) && wait_ge(upd + it.i * NB + it.q, it.q, p);
            } else if (it.kind == K_U) {
                ok = wait_ge(tdone + it.i * NB + it.q, 1, p) && wait_ge(tdone + it.j * NB + it.q, 1, p) &&
                     wait_ge(upd + it.i * NB + it.j, it.q, p);
            } else if (it.kind == K_I1 || it.kind == K_I2) {
                const int nb = 1 << it.level, r0 = 2 * it.pair * nb, half = nb / 2;
                // X of the pair's first (I1) or second (I2) half: the P item at
                // level 0, else all step-2 items of that half one level down
                const int sub = (it.kind == K_I1) ? 0 : 1;
                ok = (it.level == 0) ? wait_ge(pdone + r0 + sub, 1, p)
                                     : wait_ge(ctr_i2done(p) + pair_slot(p, it.level - 1, 2 * it.pair + sub),
                                               half * half, p);
                if (it.kind == K_I1) {
                    // row a of L_21, columns c .. nb - 1
                    for (int k = it.c; k < nb && ok; ++k) ok = wait_ge(tdone + (r0 + nb + it.a) * NB + r0 + k, 1, p);
                } else {
                    ok = ok && wait_ge(ctr_i1done(p) + pair_slot(p, it.level, it.pair), nb * nb, p);
                }
            } else if (it.j == it.i) {
                ok = wait_ge(pdone + it.i, 1, p);  // diagonal block of X
            } else if (it.j < it.i) {
                // block (i, j) of X is written by the step-2 items of the pair in
                // which i and j first fall into different halves
                const int l = 31 - __clz(it.i ^ it.j), nb = 1 << l;
                ok = wait_ge(ctr_i2done(p) + pair_slot(p, l, it.i >> (l + 1)), nb * nb, p);
            }  // blocks above the diagonal are zero from the start
            ok_s = ok ? 1 : 0;
        }
        __syncthreads();
        if (!ok_s) break;
        float acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = 0.f;
        if (it.kind == K_P) {
            if (it.q > 0) {
                // L_q,q-1 = A_q,q-1 X_q-1,q-1^T, published for the U items of column q-1
                const int q = it.q;
                float *c = p.W + (int64_t)q * DB * b + (q - 1) * DB;
                // A_q,q-1 (final since the updates of columns 0 .. q-2) comes in
                // while P(q-1) may still be running
                load_blk(s.a, c, b, false);
                __syncthreads();  // every thread has read the previous ok_s
                if (threadIdx.x == 0)
                    ok_s = (wait_ge(ctr_pdone(p) + q - 1, 1, p) && wait_ge(ctr_upd(p) + q * NB + q, q - 1, p)) ? 1 : 0;
                __syncthreads();
                if (!ok_s) break;
                load_blk(s.b, p.X + (int64_t)(q - 1) * DB * b + (q - 1) * DB, b, true);
                __syncthreads();
                mac_blk(s, acc);
                __syncthreads();
                store_blk(c, b, acc, 1.f, 0.f);
                // L_q,q-1 into s.a and, transposed, into s.b; then L L^T
                const int gx = threadIdx.x & 15, gy = threadIdx.x >> 4;
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        s.a[gy + 16 * u][gx + 16 * v] = acc[u][v];
                        s.b[gx + 16 * v][gy + 16 * u] = acc[u][v];
                        acc[u][v] = 0.f;
                    }
                __syncthreads();
                if (threadIdx.x == 0) signal(ctr_tdone(p) + q * NB + q - 1);
                mac_blk(s, acc);
                __syncthreads();
                potrf_inv_block(p, q, s, acc);
            } else {
                potrf_inv_block(p, it.q, s);
            }
        } else if (it.kind == K_T) {
            // L_iq = A_iq X_qq^T, in place
            float *c = p.W + (int64_t)it.i * DB * b + it.q * DB;
            load_blk(s.a, c, b, false);
            load_blk(s.b, p.X + (int64_t)it.q * DB * b + it.q * DB, b, true);
            __syncthreads();
            mac_blk(s, acc);
            __syncthreads();
            store_blk(c, b, acc, 1.f, 0.f);
        } else if (it.kind == K_U) {
            // A_ij -= L_iq L_jq^T
            load_blk(s.a, p.W + (int64_t)it.i * DB * b + it.q * DB, b, false);
            load_blk(s.b, p.W + (int64_t)it.j * DB * b + it.q * DB, b, true);
            __syncthreads();
            mac_blk(s, acc);
            __syncthreads();
            store_blk(p.W + (int64_t)it.i * DB * b + it.j * DB, b, acc, -1.f, 1.f);
        } else if (it.kind == K_I1 || it.kind == K_I2) {
            const int64_t nb = (int64_t)1 << it.level, sz = nb * DB, base = 2 * it.pair * sz;
            // products of level l after those of levels 0 .. l - 1 (each level
            // NB * 2^l * DB * DB / 2 floats): levels run concurrently
            float *tp = p.tmp + (int64_t)p.NB * (nb - 1) * (DB * DB / 2) + (int64_t)it.pair * sz * sz;
            if (it.kind == K_I1) {
                // T_p[a][c] = sum_{k >= c} L21[a][k] X11[k][c]
                for (int64_t kk = it.c; kk < nb; ++kk) {
                    load_blk(s.a, p.W + (base + sz + it.a * DB) * b + base + kk * DB, b, false);
                    load_blk(s.b, p.X + (base + kk * DB) * b + base + it.c * DB, b, false);
                    __syncthreads();
                    mac_blk(s, acc);
                    __syncthreads();
                }
                store_blk(tp + (int64_t)it.a * DB * sz + it.c * DB, sz, acc, 1.f, 0.f);
            } else {
                // X21[a][c] = -sum_{k <= a} X22[a][k] T_p[k][c]
                for (int64_t kk = 0; kk <= it.a; ++kk) {
                    load_blk(s.a, p.X + (base + sz + it.a * DB) * b + base + sz + kk * DB, b, false);
                    load_blk(s.b, tp + kk * DB * sz + it.c * DB, sz, false);
                    __syncthreads();
                    mac_blk(s, acc);
                    __syncthreads();
                }
                store_blk(p.X + (base + sz + it.a * DB) * b + base + it.c * DB, b, acc, -1.f, 0.f);
            }
        } else {
            // block (r, cb) of X: transpose into X^T and the FP16 split
            const int r = it.i, cb = it.j;
            const float *src = p.X + (int64_t)r * DB * b + cb * DB;
            load_blk(s.a, src, b, false);
            __syncthreads();
            for (int e = threadIdx.x; e < DB * DB; e += DT) {
                const int rr = e / DB, cc = e % DB;
                // X^T block (cb, r): element (cc, rr) = X (rr, cc)
                __stcg(p.XT + ((int64_t)cb * DB + rr) * b + r * DB + cc, s.a[cc][rr]);
                if (p.hi) {
                    const float v = s.a[rr][cc];
                    const __half h = __float2half_rn(v);
                    const int64_t o = ((int64_t)r * DB + rr) * b + cb * DB + cc;
                    p.hi[o] = h;
                    p.lo[o] = __float2half_rn(v - __half2float(h));
                }
            }
        }
        __syncthreads();
        // ---- publish
        if (threadIdx.x == 0) {
            if (it.kind == K_P) {
                signal(ctr_pdone(p) + it.q);
            } else if (it.kind == K_T) {
                signal(ctr_tdone(p) + it.i * NB + it.q);
            } else if (it.kind == K_U) {
                signal(ctr_upd(p) + it.i * NB + it.j);
            } else if (it.kind == K_I1) {
                signal(ctr_i1done(p) + pair_slot(p, it.level, it.pair));
            } else if (it.kind == K_I2) {
                signal(ctr_i2done(p) + pair_slot(p, it.level, it.pair));
            }
        }
    }
}

}  // namespace

int64_t diag_counter_count(int64_t b) {
    const int64_t NB = b / DB;
    return 2 + NB + 2 * NB * NB + 2 * NB;
}

// Factor + inverse of diagonal tile k in FP32 (W in place, Linv, LinvT and
// the FP16 split of Linv when present).  The counters `ctr` hold
// diag_counter_count(b) ints.
krr_status launch_diag_dataflow(Ctx *c, int64_t k, float *W, float *X, float *XT, __half *hi, __half *lo,
                                float *tmp, int *ctr, double *minpiv, cudaStream_t s, int64_t cta_cap) {
    const int64_t b = c->b;
    if (b % DB != 0 || b / DB > DMAX_NB) {
        c->last_error = "diagonal step: tile edge must be a multiple of 64 and at most 4096";
        return KRR_EINVAL;
    }
    DiagParams p;
    memset(&p, 0, sizeof(p));
    p.W = W;
    p.X = X;
    p.XT = XT;
    p.hi = hi;
    p.lo = lo;
    p.tmp = tmp;
    p.b = b;
    p.NB = (int)(b / DB);
    int levels = 0;
    while (((int64_t)DB << levels) < b) ++levels;
    p.levels = levels;
    p.tile_k = k;
    p.n_factor = factor_items_for(p.NB);
    int64_t inv = 0;
    for (int l = 0; l < levels; ++l) inv += 2 * inv_step_items(p.NB, l);
    p.items = p.n_factor + inv + (int64_t)p.NB * p.NB;
    p.ctr = ctr;
    p.minpiv = minpiv;
    p.err = c->derr;
    p.wait_ns = (uint64_t)c->opt.wait_budget_ns;
    KRR_CUDA_TRY(c, cudaMemsetAsync(ctr, 0, (size_t)diag_counter_count(b) * sizeof(int), s));
    KRR_CUDA_TRY(c, cudaMemsetAsync(X, 0, (size_t)b * b * sizeof(float), s));
    int64_t gl = grid_limit(c, GL_DIAG);
    if (cta_cap > 0 && cta_cap < gl) gl = cta_cap;
    const int64_t grid = std::min<int64_t>(gl, std::max<int64_t>(p.NB * (p.NB + 1) / 2, 1));
    count_launch(), diag_kernel<<<(unsigned)grid, DT, 0, s>>>(p);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->last_error = std::string("diagonal step launch: ") + cudaGetErrorString(e);
        return KRR_ECUDA;
    }
    return KRR_OK;
}

}  // namespace krr
