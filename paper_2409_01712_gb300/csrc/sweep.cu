// Persistent dataflow kernel for the tile sweeps of the solve phase (Alg. 3:
// forward substitution L z = y, backward substitution L^T x = z) and for the
// refinement residual r = y - (K + lambda I) a.
//
// Work items (one 128-row slab s of a row block each):
//   forward   DIAG(j, s)     z_j[s] = Linv_jj[s, :] y_j            (y_j fully updated)
//             LINK(i, j, s)  y_i[s] -= L_ij[s, :] z_j, i > j       (row slab of L_ij)
//   backward  DIAG(j, s)     x_j[s] = Linv_jj^T[s, :] z_j
//             LINK(t, j, s)  z_t[s] -= L_jt[:, s]^T x_j, t < j     (column slab of L_jt)
//   residual  RES(i, s)      r_i[s] = y_i - lambda a_i - sum_j K_ij a_j; K is symmetric,
//                            so row slabs of the stored tiles (i, j <= i) and
//                            column slabs of (j > i, i)
// The right-hand side is updated in place.  Items are claimed from a device
// counter in dependency order: the forward sweep lists, for j = 0, 1, ...,
// the DIAG items of block j and then every LINK item that reads z_j (the
// backward sweep the same for j = nt - 1, ...).  Counters publish progress:
// ready[j] (DIAG slabs of block j done), done[i] (slabs of block i whose last
// LINK is done), seq[i][s] (LINKs applied to slab (i, s)); the LINKs of one
// slab apply their updates in a fixed order, so results are deterministic.
// A CTA only waits on items claimed before its own by running CTAs, so the
// sweep always progresses; every wait is still bounded (%globaltimer) and
// ends the kernel with KRR_ETIMEOUT.
//
// CTA: warp 0 produces, warps 1..8 consume.
//   producer  claims items; streams each tile slab as 16 KB chunks by TMA
//             (128-byte swizzle) into a shared-memory ring, and copies the
//             matching vector rows (cp.async) once they are published;
//   consumers FP32 FMAs from shared memory, 4 accumulated rows (row chunk)
//             or 4 columns (column chunk) per thread; 8 lanes share each row
//             or column and are summed by warp shuffles, so every output has
//             one owner thread and no shared-memory reduction is needed.
// The residual folds each tile's FP32 partial sums into FP64 (owner threads,
// shared memory) before the next tile: cancellation happens within a tile's
// row sums.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "krr_internal.h"

namespace krr {

namespace {

constexpr int SW_CONSUMERS = 256;
constexpr int SW_THREADS = 32 + SW_CONSUMERS;
constexpr int SW_SLAB = 128;        // output rows of an item
constexpr int SW_CHUNK = 16384;     // tile bytes per stage
constexpr int SW_HDR = 64;          // stage header bytes
constexpr int SW_PCMAX = 24;        // right-hand sides per launch

enum SweepJob { SW_FWD = 0, SW_BWD = 1, SW_RES = 2 };
enum ChunkKind { CK_ROW = 0, CK_COL = 1, CK_END = 3 };
enum ChunkFlags { F_FIRST = 1, F_LAST_CONTRIB = 2, F_LAST_ITEM = 4, F_SWITCH = 8, F_LAST_LINK = 16 };
enum EndOp { E_LINK = 0, E_DIAG = 1, E_RES = 2 };

struct StageHdr {
    int32_t kind, prec, flags, endop;
    int32_t blk, slab, seq;   // output block and slab; LINK: updates applied before this one
    float inv_scale, shift;
};

struct SweepParams {
    int job;
    int64_t b, nt, S, items;  // S = b / SW_SLAB slabs per block
    int pc, pcp, q0, x16;     // x16: vector rows can be copied in 16-byte pieces
    int64_t ldx;
    int stages;
    int64_t stage_bytes;
    float *rhs;               // FWD: y, BWD: z (updated in place); RES: y
    float *out;               // FWD: z; BWD: x
    const float *xv;          // RES: a
    double *r;                // RES: residual (n_pad x ldx)
    const double *shift;      // RES: shift c (device)
    const double *colsum;     // RES: 1^T a per column
    float lambda;
    const TileDesc *ltab;
    int *flags;               // [0] item counter, [1] abort, then done[nt], ready[nt], seq[nt * S]
    uint64_t wait_ns;
    DevErrors *err;
};

__host__ __device__ constexpr int esize_of(int prec) {
    return prec == KRR_PREC_FP32 ? 4 : (prec == KRR_PREC_FP16 ? 2 : 1);
}

__device__ __forceinline__ int *done_ctr(const SweepParams &p) { return p.flags + 2; }
__device__ __forceinline__ int *ready_ctr(const SweepParams &p) { return p.flags + 2 + p.nt; }
__device__ __forceinline__ int *seq_ctr(const SweepParams &p) { return p.flags + 2 + 2 * p.nt; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void record_timeout(const SweepParams &p) {
    atomicExch(&p.flags[1], 1);
    atomicCAS(&p.err->code, 0, (int)KRR_ETIMEOUT);
}

// Bounded wait on a CTA barrier; false on expiry or when the sweep aborted.
// The abort flag (global memory) and the clock are read every 32 polls only,
// so a completed phase is seen within one try_wait.
__device__ __forceinline__ bool wait_bar(uint64_t *b, uint32_t parity, const SweepParams &p) {
    if (mbar_try_wait(b, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(b, parity)) return true;
        if ((it & 31) == 0) {
            if (*(volatile int *)&p.flags[1]) return false;
            if (globaltimer() - t0 > p.wait_ns) {
                record_timeout(p);
                return false;
            }
        }
    }
}

// Bounded wait until a block counter reaches `target`.
__device__ __forceinline__ bool wait_count(const int *ctr, int target, const SweepParams &p) {
    if (ld_acquire(ctr) >= target) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (ld_acquire(ctr) >= target) return true;
        if ((it & 15) == 0) {
            if (*(volatile int *)&p.flags[1]) return false;
            if (globaltimer() - t0 > p.wait_ns) {
                record_timeout(p);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_arrive(uint64_t *b) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}

// ---------------------------------------------------------------------------
// Item decoding.
// ---------------------------------------------------------------------------
struct Item {
    int endop;
    int64_t blk, slab;   // output block and slab
    int64_t src;         // FWD/BWD: block of the vector read (LINK: j; DIAG: blk)
    int64_t seqv;        // LINK: number of updates applied to (blk, slab) before this one
    bool last_link;
    int ncontrib;
};

// Sweeps: column c (0..nt-1) of the item list holds S DIAG items and then
// S * (nt - 1 - c) LINK items; it starts at S * (c * nt - c (c - 1) / 2).
__device__ __forceinline__ int64_t col_start(int64_t S, int64_t nt, int64_t c) {
    return S * (c * nt - c * (c - 1) / 2);
}

__device__ __forceinline__ void decode_item(const SweepParams &p, int64_t t, Item &it) {
    const int64_t S = p.S, nt = p.nt;
    if (p.job == SW_RES) {
        it.endop = E_RES;
        it.blk = t / S;
        it.slab = t % S;
        it.src = 0;
        it.seqv = 0;
        it.last_link = false;
        it.ncontrib = (int)nt;
        return;
    }
    int64_t lo = 0, hi = nt - 1;  // largest c with col_start(c) <= t
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (col_start(S, nt, mid) <= t) lo = mid;
        else hi = mid - 1;
    }
    const int64_t c = lo, r = t - col_start(S, nt, c);
    const bool fwd = (p.job == SW_FWD);
    const int64_t j = fwd ? c : nt - 1 - c;  // block whose vector this column publishes / reads
    it.src = j;
    it.ncontrib = 1;
    if (r < S) {
        it.endop = E_DIAG;
        it.blk = j;
        it.slab = r;
        it.seqv = 0;
        it.last_link = false;
    } else {
        const int64_t m = (r - S) / S;   // m-th block updated from block j
        it.endop = E_LINK;
        it.slab = (r - S) % S;
        it.blk = fwd ? j + 1 + m : j - 1 - m;
        it.seqv = fwd ? j : nt - 1 - j;
        it.last_link = fwd ? (j == it.blk - 1) : (j == it.blk + 1);
    }
}

// One contribution: a tile slab streamed as chunks and the vector block it
// multiplies.
struct Contrib {
    int kind, prec, map;
    int64_t trow;        // first row of the tile in its tensor map
    float inv_scale, shift;
    const float *xsrc;   // vector rows of the contribution (block start)
    const int *dep;      // counter that must reach dep_target before reading them
    int dep_target;
};

__device__ __forceinline__ void contrib_info(const SweepParams &p, const Item &it, int e, Contrib &c) {
    const int64_t b = p.b, nt = p.nt;
    c.inv_scale = 1.f;
    c.shift = 0.f;
    c.dep = nullptr;
    c.dep_target = 0;
    if (p.job == SW_RES) {
        const int64_t i = it.blk, j = e;
        c.prec = KRR_PREC_FP32;
        c.shift = (float)*p.shift;
        c.xsrc = p.xv + j * b * p.ldx + p.q0;
        if (j <= i) {
            c.kind = CK_ROW;
            c.map = 0;
            c.trow = tri_index(i, j) * b;
        } else {
            c.kind = CK_COL;
            c.map = 1;
            c.trow = tri_index(j, i) * b;
        }
        return;
    }
    const bool fwd = (p.job == SW_FWD);
    if (it.endop == E_DIAG) {
        c.kind = CK_ROW;
        c.prec = KRR_PREC_FP32;
        c.map = 3;
        c.trow = it.blk * b;
        c.xsrc = p.rhs + it.blk * b * p.ldx + p.q0;
        const bool first = fwd ? (it.blk == 0) : (it.blk == nt - 1);
        c.dep = done_ctr(p) + it.blk;
        c.dep_target = first ? 0 : (int)p.S;
        return;
    }
    // LINK: forward reads row slab `slab` of L_{blk, src}; backward column
    // slab `slab` of L_{src, blk}
    const int64_t ti = fwd ? it.blk : it.src, tj = fwd ? it.src : it.blk;
    const TileDesc d = p.ltab[off_index(ti, tj)];
    c.kind = fwd ? CK_ROW : CK_COL;
    c.prec = d.prec;
    c.map = (d.prec == KRR_PREC_FP16) ? 0 : (d.prec == KRR_PREC_FP32 ? 1 : 2);
    c.trow = d.offset / (b * esize_of(d.prec));
    if (d.prec != KRR_PREC_FP32) c.inv_scale = 1.f / d.scale;
    c.xsrc = p.out + it.src * b * p.ldx + p.q0;
    c.dep = ready_ctr(p) + it.src;
    c.dep_target = (int)p.S;
}

// Vector rows in a stage: row r at r * pcp + (r >> vs) * 4 floats, vs =
// log2(values per 16-byte unit of the tile precision).  The skew of 16 bytes
// per group of (1 << vs) rows puts the rows that the 8 lanes of a row-chunk
// read at once (one per 16-byte unit) in different banks.
__host__ __device__ __forceinline__ int xrow_off(int r, int vs, int pcp) { return r * pcp + ((r >> vs) << 2); }
__host__ __device__ constexpr int vshift_of(int prec) {
    return prec == KRR_PREC_FP32 ? 2 : (prec == KRR_PREC_FP16 ? 3 : 4);
}

// ---------------------------------------------------------------------------
// Consumer math.  A chunk is 128-byte swizzled: byte x of 128-byte row r sits
// at r * 128 + ((x / 16) ^ (r % 8)) * 16 + x % 16.  Thread = (warp w, lane l).
//   row chunk (128 rows x 128 B): rows 4w + (l / 8) + 32u (u < 4), 16-byte
//       unit l % 8 of each; x row = column of the value.
//   column chunk (128 columns x 128 / esize rows, esize boxes of 128 / esize
//       columns): columns 16w + 4 (l % 4) + u (u < 4), rows l / 4 + 8k.
// acc[u][q] belongs to output row u of the thread's mapping.
// ---------------------------------------------------------------------------
template <int PREC>
__device__ __forceinline__ void to_f32x4(uint32_t w0, uint32_t w1, float *v);

template <int NQ>
__device__ __forceinline__ void fma4(float (&acc)[4][4 * NQ], const float (&v)[4], const float *xr) {
#pragma unroll
    for (int q4 = 0; q4 < NQ; ++q4) {
        const float4 z = *reinterpret_cast<const float4 *>(xr + 4 * q4);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            acc[u][4 * q4 + 0] = fmaf(v[u], z.x, acc[u][4 * q4 + 0]);
            acc[u][4 * q4 + 1] = fmaf(v[u], z.y, acc[u][4 * q4 + 1]);
            acc[u][4 * q4 + 2] = fmaf(v[u], z.z, acc[u][4 * q4 + 2]);
            acc[u][4 * q4 + 3] = fmaf(v[u], z.w, acc[u][4 * q4 + 3]);
        }
    }
}

// Values e of the 16-byte unit u of 4 rows: FP32 4, FP16 8, E4M3 16 per unit.
template <int PREC, int NQ>
__device__ __forceinline__ void row_chunk(const uint8_t *tile, const float *xs, int pcp, float sc, float sh,
                                          int w, int l, float (&acc)[4][4 * NQ]) {
    const int part = l & 7, r0 = 4 * w + (l >> 3);
    uint4 raw[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int r = r0 + 32 * u;
        raw[u] = *reinterpret_cast<const uint4 *>(tile + r * 128 + ((part ^ (r & 7)) << 4));
    }
    if (PREC == KRR_PREC_FP32) {
        const float *x0 = xs + part * (4 * pcp + 4);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            float v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t bits = e == 0 ? raw[u].x : e == 1 ? raw[u].y : e == 2 ? raw[u].z : raw[u].w;
                v[u] = fmaf(__uint_as_float(bits), sc, -sh);
            }
            fma4<NQ>(acc, v, x0 + e * pcp);
        }
    } else if (PREC == KRR_PREC_FP16) {
        const float *x0 = xs + part * (8 * pcp + 4);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float v0[4], v1[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t bits = h == 0 ? raw[u].x : h == 1 ? raw[u].y : h == 2 ? raw[u].z : raw[u].w;
                const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&bits));
                v0[u] = fmaf(f.x, sc, -sh);
                v1[u] = fmaf(f.y, sc, -sh);
            }
            fma4<NQ>(acc, v0, x0 + (2 * h) * pcp);
            fma4<NQ>(acc, v1, x0 + (2 * h + 1) * pcp);
        }
    } else {
        const float *x0 = xs + part * (16 * pcp + 4);
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float v[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t bits = h == 0 ? raw[u].x : h == 1 ? raw[u].y : h == 2 ? raw[u].z : raw[u].w;
                const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(bits & 0xffffu), __NV_E4M3);
                const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(bits >> 16), __NV_E4M3);
                const float2 a = __half22float2(__half2(lo)), c = __half22float2(__half2(hi));
                v[0][u] = fmaf(a.x, sc, -sh);
                v[1][u] = fmaf(a.y, sc, -sh);
                v[2][u] = fmaf(c.x, sc, -sh);
                v[3][u] = fmaf(c.y, sc, -sh);
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) fma4<NQ>(acc, v[e], x0 + (4 * h + e) * pcp);
        }
    }
}

template <int PREC, int NQ>
__device__ __forceinline__ void col_chunk(const uint8_t *tile, const float *xs, int pcp, float sc, float sh,
                                          int w, int l, float (&acc)[4][4 * NQ]) {
    constexpr int ES = esize_of(PREC), RR = 128 / ES;   // rows of the chunk = columns per box
    constexpr int VS = (PREC == KRR_PREC_FP32) ? 2 : (PREC == KRR_PREC_FP16 ? 3 : 4);
    const int c0 = 16 * w + 4 * (l & 3), rp = l >> 2;
    const int box = c0 / RR, within = (c0 % RR) * ES, unit = within >> 4, boff = within & 15;
    const uint8_t *bb = tile + box * (RR * 128) + boff;
#pragma unroll 4
    for (int k = 0; k < RR / 8; ++k) {
        const int r = rp + 8 * k;
        const uint8_t *pe = bb + r * 128 + ((unit ^ (r & 7)) << 4);
        float v[4];
        if (PREC == KRR_PREC_FP32) {
            const float4 f = *reinterpret_cast<const float4 *>(pe);
            v[0] = f.x; v[1] = f.y; v[2] = f.z; v[3] = f.w;
        } else if (PREC == KRR_PREC_FP16) {
            const uint2 u2 = *reinterpret_cast<const uint2 *>(pe);
            const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&u2.x));
            const float2 c = __half22float2(*reinterpret_cast<const __half2 *>(&u2.y));
            v[0] = a.x; v[1] = a.y; v[2] = c.x; v[3] = c.y;
        } else {
            const uint32_t bits = *reinterpret_cast<const uint32_t *>(pe);
            const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(bits & 0xffffu), __NV_E4M3);
            const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(bits >> 16), __NV_E4M3);
            const float2 a = __half22float2(__half2(lo)), c = __half22float2(__half2(hi));
            v[0] = a.x; v[1] = a.y; v[2] = c.x; v[3] = c.y;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = fmaf(v[u], sc, -sh);
        fma4<NQ>(acc, v, xs + xrow_off(r, VS, pcp));
    }
}

// Sums the 8 lanes that share each output (row chunk: lanes l % 8; column
// chunk: lanes l / 4) into the owner lane (l % 8 == 0, resp. l < 4).
template <int NQ>
__device__ __forceinline__ void reduce_lanes(int kind, float (&acc)[4][4 * NQ]) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int q = 0; q < 4 * NQ; ++q) {
            float v = acc[u][q];
            if (kind == CK_ROW) {
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                v += __shfl_xor_sync(0xffffffffu, v, 4);
            } else {
                v += __shfl_xor_sync(0xffffffffu, v, 4);
                v += __shfl_xor_sync(0xffffffffu, v, 8);
                v += __shfl_xor_sync(0xffffffffu, v, 16);
            }
            acc[u][q] = v;
        }
}

__device__ __forceinline__ bool is_owner(int kind, int l) { return kind == CK_ROW ? (l & 7) == 0 : l < 4; }
// Output row (0..127 within the slab) of acc[u] for the owner thread.
__device__ __forceinline__ int owner_row(int kind, int w, int l, int u) {
    return kind == CK_ROW ? 4 * w + (l >> 3) + 32 * u : 16 * w + 4 * (l & 3) + u;
}

// One CTA per SM.  9 warps put 3 warps on one SM sub-partition, whose 16K
// registers then cap a thread at 168.
template <int NQ>
__global__ void __launch_bounds__(SW_THREADS, 1)
    sweep_kernel(const __grid_constant__ CUtensorMap m0, const __grid_constant__ CUtensorMap m1,
                 const __grid_constant__ CUtensorMap m2, const __grid_constant__ CUtensorMap m3,
                 const SweepParams p) {
    extern __shared__ __align__(1024) uint8_t sw_smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(sw_smem_raw) + 1023) & ~uintptr_t(1023));
    const int NS = p.stages;
    const int64_t SB = p.stage_bytes;
    // layout: stages x [chunk 16 KB | header | vector rows], FP64 row sums, barriers
    double *acc64 = reinterpret_cast<double *>(smem + NS * SB);
    uint64_t *bars = reinterpret_cast<uint64_t *>(acc64 + SW_SLAB * p.pcp);
    uint64_t *full = bars, *empty = bars + NS, *cbar = bars + 2 * NS;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1 + 32);
            mbar_init(&empty[s], SW_CONSUMERS / 32);
        }
        mbar_init(cbar, SW_CONSUMERS);  // consumer-group barrier
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&m0)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&m1)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&m2)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&m3)) : "memory");
    }
    __syncthreads();

    if (warp == 0) {
        // ------------------------------ producer ------------------------------
        const CUtensorMap *maps[4] = {&m0, &m1, &m2, &m3};
        int s = 0;
        uint32_t ph = 0;
        int issued = 0;
        bool ok = true;
        // vector-row copies: a row is `per_row` pieces of 16 (x16) or 4 bytes;
        // lanes take fixed (row offset, piece) pairs
        const int per_row = p.x16 ? p.pc / 4 : p.pc;
        const int rows_per_pass = 32 / per_row;
        const int lane_row = lane / per_row, lane_q = (lane % per_row) * (p.x16 ? 4 : 1);
        // emits one stage (TMA chunk + vector rows); false on abort
        auto next_stage = [&](const StageHdr &h, const CUtensorMap *map, int nbox, int bx_step, int x0, int y0,
                              int box_bytes, const float *xrows, int xr, const int *dep, int dep_target) -> bool {
            const int vs = vshift_of(h.prec);
            // every lane waits (acquire); the vote keeps the warp's decision uniform
            if (!__all_sync(0xffffffffu, wait_bar(&empty[s], ph ^ 1, p))) return false;
            uint8_t *st = smem + s * SB;
            if (lane == 0) {
                *reinterpret_cast<StageHdr *>(st + SW_CHUNK) = h;
                if (map) {
                    mbar_arrive_expect_tx(&full[s], (uint32_t)(nbox * box_bytes));
                    for (int bx = 0; bx < nbox; ++bx)
                        tma_load_2d(st + bx * box_bytes, map, x0 + bx * bx_step, y0, &full[s]);
                } else {
                    mbar_arrive(&full[s]);
                }
            }
            bool dep_ok = true;
            if (dep) {
                int okl = 1;
                if (lane == 0) okl = wait_count(dep, dep_target, p) ? 1 : 0;
                dep_ok = __shfl_sync(0xffffffffu, okl, 0) != 0;
                if (dep_ok) (void)ld_acquire(dep);  // every lane acquires before its copies
            }
            if (xrows && dep_ok && lane_row < rows_per_pass) {
                // lane (lane_row, lane_q) copies piece lane_q of rows lane_row, + rows_per_pass, ...
                float *xs = reinterpret_cast<float *>(st + SW_CHUNK + SW_HDR) + lane_q;
                const float *src = xrows + (int64_t)lane_row * p.ldx + lane_q;
                const int64_t sstep = (int64_t)rows_per_pass * p.ldx;
                if (p.x16) {
                    for (int r = lane_row; r < xr; r += rows_per_pass, src += sstep)
                        cp_async16(xs + xrow_off(r, vs, p.pcp), src);
                } else {
                    for (int r = lane_row; r < xr; r += rows_per_pass, src += sstep)
                        cp_async4(xs + xrow_off(r, vs, p.pcp), src);
                }
            }
            cp_async_arrive(&full[s]);
            ++issued;
            if (++s == NS) { s = 0; ph ^= 1; }
            return dep_ok;
        };
        while (ok) {
            int64_t t = 0;
            if (lane == 0) t = atomicAdd(&p.flags[0], 1);
            t = __shfl_sync(0xffffffffu, t, 0);
            if (t >= p.items) break;
            Item it;
            decode_item(p, t, it);
            StageHdr h;
            h.endop = it.endop;
            h.blk = (int)it.blk;
            h.slab = (int)it.slab;
            h.seq = (int)it.seqv;
            int prev_kind = -1;
            for (int e = 0; e < it.ncontrib && ok; ++e) {
                Contrib c;
                contrib_info(p, it, e, c);
                const int ES = esize_of(c.prec);
                const int span = 128 / ES;                 // chunk columns (row) / rows (column)
                const int nchunk = (int)(p.b / span);
                h.kind = c.kind;
                h.prec = c.prec;
                h.inv_scale = c.inv_scale;
                h.shift = c.shift;
                const int sw = (prev_kind >= 0 && prev_kind != c.kind) ? F_SWITCH : 0;
                prev_kind = c.kind;
                for (int k = 0; k < nchunk && ok; ++k) {
                    h.flags = ((e == 0 && k == 0) ? F_FIRST : 0) | (k == nchunk - 1 ? sw | F_LAST_CONTRIB : 0) |
                              ((e == it.ncontrib - 1 && k == nchunk - 1) ? F_LAST_ITEM : 0) |
                              (it.last_link ? F_LAST_LINK : 0);
                    const int64_t xr0 = (int64_t)k * span;   // vector rows of this chunk within the block
                    const float *xrows = c.xsrc + xr0 * p.ldx;
                    const int *dep = (k == 0) ? c.dep : nullptr;
                    if (c.kind == CK_ROW) {
                        // rows [slab * 128, +128) of the tile, columns [xr0, xr0 + span)
                        ok = next_stage(h, maps[c.map], 1, 0, (int)xr0, (int)(c.trow + it.slab * SW_SLAB),
                                        SW_CHUNK, xrows, span, dep, c.dep_target);
                    } else {
                        // columns [slab * 128, +128) as ES boxes of span columns, rows [xr0, xr0 + span)
                        ok = next_stage(h, maps[c.map], ES, span, (int)(it.slab * SW_SLAB), (int)(c.trow + xr0),
                                        SW_CHUNK / ES, xrows, span, dep, c.dep_target);
                    }
                }
            }
        }
        if (ok) {
            StageHdr h;
            memset(&h, 0, sizeof(h));
            h.kind = CK_END;
            ok = next_stage(h, nullptr, 0, 0, 0, 0, 0, nullptr, 0, nullptr, 0);
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
        if (!ok && lane == 0) {
            // drain: wait (bounded) for the copies of the last stages to land
            int n = issued < NS ? issued : NS;
            int ss = s;
            uint32_t pp = ph;
            for (int e = 0; e < n; ++e) {
                if (--ss < 0) { ss = NS - 1; pp ^= 1; }
                const uint64_t t0 = globaltimer();
                while (!mbar_try_wait(&full[ss], pp) && globaltimer() - t0 < drain_limit(p.wait_ns)) {}
            }
        }
    } else {
        // ------------------------------ consumers ------------------------------
        // Group synchronisation uses an mbarrier with bounded waits (not
        // bar.sync), so a consumer that gives up cannot strand the others.
        const int w = warp - 1, ct = threadIdx.x - 32;
        const int pc = p.pc, pcp = p.pcp;
        uint32_t cph = 0;
        auto csync = [&]() -> bool {
            mbar_arrive(cbar);
            const bool r = __all_sync(0xffffffffu, wait_bar(cbar, cph, p));
            cph ^= 1;
            return r;
        };
        float acc[4][4 * NQ];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int q = 0; q < 4 * NQ; ++q) acc[u][q] = 0.f;
        int s = 0;
        uint32_t ph = 0;
        while (true) {
            if (!__all_sync(0xffffffffu, wait_bar(&full[s], ph, p))) break;
            const uint8_t *st = smem + s * SB;
            const StageHdr h = *reinterpret_cast<const StageHdr *>(st + SW_CHUNK);
            if (h.kind == CK_END) break;
            if ((h.flags & F_FIRST) && h.endop == E_RES) {
                // the previous item's last readers of acc64 passed a csync
                for (int e = ct; e < SW_SLAB * pcp; e += SW_CONSUMERS) acc64[e] = 0.0;
                if (!csync()) break;
            }
            const float *xs = reinterpret_cast<const float *>(st + SW_CHUNK + SW_HDR);
            if (h.kind == CK_ROW) {
                if (h.prec == KRR_PREC_FP16) row_chunk<KRR_PREC_FP16, NQ>(st, xs, pcp, h.inv_scale, h.shift, w, lane, acc);
                else if (h.prec == KRR_PREC_FP32) row_chunk<KRR_PREC_FP32, NQ>(st, xs, pcp, h.inv_scale, h.shift, w, lane, acc);
                else row_chunk<KRR_PREC_E4M3, NQ>(st, xs, pcp, h.inv_scale, h.shift, w, lane, acc);
            } else {
                if (h.prec == KRR_PREC_FP16) col_chunk<KRR_PREC_FP16, NQ>(st, xs, pcp, h.inv_scale, h.shift, w, lane, acc);
                else if (h.prec == KRR_PREC_FP32) col_chunk<KRR_PREC_FP32, NQ>(st, xs, pcp, h.inv_scale, h.shift, w, lane, acc);
                else col_chunk<KRR_PREC_E4M3, NQ>(st, xs, pcp, h.inv_scale, h.shift, w, lane, acc);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);  // the stage is free again
            if (++s == NS) { s = 0; ph ^= 1; }
            if (!(h.flags & F_LAST_CONTRIB)) continue;
            reduce_lanes<NQ>(h.kind, acc);
            const bool own = is_owner(h.kind, lane);
            const int64_t row0 = (int64_t)h.blk * p.b + (int64_t)h.slab * SW_SLAB;
            bool ok = true;
            if (h.endop == E_RES) {
                // the owners of a row change when the tiles switch from row to
                // column slabs: order the earlier owners' FP64 updates first
                if ((h.flags & F_SWITCH) && !csync()) break;
                if (own) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        double *a64 = acc64 + owner_row(h.kind, w, lane, u) * pcp;
#pragma unroll
                        for (int q = 0; q < 4 * NQ; ++q)
                            if (q < pc) a64[q] += (double)acc[u][q];
                    }
                    if (h.flags & F_LAST_ITEM) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int row = owner_row(h.kind, w, lane, u);
                            const int64_t gi = (row0 + row) * p.ldx + p.q0;
                            for (int q = 0; q < pc; ++q)
                                p.r[gi + q] = ((double)p.rhs[gi + q] - (double)p.lambda * (double)p.xv[gi + q]) -
                                              acc64[row * pcp + q] - (*p.shift) * p.colsum[p.q0 + q];
                        }
                    }
                }
                if ((h.flags & F_LAST_ITEM) && !csync()) break;  // acc64 is free for the next item
            } else if (h.endop == E_DIAG) {
                if (own) {
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int64_t gi = (row0 + owner_row(h.kind, w, lane, u)) * p.ldx + p.q0;
#pragma unroll
                        for (int q = 0; q < 4 * NQ; ++q)
                            if (q < pc) __stcg(p.out + gi + q, acc[u][q]);
                    }
                }
                ok = csync();
                if (ok && ct == 0) {
                    __threadfence();
                    atomicAdd(ready_ctr(p) + h.blk, 1);
                }
            } else {  // E_LINK: y_blk[slab] -= sum, after the earlier updates of this slab
                int *sq = seq_ctr(p) + (int64_t)h.blk * p.S + h.slab;
                int okw = 1;
                if (lane == 0) okw = wait_count(sq, h.seq, p) ? 1 : 0;
                ok = __shfl_sync(0xffffffffu, okw, 0) != 0;
                if (ok) {
                    (void)ld_acquire(sq);
                    if (own) {
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int64_t gi = (row0 + owner_row(h.kind, w, lane, u)) * p.ldx + p.q0;
#pragma unroll
                            for (int q = 0; q < 4 * NQ; ++q)
                                if (q < pc) __stcg(p.rhs + gi + q, __ldcg(p.rhs + gi + q) - acc[u][q]);
                        }
                    }
                }
                ok = csync() && ok;
                if (ok && ct == 0) {
                    __threadfence();
                    atomicAdd(sq, 1);
                    if (h.flags & F_LAST_LINK) atomicAdd(done_ctr(p) + h.blk, 1);
                }
            }
            if (!ok) break;
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int q = 0; q < 4 * NQ; ++q) acc[u][q] = 0.f;
        }
    }
}

// Encoder of TMA descriptors (driver entry point, looked up once).
typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                             const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                             CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn encoder(Ctx *c) {
    static EncodeFn fn = nullptr;
    if (fn) return fn;
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !f) {
        cudaGetLastError();
        c->last_error = "cuTensorMapEncodeTiled is not available from the driver";
        return nullptr;
    }
    fn = (EncodeFn)f;
    return fn;
}

// Row-major matrix of `rows` rows of `cols` elements, boxes of
// (128 bytes of columns) x box_rows, 128-byte swizzle.
krr_status map_rows(Ctx *c, CUtensorMap *m, const void *base, int prec, int64_t rows, int64_t cols, int box_rows) {
    EncodeFn enc = encoder(c);
    if (!enc) return KRR_ECUDA;
    const int es = esize_of(prec);
    const CUtensorMapDataType dt = prec == KRR_PREC_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : prec == KRR_PREC_FP16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                           : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(cols * es)};
    const cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(m, dt, 2, const_cast<void *>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        c->last_error = "cuTensorMapEncodeTiled (sweep) failed with code " + std::to_string((int)r);
        return KRR_ECUDA;
    }
    return KRR_OK;
}

constexpr size_t smem_limit() { return 227 * 1024; }

// Dynamic shared memory: stages, FP64 row sums, barriers, alignment slack.
size_t smem_bytes(int stages, int64_t stage_bytes, int pcp) {
    return (size_t)stages * stage_bytes + (size_t)SW_SLAB * pcp * 8 + (size_t)(2 * stages + 1) * 8 + 1024;
}

template <int NQ>
krr_status launch_nq(Ctx *c, const CUtensorMap (&m)[4], const SweepParams &p, size_t smem) {
    static PerDevice attr;
    if (!attr.has(c->device)) {
        const cudaError_t e =
            cudaFuncSetAttribute(sweep_kernel<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_limit());
        if (e != cudaSuccess) {
            c->last_error = std::string("cudaFuncSetAttribute (sweep): ") + cudaGetErrorString(e);
            return KRR_ECUDA;
        }
        attr.put(c->device);
    }
    const int64_t grid = std::min<int64_t>(p.items, grid_limit(c));
    count_launch(), sweep_kernel<NQ><<<(unsigned)grid, SW_THREADS, smem, c->stream>>>(m[0], m[1], m[2], m[3], p);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->last_error = std::string("sweep launch: ") + cudaGetErrorString(e);
        return KRR_ECUDA;
    }
    return KRR_OK;
}

int64_t flag_count(const Ctx *c) { return 2 + 2 * c->nt + c->nt * (c->b / SW_SLAB); }

krr_status ensure_sweep_buffers(Ctx *c) {
    const int64_t nflags = flag_count(c);
    if (c->sw_flags_cap < nflags) {
        if (c->sw_flags) cudaFree(c->sw_flags);
        c->sw_flags = nullptr;
        c->sw_flags_cap = 0;
        if (cudaMalloc((void **)&c->sw_flags, nflags * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            c->last_error = "cudaMalloc failed for the sweep counters";
            return KRR_ENOMEM;
        }
        c->sw_flags_cap = nflags;
    }
    return KRR_OK;
}

krr_status run_job(Ctx *c, int job, float *rhs, float *out, const float *xv, double *r, int64_t p) {
    const int64_t b = c->b, nt = c->nt;
    if (b % SW_SLAB != 0) {
        c->last_error = "sweep: the tile edge must be a multiple of 128";
        return KRR_EINVAL;
    }
    KRR_TRY(ensure_sweep_buffers(c));
    CUtensorMap m[4];
    if (job == SW_RES) {
        const int64_t rows = nt * (nt + 1) / 2 * b;
        KRR_TRY(map_rows(c, &m[0], c->Kd, KRR_PREC_FP32, rows, b, 128));
        KRR_TRY(map_rows(c, &m[1], c->Kd, KRR_PREC_FP32, rows, b, 32));
        m[2] = m[0];
        m[3] = m[0];
    } else {
        const bool fwd = (job == SW_FWD);
        const size_t pb = c->pool_bytes;
        KRR_TRY(map_rows(c, &m[0], c->pool, KRR_PREC_FP16, (int64_t)(pb / (2 * b)), b, fwd ? 128 : 64));
        KRR_TRY(map_rows(c, &m[1], c->pool, KRR_PREC_FP32, (int64_t)(pb / (4 * b)), b, fwd ? 128 : 32));
        KRR_TRY(map_rows(c, &m[2], c->pool, KRR_PREC_E4M3, (int64_t)(pb / b), b, 128));
        KRR_TRY(map_rows(c, &m[3], fwd ? c->Linv : c->LinvT, KRR_PREC_FP32, nt * b, b, 128));
    }
    for (int64_t q0 = 0; q0 < p; q0 += SW_PCMAX) {
        SweepParams sp;
        memset(&sp, 0, sizeof(sp));
        sp.job = job;
        sp.b = b;
        sp.nt = nt;
        sp.S = b / SW_SLAB;
        sp.items = (job == SW_RES) ? nt * sp.S : sp.S * nt * (nt + 1) / 2;
        sp.pc = (int)std::min<int64_t>(SW_PCMAX, p - q0);
        sp.pcp = (sp.pc + 3) & ~3;
        sp.q0 = (int)q0;
        sp.ldx = p;
        sp.x16 = (p % 4 == 0 && sp.pc % 4 == 0) ? 1 : 0;
        // vector rows per stage: 32 (FP32 tiles) up to 128 (E4M3 tiles)
        const int64_t xrows = (job == SW_RES) ? 32 : 128;
        sp.stage_bytes = (SW_CHUNK + SW_HDR + xrows * sp.pcp * 4 + 128 + 1023) / 1024 * 1024;
        int stages = 8;
        while (stages > 2 && smem_bytes(stages, sp.stage_bytes, sp.pcp) > smem_limit()) --stages;
        sp.stages = stages;
        sp.rhs = rhs;
        sp.out = out;
        sp.xv = xv;
        sp.r = r;
        sp.shift = c->red + RED_KSHIFT;
        sp.colsum = c->colsum;
        sp.lambda = (float)c->lambda;
        sp.ltab = c->ltab;
        sp.flags = c->sw_flags;
        sp.wait_ns = (uint64_t)c->opt.wait_budget_ns;
        sp.err = c->derr;
        KRR_CUDA_TRY(c, cudaMemsetAsync(c->sw_flags, 0, (size_t)flag_count(c) * sizeof(int), c->stream));
        const size_t smem = smem_bytes(stages, sp.stage_bytes, sp.pcp);
        krr_status st;
        switch (sp.pcp / 4) {
            case 1: st = launch_nq<1>(c, m, sp, smem); break;
            case 2: st = launch_nq<2>(c, m, sp, smem); break;
            case 3: st = launch_nq<3>(c, m, sp, smem); break;
            case 4: st = launch_nq<4>(c, m, sp, smem); break;
            case 5: st = launch_nq<5>(c, m, sp, smem); break;
            default: st = launch_nq<6>(c, m, sp, smem); break;
        }
        KRR_TRY(st);
    }
    return KRR_OK;
}

}  // namespace

// x (n_pad x p) <- (L L^T)^-1 x with the stored factor: the forward sweep
// updates x in place and writes z to tmp, the backward sweep updates tmp in
// place and writes the solution to x.
krr_status sweep_solve(Ctx *c, float *x, float *tmp, int64_t p) {
    KRR_TRY(run_job(c, SW_FWD, x, tmp, nullptr, nullptr, p));
    return run_job(c, SW_BWD, tmp, x, nullptr, nullptr, p);
}

// r = y - lambda a - (K - c 1 1^T) a - c 1 (1^T a); the column sums 1^T a
// must be in c->colsum.
krr_status sweep_residual(Ctx *c, const float *y, const float *a, double *r, int64_t p) {
    return run_job(c, SW_RES, const_cast<float *>(y), nullptr, a, r, p);
}

}  // namespace krr
