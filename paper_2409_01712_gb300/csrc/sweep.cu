// Persistent dataflow kernel for the tile sweeps of the solve phase (Alg. 3:
// forward substitution L z = y, backward substitution L^T x = z) and for the
// refinement residual r = y - (K + lambda I) a.
//
// Work is cut into items that each own 128 output rows ("slab" s of row
// block i) and read every tile that contributes to them:
//   forward   ACC(i, s)    acc_i = y_i - sum_{j<i} L_ij z_j     (row slabs of L_ij)
//             DIAG(i, s)   z_i   = Linv_ii acc_i                 (row slab of Linv_ii)
//   backward  ACC(j, s)    acc_j = z_j - sum_{i>j} L_ij^T x_i   (column slabs of L_ij)
//             DIAG(j, s)   x_j   = Linv_jj^T acc_j               (row slab of Linv_jj^T)
//   residual  RES(i, s)    r_i = y_i - lambda a_i - sum_j K_ij a_j, K symmetric:
//             row slabs of the stored tiles (i, j <= i), column slabs of (j > i, i)
// Items are claimed in an order that respects the dependencies (all items of
// block i before block i + 1 forward, the reverse backward), from a device
// counter, by whichever CTA is free.  Readiness is published per block with
// counters: done[i] counts finished ACC slabs of block i, ready[i] finished
// DIAG slabs.  A CTA only waits for items that were claimed before its own,
// by CTAs that are running, so the sweep always progresses; every wait is
// still bounded (%globaltimer) and ends the kernel with KRR_ETIMEOUT.
//
// CTA layout: warp 0 produces, warps 1..8 consume.
//   producer  claims items, streams the tile data of each contribution as
//             16 KB chunks into a shared-memory ring with TMA (128-byte
//             swizzle), and copies the matching rows of the input vectors
//             (cp.async) once their producer item has published them;
//   consumers 256 threads, FP32 FMAs from shared memory.  A row chunk (128
//             rows x 128 bytes) gives each thread 2 rows and a quarter of the
//             columns; a column chunk (128 columns x 128 bytes per row) gives
//             each thread 2 columns and a quarter of the rows.  Partial sums
//             of the four quarters are added in a fixed order (deterministic).
// The residual folds every tile's FP32 partial into FP64 before the next tile,
// as the row sums of one tile are where cancellation happens.
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
constexpr int SW_PCMAX = 32;        // right-hand sides per launch

enum SweepJob { SW_FWD = 0, SW_BWD = 1, SW_RES = 2 };
enum ChunkKind { CK_ROW = 0, CK_COL = 1, CK_NONE = 2, CK_END = 3 };
enum ChunkFlags { F_FIRST = 1, F_LAST_CONTRIB = 2, F_LAST_ITEM = 4 };
enum EndOp { E_ACC = 0, E_DIAG = 1, E_RES = 2 };

struct StageHdr {
    int32_t kind, prec, flags, endop;
    int32_t blk, slab;
    float inv_scale, shift;
};

struct SweepParams {
    int job;
    int64_t b, nt, S, items;  // S = b / SW_SLAB slabs per block
    int pc, pcp, q0, x16;     // x16: vector rows can be copied in 16-byte pieces
    int64_t ldx;
    int stages;
    int64_t stage_bytes;
    const float *rhs;         // FWD: y; BWD: z; RES: y
    float *acc;               // FWD / BWD: partial results (n_pad x ldx)
    float *out;               // FWD: z; BWD: x
    const float *xv;          // RES: a
    double *r;                // RES: residual (n_pad x ldx)
    const double *shift;      // RES: shift c (device)
    const double *colsum;     // RES: 1^T a per column
    float lambda;
    const TileDesc *ltab;
    int *flags;               // [0] item counter, [1] abort, [2 + i] done[i], [2 + nt + i] ready[i]
    uint64_t wait_ns;
    DevErrors *err;
};

__host__ __device__ constexpr int esize_of(int prec) {
    return prec == KRR_PREC_FP32 ? 4 : (prec == KRR_PREC_FP16 ? 2 : 1);
}

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
__device__ __forceinline__ bool wait_bar(uint64_t *b, uint32_t parity, const SweepParams &p) {
    if (mbar_try_wait(b, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (true) {
        if (mbar_try_wait(b, parity)) return true;
        if (*(volatile int *)&p.flags[1]) return false;
        if (globaltimer() - t0 > p.wait_ns) {
            record_timeout(p);
            return false;
        }
    }
}

// Bounded wait until a block counter reaches `target`.
__device__ __forceinline__ bool wait_count(const int *ctr, int target, const SweepParams &p) {
    if (ld_acquire(ctr) >= target) return true;
    const uint64_t t0 = globaltimer();
    while (true) {
        __nanosleep(64);
        if (ld_acquire(ctr) >= target) return true;
        if (*(volatile int *)&p.flags[1]) return false;
        if (globaltimer() - t0 > p.wait_ns) {
            record_timeout(p);
            return false;
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

// One contribution of an item: a tile streamed as chunks plus the vector
// block it multiplies.
struct Contrib {
    int kind;          // CK_ROW / CK_COL
    int prec;
    int map;           // tensor map index 0..3
    int64_t trow;      // first row of the tile in its tensor map
    float inv_scale, shift;
    int64_t xblk;      // vector block
    const float *xsrc; // vector base (n_pad x ldx)
    const int *dep;    // counter to wait for before reading the vector (or null)
};

struct ItemInfo {
    int endop;
    int64_t blk, slab;
    int ncontrib;      // contributions
};

// Decodes item t: the end operation and output location.
__device__ __forceinline__ void item_info(const SweepParams &p, int64_t t, ItemInfo &it) {
    if (p.job == SW_RES) {
        it.endop = E_RES;
        it.blk = t / p.S;
        it.slab = t % p.S;
        it.ncontrib = (int)p.nt;
        return;
    }
    const int64_t q = t / (2 * p.S), r = t % (2 * p.S);
    it.blk = (p.job == SW_FWD) ? q : p.nt - 1 - q;
    if (r < p.S) {
        it.endop = E_ACC;
        it.slab = r;
        it.ncontrib = (int)((p.job == SW_FWD) ? it.blk : p.nt - 1 - it.blk);
    } else {
        it.endop = E_DIAG;
        it.slab = r - p.S;
        it.ncontrib = 1;
    }
}

// Contribution e (0-based, in processing order) of an item.
__device__ __forceinline__ void contrib_info(const SweepParams &p, const ItemInfo &it, int e, Contrib &c) {
    const int64_t b = p.b, nt = p.nt;
    c.shift = 0.f;
    c.inv_scale = 1.f;
    const int *done = p.flags + 2, *ready = p.flags + 2 + nt;
    if (p.job == SW_RES) {
        const int64_t i = it.blk, j = e;
        c.prec = KRR_PREC_FP32;
        c.shift = (float)*p.shift;
        c.xblk = j;
        c.xsrc = p.xv;
        c.dep = nullptr;
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
    if (it.endop == E_DIAG) {
        c.kind = CK_ROW;
        c.prec = KRR_PREC_FP32;
        c.map = 3;
        c.trow = it.blk * b;
        c.xblk = it.blk;
        c.xsrc = p.acc;
        c.dep = done + it.blk;
        return;
    }
    int64_t i, j, vb;
    if (p.job == SW_FWD) {
        i = it.blk;
        j = e;
        vb = j;
        c.kind = CK_ROW;
    } else {
        j = it.blk;
        i = nt - 1 - e;
        vb = i;
        c.kind = CK_COL;
    }
    const TileDesc d = p.ltab[off_index(i, j)];
    c.prec = d.prec;
    c.map = (d.prec == KRR_PREC_FP16) ? 0 : (d.prec == KRR_PREC_FP32 ? 1 : 2);
    c.trow = d.offset / (b * esize_of(d.prec));
    if (d.prec != KRR_PREC_FP32) c.inv_scale = 1.f / d.scale;
    c.xblk = vb;
    c.xsrc = p.out;
    c.dep = ready + vb;
}

// ---------------------------------------------------------------------------
// Consumer math.  The tile chunk is 128-byte swizzled: byte `x` of row `r`
// (128-byte rows) sits at r * 128 + ((x / 16) ^ (r % 8)) * 16 + x % 16.
// ---------------------------------------------------------------------------
template <int PREC>
__device__ __forceinline__ void unpack16(const uint4 &u, float *v) {
    if (PREC == KRR_PREC_FP32) {
        v[0] = __uint_as_float(u.x); v[1] = __uint_as_float(u.y);
        v[2] = __uint_as_float(u.z); v[3] = __uint_as_float(u.w);
    } else if (PREC == KRR_PREC_FP16) {
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w[k]));
            v[2 * k] = f.x;
            v[2 * k + 1] = f.y;
        }
    } else {
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[k] & 0xffffu), __NV_E4M3);
            const __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w[k] >> 16), __NV_E4M3);
            const float2 a = __half22float2(__half2(lo)), c = __half22float2(__half2(hi));
            v[4 * k] = a.x; v[4 * k + 1] = a.y; v[4 * k + 2] = c.x; v[4 * k + 3] = c.y;
        }
    }
}

// Row chunk: 128 rows x (128 / esize) columns.  Thread ct: rows ra = ct % 64
// and ra + 64, columns of quarter ct / 64 (32 bytes of every row).
template <int PREC, int NQ>
__device__ __forceinline__ void row_chunk(const uint8_t *tile, const float *xs, int pcp, float inv_scale,
                                          float shift, int ct, float (&acc)[2][4 * NQ]) {
    constexpr int ES = esize_of(PREC), VPU = 16 / ES;  // values per 16-byte unit
    const int qq = ct >> 6, ra = ct & 63, rb = ra + 64;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int unit = 2 * qq + h;
        const uint4 ua = *reinterpret_cast<const uint4 *>(tile + ra * 128 + ((unit ^ (ra & 7)) << 4));
        const uint4 ub = *reinterpret_cast<const uint4 *>(tile + rb * 128 + ((unit ^ (rb & 7)) << 4));
        float va[VPU], vb[VPU];
        unpack16<PREC>(ua, va);
        unpack16<PREC>(ub, vb);
#pragma unroll
        for (int e = 0; e < VPU; ++e) {
            const float a = fmaf(va[e], inv_scale, -shift), c = fmaf(vb[e], inv_scale, -shift);
            const float *xr = xs + (unit * VPU + e) * pcp;
#pragma unroll
            for (int q4 = 0; q4 < NQ; ++q4) {
                const float4 z = *reinterpret_cast<const float4 *>(xr + 4 * q4);
                acc[0][4 * q4 + 0] = fmaf(a, z.x, acc[0][4 * q4 + 0]);
                acc[0][4 * q4 + 1] = fmaf(a, z.y, acc[0][4 * q4 + 1]);
                acc[0][4 * q4 + 2] = fmaf(a, z.z, acc[0][4 * q4 + 2]);
                acc[0][4 * q4 + 3] = fmaf(a, z.w, acc[0][4 * q4 + 3]);
                acc[1][4 * q4 + 0] = fmaf(c, z.x, acc[1][4 * q4 + 0]);
                acc[1][4 * q4 + 1] = fmaf(c, z.y, acc[1][4 * q4 + 1]);
                acc[1][4 * q4 + 2] = fmaf(c, z.z, acc[1][4 * q4 + 2]);
                acc[1][4 * q4 + 3] = fmaf(c, z.w, acc[1][4 * q4 + 3]);
            }
        }
    }
}

// Column chunk: 128 columns x (128 / esize) rows, stored as esize boxes of
// (128 / esize) columns.  Thread ct: columns 2 (ct % 64) and 2 (ct % 64) + 1,
// rows of quarter ct / 64.
template <int PREC, int NQ>
__device__ __forceinline__ void col_chunk(const uint8_t *tile, const float *xs, int pcp, float inv_scale,
                                          float shift, int ct, float (&acc)[2][4 * NQ]) {
    constexpr int ES = esize_of(PREC), RR = 128 / ES, RQ = RR / 4;
    const int qq = ct >> 6, c0 = 2 * (ct & 63);
    const int box = c0 / RR, within = (c0 % RR) * ES, unit = within >> 4, boff = within & 15;
    const uint8_t *bbase = tile + box * (RR * 128) + boff;
#pragma unroll 4
    for (int rr = 0; rr < RQ; ++rr) {
        const int r = qq * RQ + rr;
        const uint8_t *pe = bbase + r * 128 + ((unit ^ (r & 7)) << 4);
        float v0, v1;
        if (PREC == KRR_PREC_FP32) {
            const float2 f = *reinterpret_cast<const float2 *>(pe);
            v0 = f.x;
            v1 = f.y;
        } else if (PREC == KRR_PREC_FP16) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(pe));
            v0 = f.x;
            v1 = f.y;
        } else {
            const uint16_t w = *reinterpret_cast<const uint16_t *>(pe);
            const __half2_raw h = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)w, __NV_E4M3);
            const float2 f = __half22float2(__half2(h));
            v0 = f.x;
            v1 = f.y;
        }
        v0 = fmaf(v0, inv_scale, -shift);
        v1 = fmaf(v1, inv_scale, -shift);
        const float *xr = xs + r * pcp;
#pragma unroll
        for (int q4 = 0; q4 < NQ; ++q4) {
            const float4 z = *reinterpret_cast<const float4 *>(xr + 4 * q4);
            acc[0][4 * q4 + 0] = fmaf(v0, z.x, acc[0][4 * q4 + 0]);
            acc[0][4 * q4 + 1] = fmaf(v0, z.y, acc[0][4 * q4 + 1]);
            acc[0][4 * q4 + 2] = fmaf(v0, z.z, acc[0][4 * q4 + 2]);
            acc[0][4 * q4 + 3] = fmaf(v0, z.w, acc[0][4 * q4 + 3]);
            acc[1][4 * q4 + 0] = fmaf(v1, z.x, acc[1][4 * q4 + 0]);
            acc[1][4 * q4 + 1] = fmaf(v1, z.y, acc[1][4 * q4 + 1]);
            acc[1][4 * q4 + 2] = fmaf(v1, z.z, acc[1][4 * q4 + 2]);
            acc[1][4 * q4 + 3] = fmaf(v1, z.w, acc[1][4 * q4 + 3]);
        }
    }
}

// Writes the thread's partials into red[quarter][row][q] (rows of the item).
template <int NQ>
__device__ __forceinline__ void spill_partials(int kind, int ct, int pc, int pcp, const float (&acc)[2][4 * NQ],
                                               float *red) {
    const int qq = ct >> 6;
    int r0, r1;
    if (kind == CK_ROW) {
        r0 = ct & 63;
        r1 = r0 + 64;
    } else {
        r0 = 2 * (ct & 63);
        r1 = r0 + 1;
    }
    float *d0 = red + (qq * SW_SLAB + r0) * pcp, *d1 = red + (qq * SW_SLAB + r1) * pcp;
#pragma unroll
    for (int q = 0; q < 4 * NQ; ++q) {
        if (q < pc) {
            d0[q] = acc[0][q];
            d1[q] = acc[1][q];
        }
    }
}

template <int NQ>
__global__ void __launch_bounds__(SW_THREADS, 1)
    sweep_kernel(const __grid_constant__ CUtensorMap m0, const __grid_constant__ CUtensorMap m1,
                 const __grid_constant__ CUtensorMap m2, const __grid_constant__ CUtensorMap m3,
                 const SweepParams p) {
    extern __shared__ __align__(1024) uint8_t sw_smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(sw_smem_raw) + 1023) & ~uintptr_t(1023));
    const int NS = p.stages;
    const int64_t SB = p.stage_bytes;
    // layout: stages x [chunk 16 KB | header 64 B | vector rows], red, acc64, barriers
    float *red = reinterpret_cast<float *>(smem + NS * SB);
    double *acc64 = reinterpret_cast<double *>(red + 4 * SW_SLAB * p.pcp);
    uint64_t *bars = reinterpret_cast<uint64_t *>(acc64 + SW_SLAB * p.pcp);
    uint64_t *full = bars, *empty = bars + NS;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1 + 32);
            mbar_init(&empty[s], SW_CONSUMERS / 32);
        }
        mbar_init(&bars[2 * NS], SW_CONSUMERS);  // consumer-group barrier
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
        // emits one stage: optional TMA chunk + vector rows; returns false on abort
        auto next_stage = [&](StageHdr h, const CUtensorMap *map, int nbox, int bx_step, int x0, int y0,
                              int box_bytes, const float *xrows, int xr, const int *dep) -> bool {
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
            if (xrows && dep) {
                int okl = 1;
                if (lane == 0) okl = wait_count(dep, (int)p.S, p) ? 1 : 0;
                okl = __shfl_sync(0xffffffffu, okl, 0);
                dep_ok = okl != 0;
                if (dep_ok) (void)ld_acquire(dep);  // every lane acquires before its copies
            }
            if (xrows && dep_ok) {
                float *xs = reinterpret_cast<float *>(st + SW_CHUNK + SW_HDR);
                const int pc = p.pc, pcp = p.pcp;
                if (p.x16) {
                    const int per_row = pc / 4, total = xr * per_row;
                    for (int e = lane; e < total; e += 32) {
                        const int r = e / per_row, q = (e % per_row) * 4;
                        cp_async16(xs + r * pcp + q, xrows + (int64_t)r * p.ldx + q);
                    }
                } else {
                    const int total = xr * pc;
                    for (int e = lane; e < total; e += 32) {
                        const int r = e / pc, q = e % pc;
                        cp_async4(xs + r * pcp + q, xrows + (int64_t)r * p.ldx + q);
                    }
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
            ItemInfo it;
            item_info(p, t, it);
            StageHdr h;
            h.endop = it.endop;
            h.blk = (int)it.blk;
            h.slab = (int)it.slab;
            if (it.ncontrib == 0) {
                h.kind = CK_NONE;
                h.prec = KRR_PREC_FP32;
                h.flags = F_FIRST | F_LAST_CONTRIB | F_LAST_ITEM;
                h.inv_scale = 1.f;
                h.shift = 0.f;
                ok = next_stage(h, nullptr, 0, 0, 0, 0, 0, nullptr, 0, nullptr);
                continue;
            }
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
                for (int k = 0; k < nchunk && ok; ++k) {
                    h.flags = ((e == 0 && k == 0) ? F_FIRST : 0) | (k == nchunk - 1 ? F_LAST_CONTRIB : 0) |
                              ((e == it.ncontrib - 1 && k == nchunk - 1) ? F_LAST_ITEM : 0);
                    const int64_t xr0 = (int64_t)k * span;   // vector rows of this chunk within the block
                    const float *xrows = c.xsrc + (c.xblk * p.b + xr0) * p.ldx + p.q0;
                    const int *dep = (k == 0) ? c.dep : nullptr;
                    if (c.kind == CK_ROW) {
                        // rows [slab * 128, +128) of the tile, columns [xr0, xr0 + span)
                        ok = next_stage(h, maps[c.map], 1, 0, (int)xr0, (int)(c.trow + it.slab * SW_SLAB),
                                        SW_CHUNK, xrows, span, dep);
                    } else {
                        // columns [slab * 128, +128) as ES boxes of span columns, rows [xr0, xr0 + span)
                        ok = next_stage(h, maps[c.map], ES, span, (int)(it.slab * SW_SLAB), (int)(c.trow + xr0),
                                        SW_CHUNK / ES, xrows, span, dep);
                    }
                }
            }
        }
        if (ok) {
            StageHdr h;
            memset(&h, 0, sizeof(h));
            h.kind = CK_END;
            ok = next_stage(h, nullptr, 0, 0, 0, 0, 0, nullptr, 0, nullptr);
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
                while (!mbar_try_wait(&full[ss], pp) && globaltimer() - t0 < p.wait_ns) {}
            }
        }
    } else {
        // ------------------------------ consumers ------------------------------
        // Consumer-group synchronisation uses an mbarrier with bounded waits
        // (not bar.sync), so a consumer that gives up cannot strand the others.
        const int ct = threadIdx.x - 32;
        const int pc = p.pc, pcp = p.pcp;
        uint64_t *cbar = bars + 2 * NS;
        uint32_t cph = 0;
        auto csync = [&]() -> bool {
            mbar_arrive(cbar);
            const bool r = __all_sync(0xffffffffu, wait_bar(cbar, cph, p));
            cph ^= 1;
            return r;
        };
        float acc[2][4 * NQ];
        bool zero_next = true;
        int s = 0;
        uint32_t ph = 0;
        while (true) {
            if (!__all_sync(0xffffffffu, wait_bar(&full[s], ph, p))) break;
            const uint8_t *st = smem + s * SB;
            const StageHdr h = *reinterpret_cast<const StageHdr *>(st + SW_CHUNK);
            if (h.kind == CK_END) break;
            if ((h.flags & F_FIRST) && h.endop == E_RES)
                for (int e = ct; e < SW_SLAB * pcp; e += SW_CONSUMERS) acc64[e] = 0.0;
            if (zero_next) {
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int q = 0; q < 4 * NQ; ++q) acc[u][q] = 0.f;
                zero_next = false;
            }
            if (h.kind != CK_NONE) {
                const float *xs = reinterpret_cast<const float *>(st + SW_CHUNK + SW_HDR);
                if (h.kind == CK_ROW) {
                    if (h.prec == KRR_PREC_FP16) row_chunk<KRR_PREC_FP16, NQ>(st, xs, pcp, h.inv_scale, h.shift, ct, acc);
                    else if (h.prec == KRR_PREC_FP32) row_chunk<KRR_PREC_FP32, NQ>(st, xs, pcp, h.inv_scale, h.shift, ct, acc);
                    else row_chunk<KRR_PREC_E4M3, NQ>(st, xs, pcp, h.inv_scale, h.shift, ct, acc);
                } else {
                    if (h.prec == KRR_PREC_FP16) col_chunk<KRR_PREC_FP16, NQ>(st, xs, pcp, h.inv_scale, h.shift, ct, acc);
                    else if (h.prec == KRR_PREC_FP32) col_chunk<KRR_PREC_FP32, NQ>(st, xs, pcp, h.inv_scale, h.shift, ct, acc);
                    else col_chunk<KRR_PREC_E4M3, NQ>(st, xs, pcp, h.inv_scale, h.shift, ct, acc);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);  // the stage is free again
            if (++s == NS) { s = 0; ph ^= 1; }
            const bool item_end = (h.flags & F_LAST_ITEM) != 0;
            if (h.endop == E_RES && (h.flags & F_LAST_CONTRIB)) {
                // fold this tile's FP32 partials into the FP64 row sums
                spill_partials<NQ>(h.kind, ct, pc, pcp, acc, red);
                if (!csync()) break;
                for (int e = ct; e < SW_SLAB * pc; e += SW_CONSUMERS) {
                    const int row = e / pc, q = e % pc;
                    const float *rr = red + row * pcp + q;
                    const float sum = ((rr[0] + rr[SW_SLAB * pcp]) + rr[2 * SW_SLAB * pcp]) + rr[3 * SW_SLAB * pcp];
                    acc64[row * pcp + q] += (double)sum;
                }
                if (!csync()) break;
                zero_next = true;
            }
            if (!item_end) continue;
            const bool have = (h.kind != CK_NONE);
            if (h.endop != E_RES && have) {
                spill_partials<NQ>(h.kind, ct, pc, pcp, acc, red);
                if (!csync()) break;
            }
            const int64_t row0 = (int64_t)h.blk * p.b + (int64_t)h.slab * SW_SLAB;
            for (int e = ct; e < SW_SLAB * pc; e += SW_CONSUMERS) {
                const int row = e / pc, q = e % pc;
                const int64_t gi = (row0 + row) * p.ldx + p.q0 + q;
                if (h.endop == E_RES) {
                    p.r[gi] = ((double)p.rhs[gi] - (double)p.lambda * (double)p.xv[gi]) - acc64[row * pcp + q] -
                              (*p.shift) * p.colsum[p.q0 + q];
                    continue;
                }
                float sum = 0.f;
                if (have) {
                    const float *rr = red + row * pcp + q;
                    sum = ((rr[0] + rr[SW_SLAB * pcp]) + rr[2 * SW_SLAB * pcp]) + rr[3 * SW_SLAB * pcp];
                }
                if (h.endop == E_ACC) __stcg(p.acc + gi, __ldcg(p.rhs + gi) - sum);
                else __stcg(p.out + gi, sum);
            }
            if (!csync()) break;  // outputs written; red / acc64 free again
            if (ct == 0 && h.endop != E_RES) {
                __threadfence();
                int *ctr = (h.endop == E_ACC) ? p.flags + 2 + h.blk : p.flags + 2 + p.nt + h.blk;
                atomicAdd(ctr, 1);
            }
            zero_next = true;
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

// Dynamic shared memory of a launch: stages, partials, FP64 row sums,
// barriers, alignment slack.
size_t smem_bytes(int stages, int64_t stage_bytes, int pcp) {
    return (size_t)stages * stage_bytes + (size_t)4 * SW_SLAB * pcp * 4 + (size_t)SW_SLAB * pcp * 8 +
           (size_t)(2 * stages + 1) * 8 + 1024;
}

template <int NQ>
krr_status launch_nq(Ctx *c, const CUtensorMap (&m)[4], const SweepParams &p, size_t smem) {
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(sweep_kernel<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_limit());
        if (e != cudaSuccess) {
            c->last_error = std::string("cudaFuncSetAttribute (sweep): ") + cudaGetErrorString(e);
            return KRR_ECUDA;
        }
        attr = true;
    }
    const int64_t grid = std::min<int64_t>(p.items, c->num_sms);
    count_launch(), sweep_kernel<NQ><<<(unsigned)grid, SW_THREADS, smem, c->stream>>>(m[0], m[1], m[2], m[3], p);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->last_error = std::string("sweep launch: ") + cudaGetErrorString(e);
        return KRR_ECUDA;
    }
    return KRR_OK;
}


krr_status ensure_sweep_buffers(Ctx *c, int64_t p) {
    const int64_t nflags = 2 + 2 * c->nt;
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
    const int64_t cnt = c->n_pad * p;
    if (c->sw_acc_cap < cnt) {
        if (c->sw_acc) cudaFree(c->sw_acc);
        c->sw_acc = nullptr;
        c->sw_acc_cap = 0;
        if (cudaMalloc((void **)&c->sw_acc, cnt * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            c->last_error = "cudaMalloc failed for the sweep partial vectors";
            return KRR_ENOMEM;
        }
        c->sw_acc_cap = cnt;
    }
    return KRR_OK;
}

krr_status run_job(Ctx *c, int job, const float *rhs, float *out, const float *xv, double *r, int64_t p) {
    const int64_t b = c->b, nt = c->nt;
    if (b % SW_SLAB != 0) {
        c->last_error = "sweep: the tile edge must be a multiple of 128";
        return KRR_EINVAL;
    }
    KRR_TRY(ensure_sweep_buffers(c, p));
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
        sp.items = (job == SW_RES) ? nt * sp.S : 2 * nt * sp.S;
        sp.pc = (int)std::min<int64_t>(SW_PCMAX, p - q0);
        sp.pcp = (sp.pc + 3) & ~3;
        sp.q0 = (int)q0;
        sp.ldx = p;
        sp.x16 = (p % 4 == 0 && sp.pc % 4 == 0) ? 1 : 0;
        // vector rows per stage: 32 (FP32 tiles) up to 128 (E4M3 tiles)
        const int64_t xrows = (job == SW_RES) ? 32 : 128;
        sp.stage_bytes = (SW_CHUNK + SW_HDR + xrows * sp.pcp * 4 + 1023) / 1024 * 1024;
        int stages = 6;
        while (stages > 2 && smem_bytes(stages, sp.stage_bytes, sp.pcp) > smem_limit()) --stages;
        sp.stages = stages;
        sp.rhs = rhs;
        sp.acc = c->sw_acc;
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
        KRR_CUDA_TRY(c, cudaMemsetAsync(c->sw_flags, 0, (size_t)(2 + 2 * nt) * sizeof(int), c->stream));
        const size_t smem = smem_bytes(stages, sp.stage_bytes, sp.pcp);
        krr_status st;
        switch (sp.pcp / 4) {
            case 1: st = launch_nq<1>(c, m, sp, smem); break;
            case 2: st = launch_nq<2>(c, m, sp, smem); break;
            case 3: st = launch_nq<3>(c, m, sp, smem); break;
            case 4: st = launch_nq<4>(c, m, sp, smem); break;
            case 5: st = launch_nq<5>(c, m, sp, smem); break;
            case 6: st = launch_nq<6>(c, m, sp, smem); break;
            case 7: st = launch_nq<7>(c, m, sp, smem); break;
            default: st = launch_nq<8>(c, m, sp, smem); break;
        }
        KRR_TRY(st);
    }
    return KRR_OK;
}

}  // namespace

// x (n_pad x p) <- (L L^T)^-1 x with the stored factor: forward sweep into
// tmp (z), backward sweep back into x.
krr_status sweep_solve(Ctx *c, float *x, float *tmp, int64_t p) {
    KRR_TRY(run_job(c, SW_FWD, x, tmp, nullptr, nullptr, p));
    return run_job(c, SW_BWD, tmp, x, nullptr, nullptr, p);
}

// r = y - lambda a - (K - c 1 1^T) a - c 1 (1^T a); the column sums 1^T a
// must be in c->colsum.
krr_status sweep_residual(Ctx *c, const float *y, const float *a, double *r, int64_t p) {
    return run_job(c, SW_RES, y, nullptr, a, r, p);
}

}  // namespace krr
