// Tensor-core tile sweeps of the solve phase (Alg. 3: forward substitution
// L z = y, backward substitution L^T x = z) for the mixed-precision factor.
//
// Work items (one 128-row slab s of a row block each), as in the paper's tile
// Cholesky solve, right-looking:
//   forward   DIAG(j, s)     z_j[s] = Linv_jj[s, :] y_j             (y_j final)
//             LINK(i, j, s)  y_i[s] -= L_ij[s, :] z_j,  i > j        (row slab of L_ij)
//   backward  DIAG(j, s)     x_j[s] = (Linv_jj^T)[s, :] z_j
//             LINK(t, j, s)  z_t[s] -= (L_jt^T)[s, :] x_j,  t < j    (column slab of L_jt)
// Every item is one tcgen05.mma chain D[128 x NP] = A[128 x b] B[NP x b]^T with
// FP32 accumulation in TMEM:
//   A  a 128-row slab of a factor tile in FP16 (K-major by TMA for the forward
//      sweep; MN-major -- the tile's columns -- for the backward sweep, so no
//      transposed copy of the factor is kept).  FP32-class tiles are stored as
//      an exact FP16 pair (hi, lo) and contribute two A phases; E4M3 tiles are
//      read from their FP16 copy; the diagonal inverses from their FP16 split.
//   B  the vector block as an FP16 pair (hi, lo) with one power-of-two scale
//      per block and column, K-major ([column][row]); both halves are
//      multiplied, so B carries about 22 significant bits.
// The right-hand side is updated in place; a LINK applies its update after the
// earlier ones of the same slab (fixed order: deterministic results).  A slab
// whose rows become final (a DIAG slab, the last LINK of a slab) writes them
// at once as the FP16 pair with a scale predicted from the previous block; the
// last slab of the block checks the prediction against the block's maximum
// (converting the whole block again with the exact scale if it fails) and
// publishes the block.
//
// Items are claimed from a device counter in dependency order (item 0 converts
// the first block; then, per column, its S DIAG items, its head LINK items and
// the LINK items of the column before; see "Items" below).  An item only waits
// for items claimed before it by running CTAs; every wait is bounded
// (%globaltimer) and ends the kernel with KRR_ETIMEOUT.
//
// CTA (192 threads, one per SM):
//   warp 0      producer: claims items, TMA loads of A (16 KB per stage) and B
//               into a shared-memory ring; B only after the block it reads has
//               been published (the A loads of the first stages go out first);
//   warp 1      TMEM allocation and the single MMA-issuing thread;
//   warps 2..5  epilogue: TMEM -> registers, scales, the in-place update or the
//               DIAG store, progress counters and block conversions.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <string>

#include "krr_internal.h"

namespace krr {

namespace {

constexpr int TS_THREADS = 192;
constexpr int TS_EPI = 128;
constexpr int TS_SLAB = 128;             // output rows of an item (MMA M)
constexpr int TS_KC = 64;                // K elements of a stage (128 bytes of FP16)
constexpr int TS_ABYTES = TS_SLAB * 128;  // A bytes of a stage
constexpr int TS_NPMAX = 32;             // right-hand sides per launch
constexpr int TS_IRING = 4;              // item header slots

enum { TS_FWD = 0, TS_BWD = 1 };
enum { IT_CONV = 0, IT_DIAG = 1, IT_LINK = 2, IT_END = 3 };
// A operand maps
enum { AM_POOL = 0, AM_WSH = 1, AM_LHI = 2, AM_LLO = 3 };

struct TsParams {
    int job;
    int64_t b, nt, S, KC, items, n_pad;
    int np, pc, q0;
    int64_t rs, cs;           // vector element (row, column q0 + q) at row * rs + (q0 + q) * cs
    float *rhs;               // FWD: y, BWD: z (updated in place)
    float *out;               // FWD: z, BWD: x
    float *mx_in, *mx_out;    // per-slab column maxima of rhs / out blocks, [nt][S][TS_NPMAX]
    float *bm_in, *bm_out;    // their block column maxima, [nt][TS_NPMAX]
    __half *vin, *vout;       // FP16 pairs of rhs / out blocks: [2 np][n_pad] (hi rows, then lo rows)
    float *sin, *sout;        // their scales, [nt][np]
    const TileDesc *ltab;
    int *flags;               // [0] items, [1] abort, cin[nt], cout[nt], done[nt], ready[nt], seq[nt * S]
    int stages, stage_bytes;
    uint32_t idesc;
    uint64_t wait_ns;
    DevErrors *err;
};

struct ItemHdr {
    int type;
    int blk, slab, src;      // output block and slab; block of the vector read
    int seqv;                // LINK: updates applied to (blk, slab) before this one
    int last_link;
    int nph;                 // A phases (1 or 2)
    int amap[2];
    int arow[2];             // first row of the tile (phase) in its map
    float inv_tscale;        // 1 / tile scale
};

__device__ __forceinline__ int *cin_ctr(const TsParams &p) { return p.flags + 2; }
__device__ __forceinline__ int *cout_ctr(const TsParams &p) { return p.flags + 2 + p.nt; }
__device__ __forceinline__ int *done_ctr(const TsParams &p) { return p.flags + 2 + 2 * p.nt; }
__device__ __forceinline__ int *ready_ctr(const TsParams &p) { return p.flags + 2 + 3 * p.nt; }
__device__ __forceinline__ int *seq_ctr(const TsParams &p) { return p.flags + 2 + 4 * p.nt; }

__device__ __forceinline__ uint32_t smem_u32(const void *ptr) {
    return (uint32_t)__cvta_generic_to_shared(ptr);
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ int ld_acquire(const int *ptr) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(ptr) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(int *ptr, int v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(ptr), "r"(v) : "memory");
}

// Orders this thread's generic-proxy global accesses with later async-proxy
// (TMA) accesses.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

__device__ __forceinline__ void record_timeout(const TsParams &p) {
    atomicExch(&p.flags[1], 1);
    atomicCAS(&p.err->code, 0, (int)KRR_ETIMEOUT);
}

__device__ __forceinline__ bool aborted(const TsParams &p) { return *(volatile int *)&p.flags[1] != 0; }

// Bounded wait on a CTA barrier; false on expiry or when the sweep aborted.
__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity, const TsParams &p) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 31) == 0) {
            if (aborted(p)) return false;
            if (globaltimer() - t0 > p.wait_ns) {
                record_timeout(p);
                return false;
            }
        }
    }
}

// Bounded wait until a progress counter reaches `target`.
// Polls back off exponentially (32 ns up to 256 ns) so that many waiting
// CTAs do not flood the L2 slice holding the counter.
__device__ __forceinline__ bool wait_count(const int *ctr, int target, const TsParams &p) {
    if (ld_acquire(ctr) >= target) return true;
    const uint64_t t0 = globaltimer();
    uint32_t nap = 32;
    for (uint32_t it = 1;; ++it) {
        __nanosleep(nap);
        if (nap < 256) nap <<= 1;
        if (ld_acquire(ctr) >= target) return true;
        if ((it & 15) == 0) {
            if (aborted(p)) return false;
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

// Shared-memory matrix descriptors, 128-byte swizzle (tcgen05 version 1).
// K-major: 8-row groups of 128-byte rows, 1024 bytes apart (SBO); the
// leading offset is unused.
__device__ __forceinline__ uint64_t desc_kmajor(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}
// MN-major: every 128-byte row holds 64 consecutive M elements of one K
// index; 8-row K groups are 1024 bytes apart (SBO) and the two 64-wide M
// halves of the slab are 8192 bytes apart (LBO, one TMA box each).
__device__ __forceinline__ uint64_t desc_mnmajor(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(8192 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ void mma_f16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(r[e]);
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 128;" ::: "memory"); }

// ---------------------------------------------------------------------------
// Items.  Positions count from the start of the sweep: block position c is
// block c (forward) or nt - 1 - c (backward); LINK(c', p) applies column c'
// to block position p > c'.  Item 0 converts the first block of the
// right-hand side; then section c (0..nt-1) lists, S slabs each:
//   DIAG(c);
//   LINK(c - 1, c + 1)                 (1 <= c <= nt - 2)
//   LINK(c, c + 1), the head           (c <= nt - 2)
//   LINK(c - 1, p) for p = c + 2 .. nt - 1.
// The updates of a slab apply in column order, the head last, as with a plain
// column-by-column order; but DIAG(c + 1) is claimed before the bulk of
// column c's updates (listed one section later), so the chain DIAG -> head ->
// DIAG of consecutive columns does not wait for those to be claimed.  Every
// item depends only on items listed before it.  Section sizes: 2S (c = 0,
// nt > 1), S (nt + 1 - c) (0 < c < nt - 1), S (c = nt - 1).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t sec_start(int64_t S, int64_t nt, int64_t c) {
    if (c == 0) return 0;
    const int64_t first = (nt > 1) ? 2 * S : S;
    return first + S * ((c - 1) * (nt + 1) - (c - 1) * c / 2);
}

__device__ void decode_item(const TsParams &p, int64_t t, ItemHdr &h) {
    const int64_t S = p.S, nt = p.nt, b = p.b;
    const bool fwd = (p.job == TS_FWD);
    h.seqv = 0;
    h.last_link = 0;
    h.inv_tscale = 1.f;
    h.nph = 0;
    h.amap[0] = h.amap[1] = 0;
    h.arow[0] = h.arow[1] = 0;
    if (t == 0) {
        h.type = IT_CONV;
        h.blk = fwd ? 0 : (int)(nt - 1);
        h.slab = 0;
        h.src = h.blk;
        return;
    }
    const int64_t u = t - 1;
    int64_t lo = 0, hi = nt - 1;  // largest c with sec_start(c) <= u
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (sec_start(S, nt, mid) <= u) lo = mid;
        else hi = mid - 1;
    }
    const int64_t c = lo;
    int64_t r = u - sec_start(S, nt, c);
    if (r < S) {
        const int64_t j = fwd ? c : nt - 1 - c;
        h.type = IT_DIAG;
        h.blk = (int)j;
        h.src = (int)j;
        h.slab = (int)r;
        h.nph = 2;
        h.amap[0] = AM_LHI;
        h.amap[1] = AM_LLO;
        h.arow[0] = h.arow[1] = (int)(j * b);
        return;
    }
    r -= S;
    int64_t col, pos, slab;  // LINK: column and block positions
    const bool pre = (c >= 1 && c <= nt - 2), head = (c <= nt - 2);
    if (pre && r < S) {
        col = c - 1, pos = c + 1, slab = r;
    } else {
        if (pre) r -= S;
        if (head && r < S) {
            col = c, pos = c + 1, slab = r;
        } else {
            if (head) r -= S;
            col = c - 1, pos = c + 2 + r / S, slab = r % S;
        }
    }
    const int64_t j = fwd ? col : nt - 1 - col;  // block of the vector read
    const int64_t blk = fwd ? pos : nt - 1 - pos;
    h.type = IT_LINK;
    h.src = (int)j;
    h.blk = (int)blk;
    h.slab = (int)slab;
    h.seqv = (int)col;
    h.last_link = (col == pos - 1) ? 1 : 0;
    // forward reads L_{blk, j}, backward L_{j, blk}
    const int64_t ti = fwd ? blk : j, tj = fwd ? j : blk;
    const int64_t off = off_index(ti, tj);
    const TileDesc d = p.ltab[off];
    h.inv_tscale = 1.f / d.scale;
    if (d.prec == KRR_PREC_E4M3) {
        // FP16 copy of the E4M3 tile in the tile's (spent) trailing slot
        h.nph = 1;
        h.amap[0] = AM_WSH;
        h.arow[0] = (int)(off * b);
    } else {
        const int row0 = (int)(d.offset / (2 * b));
        h.amap[0] = h.amap[1] = AM_POOL;
        h.arow[0] = row0;
        h.arow[1] = row0 + (int)b;  // FP32 class: the lo half follows the hi half
        h.nph = (d.prec == KRR_PREC_FP32) ? 2 : 1;
    }
}

// ---------------------------------------------------------------------------
// Block conversion (128 epilogue threads): v rows [blk b, +b), columns
// [q0, q0 + pc) -> FP16 terms with the power-of-two scale s_q putting the
// column maximum in [4096, 8192) (8x headroom below the FP16 maximum):
// two terms hi = fp16(s v), lo = fp16(s v - hi) (about 22 significant bits),
// or three, hi, mid = fp16(s v - hi), lo = fp16(s v - hi - mid), which hold
// an FP32 value exactly down to 2^-14 of the column maximum (below that the
// absolute error stays under 2^-38 of the maximum).  Planes of np rows each;
// padding columns [pc, np) are zero.
// ---------------------------------------------------------------------------
__device__ void convert_block(const TsParams &p, const float *v, int64_t blk, __half *vb, float *sv,
                              float *smax, float *sscale, int tid, int terms = 2, const float *slabmax = nullptr,
                              float *bmax = nullptr) {
    const int64_t b = p.b, n_pad = p.n_pad, rs = p.rs, cs = p.cs;
    const int pc = p.pc, np = p.np;
    if (slabmax) {
        // column maxima published by the slabs of the block
        if (tid < pc) {
            float m = 0.f;
            for (int64_t sl = 0; sl < p.S; ++sl) m = fmaxf(m, __ldcg(slabmax + (blk * p.S + sl) * TS_NPMAX + tid));
            smax[tid] = m;
            smax[TS_NPMAX + tid] = smax[2 * TS_NPMAX + tid] = smax[3 * TS_NPMAX + tid] = 0.f;
        }
    } else {
        float mx[TS_NPMAX];
#pragma unroll
        for (int q = 0; q < TS_NPMAX; ++q) mx[q] = 0.f;
        for (int64_t r = tid; r < b; r += TS_EPI) {
            const float *row = v + (blk * b + r) * rs + p.q0 * cs;
#pragma unroll
            for (int q = 0; q < TS_NPMAX; ++q) {
                if (q < pc) {
                    mx[q] = fmaxf(mx[q], fabsf(__ldcg(row)));
                    row += cs;
                }
            }
        }
        const int wq = tid >> 5, lane = tid & 31;
#pragma unroll
        for (int q = 0; q < TS_NPMAX; ++q) {
            if (q < pc) {
                float m = mx[q];
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
                if (lane == 0) smax[wq * TS_NPMAX + q] = m;
            }
        }
    }
    epi_sync();
    if (tid < np) {
        float s = 1.f;
        if (tid < pc) {
            const float m = fmaxf(fmaxf(smax[tid], smax[TS_NPMAX + tid]),
                                  fmaxf(smax[2 * TS_NPMAX + tid], smax[3 * TS_NPMAX + tid]));
            if (m > 0.f && m < 3.0e38f) {
                int e;
                frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
                s = ldexpf(1.f, max(-126, min(126, 13 - e)));
            }
            if (bmax) bmax[blk * TS_NPMAX + tid] = m;
        }
        sscale[tid] = s;
        sv[blk * np + tid] = s;
    }
    epi_sync();
    for (int64_t r = tid; r < b; r += TS_EPI) {
        const int64_t grow = blk * b + r;
        const float *row = v + grow * rs + p.q0 * cs;
        // the row's loads first (the FP16 stores below may alias them)
        float xv[TS_NPMAX];
#pragma unroll
        for (int q = 0; q < TS_NPMAX; ++q) {
            if (q < pc) {
                xv[q] = __ldcg(row);
                row += cs;
            }
        }
#pragma unroll
        for (int q = 0; q < TS_NPMAX; ++q) {
            if (q < np) {
                const float x = (q < pc) ? xv[q] * sscale[q] : 0.f;
                const __half hh = __float2half_rn(x);
                const float r1 = x - __half2float(hh);  // exact
                const __half m = __float2half_rn(r1);
                vb[(int64_t)q * n_pad + grow] = hh;
                vb[(int64_t)(np + q) * n_pad + grow] = m;
                if (terms == 3) vb[(int64_t)(2 * np + q) * n_pad + grow] = __float2half_rn(r1 - __half2float(m));
            }
        }
    }
    // publish: the block is read next by TMA (async proxy) on other SMs; the
    // caller's thread 0 releases the flag after this barrier
    epi_sync();
    if (tid == 0) {
        __threadfence();
        fence_proxy_async_global();
    }
}

// Column maxima of |x| over the 128 rows of a slab (x one row per thread) into
// dst[TS_NPMAX] (one block of the per-slab array).
__device__ __forceinline__ void slab_max(const float (&x)[TS_NPMAX], int pc, float *smax, int tid, float *dst) {
    const int wq = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int q = 0; q < TS_NPMAX; ++q) {
        if (q < pc) {
            float m = fabsf(x[q]);
            for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0) smax[wq * TS_NPMAX + q] = m;
        }
    }
    epi_sync();
    if (tid < pc)
        dst[tid] = fmaxf(fmaxf(smax[tid], smax[TS_NPMAX + tid]), fmaxf(smax[2 * TS_NPMAX + tid], smax[3 * TS_NPMAX + tid]));
}

// Predicted scale of a block from the column maximum m of the block before
// it in the sweep: puts m in [256, 512).  Blocks of one vector have similar
// magnitudes, so each slab converts its own rows with this scale as soon as
// they are final; the block keeps it if its own maximum lands in
// [PRED_LO, PRED_HI) (about 22 significant bits relative to the maximum, as
// with the exact scale, and 2x headroom below the FP16 maximum), else the last
// slab converts the whole block again with the exact scale.
constexpr float PRED_LO = 8.f, PRED_HI = 32768.f;

__device__ __forceinline__ float pred_scale(float m) {
    if (!(m > 0.f) || !(m < 3.0e38f)) return 1.f;
    int e;
    frexpf(m, &e);
    return ldexpf(1.f, max(-126, min(126, 9 - e)));
}

// One row (one element per column, already final) as an FP16 pair with the
// per-column scales sscale: planes q (hi) and np + q (lo); padding columns zero.
__device__ __forceinline__ void store_pair_row(const TsParams &p, __half *vb, int64_t grow, const float (&x)[TS_NPMAX],
                                               const float *sscale) {
    const int pc = p.pc, np = p.np;
    const int64_t n_pad = p.n_pad;
#pragma unroll
    for (int q = 0; q < TS_NPMAX; ++q) {
        if (q < np) {
            const float xs = (q < pc) ? x[q] * sscale[q] : 0.f;
            const __half hh = __float2half_rn(xs);
            vb[(int64_t)q * n_pad + grow] = hh;
            vb[(int64_t)(np + q) * n_pad + grow] = __float2half_rn(xs - __half2float(hh));
        }
    }
}

// Last slab of a block (128 epilogue threads): block column maxima from the
// slab maxima into bmax; true (for every thread) if the predicted scales in
// sscale hold for every column, and then they become the block's scales sv.
__device__ bool accept_block(const TsParams &p, const float *slabmax, int64_t blk, const float *sscale, float *sv,
                             float *bmax, int *sflag, int tid) {
    if (tid == 0) sflag[3] = 1;
    epi_sync();
    if (tid < p.pc) {
        float m = 0.f;
        for (int64_t sl = 0; sl < p.S; ++sl) m = fmaxf(m, __ldcg(slabmax + (blk * p.S + sl) * TS_NPMAX + tid));
        bmax[blk * TS_NPMAX + tid] = m;
        const float ms = m * sscale[tid];
        if (!(m == 0.f || (ms >= PRED_LO && ms < PRED_HI))) sflag[3] = 0;
    }
    epi_sync();
    const bool ok = sflag[3] != 0;
    if (ok && tid < p.np) sv[blk * p.np + tid] = sscale[tid];
    epi_sync();
    return ok;
}

__global__ void __launch_bounds__(TS_THREADS, 1)
    tcsweep_kernel(const __grid_constant__ CUtensorMap mPool, const __grid_constant__ CUtensorMap mWsh,
                   const __grid_constant__ CUtensorMap mLhi, const __grid_constant__ CUtensorMap mLlo,
                   const __grid_constant__ CUtensorMap mVin, const __grid_constant__ CUtensorMap mVout,
                   const TsParams p) {
    extern __shared__ __align__(1024) uint8_t ts_smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(ts_smem_raw) + 1023) & ~uintptr_t(1023));
    const int NS = p.stages, SB = p.stage_bytes;
    ItemHdr *hdrs = reinterpret_cast<ItemHdr *>(smem + NS * SB);
    float *smax = reinterpret_cast<float *>(hdrs + TS_IRING);    // [4][TS_NPMAX]
    float *sscale = smax + 4 * TS_NPMAX;                          // [TS_NPMAX]
    float *smul = sscale + TS_NPMAX;                              // [TS_NPMAX]
    int *sflag = reinterpret_cast<int *>(smul + TS_NPMAX);        // [4]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sflag + 4);
    uint64_t *full = bars, *empty = bars + NS, *tfull = bars + 2 * NS, *tempty = bars + 2 * NS + 2,
             *ifull = bars + 2 * NS + 4, *iempty = bars + 2 * NS + 4 + TS_IRING,
             *drain = bars + 2 * NS + 4 + 2 * TS_IRING;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int np = p.np;
    // two accumulators of 2 np columns: products with the hi half of B, then
    // with the lo half (one MMA of N = 2 np per K step reads A once)
    const uint32_t tcols = (np * 4 <= 32) ? 32u : (np * 4 <= 64 ? 64u : (np * 4 <= 128 ? 128u : 256u));
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], TS_EPI / 32);
        }
        for (int q = 0; q < TS_IRING; ++q) {
            mbar_init(&ifull[q], 1);
            mbar_init(&iempty[q], TS_EPI / 32 + 1);  // epilogue warps and the MMA thread
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mPool)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mWsh)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mLhi)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mLlo)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mVin)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mVout)) : "memory");
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const bool fwd = (p.job == TS_FWD);
    const uint32_t bbytes = (uint32_t)(2 * np * 128);
    const int KC = (int)p.KC;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------ producer ------------------------------
            const CUtensorMap *amaps[4] = {&mPool, &mWsh, &mLhi, &mLlo};
            int s = 0;
            uint32_t ph = 0;
            int slot = 0;
            uint32_t sph = 0;
            int issued = 0;
            bool ok = true;
            // A chunk c of the item (phase c / KC, K chunk c % KC) into stage st
            auto load_a = [&](const ItemHdr &h, int c, uint8_t *st, uint64_t *bar) {
                const int q = c / KC, kc = c % KC;
                const CUtensorMap *m = amaps[h.amap[q]];
                if (fwd) {
                    tma_load_2d(st, m, kc * TS_KC, h.arow[q] + h.slab * TS_SLAB, bar);
                } else {
                    const int y = h.arow[q] + kc * TS_KC;
                    tma_load_2d(st, m, h.slab * TS_SLAB, y, bar);
                    tma_load_2d(st + TS_ABYTES / 2, m, h.slab * TS_SLAB + 64, y, bar);
                }
            };
            auto load_b = [&](const ItemHdr &h, int c, uint8_t *st, uint64_t *bar) {
                const int kc = c % KC;
                const CUtensorMap *m = (h.type == IT_DIAG) ? &mVin : &mVout;
                tma_load_2d(st + TS_ABYTES, m, (int)(h.src * p.b) + kc * TS_KC, 0, bar);
            };
            while (ok) {
                int64_t t = atomicAdd(&p.flags[0], 1);
                ItemHdr h;
                if (t >= p.items) {
                    memset(&h, 0, sizeof(h));
                    h.type = IT_END;
                } else {
                    decode_item(p, t, h);
                }
                if (!wait_bar(&iempty[slot], sph ^ 1, p)) { ok = false; break; }
                hdrs[slot] = h;
                mbar_arrive(&ifull[slot]);
                if (++slot == TS_IRING) { slot = 0; sph ^= 1; }
                if (h.type == IT_END) break;
                if (h.type == IT_CONV) continue;
                const int nch = h.nph * KC;
                // the first stages' A loads go out before the dependency wait
                const int npre = min(NS, nch);
                int pst[8];
                for (int c = 0; c < npre && ok; ++c) {
                    if (!wait_bar(&empty[s], ph ^ 1, p)) { ok = false; break; }
                    uint8_t *st = smem + s * SB;
                    mbar_arrive_expect_tx(&full[s], (uint32_t)TS_ABYTES + bbytes);
                    load_a(h, c, st, &full[s]);
                    pst[c] = s;
                    ++issued;
                    if (++s == NS) { s = 0; ph ^= 1; }
                }
                if (!ok) break;
                const int *dep = (h.type == IT_DIAG) ? done_ctr(p) + h.blk : ready_ctr(p) + h.src;
                ok = wait_count(dep, 1, p);
                fence_proxy_async_global();
                // (after an abort too, so every issued stage completes and can be drained)
                for (int c = 0; c < npre; ++c) load_b(h, c, smem + pst[c] * SB, &full[pst[c]]);
                for (int c = npre; c < nch && ok; ++c) {
                    if (!wait_bar(&empty[s], ph ^ 1, p)) { ok = false; break; }
                    uint8_t *st = smem + s * SB;
                    mbar_arrive_expect_tx(&full[s], (uint32_t)TS_ABYTES + bbytes);
                    load_a(h, c, st, &full[s]);
                    load_b(h, c, st, &full[s]);
                    ++issued;
                    if (++s == NS) { s = 0; ph ^= 1; }
                }
            }
            if (!ok) {
                // drain: wait (bounded) for the loads of the last stages to land
                const int n = issued < NS ? issued : NS;
                int ss = s;
                uint32_t pp = ph;
                for (int e = 0; e < n; ++e) {
                    if (--ss < 0) { ss = NS - 1; pp ^= 1; }
                    const uint64_t t0 = globaltimer();
                    while (!mbar_try_wait(&full[ss], pp) && globaltimer() - t0 < drain_limit(p.wait_ns)) {}
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------ MMA issuer ------------------------------
            int s = 0;
            uint32_t ph = 0;
            int slot = 0;
            uint32_t sph = 0;
            int acc = 0;
            uint32_t aph = 0;
            bool ok = true, any = false;
            while (ok) {
                if (!wait_bar(&ifull[slot], sph, p)) { ok = false; break; }
                const ItemHdr h = hdrs[slot];
                mbar_arrive(&iempty[slot]);
                if (++slot == TS_IRING) { slot = 0; sph ^= 1; }
                if (h.type == IT_END) break;
                if (h.type == IT_CONV) continue;
                if (!wait_bar(&tempty[acc], aph ^ 1, p)) { ok = false; break; }
                tmem_fence_after();
                const uint32_t tacc = tmem_base + (uint32_t)(acc * 2 * np);
                const int nch = h.nph * KC;
                for (int c = 0; c < nch; ++c) {
                    if (!wait_bar(&full[s], ph, p)) { ok = false; break; }
                    tmem_fence_after();
                    const uint32_t sa = smem_u32(smem + s * SB), sb = sa + TS_ABYTES;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t ad = fwd ? desc_kmajor(sa + kk * 32) : desc_mnmajor(sa + kk * 2048);
                        // B rows [0, np) = hi half, [np, 2 np) = lo half
                        mma_f16(tacc, ad, desc_kmajor(sb + kk * 32), p.idesc, (c > 0 || kk > 0) ? 1u : 0u);
                    }
                    any = true;
                    mma_commit(&empty[s]);
                    if (++s == NS) { s = 0; ph ^= 1; }
                }
                if (!ok) break;
                mma_commit(&tfull[acc]);
                if (++acc == 2) { acc = 0; aph ^= 1; }
            }
            if (!ok && any) {
                mma_commit(drain);
                const uint64_t t0 = globaltimer();
                while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < drain_limit(p.wait_ns)) {}
            }
        }
    } else {
        // ------------------------------ epilogue ------------------------------
        const int tid = threadIdx.x - 64;
        const int row = ((warp & 3) << 5) + lane;  // TMEM lane quarter of this warp
        int slot = 0;
        uint32_t sph = 0;
        int acc = 0;
        uint32_t aph = 0;
        const int pc = p.pc;
        const int64_t b = p.b, S = p.S;
        // one thread waits, the group follows its decision
        auto group_wait_bar = [&](uint64_t *bar, uint32_t parity) -> bool {
            if (tid == 0) sflag[0] = wait_bar(bar, parity, p) ? 1 : 0;
            epi_sync();
            const bool r = sflag[0] != 0;
            epi_sync();
            return r;
        };
        while (true) {
            if (!group_wait_bar(&ifull[slot], sph)) break;
            const ItemHdr h = hdrs[slot];
            epi_sync();
            if (lane == 0) mbar_arrive(&iempty[slot]);
            if (++slot == TS_IRING) { slot = 0; sph ^= 1; }
            if (h.type == IT_END) break;
            if (h.type == IT_CONV) {
                convert_block(p, p.rhs, h.blk, p.vin, p.sin, smax, sscale, tid, 2, nullptr, p.bm_in);
                if (tid == 0) st_release(done_ctr(p) + h.blk, 1);
                continue;
            }
            const int64_t grow = (int64_t)h.blk * b + (int64_t)h.slab * TS_SLAB + row;
            // LINK: once the earlier updates of this slab are in, load the rows
            // to update before waiting for the accumulator (the L2 round trip
            // overlaps the MMAs)
            float yv[TS_NPMAX];
            float *y = p.rhs + grow * p.rs + p.q0 * p.cs;
            int *sq = seq_ctr(p) + (int64_t)h.blk * S + h.slab;
            if (h.type == IT_LINK) {
                if (tid == 0) sflag[2] = wait_count(sq, h.seqv, p) ? 1 : 0;
                epi_sync();
                if (!sflag[2]) break;
                const float *yp = y;
#pragma unroll
                for (int q = 0; q < TS_NPMAX; ++q) {
                    if (q < pc) {
                        yv[q] = __ldcg(yp);
                        yp += p.cs;
                    }
                }
            }
            if (!group_wait_bar(&tfull[acc], aph)) break;
            tmem_fence_after();
            float v[TS_NPMAX];
            const uint32_t tacc = tmem_base + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(acc * 2 * np);
#pragma unroll
            for (int c16 = 0; c16 < TS_NPMAX / 16; ++c16) {
                if (c16 * 16 < np) {
                    float hv[16], lv[16];
                    tmem_ld16(tacc + c16 * 16, hv);
                    tmem_ld16(tacc + np + c16 * 16, lv);
#pragma unroll
                    for (int e = 0; e < 16; ++e) v[c16 * 16 + e] = hv[e] + lv[e];
                }
            }
            tmem_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[acc]);
            if (++acc == 2) { acc = 0; aph ^= 1; }
            // column multipliers: 1 / (tile scale * vector block scale)
            const float *sv = (h.type == IT_DIAG) ? p.sin + (int64_t)h.blk * np : p.sout + (int64_t)h.src * np;
            if (tid < pc) smul[tid] = h.inv_tscale / __ldcg(sv + tid);
            // predicted scale of the block this item finishes: from the block
            // before it in the sweep (the right-hand side's own block for the
            // first solution block)
            const int64_t prev = fwd ? (int64_t)h.blk - 1 : (int64_t)h.blk + 1;
            const bool first = fwd ? (h.blk == 0) : (h.blk == p.nt - 1);
            if ((h.type == IT_DIAG || h.last_link) && tid < np) {
                const float *bm = (h.type == IT_LINK) ? p.bm_in + prev * TS_NPMAX
                                  : first            ? p.bm_in + (int64_t)h.blk * TS_NPMAX
                                                     : p.bm_out + prev * TS_NPMAX;
                sscale[tid] = (tid < pc) ? pred_scale(__ldcg(bm + tid)) : 1.f;
            }
            if (h.type == IT_DIAG) {
                epi_sync();
                float *o = p.out + grow * p.rs + p.q0 * p.cs;
                {
                    float *op = o;
#pragma unroll
                    for (int q = 0; q < TS_NPMAX; ++q) {
                        if (q < pc) {
                            v[q] *= smul[q];
                            __stcg(op, v[q]);
                            op += p.cs;
                        }
                    }
                }
                store_pair_row(p, p.vout, grow, v, sscale);
                slab_max(v, pc, smax, tid, p.mx_out + ((int64_t)h.blk * S + h.slab) * TS_NPMAX);
                epi_sync();
                if (tid == 0) {
                    __threadfence();
                    fence_proxy_async_global();  // the FP16 rows are read by TMA on other SMs
                    const bool last = atomicAdd(cout_ctr(p) + h.blk, 1) == (int)S - 1;
                    if (last) __threadfence();  // the other slabs' rows and maxima are read next
                    sflag[1] = last ? 1 : 0;
                }
                epi_sync();
                if (sflag[1]) {
                    if (!accept_block(p, p.mx_out, h.blk, sscale, p.sout, p.bm_out, sflag, tid))
                        convert_block(p, p.out, h.blk, p.vout, p.sout, smax, sscale, tid, 2, p.mx_out, p.bm_out);
                    if (tid == 0) {
                        __threadfence();
                        st_release(ready_ctr(p) + h.blk, 1);
                    }
                }
            } else {
                // LINK: the rows were loaded before the accumulator wait
                epi_sync();  // smul
                {
                    float *ys = y;
#pragma unroll
                    for (int q = 0; q < TS_NPMAX; ++q) {
                        if (q < pc) {
                            yv[q] -= v[q] * smul[q];
                            __stcg(ys, yv[q]);
                            ys += p.cs;
                        }
                    }
                }
                if (h.last_link) {
                    store_pair_row(p, p.vin, grow, yv, sscale);
                    slab_max(yv, pc, smax, tid, p.mx_in + ((int64_t)h.blk * S + h.slab) * TS_NPMAX);
                }
                epi_sync();
                if (tid == 0) {
                    __threadfence();
                    if (h.last_link) fence_proxy_async_global();
                    atomicAdd(sq, 1);
                    const bool last = h.last_link && atomicAdd(cin_ctr(p) + h.blk, 1) == (int)S - 1;
                    if (last) __threadfence();  // the other slabs' rows are read next
                    sflag[1] = last ? 1 : 0;
                }
                epi_sync();
                if (sflag[1]) {
                    if (!accept_block(p, p.mx_in, h.blk, sscale, p.sin, p.bm_in, sflag, tid))
                        convert_block(p, p.rhs, h.blk, p.vin, p.sin, smax, sscale, tid, 2, p.mx_in, p.bm_in);
                    if (tid == 0) {
                        __threadfence();
                        st_release(done_ctr(p) + h.blk, 1);
                    }
                }
            }
        }
    }
    tmem_fence_before();
    __syncthreads();
    if (warp == 1) {
        tmem_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(tcols) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Refinement residual on the tensor cores:
//   r = y - lambda a - sum_j (K_ij - c) a_j - c 1 (1^T a)      (FP64 output)
// with K the FP32 kernel tiles (lower triangle; block row i reads the row
// slabs of tiles (i, j <= i) and the column slabs of tiles (j > i, i)) and c
// the shift (mean off-diagonal entry of K), which keeps the products small.
// Item (i, s) = 128 rows of block i, one accumulation per tile j:
//   warp 0      producer: TMA of the FP32 K chunk (128 x 64 rows x columns, or
//               64 x 128 for a column slab) into a staging ring, and of the
//               FP16 terms of a_j (B) into a ring of their own;
//   warps 6..9  converters: (K - c) 2^12 -> FP16 pair (hi, lo), written in
//               place over the staged FP32 chunk (each thread overwrites only
//               the bytes its own warp read) in the MMA's K-major or MN-major
//               128-byte-swizzled layout, so the staging ring is also the
//               operand ring;
//   warp 1      MMA: A_hi x [B_hi; B_mid; B_lo] (N = 3 np) and A_lo x [B_hi;
//               B_mid] (N = 2 np); a is split into three FP16 terms (exact for
//               FP32 values), K - c into two (about 22 bits of a quantity
//               already small); the dropped products are below 2^-33;
//   warps 2..5  epilogue: per 64-wide chunk, the three FP32 accumulator
//               parts are summed, de-scaled exactly (powers of two) and added
//               to a two-term FP32 (TwoSum) accumulator, so each FP32 sum in
//               TMEM spans only 64 products.
// Operands exactly representing the FP32 inputs, exact FP16 products and
// FP32 accumulation: the residual keeps FP32 accuracy.
// Every wait is bounded and ends the kernel with KRR_ETIMEOUT.
// ---------------------------------------------------------------------------
constexpr int RS_THREADS = 320;
constexpr int RS_STG = 32768;      // FP32 chunk: 128 x 64 or 64 x 128
constexpr int RS_NSTG = 5;         // staging ring (FP32 K chunks by TMA, converted in place)
constexpr int RS_NB = 3;           // B ring (FP16 terms of a, TMA): loads run ahead of the A ring
// (K - c) s in FP16 with the power of two s = 2^(e - 1) <= 8192 / (max|K| + |c|):
// |(K - c) s| <= 8192, far below the FP16 maximum (s = 2^12 for the Gaussian
// kernel, whose entries lie in (0, 1]).
__device__ __forceinline__ float rs_kscale(const double *kbound, const double *shift) {
    int e;
    frexpf(8192.f / (float)(*kbound + fabs(*shift)), &e);
    return ldexpf(1.f, e - 1);
}

struct RsParams {
    int64_t b, nt, S, KC, items, n_pad;
    int np, pc, q0;
    int64_t ldx;
    const float *y, *a;
    double *r;
    const double *shift, *colsum;
    const double *kbound;   // max |K_ij| (the residual operand's scale follows from it)
    float lambda;
    const float *sa;        // scales of the FP16 pair of a, [nt][np]
    int *flags;             // [0] item counter, [1] abort
    int b_bytes;            // one B chunk: 3 np rows of 128 bytes
    uint32_t idesc_k, idesc_mn, idesc_k2, idesc_mn2;  // N = 3 np and N = 2 np
    uint64_t wait_ns;
    DevErrors *err;
};

__device__ __forceinline__ bool rs_aborted(const RsParams &p) { return *(volatile int *)&p.flags[1] != 0; }

__device__ __forceinline__ bool rs_wait(uint64_t *bar, uint32_t parity, const RsParams &p) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 31) == 0) {
            if (rs_aborted(p)) return false;
            if (globaltimer() - t0 > p.wait_ns) {
                atomicExch(&p.flags[1], 1);
                atomicCAS(&p.err->code, 0, (int)KRR_ETIMEOUT);
                return false;
            }
        }
    }
}

__global__ void __launch_bounds__(RS_THREADS, 1)
    tcres_kernel(const __grid_constant__ CUtensorMap mK128, const __grid_constant__ CUtensorMap mK64,
                 const __grid_constant__ CUtensorMap mA, const RsParams p) {
    extern __shared__ __align__(1024) uint8_t rs_smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(rs_smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *stg = smem;                                   // RS_NSTG x 32 KB
    uint8_t *bst = smem + RS_NSTG * RS_STG;                // RS_NB x b_bytes
    int64_t *items = reinterpret_cast<int64_t *>(bst + RS_NB * p.b_bytes);  // item ring
    uint64_t *bars = reinterpret_cast<uint64_t *>(items + TS_IRING);
    // sfull: FP32 chunk landed; cfull: converted in place; sempty: MMAs done
    uint64_t *sfull = bars, *sempty = bars + RS_NSTG, *cfull = bars + 2 * RS_NSTG,
             *bfull = cfull + RS_NSTG, *bempty = bfull + RS_NB,
             *tfull = bempty + RS_NB, *tempty = tfull + 2, *ifull = tempty + 2, *iempty = ifull + TS_IRING,
             *drain = iempty + TS_IRING;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(drain + 1);
    // epilogue: low halves of the two-term column sums, [TS_NPMAX][128 threads]
    float *alo_s = reinterpret_cast<float *>(tmem_slot + 4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int np = p.np;
    const uint32_t tcols = (np * 6 <= 128) ? 128u : 256u;  // two accumulators of 3 np columns
    if (threadIdx.x == 0) {
        for (int q = 0; q < RS_NSTG; ++q) {
            mbar_init(&sfull[q], 1);
            mbar_init(&sempty[q], 1);      // MMA commit
            mbar_init(&cfull[q], 4);       // converter warps
        }
        for (int q = 0; q < RS_NB; ++q) {
            mbar_init(&bfull[q], 1);       // producer (B bytes)
            mbar_init(&bempty[q], 1);      // MMA commit
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], 4);      // epilogue warps
        }
        for (int q = 0; q < TS_IRING; ++q) {
            mbar_init(&ifull[q], 1);
            mbar_init(&iempty[q], 4 + 4 + 1);  // epilogue, converter warps, MMA thread
        }
        mbar_init(drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(tcols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mK128)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mK64)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mA)) : "memory");
    }
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const int64_t b = p.b, nt = p.nt, S = p.S;
    const int KC = (int)p.KC;
    const uint32_t bbytes = (uint32_t)p.b_bytes;

    if (warp == 0) {
        if (lane == 0) {
            // ------------------------------ producer ------------------------------
            int ss = 0, os = 0, slot = 0;
            uint32_t sph = 0, oph = 0, iph = 0;
            int issued_s = 0, issued_o = 0;
            bool ok = true;
            while (ok) {
                const int64_t t = atomicAdd(&p.flags[0], 1);
                if (!rs_wait(&iempty[slot], iph ^ 1, p)) { ok = false; break; }
                items[slot] = (t < p.items) ? t : -1;
                mbar_arrive(&ifull[slot]);
                if (++slot == TS_IRING) { slot = 0; iph ^= 1; }
                if (t >= p.items) break;
                const int64_t i = t / S, sl = t % S;
                for (int64_t j = 0; j < nt && ok; ++j) {
                    for (int kc = 0; kc < KC && ok; ++kc) {
                        if (!rs_wait(&sempty[ss], sph ^ 1, p)) { ok = false; break; }
                        uint8_t *st = stg + ss * RS_STG;
                        mbar_arrive_expect_tx(&sfull[ss], RS_STG);
                        if (j <= i) {
                            // row slab of tile (i, j): rows [sl 128, +128), columns [kc 64, +64)
                            const int y = (int)(tri_index(i, j) * b + sl * TS_SLAB);
                            tma_load_2d(st, &mK128, kc * 64, y, &sfull[ss]);
                            tma_load_2d(st + RS_STG / 2, &mK128, kc * 64 + 32, y, &sfull[ss]);
                        } else {
                            // column slab of tile (j, i): rows [kc 64, +64), columns [sl 128, +128)
                            const int y = (int)(tri_index(j, i) * b + kc * 64);
                            for (int e = 0; e < 4; ++e)
                                tma_load_2d(st + e * (RS_STG / 4), &mK64, (int)(sl * TS_SLAB) + 32 * e, y, &sfull[ss]);
                        }
                        ++issued_s;
                        if (++ss == RS_NSTG) { ss = 0; sph ^= 1; }
                        if (!rs_wait(&bempty[os], oph ^ 1, p)) { ok = false; break; }
                        mbar_arrive_expect_tx(&bfull[os], bbytes);
                        tma_load_2d(bst + os * p.b_bytes, &mA, (int)(j * b) + kc * 64, 0, &bfull[os]);
                        ++issued_o;
                        if (++os == RS_NB) { os = 0; oph ^= 1; }
                    }
                }
            }
            if (!ok) {
                // drain the copies in flight (bounded)
                int n = issued_s < RS_NSTG ? issued_s : RS_NSTG;
                int q = ss;
                uint32_t pp = sph;
                for (int e = 0; e < n; ++e) {
                    if (--q < 0) { q = RS_NSTG - 1; pp ^= 1; }
                    const uint64_t t0 = globaltimer();
                    while (!mbar_try_wait(&sfull[q], pp) && globaltimer() - t0 < drain_limit(p.wait_ns)) {}
                }
                n = issued_o < RS_NB ? issued_o : RS_NB;
                q = os;
                pp = oph;
                for (int e = 0; e < n; ++e) {
                    if (--q < 0) { q = RS_NB - 1; pp ^= 1; }
                    const uint64_t t0 = globaltimer();
                    while (!mbar_try_wait(&bfull[q], pp) && globaltimer() - t0 < drain_limit(p.wait_ns)) {}
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ------------------------------ MMA issuer ------------------------------
            int ss = 0, bs = 0, slot = 0, acc = 0;
            uint32_t sph = 0, bph = 0, iph = 0, aph = 0;
            bool ok = true, any = false;
            while (ok) {
                if (!rs_wait(&ifull[slot], iph, p)) { ok = false; break; }
                const int64_t t = items[slot];
                mbar_arrive(&iempty[slot]);
                if (++slot == TS_IRING) { slot = 0; iph ^= 1; }
                if (t < 0) break;
                const int64_t i = t / S;
                for (int64_t j = 0; j < nt && ok; ++j) {
                    const bool kmaj = (j <= i);
                    for (int kc = 0; kc < KC; ++kc) {
                        // one accumulation per 64-wide chunk, folded into FP64
                        // by the epilogue: the FP32 sums in TMEM stay short
                        if (!rs_wait(&tempty[acc], aph ^ 1, p)) { ok = false; break; }
                        tmem_fence_after();
                        const uint32_t tacc = tmem_base + (uint32_t)(acc * 3 * np);
                        if (!rs_wait(&cfull[ss], sph, p)) { ok = false; break; }
                        if (!rs_wait(&bfull[bs], bph, p)) { ok = false; break; }
                        tmem_fence_after();
                        const uint32_t sa = smem_u32(stg + ss * RS_STG), sb = smem_u32(bst + bs * p.b_bytes);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t bd = desc_kmajor(sb + kk * 32);
                            if (kmaj) {
                                mma_f16(tacc, desc_kmajor(sa + kk * 32), bd, p.idesc_k, kk > 0 ? 1u : 0u);
                                mma_f16(tacc, desc_kmajor(sa + 16384 + kk * 32), bd, p.idesc_k2, 1u);
                            } else {
                                mma_f16(tacc, desc_mnmajor(sa + kk * 2048), bd, p.idesc_mn, kk > 0 ? 1u : 0u);
                                mma_f16(tacc, desc_mnmajor(sa + 16384 + kk * 2048), bd, p.idesc_mn2, 1u);
                            }
                        }
                        any = true;
                        mma_commit(&sempty[ss]);  // the stage takes the next TMA load
                        mma_commit(&bempty[bs]);
                        if (++ss == RS_NSTG) { ss = 0; sph ^= 1; }
                        if (++bs == RS_NB) { bs = 0; bph ^= 1; }
                        mma_commit(&tfull[acc]);
                        if (++acc == 2) { acc = 0; aph ^= 1; }
                    }
                }
            }
            if (!ok && any) {
                mma_commit(drain);
                const uint64_t t0 = globaltimer();
                while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < drain_limit(p.wait_ns)) {}
            }
        }
    } else if (warp >= 6) {
        // ------------------------------ converters ------------------------------
        const int ct = threadIdx.x - 192;
        const float c = (float)*p.shift;
        const float kscale = rs_kscale(p.kbound, p.shift);
        int ss = 0, slot = 0;
        uint32_t sph = 0, iph = 0;
        bool ok = true;
        while (ok) {
            if (!__all_sync(0xffffffffu, rs_wait(&ifull[slot], iph, p))) break;
            const int64_t t = items[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&iempty[slot]);
            if (++slot == TS_IRING) { slot = 0; iph ^= 1; }
            if (t < 0) break;
            const int64_t i = t / S;
            for (int64_t j = 0; j < nt && ok; ++j) {
                const bool kmaj = (j <= i);
                // thread -> (row r of the staged chunk, 64-value half h)
                const int r = kmaj ? ct : (ct >> 1), h = kmaj ? 0 : (ct & 1);
                const int boxb = kmaj ? RS_STG / 2 : RS_STG / 4;
                for (int kc = 0; kc < KC; ++kc) {
                    if (!__all_sync(0xffffffffu, rs_wait(&sfull[ss], sph, p))) { ok = false; break; }
                    const uint8_t *src = stg + ss * RS_STG + r * 128;
                    uint8_t *dst = stg + ss * RS_STG + h * 8192 + r * 128;
                    float v[64];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const float4 f = *reinterpret_cast<const float4 *>(src + (2 * h + e) * boxb + ((u ^ (r & 7)) << 4));
                            v[e * 32 + 4 * u] = f.x; v[e * 32 + 4 * u + 1] = f.y;
                            v[e * 32 + 4 * u + 2] = f.z; v[e * 32 + 4 * u + 3] = f.w;
                        }
                    }
                    // the FP16 rows overwrite FP32 rows that lanes of this warp
                    // read (thread (r, 0) writes over box 2 row r of thread (r, 1))
                    __syncwarp();
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        uint4 hv, lv;
                        __half2 *hh = reinterpret_cast<__half2 *>(&hv), *ll = reinterpret_cast<__half2 *>(&lv);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float x0 = (v[8 * u + 2 * e] - c) * kscale, x1 = (v[8 * u + 2 * e + 1] - c) * kscale;
                            const __half2 hx = __floats2half2_rn(x0, x1);
                            const float2 hf = __half22float2(hx);
                            hh[e] = hx;
                            ll[e] = __floats2half2_rn(x0 - hf.x, x1 - hf.y);
                        }
                        const int off = (u ^ (r & 7)) << 4;
                        *reinterpret_cast<uint4 *>(dst + off) = hv;
                        *reinterpret_cast<uint4 *>(dst + 16384 + off) = lv;
                    }
                    // generic-proxy writes, read next by the tensor cores
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&cfull[ss]);
                    if (++ss == RS_NSTG) { ss = 0; sph ^= 1; }
                }
            }
        }
    } else {
        // ------------------------------ epilogue ------------------------------
        const int row = ((warp & 3) << 5) + lane;
        int slot = 0, acc = 0;
        uint32_t iph = 0, aph = 0;
        const int pc = p.pc;
        while (true) {
            if (!__all_sync(0xffffffffu, rs_wait(&ifull[slot], iph, p))) break;
            const int64_t t = items[slot];
            __syncwarp();
            if (lane == 0) mbar_arrive(&iempty[slot]);
            if (++slot == TS_IRING) { slot = 0; iph ^= 1; }
            if (t < 0) break;
            const int64_t i = t / S, sl = t % S;
            // per column a two-term FP32 sum (hi, lo) grown by error-free
            // transformations (TwoSum): about 48 significant bits without
            // FP64 arithmetic, which runs at a small fraction of the FP32 rate
            const int et = threadIdx.x - 64;  // epilogue thread 0..127
            float ahi[TS_NPMAX];
#pragma unroll
            for (int q = 0; q < TS_NPMAX; ++q) {
                ahi[q] = 0.f;
                alo_s[q * 128 + et] = 0.f;
            }
            bool ok = true;
            const float kscale = rs_kscale(p.kbound, p.shift);
            float mlane = 0.f;  // lane q: 1 / (kscale * scale of column q of a_j)
            for (int64_t jc = 0; jc < nt * KC; ++jc) {
                const int64_t j = jc / KC;
                if (jc % KC == 0) mlane = (lane < pc) ? 1.f / (kscale * __ldg(p.sa + j * np + lane)) : 0.f;
                if (!__all_sync(0xffffffffu, rs_wait(&tfull[acc], aph, p))) { ok = false; break; }
                tmem_fence_after();
                const uint32_t tacc = tmem_base + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(acc * 3 * np);
                float v[TS_NPMAX];
#pragma unroll
                for (int c16 = 0; c16 < TS_NPMAX / 16; ++c16) {
                    if (c16 * 16 < np) {
                        float hv[16], mv[16], lv[16];
                        tmem_ld16(tacc + c16 * 16, hv);
                        tmem_ld16(tacc + np + c16 * 16, mv);
                        tmem_ld16(tacc + 2 * np + c16 * 16, lv);
#pragma unroll
                        for (int e = 0; e < 16; ++e) v[c16 * 16 + e] = hv[e] + (mv[e] + lv[e]);
                    }
                }
                tmem_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&tempty[acc]);
                if (++acc == 2) { acc = 0; aph ^= 1; }
#pragma unroll
                for (int q = 0; q < TS_NPMAX; ++q) {
                    const float mq = __shfl_sync(0xffffffffu, mlane, q);
                    if (q < pc) {
                        const float xq = v[q] * mq;  // exact: powers of two
                        const float s2 = ahi[q] + xq, bp = s2 - ahi[q];
                        alo_s[q * 128 + et] += (ahi[q] - (s2 - bp)) + (xq - bp);
                        ahi[q] = s2;
                    }
                }
            }
            if (!ok) break;
            const int64_t grow = i * b + sl * TS_SLAB + row;
            const int64_t gi = grow * p.ldx + p.q0;
            const double c = *p.shift;
#pragma unroll
            for (int q = 0; q < TS_NPMAX; ++q)
                if (q < pc)
                    p.r[gi + q] = ((double)p.y[gi + q] - (double)p.lambda * (double)p.a[gi + q]) -
                                  ((double)ahi[q] + (double)alo_s[q * 128 + et]) - c * p.colsum[p.q0 + q];
        }
    }
    tmem_fence_before();
    __syncthreads();
    if (warp == 1) {
        tmem_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(tcols) : "memory");
    }
}

// FP16 pairs of every block of v (one CTA of 128 threads per block).
__global__ void __launch_bounds__(TS_EPI) convert_all_kernel(const TsParams p, const float *v, __half *vb, float *sv,
                                                              int terms) {
    __shared__ float smax[4 * TS_NPMAX], sscale[TS_NPMAX];
    convert_block(p, v, blockIdx.x, vb, sv, smax, sscale, threadIdx.x, terms);
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

// FP16 row-major matrix (rows x cols), boxes of 64 columns (128 bytes) x
// box_rows, 128-byte swizzle.
krr_status map_f16(Ctx *c, CUtensorMap *m, const void *base, int64_t rows, int64_t cols, int box_rows) {
    EncodeFn enc = encoder(c);
    if (!enc) return KRR_ECUDA;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(cols * 2)};
    const cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        c->last_error = "cuTensorMapEncodeTiled (tensor-core sweep) failed with code " + std::to_string((int)r);
        return KRR_ECUDA;
    }
    return KRR_OK;
}

constexpr size_t ts_smem_limit() { return 227 * 1024; }

size_t ts_smem_bytes(int stages, int stage_bytes) {
    return (size_t)stages * stage_bytes + TS_IRING * sizeof(ItemHdr) + (6 * TS_NPMAX + 4) * 4 +
           (size_t)(2 * stages + 5 + 2 * TS_IRING) * 8 + 16 + 1024;
}

int64_t ts_flag_count(const Ctx *c) { return 2 + 4 * c->nt + c->nt * (c->b / TS_SLAB); }

// Auxiliary buffer: block scales of the two FP16 vector buffers ([nt][TS_NPMAX]
// each), per-slab column maxima of the two ([nt][S][TS_NPMAX] each), their
// block column maxima ([nt][TS_NPMAX] each), then the progress counters.
int64_t ts_scale_count(const Ctx *c) { return c->nt * TS_NPMAX; }
int64_t ts_max_count(const Ctx *c) { return c->nt * (c->b / TS_SLAB) * TS_NPMAX; }

krr_status ensure_ts_buffers(Ctx *c, int64_t p) {
    const size_t vbytes = (size_t)3 * TS_NPMAX * c->n_pad * sizeof(__half);
    if (c->ts_vcap < vbytes) {
        for (__half **v : {&c->ts_v0, &c->ts_v1}) {
            if (*v) cudaFree(*v);
            *v = nullptr;
            if (cudaMalloc((void **)v, vbytes) != cudaSuccess) {
                cudaGetLastError();
                c->ts_vcap = 0;
                c->last_error = "cudaMalloc failed for the sweep vector blocks";
                return KRR_ENOMEM;
            }
        }
        c->ts_vcap = vbytes;
    }
    const size_t abytes = (size_t)(4 * ts_scale_count(c) + 2 * ts_max_count(c)) * sizeof(float) +
                          (size_t)ts_flag_count(c) * sizeof(int);
    if (c->ts_aux_cap < abytes) {
        if (c->ts_aux) cudaFree(c->ts_aux);
        c->ts_aux = nullptr;
        if (cudaMalloc(&c->ts_aux, abytes) != cudaSuccess) {
            cudaGetLastError();
            c->ts_aux_cap = 0;
            c->last_error = "cudaMalloc failed for the sweep counters";
            return KRR_ENOMEM;
        }
        c->ts_aux_cap = abytes;
    }
    const size_t xbytes = (size_t)c->n_pad * p * sizeof(float);
    if (p > 0 && c->ts_xcap < xbytes) {
        if (c->ts_xt) cudaFree(c->ts_xt);
        c->ts_xt = nullptr;
        if (cudaMalloc((void **)&c->ts_xt, xbytes) != cudaSuccess) {
            cudaGetLastError();
            c->ts_xcap = 0;
            c->last_error = "cudaMalloc failed for the sweep vector copy";
            return KRR_ENOMEM;
        }
        c->ts_xcap = xbytes;
    }
    return KRR_OK;
}

float *ts_scales(Ctx *c) { return (float *)c->ts_aux; }
float *ts_maxima(Ctx *c) { return ts_scales(c) + 2 * ts_scale_count(c); }
float *ts_block_maxima(Ctx *c) { return ts_maxima(c) + 2 * ts_max_count(c); }
int *ts_flags(Ctx *c) { return (int *)(ts_block_maxima(c) + 2 * ts_scale_count(c)); }

// dst (cols x rows, row-major) = src^T, src rows x cols row-major.
__global__ void transpose_kernel(const float *__restrict__ src, int64_t rows, int64_t cols, float *__restrict__ dst) {
    __shared__ float t[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int64_t r = r0 + k, cc = c0 + threadIdx.x;
        if (r < rows && cc < cols) t[k][threadIdx.x] = src[r * cols + cc];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int64_t cc = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && cc < cols) dst[cc * rows + r] = t[threadIdx.x][k];
    }
}

void launch_transpose(const float *src, int64_t rows, int64_t cols, float *dst, cudaStream_t s) {
    const dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
    count_launch(), transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(src, rows, cols, dst);
}

krr_status run_ts(Ctx *c, int job, float *rhs, float *out, int64_t p) {
    const int64_t b = c->b, nt = c->nt;
    if (b % TS_SLAB != 0) {
        c->last_error = "tensor-core sweep: the tile edge must be a multiple of 128";
        return KRR_EINVAL;
    }
    KRR_TRY(ensure_ts_buffers(c, p));
    const bool fwd = (job == TS_FWD);
    const int abox = fwd ? 128 : 64;
    const int64_t noff = nt * (nt - 1) / 2;
    CUtensorMap mp, mw, mlh, mll, mvi, mvo;
    KRR_TRY(map_f16(c, &mp, c->pool, (int64_t)(c->pool_bytes / (2 * b)), b, abox));
    // the E4M3 copies live in the trailing tiles (only read when such tiles exist)
    KRR_TRY(map_f16(c, &mw, noff > 0 ? c->W : c->Linv_hi, (noff > 0 ? noff : 1) * b, b, abox));
    KRR_TRY(map_f16(c, &mlh, c->Linv_hi, nt * b, b, abox));
    KRR_TRY(map_f16(c, &mll, c->Linv_lo, nt * b, b, abox));
    float *sbase = ts_scales(c);
    int *flags = ts_flags(c);
    static PerDevice attr;
    if (!attr.has(c->device)) {
        const cudaError_t e =
            cudaFuncSetAttribute(tcsweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ts_smem_limit());
        if (e != cudaSuccess) {
            c->last_error = std::string("cudaFuncSetAttribute (tensor-core sweep): ") + cudaGetErrorString(e);
            return KRR_ECUDA;
        }
        attr.put(c->device);
    }
    for (int64_t q0 = 0; q0 < p; q0 += TS_NPMAX) {
        TsParams sp;
        memset(&sp, 0, sizeof(sp));
        sp.job = job;
        sp.b = b;
        sp.nt = nt;
        sp.S = b / TS_SLAB;
        sp.KC = b / TS_KC;
        sp.n_pad = c->n_pad;
        sp.items = 1 + sp.S * nt * (nt + 1) / 2;  // sum of the section sizes
        sp.pc = (int)std::min<int64_t>(TS_NPMAX, p - q0);
        sp.np = (sp.pc + 15) & ~15;
        sp.q0 = (int)q0;
        // column-major vectors ([p][n_pad]): one row per epilogue thread gives
        // coalesced accesses for every column
        sp.rs = 1;
        sp.cs = c->n_pad;
        sp.rhs = rhs;
        sp.out = out;
        sp.mx_in = ts_maxima(c);
        sp.mx_out = ts_maxima(c) + ts_max_count(c);
        sp.bm_in = ts_block_maxima(c);
        sp.bm_out = ts_block_maxima(c) + ts_scale_count(c);
        sp.vin = c->ts_v0;
        sp.vout = c->ts_v1;
        sp.sin = sbase;
        sp.sout = sbase + ts_scale_count(c);
        sp.ltab = c->ltab;
        sp.flags = flags;
        sp.stage_bytes = TS_ABYTES + 2 * sp.np * 128;
        int stages = 8;
        while (stages > 2 && ts_smem_bytes(stages, sp.stage_bytes) > ts_smem_limit()) --stages;
        sp.stages = stages;
        // kind::f16, D = F32, A = B = F16, A K-major (forward) or MN-major
        // (backward), B K-major, N = 2 np (hi and lo halves), M = 128
        sp.idesc = (1u << 4) | ((fwd ? 0u : 1u) << 15) | ((uint32_t)((2 * sp.np) >> 3) << 17) |
                   ((uint32_t)(TS_SLAB >> 4) << 24);
        sp.wait_ns = (uint64_t)c->opt.wait_budget_ns;
        sp.err = c->derr;
        KRR_TRY(map_f16(c, &mvi, c->ts_v0, 2 * sp.np, c->n_pad, 2 * sp.np));
        KRR_TRY(map_f16(c, &mvo, c->ts_v1, 2 * sp.np, c->n_pad, 2 * sp.np));
        KRR_CUDA_TRY(c, cudaMemsetAsync(flags, 0, (size_t)ts_flag_count(c) * sizeof(int), c->stream));
        const size_t smem = ts_smem_bytes(stages, sp.stage_bytes);
        const int64_t grid = std::min<int64_t>(sp.items, grid_limit(c, GL_SWEEP));
        count_launch(), tcsweep_kernel<<<(unsigned)grid, TS_THREADS, smem, c->stream>>>(mp, mw, mlh, mll, mvi, mvo, sp);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            c->last_error = std::string("tensor-core sweep launch: ") + cudaGetErrorString(e);
            return KRR_ECUDA;
        }
    }
    return KRR_OK;
}

}  // namespace

// x (n_pad x p) <- (L L^T)^-1 x with the stored mixed-precision factor on the
// tensor cores: the forward sweep updates x in place and writes z to tmp, the
// backward sweep updates tmp in place and writes the solution to x.
krr_status tc_sweep_solve(Ctx *c, float *x, float *tmp, int64_t p) {
    KRR_TRY(ensure_ts_buffers(c, p));
    // the sweeps work on column-major copies: x^T in ts_xt, z^T in tmp
    float *xt = c->ts_xt;
    launch_transpose(x, c->n_pad, p, xt, c->stream);
    KRR_TRY(run_ts(c, TS_FWD, xt, tmp, p));
    KRR_TRY(run_ts(c, TS_BWD, tmp, xt, p));
    launch_transpose(xt, p, c->n_pad, x, c->stream);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->last_error = std::string("sweep transposes: ") + cudaGetErrorString(e);
        return KRR_ECUDA;
    }
    return KRR_OK;
}

namespace {

// FP32 row-major matrix, boxes of 32 columns (128 bytes) x box_rows, 128-byte swizzle.
krr_status map_f32(Ctx *c, CUtensorMap *m, const void *base, int64_t rows, int64_t cols, int box_rows) {
    EncodeFn enc = encoder(c);
    if (!enc) return KRR_ECUDA;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(cols * 4)};
    const cuuint32_t box[2] = {32u, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void *>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        c->last_error = "cuTensorMapEncodeTiled (tensor-core residual) failed with code " + std::to_string((int)r);
        return KRR_ECUDA;
    }
    return KRR_OK;
}

size_t rs_smem_bytes(int b_bytes) {
    return (size_t)RS_NSTG * RS_STG + (size_t)RS_NB * b_bytes + TS_IRING * 8 +
           (size_t)(3 * RS_NSTG + 2 * RS_NB + 4 + 2 * TS_IRING + 1) * 8 + 16 +
           (size_t)TS_NPMAX * 128 * 4 + 1024;
}

}  // namespace

// r = y - (K + lambda I) a on the tensor cores (mixed mode), given the column
// sums of a in c->colsum and the shift in c->red[RED_KSHIFT].
krr_status tc_residual(Ctx *c, const float *y, const float *a, double *r, int64_t p) {
    const int64_t b = c->b, nt = c->nt;
    KRR_TRY(ensure_ts_buffers(c, 0));
    float *sbase = ts_scales(c);
    int *flags = ts_flags(c);
    const int64_t ntri = nt * (nt + 1) / 2;
    CUtensorMap mk128, mk64, ma;
    KRR_TRY(map_f32(c, &mk128, c->Kd, ntri * b, b, 128));
    KRR_TRY(map_f32(c, &mk64, c->Kd, ntri * b, b, 64));
    static PerDevice attr;
    if (!attr.has(c->device)) {
        const cudaError_t e =
            cudaFuncSetAttribute(tcres_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ts_smem_limit());
        if (e != cudaSuccess) {
            c->last_error = std::string("cudaFuncSetAttribute (tensor-core residual): ") + cudaGetErrorString(e);
            return KRR_ECUDA;
        }
        attr.put(c->device);
    }
    for (int64_t q0 = 0; q0 < p; q0 += TS_NPMAX) {
        // the FP16 pair of a with per-block scales (B operand)
        TsParams cp;
        memset(&cp, 0, sizeof(cp));
        cp.b = b;
        cp.nt = nt;
        cp.n_pad = c->n_pad;
        cp.pc = (int)std::min<int64_t>(TS_NPMAX, p - q0);
        cp.np = (cp.pc + 15) & ~15;
        cp.q0 = (int)q0;
        cp.S = b / TS_SLAB;
        cp.rs = p;  // a is row-major here
        cp.cs = 1;
        count_launch(), convert_all_kernel<<<(unsigned)nt, TS_EPI, 0, c->stream>>>(cp, a, c->ts_v0, sbase, 3);
        KRR_TRY(map_f16(c, &ma, c->ts_v0, 3 * cp.np, c->n_pad, 3 * cp.np));
        RsParams rp;
        memset(&rp, 0, sizeof(rp));
        rp.b = b;
        rp.nt = nt;
        rp.S = b / TS_SLAB;
        rp.KC = b / TS_KC;
        rp.items = nt * rp.S;
        rp.n_pad = c->n_pad;
        rp.np = cp.np;
        rp.pc = cp.pc;
        rp.q0 = cp.q0;
        rp.ldx = p;
        rp.y = y;
        rp.a = a;
        rp.r = r;
        rp.shift = c->red + RED_KSHIFT;
        rp.kbound = c->red + RED_KBOUND;
        rp.colsum = c->colsum;
        rp.lambda = (float)c->lambda;
        rp.sa = sbase;
        rp.flags = flags;
        rp.b_bytes = 3 * rp.np * 128;
        rp.idesc_k = (1u << 4) | ((uint32_t)((3 * rp.np) >> 3) << 17) | ((uint32_t)(TS_SLAB >> 4) << 24);
        rp.idesc_mn = rp.idesc_k | (1u << 15);
        rp.idesc_k2 = (1u << 4) | ((uint32_t)((2 * rp.np) >> 3) << 17) | ((uint32_t)(TS_SLAB >> 4) << 24);
        rp.idesc_mn2 = rp.idesc_k2 | (1u << 15);
        rp.wait_ns = (uint64_t)c->opt.wait_budget_ns;
        rp.err = c->derr;
        KRR_CUDA_TRY(c, cudaMemsetAsync(flags, 0, 2 * sizeof(int), c->stream));
        const size_t smem = rs_smem_bytes(rp.b_bytes);
        const int64_t grid = std::min<int64_t>(rp.items, grid_limit(c, GL_RESIDUAL));
        count_launch(), tcres_kernel<<<(unsigned)grid, RS_THREADS, smem, c->stream>>>(mk128, mk64, ma, rp);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            c->last_error = std::string("tensor-core residual launch: ") + cudaGetErrorString(e);
            return KRR_ECUDA;
        }
    }
    return KRR_OK;
}

}  // namespace krr
