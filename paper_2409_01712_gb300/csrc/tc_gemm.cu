// Tensor-core (tcgen05) kernels of the KRR engine for sm_103a.
//
// One persistent, warp-specialised kernel template computes 128 x 256 output
// blocks of C = A B^T with both operands K-major in global memory:
//   warp 0      TMA producer: 128-byte-swizzled A (128 rows) and B (256 rows)
//               slabs of 128 bytes along K into a shared-memory ring (4 stages
//               of 48 KB; 6 of 32 KB in pair mode, below);
//   warp 1      TMEM allocator and MMA issuer (one thread): tcgen05.mma
//               M = 128, N = 256 into one of two TMEM accumulators;
//   warps 2..9  epilogue: tcgen05.ld of the accumulator, fused per-op math,
//               stores to global memory.
// Every mbarrier wait is bounded by the context's wait budget
// (%globaltimer); on expiry the kernel records KRR_ETIMEOUT, drains its own
// copies and MMAs in flight, frees TMEM and returns.
//
// Ops (the paper's phases):
//   OP_DIST    Build (Alg. 2, Gaussian kernel of Alg. 5) with the distance
//              form of Sec. IV-B: S = G_I G_J^T on E4M3 operands (genotypes
//              0/1/2 are exact), d = n_i + n_j - 2 S, K = exp(-gamma d).
//   OP_PREDICT Predict (Alg. 4): the same distance tile for test x training
//              rows, exponentiated and multiplied by the matching 256 rows of
//              the weights; per-block partial products.
//   OP_TRSM    Factorize (Alg. 3), panel solve of tile column k:
//              L_ik = W_ik Linv_kk^T with FP16 hi/lo operand splits.
//   OP_GRADT   Gradient of the held-out loss (not in the paper): the test x
//              training distance tile again, contracted as
//              sum_j d_tj K_tj <G_p,t, A_j> per block.
//   OP_GRADK   Same over the lower-triangle training tiles:
//              sum_ij d_ij K_ij <Z_i, A_j> (both triangles through symmetry).
//   OP_UPDATE  Factorize (Alg. 3), trailing update of step k:
//              W_ij -= L_ik L_jk^T for k < j <= i, FP16 operands (hi/lo
//              phases for tiles stored at FP32 accuracy), FP32 accumulation;
//              a block whose two factor tiles are both stored E4M3 runs as
//              kind::f8f6f4 on the stored E4M3 bytes (twice the FP16 rate,
//              half the operand bytes, the same exact products).
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "krr_internal.h"

namespace krr {

namespace {

constexpr int OP_DIST = 0, OP_PREDICT = 1, OP_TRSM = 2, OP_UPDATE = 3, OP_GRADT = 4, OP_GRADK = 5;
constexpr int GRAD_MAX_P = 16;
constexpr int KIND_F16 = 0, KIND_F8 = 1;

constexpr int BM = 128, BN = 256;       // output block
constexpr int SLAB = 128;               // bytes of K per stage and row
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * SLAB;      // 16 KB
constexpr int B_BYTES = BN * SLAB;      // 32 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int NUM_THREADS = 320;        // 2 control warps + 8 epilogue warps
constexpr int EPI_THREADS = 256;
constexpr int TMEM_COLS = 512;          // two 256-column FP32 accumulators
constexpr int PRED_MAX_P = 32;
constexpr uint64_t DRAIN_GRACE_NS = 200000;  // 0.2 ms

// Instruction descriptor (kind::f16 with F16 operands, kind::f8f6f4 with
// E4M3 operands -- both formats encode as 0): D = F32, A and B K-major,
// N = 256, M = 128.
constexpr uint32_t IDESC = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);

// Pair mode (PAIR = 2; the panel solve and the trailing update): two CTAs of a
// cluster run one tcgen05.mma with cta_group::2 over a 256 x 256 block,
// M = 256: each CTA stages its own 128 A rows and one 128-row half of B, and
// keeps its 128 output rows in its TMEM.  A stage is 32 KB instead of 48 KB.
constexpr int BOX_BYTES = BM * 128;     // one 64-column box of an FP16 target block

template <int PAIR>
struct PairCfg {
    static constexpr int stages = (PAIR == 2) ? 6 : STAGES;
    // pair mode (trailing update): the FP16 target block (128 x 256) passes
    // through shared memory as four 64-column boxes in two buffers (TMA load,
    // update in place, TMA store)
    static constexpr int cbuf_bytes = (PAIR == 2) ? 2 * BOX_BYTES : 0;
    static constexpr int stage_bytes = (PAIR == 2) ? 2 * A_BYTES : STAGE_BYTES;
    static constexpr uint32_t idesc = (PAIR == 2)
        ? (1u << 4) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)((2 * BM) >> 4) << 24)
        : IDESC;
};

struct TcParams {
    // n: real training rows; n_pad: padded training rows; n_test / test_rows:
    // real / padded test rows; p / ldaw: weight columns in this launch and the
    // leading dimension of the weights.
    int64_t n, n_pad, n_test, test_rows, b, nt, k, m_pad, items, p, ldaw;
    // index of the launch's first item (a whole number of tiles): a launch
    // covers items [item0, item0 + items) of its operation
    int64_t item0;
    int lb;  // log2 b (the tile edge is a power of two)
    float gamma, lambda;
    const int32_t *norms_a, *norms_b;
    float *Kd;
    uint32_t *Dd;
    double *knorm_part;
    __half *W;
    float *Wd;
    const TileDesc *ltab;
    float *colbuf;
    const float *aw;
    float *part;
    const float *zw;   // OP_GRADK: Z = (K + lambda I)^-1 K_t^T G_p, n_pad x ldaw
    const float *gp;   // OP_GRADT: G_p, padded test rows x ldaw
    double *gpart;     // OP_GRADT / OP_GRADK: one partial sum per block
    const double *kshift;  // OP_PREDICT: shift c subtracted from every K entry (nullptr: none)
    KernelFn kf;           // OP_DIST / OP_PREDICT: kernel function of the distance
    // OP_DIST / OP_PREDICT: confounders of the A rows and the B rows
    // (rows x CONF_MAX), nconf of them (0: none)
    const float *conf_a, *conf_b;
    int nconf;
    uint64_t wait_ns;
    DevErrors *err;
};

// One 128 x 256 output block: up to three operand phases, each nkb slabs.
struct Work {
    int nph, nkb;
    int kind8;  // pair-mode update: both operands E4M3 (kind::f8f6f4, 128 K per stage)
    int amap[3], bmap[3];
    int arow[3], brow[3];
    // epilogue coordinates
    int64_t i, j, sm, sn;
    int64_t t;  // item index
};

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
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ uint32_t mbar_try_wait(uint64_t *b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, P;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok;
}

// Bounded wait; false when the budget ran out or another role aborted.
__device__ __forceinline__ bool wait_bar(uint64_t *b, uint32_t parity, uint64_t budget,
                                         volatile int *abort_flag, DevErrors *err) {
    if (mbar_try_wait(b, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (true) {
        if (mbar_try_wait(b, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer() - t0 > budget) {
            *abort_flag = 1;
            atomicCAS(&err->code, 0, (int)KRR_ETIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Pair mode: the box lands in this CTA's shared memory and completes on the
// barrier `bar_cluster` (a shared::cluster address, possibly in the peer CTA).
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, int x, int y,
                                                 uint32_t bar_cluster) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes.cta_group::2"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar_cluster)
        : "memory");
}

// L2 prefetch of a tensor-map box (no shared memory, no completion).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap *map, int x, int y) {
    asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y)
                 : "memory");
}

__device__ __forceinline__ void tma_store_2d(const CUtensorMap *map, int x, int y, const void *src) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
}
// Element-wise add of a shared-memory box into global memory (the L2 performs
// the read-modify-write; the element type is the tensor map's, here FP16).
__device__ __forceinline__ void tma_reduce_add_2d(const CUtensorMap *map, int x, int y, const void *src) {
    asm volatile("cp.reduce.async.bulk.tensor.2d.global.shared::cta.add.tile.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(smem_u32(src))
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// All but the most recent bulk group have finished reading shared memory.
__device__ __forceinline__ void bulk_wait_read1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// shared::cluster address of the same shared-memory location in CTA `rank`.
__device__ __forceinline__ uint32_t map_to_rank(const void *p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster) : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address
    d |= (uint64_t)1 << 16;                   // leading byte offset (unused for SW128 K-major)
    d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                   // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                   // 128-byte swizzle
    return d;
}

template <int KIND, int PAIR = 1>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    if (PAIR == 2) {
        static_assert(PAIR != 2 || KIND == KIND_F16, "pair mode is FP16 only");
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(PairCfg<2>::idesc), "r"(acc));
    } else if (KIND == KIND_F16) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(IDESC), "r"(acc));
    }
}

// Pair mode, both operands E4M3 (the trailing update of two E4M3 tiles):
// the same descriptors and instruction descriptor (E4M3 encodes as 0, like
// F16), 32 bytes of K per instruction = 32 elements.
__device__ __forceinline__ void mma_pair_f8(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(PairCfg<2>::idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

// Pair mode: arrives on the barrier at the same offset in both CTAs of the
// pair once the pair MMAs issued so far have completed.
__device__ __forceinline__ void mma_commit_pair(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)0x3)
        : "memory");
}

__device__ __forceinline__ void tmem_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
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

__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__device__ __forceinline__ void prefetch_l2(const void *p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// ---------------------------------------------------------------------------
// Work decoding: item index -> operand phases and epilogue coordinates.
// Every role calls this with the same arguments, so all agree on the number
// of slabs of every block (zero for skipped blocks).
// ---------------------------------------------------------------------------
// Descriptor of factor tile (k + 1 + e, k) (the trailing update runs in pair
// mode only, whose shared memory has no room to stage the column's table).
__device__ __forceinline__ TileDesc col_tile(const TcParams &p, int64_t e) {
    return p.ltab[off_index(p.k + 1 + e, p.k)];
}

// Order of the trailing-update target tiles (ii, jj), jj <= ii, of one step:
// bands of UPD_BAND tile rows, and within a band blocks of UPD_BAND tile
// columns (row by row inside a block), so the tiles in flight at any time
// read the factor tiles of at most two bands' worth of rows and columns
// (about 32 MB at b = 1024) and these stay in L2 while they are reused.  A
// band covers the same tile indices as in plain row order, so the band of
// index t is found from the row-major decoding.
constexpr int64_t UPD_BAND = 8;
__device__ __forceinline__ void update_tile_order(int64_t t, int64_t u, int64_t *ii, int64_t *jj) {
    int64_t r, c;
    tri_decode(t, &r, &c);
    const int64_t r0 = r / UPD_BAND * UPD_BAND;
    const int64_t h = (u - r0 < UPD_BAND) ? u - r0 : UPD_BAND;  // rows of the band (the last may be short)
    const int64_t l = t - r0 * (r0 + 1) / 2;                    // index inside the band
    const int64_t full = h * r0;  // tiles of the band left of its diagonal block
    if (l < full) {
        const uint32_t hb = (uint32_t)(h * UPD_BAND);
        const uint32_t cb = (uint32_t)l / hb, l2 = (uint32_t)l % hb;
        *ii = r0 + l2 / UPD_BAND;
        *jj = (int64_t)cb * UPD_BAND + l2 % UPD_BAND;
    } else {
        int64_t a, bb;
        tri_decode(l - full, &a, &bb);
        *ii = r0 + a;
        *jj = r0 + bb;
    }
}

template <int OP>
__device__ __forceinline__ void decode(const TcParams &p, int64_t t, Work &w) {
    // Every role decodes every item, so this runs in 32-bit shifts and masks
    // (the tile edge b is a power of two; item counts stay below 2^31): a
    // 64-bit division costs about a hundred dependent instructions.
    const int64_t b = p.b;
    const int lsc = p.lb - 8, lst = 2 * p.lb - 15;  // log2 (b / BN), log2 ((b / BM) (b / BN))
    const uint32_t ut = (uint32_t)t;
    const int64_t t_tile = ut >> lst;
    const uint32_t t_sub = ut & ((1u << lst) - 1u);
    const int64_t t_sm = t_sub >> lsc, t_sn = t_sub & ((1u << lsc) - 1u);
    w.t = t;
    w.kind8 = 0;
    if (OP == OP_DIST || OP == OP_GRADK) {
        tri_decode(t_tile, &w.i, &w.j);
        w.sm = t_sm;
        w.sn = t_sn;
        w.nph = 1;
        w.nkb = (int)(p.m_pad / SLAB);
        w.amap[0] = 0;
        w.bmap[0] = 2;
        w.arow[0] = (int)(w.i * b + w.sm * BM);
        w.brow[0] = (int)(w.j * b + w.sn * BN);
    } else if (OP == OP_PREDICT || OP == OP_GRADT) {
        // w.i: 128-row block of the A rows (test rows), w.j: 256-row block of
        // the B rows (training rows).  The larger operand's block index varies
        // slowest, so the smaller operand is reused from L2 while each block of
        // the larger one is read from HBM once.
        const uint32_t nab = (uint32_t)(p.test_rows / BM), ncb = (uint32_t)(p.n_pad / BN);
        if (p.n_pad >= p.test_rows) {
            w.j = ut / nab;
            w.i = ut % nab;
        } else {
            w.i = ut / ncb;
            w.j = ut % ncb;
        }
        w.sm = w.sn = 0;
        w.nph = 1;
        w.nkb = (int)(p.m_pad / SLAB);
        w.amap[0] = 0;
        w.bmap[0] = 2;
        w.arow[0] = (int)(w.i * BM);
        w.brow[0] = (int)(w.j * BN);
    } else if (OP == OP_TRSM) {
        const int64_t k = p.k;
        w.i = k + 1 + t_tile;
        w.j = k;
        w.sm = t_sm;
        w.sn = t_sn;
        // Linv_kk is lower triangular: output columns < (sn + 1) * 256 need
        // K < (sn + 1) * 256 only.
        w.nkb = (int)((w.sn + 1) * BN * 2 / SLAB);
        const int arow = (k == 0) ? (int)((w.i - 1) * b + w.sm * BM)
                                  : (int)(off_index(w.i, k) * b + w.sm * BM);
        const int brow = (int)(k * b + w.sn * BN);
        if (k == 0) {
            // A = Kd column 0 split hi/lo; B = Linv hi/lo
            w.nph = 3;
            w.amap[0] = 0; w.bmap[0] = 2;
            w.amap[1] = 0; w.bmap[1] = 3;
            w.amap[2] = 1; w.bmap[2] = 2;
        } else {
            // A = FP16 trailing tile (exact in FP16); B = Linv hi/lo
            w.nph = 2;
            w.amap[0] = 0; w.bmap[0] = 2;
            w.amap[1] = 0; w.bmap[1] = 3;
        }
        for (int q = 0; q < 3; ++q) {
            w.arow[q] = arow;
            w.brow[q] = brow;
        }
    } else {  // OP_UPDATE
        const int64_t k = p.k;
        int64_t ii, jj;
        update_tile_order(t_tile, p.nt - k - 1, &ii, &jj);
        w.i = k + 1 + ii;
        w.j = k + 1 + jj;
        w.sm = t_sm;
        w.sn = t_sn;
        w.nkb = (int)(b * 2 / SLAB);
        if (w.i == w.j && w.sn * BN >= (w.sm + 1) * BM) {
            w.nph = 0;  // strictly above the diagonal of a diagonal tile
            return;
        }
        // operand maps: 0 = factor pool viewed as FP16 rows of b, 1 = FP16 (hi)
        // panel of the column, 2 = FP16 lo panel, 4 = factor pool viewed as
        // E4M3 rows of b bytes.  Two E4M3 tiles meet in one kind::f8f6f4
        // phase on their stored bytes (a stage holds 128 of their columns);
        // otherwise FP16 tiles are read from the pool directly, FP32 tiles
        // use the hi/lo split, E4M3 tiles their FP16 shadow in the hi panel.
        const TileDesc di = col_tile(p, w.i - k - 1);
        const TileDesc dj = col_tile(p, w.j - k - 1);
        if (di.prec == KRR_PREC_E4M3 && dj.prec == KRR_PREC_E4M3) {
            w.kind8 = 1;
            w.nph = 1;
            w.nkb = (int)(b / SLAB);
            w.amap[0] = 4;
            w.arow[0] = (int)((di.offset >> p.lb) + w.sm * BM);
            w.bmap[0] = 4;
            w.brow[0] = (int)((dj.offset >> p.lb) + w.sn * BN);
            return;
        }
        const int ahi_map = (di.prec == KRR_PREC_FP16) ? 0 : 1;
        const int bhi_map = (dj.prec == KRR_PREC_FP16) ? 0 : 1;
        const int ahi_row = (int)((di.prec == KRR_PREC_FP16 ? di.offset >> (p.lb + 1) : (w.i - k - 1) * b) + w.sm * BM);
        const int bhi_row = (int)((dj.prec == KRR_PREC_FP16 ? dj.offset >> (p.lb + 1) : (w.j - k - 1) * b) + w.sn * BN);
        const int alo_row = (int)((w.i - k - 1) * b + w.sm * BM);
        const int blo_row = (int)((w.j - k - 1) * b + w.sn * BN);
        int q = 0;
        w.amap[q] = ahi_map; w.arow[q] = ahi_row; w.bmap[q] = bhi_map; w.brow[q] = bhi_row; ++q;
        if (dj.prec == KRR_PREC_FP32) { w.amap[q] = ahi_map; w.arow[q] = ahi_row; w.bmap[q] = 2; w.brow[q] = blo_row; ++q; }
        if (di.prec == KRR_PREC_FP32) { w.amap[q] = 2; w.arow[q] = alo_row; w.bmap[q] = bhi_map; w.brow[q] = bhi_row; ++q; }
        w.nph = q;
    }
}

// Cluster pairs (two CTAs along M share the B operand): pair unit u covers
// the 256 x 256 region of 128 x 256 blocks (2 pm, sn) and (2 pm + 1, sn) of
// one tile; CTA `rank` of the pair takes block 2 pm + rank.  Both CTAs of a
// pair decode the same tile, phases and B rows.
__device__ __forceinline__ int64_t pair_item(const TcParams &p, int64_t u, uint32_t rank) {
    const int lsc = p.lb - 8, lpt = 2 * p.lb - 16;  // log2 (b / BN), log2 (pairs per tile)
    const uint32_t uu = (uint32_t)u;
    const uint32_t tile = uu >> lpt, pu = uu & ((1u << lpt) - 1u);
    const uint32_t sn = pu & ((1u << lsc) - 1u), pm = pu >> lsc;
    return ((int64_t)tile << (lpt + 1)) + (int64_t)(((2u * pm + rank) << lsc) + sn);
}

// ---------------------------------------------------------------------------
// Epilogues.  Eight warps: warp w (2..9) reads TMEM lane quarter w % 4, so
// thread `row` owns accumulator row `row`; `half` = (w - 2) / 4 selects
// columns [half * 128, half * 128 + 128) of the 256-column block.
// ---------------------------------------------------------------------------
constexpr int CH_PER_HALF = BN / 16 / 2;

// Issues L2 prefetches for the trailing-update input row segment of this
// thread, before it waits for the accumulator.
template <int OP>
__device__ __forceinline__ void epilogue_prefetch(const TcParams &p, const Work &w, int row, int half) {
    if (OP != OP_UPDATE) return;
    const int64_t b = p.b, k = p.k;
    const int64_t lr = w.sm * BM + row, c0 = w.sn * BN + half * 128;
    const char *ptr;
    int bytes;
    if (w.i == w.j) {
        ptr = reinterpret_cast<const char *>((k == 0 ? p.Kd + tri_index(w.i, w.i) * b * b : p.Wd + w.i * b * b) +
                                             lr * b + c0);
        bytes = 512;
    } else if (k == 0) {
        ptr = reinterpret_cast<const char *>(p.Kd + tri_index(w.i, w.j) * b * b + lr * b + c0);
        bytes = 512;
    } else {
        ptr = reinterpret_cast<const char *>(p.W + off_index(w.i, w.j) * b * b + lr * b + c0);
        bytes = 256;
    }
    for (int o = 0; o < bytes; o += 128) prefetch_l2(ptr + o);
}

// Predict: the thread's test row against 128 training columns of the block,
// exp(-gamma d) - c times the staged weights, NQ (>= p) weight columns.
template <int NQ>
__device__ __forceinline__ void predict_half(const TcParams &p, uint32_t tacc, int ch0, int64_t gi, int64_t j0,
                                             const int32_t *nb_s, const float *aw_s, float kc, float *dst) {
    const int32_t ni = p.norms_a[gi];
    const bool real_row = gi < p.n_test;
    const int nc = p.nconf;
    float ci[CONF_MAX];
#pragma unroll
    for (int q = 0; q < CONF_MAX; ++q) ci[q] = (q < nc) ? p.conf_a[gi * CONF_MAX + q] : 0.f;
    float acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = 0.f;
    for (int ch = ch0; ch < ch0 + CH_PER_HALF; ++ch) {
        float v[16];
        tmem_ld16(tacc + ch * 16, v);
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int c = ch * 16 + e;
            const int32_t d = ni + nb_s[c] - 2 * (int32_t)v[e];
            const float *ar = aw_s + c * PRED_MAX_P;
            // confounders of the training row: slots [16, 32) of its staged row (p <= 16 then)
            const float dc = nc ? conf_dist(ci, ar + 16, nc) : 0.f;
            const float kv = (real_row && j0 + c < p.n) ? p.kf.value(p.gamma, d, dc) - kc : 0.f;
#pragma unroll
            for (int q = 0; q < NQ; ++q) acc[q] = fmaf(kv, ar[q], acc[q]);
        }
    }
    const int pp = (int)p.p;
#pragma unroll
    for (int q = 0; q < NQ; ++q)
        if (q < pp) dst[q] = acc[q];
}

// Gradient contractions: sum over 128 columns of d exp(-gamma d) times the
// staged A (and, for the training tiles, Z) columns, NQ (>= p) of them, then
// the thread's dot products with its own row; returns the warp's sum.
template <int NQ, bool KTERM>
__device__ __forceinline__ double grad_half(const TcParams &p, const Work &w, uint32_t tacc, int ch0, int64_t gi,
                                            int64_t j0, const int32_t *nb_s, const float *aw_s) {
    const int64_t a_real = KTERM ? p.n : p.n_test;
    const int32_t ni = p.norms_a[gi];
    const int pp = (int)p.p;
    float accA[NQ], accZ[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) accA[q] = accZ[q] = 0.f;
    for (int ch = ch0; ch < ch0 + CH_PER_HALF; ++ch) {
        float v[16];
        tmem_ld16(tacc + ch * 16, v);
#pragma unroll
        for (int e = 0; e < 16; ++e) {
            const int c = ch * 16 + e;
            const int32_t d = ni + nb_s[c] - 2 * (int32_t)v[e];
            const float sv = (gi < a_real && j0 + c < p.n) ? (float)d * expf(-p.gamma * (float)d) : 0.f;
            const float *ar = aw_s + c * PRED_MAX_P;  // columns beyond p are zero
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                accA[q] = fmaf(sv, ar[q], accA[q]);
                if (KTERM) accZ[q] = fmaf(sv, ar[GRAD_MAX_P + q], accZ[q]);
            }
        }
    }
    double val = 0.0;
    if (gi < a_real) {
        const float *own = KTERM ? p.zw : p.gp;  // Z_i or G_p,t
#pragma unroll
        for (int q = 0; q < NQ; ++q)
            if (q < pp) val += (double)own[gi * p.ldaw + q] * (double)accA[q];
        if (KTERM && w.i != w.j) {  // mirror entry (j, i) of an off-diagonal tile
#pragma unroll
            for (int q = 0; q < NQ; ++q)
                if (q < pp) val += (double)p.aw[gi * p.ldaw + q] * (double)accZ[q];
        }
    }
    for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xffffffffu, val, o);
    return val;
}

template <int OP>
__device__ __forceinline__ void epilogue(const TcParams &p, const Work &w, uint32_t tacc, int row, int half,
                                         int32_t *nb_s, float *aw_s, double *red_s) {
    const int64_t b = p.b;
    const int ch0 = half * CH_PER_HALF;
    if (OP == OP_DIST) {
        const int64_t gi = w.i * b + w.sm * BM + row;
        const int32_t ni = p.norms_a[gi];
        const int nc = p.nconf;
        float ci[CONF_MAX];
#pragma unroll
        for (int q = 0; q < CONF_MAX; ++q) ci[q] = (q < nc) ? p.conf_a[gi * CONF_MAX + q] : 0.f;
        const int64_t tidx = tri_index(w.i, w.j);
        float *krow = p.Kd + tidx * b * b + (w.sm * BM + row) * b + w.sn * BN;
        uint32_t *drow = p.Dd ? p.Dd + tidx * b * b + (w.sm * BM + row) * b + w.sn * BN : nullptr;
        double ss = 0.0, s1 = 0.0;
        for (int ch = ch0; ch < ch0 + CH_PER_HALF; ++ch) {
            float v[16];
            tmem_ld16(tacc + ch * 16, v);
            float kv[16];
            uint32_t dv[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int c = ch * 16 + e;
                const int64_t gj = w.j * b + w.sn * BN + c;
                const int32_t d = ni + nb_s[c] - 2 * (int32_t)v[e];
                const bool real = gi < p.n && gj < p.n;
                // confounders of column c: slots [16, 32) of its staged row
                const float dc = nc ? conf_dist(ci, aw_s + c * PRED_MAX_P + 16, nc) : 0.f;
                kv[e] = real ? (p.kf.gram ? v[e] : p.kf.value(p.gamma, d, dc)) : (gi == gj ? 1.f : 0.f);
                dv[e] = real ? (uint32_t)d : 0u;
                ss += (double)kv[e] * (double)kv[e];
                s1 += (double)kv[e];
            }
            float4 *dst = reinterpret_cast<float4 *>(krow + ch * 16);
#pragma unroll
            for (int e = 0; e < 4; ++e) dst[e] = make_float4(kv[4 * e], kv[4 * e + 1], kv[4 * e + 2], kv[4 * e + 3]);
            if (drow) {
                uint4 *dd = reinterpret_cast<uint4 *>(drow + ch * 16);
#pragma unroll
                for (int e = 0; e < 4; ++e) dd[e] = make_uint4(dv[4 * e], dv[4 * e + 1], dv[4 * e + 2], dv[4 * e + 3]);
            }
        }
        // deterministic per-block sums of K^2 and K: warp sums, then the eight
        // warps in order.  Layout: all K^2 partials, then all K partials.
        for (int o = 16; o > 0; o >>= 1) {
            ss += __shfl_xor_sync(0xffffffffu, ss, o);
            s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        }
        const int ew = (threadIdx.x >> 5) - 2;
        if ((threadIdx.x & 31) == 0) {
            red_s[ew] = ss;
            red_s[8 + ew] = s1;
        }
        epi_bar();
        if (threadIdx.x == 64) {
            const int64_t sub_per_tile = (b / BM) * (b / BN);
            const int64_t slot = tidx * sub_per_tile + w.sm * (b / BN) + w.sn;
            double a0 = 0.0, a1 = 0.0;
            for (int q = 0; q < 8; ++q) {
                a0 += red_s[q];
                a1 += red_s[8 + q];
            }
            p.knorm_part[slot] = a0;
            p.knorm_part[p.items + slot] = a1;
        }
    } else if (OP == OP_PREDICT) {
        const int64_t gi = w.i * BM + row;  // test row
        const int pp = (int)p.p;
        // K - c: the entries of K concentrate around their mean, so the
        // shifted products are small and their FP32 sums lose far less to
        // cancellation; the reduction adds c (1^T A) back in FP64.  Padding
        // columns hold zero weights.
        const float kc = p.kshift ? (float)*p.kshift : 0.f;
        // partials: [128-column block][padded test row][p]
        float *dst = p.part + ((2 * w.j + half) * p.test_rows + gi) * p.p;
        // as many weight columns as the call has, rounded up to 8 (the staged
        // weights beyond p are zero)
        if (pp <= 8)
            predict_half<8>(p, tacc, ch0, gi, w.j * BN, nb_s, aw_s, kc, dst);
        else if (pp <= 16)
            predict_half<16>(p, tacc, ch0, gi, w.j * BN, nb_s, aw_s, kc, dst);
        else if (pp <= 24)
            predict_half<24>(p, tacc, ch0, gi, w.j * BN, nb_s, aw_s, kc, dst);
        else
            predict_half<32>(p, tacc, ch0, gi, w.j * BN, nb_s, aw_s, kc, dst);
    } else if (OP == OP_GRADT || OP == OP_GRADK) {
        // d K-weighted contractions for the hyperparameter gradient
        constexpr bool kterm = (OP == OP_GRADK);
        const int64_t gi = kterm ? w.i * b + w.sm * BM + row : w.i * BM + row;
        const int64_t j0 = kterm ? w.j * b + w.sn * BN : w.j * BN;
        const double val = (p.p <= 8) ? grad_half<8, kterm>(p, w, tacc, ch0, gi, j0, nb_s, aw_s)
                                      : grad_half<GRAD_MAX_P, kterm>(p, w, tacc, ch0, gi, j0, nb_s, aw_s);
        const int ew = (threadIdx.x >> 5) - 2;
        if ((threadIdx.x & 31) == 0) red_s[ew] = val;
        epi_bar();
        if (threadIdx.x == 64) {
            double a0 = 0.0;
            for (int q = 0; q < 8; ++q) a0 += red_s[q];
            p.gpart[w.t] = a0;
        }
    } else if (OP == OP_TRSM) {
        float *orow = p.colbuf + (w.i - p.k - 1) * b * b + (w.sm * BM + row) * b + w.sn * BN;
        float mx = 0.f;
        for (int ch = ch0; ch < ch0 + CH_PER_HALF; ++ch) {
            float v[16];
            tmem_ld16(tacc + ch * 16, v);
            float4 *dst = reinterpret_cast<float4 *>(orow + ch * 16);
#pragma unroll
            for (int e = 0; e < 4; ++e) dst[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
#pragma unroll
            for (int e = 0; e < 16; ++e) mx = fmaxf(mx, fabsf(v[e]));
        }
        // max |L_ik| of the block for the adaptive-precision rule: warp
        // maxima, then the eight warps; one partial per block of the tile
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const int ew = (threadIdx.x >> 5) - 2;
        if ((threadIdx.x & 31) == 0) red_s[ew] = (double)mx;
        epi_bar();
        if (threadIdx.x == 64) {
            double m8 = 0.0;
            for (int q = 0; q < 8; ++q) m8 = fmax(m8, red_s[q]);
            const int64_t per_tile = (b / BM) * (b / BN);
            p.part[(w.i - p.k - 1) * per_tile + w.sm * (b / BN) + w.sn] = (float)m8;
        }
    } else {  // OP_UPDATE
        const int64_t k = p.k;
        const float sc = 1.f / (col_tile(p, w.i - k - 1).scale * col_tile(p, w.j - k - 1).scale);
        const int64_t lr = w.sm * BM + row;
        const bool diag = (w.i == w.j);
        const float *cin32 = nullptr;
        float *out32 = nullptr;
        __half *io16 = nullptr;
        if (diag) {
            out32 = p.Wd + w.i * b * b + lr * b + w.sn * BN;
            cin32 = (k == 0) ? p.Kd + tri_index(w.i, w.i) * b * b + lr * b + w.sn * BN : out32;
        } else {
            io16 = p.W + off_index(w.i, w.j) * b * b + lr * b + w.sn * BN;
            if (k == 0) cin32 = p.Kd + tri_index(w.i, w.j) * b * b + lr * b + w.sn * BN;
        }
#pragma unroll
        for (int cc = 0; cc < CH_PER_HALF; ++cc) {
            const int ch = ch0 + cc;
            float v[16];
            tmem_ld16(tacc + ch * 16, v);
            float cin[16];
            if (cin32) {
                const float4 *src = reinterpret_cast<const float4 *>(cin32 + ch * 16);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float4 t4 = src[e];
                    cin[4 * e] = t4.x; cin[4 * e + 1] = t4.y; cin[4 * e + 2] = t4.z; cin[4 * e + 3] = t4.w;
                }
            } else {
                const uint4 *src = reinterpret_cast<const uint4 *>(io16 + ch * 16);
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    uint4 u = src[e];
                    const __half2 *h2 = reinterpret_cast<const __half2 *>(&u);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        float2 f = __half22float2(h2[q]);
                        cin[8 * e + 2 * q] = f.x;
                        cin[8 * e + 2 * q + 1] = f.y;
                    }
                }
            }
            float out[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                float c0 = cin[e];
                if (k == 0 && diag && lr == w.sn * BN + ch * 16 + e) c0 += p.lambda;
                out[e] = c0 - v[e] * sc;
            }
            if (diag) {
                float4 *dst = reinterpret_cast<float4 *>(out32 + ch * 16);
#pragma unroll
                for (int e = 0; e < 4; ++e) dst[e] = make_float4(out[4 * e], out[4 * e + 1], out[4 * e + 2], out[4 * e + 3]);
            } else {
                uint4 pk[2];
                __half2 *h2 = reinterpret_cast<__half2 *>(pk);
#pragma unroll
                for (int q = 0; q < 8; ++q) h2[q] = __floats2half2_rn(out[2 * q], out[2 * q + 1]);
                uint4 *dst = reinterpret_cast<uint4 *>(io16 + ch * 16);
                dst[0] = pk[0];
                dst[1] = pk[1];
            }
        }
    }
}

// Trailing update, FP16 target: the update of box bx (columns [64 bx,
// 64 bx + 64)) of the block, -scale * accumulator rounded to FP16, written
// 128-byte swizzled into `box` (128 rows of 128 bytes) for a TMA reduce-add
// into the target: thread `row` takes columns [32 hh, 32 hh + 32) of the box.
__device__ __forceinline__ void delta_box(uint32_t tacc, int row, int hh, int bx, uint8_t *box, float nsc) {
#pragma unroll
    for (int cc = 0; cc < 2; ++cc) {
        const int col = hh * 32 + cc * 16, u0 = col >> 3;
        float v[16];
        tmem_ld16(tacc + bx * 64 + col, v);
        uint8_t *rp = box + row * 128;
        uint4 u[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            __half2 *h2 = reinterpret_cast<__half2 *>(&u[e]);
#pragma unroll
            for (int qq = 0; qq < 4; ++qq)
                h2[qq] = __floats2half2_rn(v[8 * e + 2 * qq] * nsc, v[8 * e + 2 * qq + 1] * nsc);
        }
        *reinterpret_cast<uint4 *>(rp + ((u0 ^ (row & 7)) << 4)) = u[0];
        *reinterpret_cast<uint4 *>(rp + (((u0 + 1) ^ (row & 7)) << 4)) = u[1];
    }
}

// Named barrier 1 of the 256 epilogue threads with the OR of `fail` over
// them: all threads get the same answer, so they leave their loops together.
__device__ __forceinline__ bool epi_any(bool fail) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, 256, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)fail)
        : "memory");
    return r != 0;
}

// Per-block epilogue inputs staged in shared memory by the epilogue warps.
template <int OP>
__device__ __forceinline__ void epilogue_stage(const TcParams &p, const Work &w, int row,
                                               int32_t *nb_s, float *aw_s) {
    if (OP == OP_DIST) {
        const int64_t j0 = w.j * p.b + w.sn * BN;
        for (int c = row; c < BN; c += EPI_THREADS) nb_s[c] = p.norms_b[j0 + c];
        if (p.nconf) {  // confounders of the block's columns: slots [16, 32) of each staged row
            for (int e = row; e < BN * CONF_MAX; e += EPI_THREADS) {
                const int c = e / CONF_MAX, q = e % CONF_MAX;
                aw_s[c * PRED_MAX_P + 16 + q] = p.conf_b[(j0 + c) * CONF_MAX + q];
            }
        }
    } else if (OP == OP_GRADK) {
        // columns j of the block: norms, A_j in slots [0, 16), Z_j in [16, 32)
        const int64_t j0 = w.j * p.b + w.sn * BN;
        for (int c = row; c < BN; c += EPI_THREADS) nb_s[c] = p.norms_b[j0 + c];
        for (int e = row; e < BN * PRED_MAX_P; e += EPI_THREADS) {
            const int c = e / PRED_MAX_P, q = e % PRED_MAX_P;
            float v = 0.f;
            if (q < GRAD_MAX_P) {
                if (q < p.p) v = p.aw[(j0 + c) * p.ldaw + q];
            } else if (q - GRAD_MAX_P < p.p) {
                v = p.zw[(j0 + c) * p.ldaw + (q - GRAD_MAX_P)];
            }
            aw_s[e] = v;
        }
    } else if (OP == OP_PREDICT || OP == OP_GRADT) {
        for (int c = row; c < BN; c += EPI_THREADS) nb_s[c] = p.norms_b[w.j * BN + c];
        // weights of the block's 256 rows: thread `row` takes element q = row %
        // 32 of rows row / 32 + 8 k; all 32 loads are in flight before the
        // (bank-conflict-free) stores
        constexpr int PER = BN * PRED_MAX_P / EPI_THREADS;
        const int q = row % PRED_MAX_P;
        float v[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int c = row / PRED_MAX_P + k * (EPI_THREADS / PRED_MAX_P);
            v[k] = (q < p.p) ? __ldg(p.aw + (w.j * BN + c) * p.ldaw + q) : 0.f;
            // with confounders (p <= 16) slots [16, 32) hold the training row's confounders
            if (OP == OP_PREDICT && p.nconf && q >= 16) v[k] = __ldg(p.conf_b + (w.j * BN + c) * CONF_MAX + (q - 16));
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) aw_s[row + k * EPI_THREADS] = v[k];
    }
}

// PAIR = 2: clusters of two CTAs, one cta_group::2 MMA per 256 x 256 region
// (rank 0 issues it).  Each CTA loads its own 128 A rows and B rows
// [rank * 128, +128) into its own ring; both loads complete on rank 0's
// `full` barrier, rank 0's commits free the stage in both CTAs and mark the
// accumulator full in both, and both CTAs' epilogues release the accumulator
// on rank 0's `tempty` barrier.
template <int KIND, int OP, int PAIR>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    tc_kernel(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
              const __grid_constant__ CUtensorMap mB0, const __grid_constant__ CUtensorMap mB1,
              const __grid_constant__ CUtensorMap mX, const TcParams p) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    constexpr int NST = PairCfg<PAIR>::stages, SBYTES = PairCfg<PAIR>::stage_bytes;
    uint8_t *stage_base = smem;
    uint8_t *cbuf = smem + NST * SBYTES;  // pair mode: staged target block
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + NST * SBYTES + PairCfg<PAIR>::cbuf_bytes);
    uint64_t *full = bars, *empty = bars + NST, *tfull = bars + 2 * NST,
             *tempty = bars + 2 * NST + 2, *drain = bars + 2 * NST + 4, *cfull = bars + 2 * NST + 5;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * NST + 7);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    double *red_s = reinterpret_cast<double *>(tmem_slot + 2);
    int32_t *nb_s = reinterpret_cast<int32_t *>(red_s + 16);
    float *aw_s = reinterpret_cast<float *>(nb_s + BN);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = (PAIR == 2) ? cluster_rank() : 0u;
    // work units: blocks (PAIR = 1) or pairs of blocks (PAIR = 2)
    const int64_t nunits = p.items / PAIR;
    const int64_t ustart = blockIdx.x / PAIR, ustep = gridDim.x / PAIR;
    auto unit_item = [&](int64_t u) -> int64_t { return p.item0 + ((PAIR == 2) ? pair_item(p, u, rank) : u); };
    if (threadIdx.x == 0) {
        for (int s = 0; s < NST; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(&tfull[a], 1);
            mbar_init(&tempty[a], PAIR * (EPI_THREADS / 32));  // one arrival per epilogue warp
        }
        mbar_init(drain, 1);
        mbar_init(&cfull[0], 1);
        mbar_init(&cfull[1], 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        if (PAIR == 2) {  // both CTAs of the pair allocate together
            asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
        } else {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(tmem_slot)),
                         "r"(TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
    }
    if (warp == 0 && lane == 0) {
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mA0)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mA1)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mB0)) : "memory");
        asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mB1)) : "memory");
        if (OP == OP_UPDATE)
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mX)) : "memory");
    }
    tmem_fence_before();
    __syncthreads();
    if (PAIR == 2) cluster_sync();  // both CTAs' barriers and TMEM are ready before any pair traffic
    tmem_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    const uint64_t budget = p.wait_ns;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- TMA producer ----------------
            const CUtensorMap *maps[5] = {&mA0, &mA1, &mB0, &mB1, &mX};
            int s = 0;
            uint32_t ph = 0;
            int issued = 0;
            uint64_t last_issue = 0;
            bool ok = true;
            for (int64_t u = ustart; u < nunits && ok; u += ustep) {
                Work w;
                decode<OP>(p, unit_item(u), w);
                for (int q = 0; q < w.nph && ok; ++q) {
                    for (int kb = 0; kb < w.nkb; ++kb) {
                        if (!wait_bar(&empty[s], ph ^ 1, budget, abort_flag, p.err)) { ok = false; break; }
                        uint8_t *sa = stage_base + s * SBYTES;
                        uint8_t *sb = sa + A_BYTES;
                        const int x = (KIND == KIND_F16 && !w.kind8) ? kb * (SLAB / 2) : kb * SLAB;
                        if (PAIR == 2) {
                            // rank 0 expects both CTAs' bytes; B rows [rank * 128, +128)
                            const uint32_t fbar = map_to_rank(&full[s], 0);
                            if (rank == 0) mbar_arrive_expect_tx(&full[s], 2 * SBYTES);
                            tma_load_2d_pair(sa, maps[w.amap[q]], x, w.arow[q], fbar);
                            tma_load_2d_pair(sb, maps[w.bmap[q]], x, w.brow[q] + (int)rank * BM, fbar);
                        } else {
                            mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                            tma_load_2d(sa, maps[w.amap[q]], x, w.arow[q], &full[s]);
                            tma_load_2d(sb, maps[w.bmap[q]], x, w.brow[q], &full[s]);
                            tma_load_2d(sb + A_BYTES, maps[w.bmap[q]], x, w.brow[q] + BM, &full[s]);
                        }
                        ++issued;
                        last_issue = globaltimer();
                        if (++s == NST) { s = 0; ph ^= 1; }
                    }
                }
            }
            if (!ok && (PAIR == 1 || rank == 0)) {
                // drain: wait (bounded) for the last loads issued to land
                // (in pair mode they complete on rank 0's barriers)
                int n = issued < NST ? issued : NST;
                int ss = s;
                uint32_t pp = ph;
                for (int e = 0; e < n; ++e) {
                    if (--ss < 0) { ss = NST - 1; pp ^= 1; }
                    const uint64_t t0 = globaltimer();
                    while (!mbar_try_wait(&full[ss], pp) && globaltimer() - t0 < drain_limit(budget)) {}
                }
            } else if (PAIR == 2 && issued > 0 && (!ok || atomicAdd(&p.err->code, 0) != 0)) {
                // pair mode, rank 1, after a wait ran out anywhere: its loads
                // complete on rank 0's barriers, which it cannot poll, and near
                // the abort it may have issued a stage rank 0 no longer waits
                // for.  Such a copy lands within microseconds: give it a grace
                // period far beyond that before the CTA leaves.
                while (globaltimer() - last_issue < DRAIN_GRACE_NS) __nanosleep(1000);
            }
        }
    } else if (warp == 1) {
        if (lane == 0 && (PAIR == 1 || rank == 0)) {
            // ---------------- MMA issuer ----------------
            int s = 0;
            uint32_t ph = 0;
            int acc = 0;
            uint32_t aph = 0;
            bool ok = true;
            bool any = false;
            for (int64_t u = ustart; u < nunits && ok; u += ustep) {
                Work w;
                decode<OP>(p, unit_item(u), w);
                const int total = w.nph * w.nkb;
                if (total == 0) continue;
                if (!wait_bar(&tempty[acc], aph ^ 1, budget, abort_flag, p.err)) { ok = false; break; }
                tmem_fence_after();
                const uint32_t tacc = tmem_base + (uint32_t)(acc * BN);
                for (int it = 0; it < total; ++it) {
                    if (!wait_bar(&full[s], ph, budget, abort_flag, p.err)) { ok = false; break; }
                    tmem_fence_after();
                    const uint32_t sa = smem_u32(stage_base + s * SBYTES);
                    const uint32_t sb = sa + A_BYTES;
                    if (PAIR == 2 && w.kind8) {
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_pair_f8(tacc, smem_desc_sw128(sa + kk * 32), smem_desc_sw128(sb + kk * 32),
                                        (it > 0 || kk > 0) ? 1u : 0u);
                    } else {
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma<KIND, PAIR>(tacc, smem_desc_sw128(sa + kk * 32), smem_desc_sw128(sb + kk * 32),
                                            (it > 0 || kk > 0) ? 1u : 0u);
                    }
                    any = true;
                    if (PAIR == 2) mma_commit_pair(&empty[s]);  // frees the stage in both CTAs
                    else mma_commit(&empty[s]);
                    if (++s == NST) { s = 0; ph ^= 1; }
                }
                if (!ok) break;
                if (PAIR == 2) mma_commit_pair(&tfull[acc]);
                else mma_commit(&tfull[acc]);
                if (++acc == 2) { acc = 0; aph ^= 1; }
            }
            if (!ok && any) {
                if (PAIR == 2) mma_commit_pair(drain);
                else mma_commit(drain);
                const uint64_t t0 = globaltimer();
                while (!mbar_try_wait(drain, 0) && globaltimer() - t0 < drain_limit(budget)) {}
            }
        }
    } else {
        // ---------------- epilogue warps ----------------
        const int row = ((warp & 3) << 5) + lane;  // TMEM lane quarter of this warp
        const int half = (warp - 2) >> 2;          // column half of the block
        const int hh = (warp - 2) >> 2;            // 32-column half of a target box
        int acc = 0;
        uint32_t aph = 0;
        for (int64_t u = ustart; u < nunits; u += ustep) {
            Work w;
            decode<OP>(p, unit_item(u), w);
            if (w.nph * w.nkb == 0) continue;
            // pair mode, FP16 target: the update goes back box by box as a TMA
            // reduce-add of its FP16 value (the L2 adds it to the target; the
            // target is never loaded into the SM); the target boxes are
            // prefetched into L2 while the MMAs run
            const bool cstage = (PAIR == 2 && OP == OP_UPDATE) && p.k > 0 && w.i != w.j;
            const int ybox = (int)(off_index(w.i, w.j) * p.b + w.sm * BM);
            if (cstage && threadIdx.x == 64)
                for (int bx = 0; bx < BN / 64; ++bx) tma_prefetch_2d(&mB1, (int)(w.sn * BN + bx * 64), ybox);
            epi_bar();
            epilogue_stage<OP>(p, w, threadIdx.x - 64, nb_s, aw_s);
            if (!cstage) epilogue_prefetch<OP>(p, w, row, half);
            epi_bar();
            // a collective decision: a wait that ran out in any thread ends the
            // loop in all of them
            const bool got = wait_bar(&tfull[acc], aph, budget, abort_flag, p.err);
            if (epi_any(!got)) break;
            tmem_fence_after();
            const uint32_t tacc = tmem_base + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(acc * BN);
            if (cstage) {
                const float nsc = -1.f / (col_tile(p, w.i - p.k - 1).scale * col_tile(p, w.j - p.k - 1).scale);
                for (int bx = 0; bx < BN / 64; ++bx) {
                    const int bi = bx & 1;
                    // buffer bi is free once the reduce that last used it has
                    // read it: at box 0 every earlier group (the previous
                    // block's boxes), later all but the newest (box bx - 1)
                    if (threadIdx.x == 64) {
                        if (bx == 0) bulk_wait_read();
                        else if (bx >= 2) bulk_wait_read1();
                    }
                    epi_bar();
                    delta_box(tacc, row, hh, bx, cbuf + bi * BOX_BYTES, nsc);
                    // generic-proxy writes become visible to the TMA reduce
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    epi_bar();
                    if (threadIdx.x == 64) {
                        tma_reduce_add_2d(&mB1, (int)(w.sn * BN + bx * 64), ybox, cbuf + bi * BOX_BYTES);
                        bulk_commit();
                    }
                }
            } else {
                epilogue<OP>(p, w, tacc, row, half, nb_s, aw_s, red_s);
            }
            tmem_fence_before();
            __syncwarp();
            if (lane == 0) {
                if (PAIR == 2) mbar_arrive_cluster(map_to_rank(&tempty[acc], 0));
                else mbar_arrive(&tempty[acc]);
            }
            if (++acc == 2) { acc = 0; aph ^= 1; }
        }
        if (PAIR == 2 && threadIdx.x == 64) bulk_wait_all();  // reduces finished before the CTA leaves
    }
    tmem_fence_before();
    __syncthreads();
    // no CTA leaves while its peer may still multicast into it or arrive on
    // its barriers
    if (PAIR == 2) cluster_sync();
    tmem_fence_after();
    if (warp == 1) {
        __syncwarp();
        if (PAIR == 2)
            asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                         : "memory");
        else
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                         : "memory");
    }
}

// Shared memory: ring + barriers/slots + norms + predict weights + alignment slack.
constexpr size_t SMEM_BYTES = (size_t)STAGES * STAGE_BYTES + 256 + BN * 4 + BN * PRED_MAX_P * 4 + 1024;
// Pair mode (trailing update only) needs no norms, weights or staged
// descriptors: ring, target block, barriers and slots.
template <int PAIR>
constexpr size_t smem_bytes_of() {
    return (PAIR == 2) ? (size_t)PairCfg<PAIR>::stages * PairCfg<PAIR>::stage_bytes + PairCfg<PAIR>::cbuf_bytes + 256 + 1024
                       : (size_t)PairCfg<PAIR>::stages * PairCfg<PAIR>::stage_bytes + PairCfg<PAIR>::cbuf_bytes + 256 +
                             BN * 4 + BN * PRED_MAX_P * 4 + 1024;
}
static_assert(smem_bytes_of<2>() <= 227 * 1024, "pair-mode shared memory");

__global__ void split_col0_kernel(const float *Kd, int64_t nt, int64_t b, __half *hi, __half *lo) {
    const int64_t tile = 1 + blockIdx.y;  // tile row i >= 1 of column 0
    const float *src = Kd + tri_index(tile, 0) * b * b;
    __half *h = hi + (tile - 1) * b * b;
    __half *l = lo + (tile - 1) * b * b;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < b * b;
         e += (int64_t)gridDim.x * blockDim.x) {
        const float v = src[e];
        const __half x = __float2half_rn(v);
        h[e] = x;
        l[e] = __float2half_rn(v - __half2float(x));
    }
}

// ---------------------------------------------------------------------------
// Host side: tensor maps and launches.
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

struct TcState {
    EncodeTiledFn encode = nullptr;
    CUtensorMap g_map;                     // packed training genotypes
    CUtensorMap w_map, hi_map, lo_map;     // trailing tiles, column panels
    CUtensorMap pool_map;                  // factor pool viewed as FP16 rows of b
    CUtensorMap pool8_map;                 // factor pool viewed as E4M3 rows of b bytes
    CUtensorMap linv_hi_map, linv_lo_map;  // diagonal inverse splits
    bool factor_maps = false;
};

krr_status make_map(Ctx *c, CUtensorMap *map, const void *base, CUtensorMapDataType dt,
                    int elem_bytes, int64_t rows, int64_t cols) {
    TcState *st = (TcState *)c->tc;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)(cols * elem_bytes)};
    const cuuint32_t box[2] = {(cuuint32_t)(SLAB / elem_bytes), (cuuint32_t)BM};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = st->encode(map, dt, 2, const_cast<void *>(base), dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        c->last_error = "cuTensorMapEncodeTiled failed with code " + std::to_string((int)r);
        return KRR_ECUDA;
    }
    return KRR_OK;
}

// cta_cap > 0 bounds the CTAs of this launch below the class limit.
template <int KIND, int OP, int PAIR = 1>
krr_status launch(Ctx *c, const CUtensorMap &a0, const CUtensorMap &a1, const CUtensorMap &b0,
                  const CUtensorMap &b1, TcParams &p, const CUtensorMap *x = nullptr, int64_t cta_cap = 0) {
    const CUtensorMap &mx = x ? *x : a0;  // fifth map: only the trailing update reads one
    if (p.items <= 0) return KRR_OK;
    static PerDevice attr, clusters_of;  // per device: smem opt-in done; clusters that fit at once
    if (!attr.has(c->device)) {
        cudaError_t e = cudaFuncSetAttribute(tc_kernel<KIND, OP, PAIR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_bytes_of<PAIR>());
        if (e != cudaSuccess) {
            c->last_error = std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e);
            return KRR_ECUDA;
        }
        attr.put(c->device);
    }
    p.wait_ns = (uint64_t)c->opt.wait_budget_ns;
    p.err = c->derr;
    if (PAIR == 1) {
        const int64_t gl = grid_limit(c, GL_SINGLE);
        const int64_t grid = p.items < gl ? p.items : gl;
        count_launch(), tc_kernel<KIND, OP, 1><<<(unsigned)grid, NUM_THREADS, SMEM_BYTES, c->stream>>>(a0, a1, b0, b1, mx, p);
    } else {
        cudaLaunchConfig_t cfg;
        memset(&cfg, 0, sizeof(cfg));
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = PAIR;
        at[0].val.clusterDim.y = 1;
        at[0].val.clusterDim.z = 1;
        cfg.blockDim = dim3(NUM_THREADS);
        cfg.dynamicSmemBytes = smem_bytes_of<PAIR>();
        cfg.stream = c->stream;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int max_clusters = clusters_of.has(c->device) ? clusters_of.get(c->device) : 0;
        if (max_clusters == 0) {
            // clusters that fit at once (SMs of a cluster share a GPC); the
            // kernel is persistent, so the grid never exceeds them
            cfg.gridDim = dim3((unsigned)(c->num_sms / PAIR * PAIR));
            int n = 0;
            if (cudaOccupancyMaxActiveClusters(&n, tc_kernel<KIND, OP, PAIR>, &cfg) != cudaSuccess || n < 1) {
                cudaGetLastError();
                n = 1;
            }
            max_clusters = n;
            clusters_of.put(c->device, n);
        }
        const int64_t units = p.items / PAIR;
        int64_t gl = grid_limit(c, GL_PAIR);
        if (cta_cap > 0 && cta_cap < gl) gl = cta_cap;
        const int64_t cap = std::min<int64_t>(max_clusters, std::max<int64_t>(gl / PAIR, 1));
        const int64_t clusters = units < cap ? units : cap;
        cfg.gridDim = dim3((unsigned)(clusters * PAIR));
        count_launch();
        cudaError_t e = cudaLaunchKernelEx(&cfg, tc_kernel<KIND, OP, PAIR>, a0, a1, b0, b1, mx, p);
        if (e != cudaSuccess) {
            cudaGetLastError();
            c->last_error = std::string("tensor-core cluster launch: ") + cudaGetErrorString(e);
            return KRR_ECUDA;
        }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->last_error = std::string("tensor-core launch: ") + cudaGetErrorString(e);
        return KRR_ECUDA;
    }
    return KRR_OK;
}

TcParams base_params(Ctx *c) {
    TcParams p;
    memset(&p, 0, sizeof(p));
    p.n = c->n;
    p.b = c->b;
    p.lb = 0;
    while ((int64_t)1 << p.lb < c->b) ++p.lb;
    p.nt = c->nt;
    p.m_pad = c->m_pad;
    p.gamma = (float)c->gamma;
    p.lambda = (float)c->lambda;
    p.kf = kernel_fn(c);
    return p;
}

krr_status ensure_factor_maps(Ctx *c) {
    TcState *st = (TcState *)c->tc;
    if (st->factor_maps) return KRR_OK;
    const int64_t b = c->b, nt = c->nt, noff = nt * (nt - 1) / 2;
    const CUtensorMapDataType f16 = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    KRR_TRY(make_map(c, &st->w_map, c->W, f16, 2, noff * b, b));
    KRR_TRY(make_map(c, &st->hi_map, c->pan_hi, f16, 2, (nt - 1) * b, b));
    KRR_TRY(make_map(c, &st->lo_map, c->pan_lo, f16, 2, (nt - 1) * b, b));
    KRR_TRY(make_map(c, &st->pool_map, c->pool, f16, 2, (int64_t)(c->pool_bytes / (2 * b)), b));
    KRR_TRY(make_map(c, &st->pool8_map, c->pool, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, (int64_t)(c->pool_bytes / b), b));
    KRR_TRY(make_map(c, &st->linv_hi_map, c->Linv_hi, f16, 2, nt * b, b));
    KRR_TRY(make_map(c, &st->linv_lo_map, c->Linv_lo, f16, 2, nt * b, b));
    st->factor_maps = true;
    return KRR_OK;
}

}  // namespace

krr_status tc_init(Ctx *c) {
    TcState *st = new (std::nothrow) TcState();
    if (!st) {
        c->last_error = "out of host memory";
        return KRR_ENOMEM;
    }
    c->tc = st;
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                     cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        cudaGetLastError();
        c->last_error = "cuTensorMapEncodeTiled is not available from the driver";
        return KRR_ECUDA;
    }
    st->encode = (EncodeTiledFn)fn;
    return KRR_OK;
}

void tc_free(Ctx *c) {
    delete (TcState *)c->tc;
    c->tc = nullptr;
}

void tc_invalidate_factor_maps(Ctx *c) {
    if (c->tc) ((TcState *)c->tc)->factor_maps = false;
}

krr_status tc_bind_genotypes(Ctx *c) {
    TcState *st = (TcState *)c->tc;
    return make_map(c, &st->g_map, c->g8, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, c->n_pad, c->m_pad);
}

krr_status tc_build(Ctx *c) {
    TcState *st = (TcState *)c->tc;
    KRR_TRY(tc_bind_genotypes(c));
    TcParams p = base_params(c);
    p.norms_a = c->norms;
    p.norms_b = c->norms;
    p.Kd = c->Kd;
    p.Dd = c->Dd;
    p.knorm_part = c->knorm2;
    p.conf_a = p.conf_b = c->conf;
    p.nconf = (int)c->nconf;
    p.n = real_rows(c);
    const int64_t ntri = c->nt * (c->nt + 1) / 2;
    p.items = ntri * (c->b / BM) * (c->b / BN);
    return launch<KIND_F8, OP_DIST>(c, st->g_map, st->g_map, st->g_map, st->g_map, p);
}

krr_status tc_trsm(Ctx *c, int64_t k) {
    TcState *st = (TcState *)c->tc;
    KRR_TRY(ensure_factor_maps(c));
    const int64_t b = c->b, nt = c->nt;
    if (k == 0) {
        count_launch(), split_col0_kernel<<<dim3(64, (unsigned)(nt - 1)), 256, 0, c->stream>>>(c->Kd, nt, b, c->pan_hi,
                                                                               c->pan_lo);
    }
    TcParams p = base_params(c);
    p.k = k;
    p.colbuf = c->colbuf;
    p.part = c->colmax;  // per-block max |L_ik|, read by the column cast
    p.items = (nt - k - 1) * (b / BM) * (b / BN);
    const CUtensorMap &a0 = (k == 0) ? st->hi_map : st->w_map;
    // CTA pairs (M = 256) share the B operand (the diagonal inverse), as in the update
    return launch<KIND_F16, OP_TRSM, 2>(c, a0, st->lo_map, st->linv_hi_map, st->linv_lo_map, p);
}

double update_flops(const Ctx *c, int64_t k, int64_t tile0, int64_t tiles) {
    // diagonal target (r0 + a, r0 + a) of the band starting at tile row r0
    // sits after the band's h * r0 tiles left of its diagonal block, at
    // triangle index a (a + 1) / 2 + a (the order of update_tile_order)
    const int64_t u = c->nt - k - 1;
    int64_t ndiag = 0;
    for (int64_t d = 0; d < u; ++d) {
        const int64_t r0 = d / UPD_BAND * UPD_BAND, a = d - r0;
        const int64_t h = (u - r0 < UPD_BAND) ? u - r0 : UPD_BAND;
        const int64_t pos = r0 * (r0 + 1) / 2 + h * r0 + a * (a + 1) / 2 + a;
        if (pos >= tile0 && pos < tile0 + tiles) ++ndiag;
    }
    const double b3 = (double)c->b * (double)c->b * (double)c->b;
    return (double)(tiles - ndiag) * 2.0 * b3 + (double)ndiag * b3;
}

krr_status tc_update(Ctx *c, int64_t k, int64_t tile0, int64_t tiles, int64_t cta_cap) {
    TcState *st = (TcState *)c->tc;
    KRR_TRY(ensure_factor_maps(c));
    const int64_t b = c->b, nt = c->nt;
    const int64_t u = nt - k - 1;
    const int64_t total = u * (u + 1) / 2;  // target tiles of the step
    if (tiles < 0) tiles = total - tile0;
    if (tile0 < 0 || tile0 + tiles > total) {
        c->last_error = "trailing update: target tile range out of bounds";
        return KRR_EINVAL;
    }
    TcParams p = base_params(c);
    p.k = k;
    p.Kd = c->Kd;
    p.W = (__half *)c->W;
    p.Wd = c->Wd;
    p.ltab = c->ltab;
    const int64_t per_tile = (b / BM) * (b / BN);
    p.item0 = tile0 * per_tile;
    p.items = tiles * per_tile;
    // mB1 = the FP16 trailing tiles: staged target blocks (TMA load and store);
    // the fifth map reads E4M3 tiles for kind::f8f6f4 blocks
    return launch<KIND_F16, OP_UPDATE, 2>(c, st->pool_map, st->hi_map, st->lo_map, st->w_map, p, &st->pool8_map,
                                          cta_cap);
}

// B = K_test^T G_p: the predict kernel with the roles of the two genotype
// sets swapped (A = training rows, B = test rows padded to 256).  part is
// (2 * test_rows256 / 256) x n_pad x p.
krr_status tc_predict_t(Ctx *c, const uint8_t *t8, const int32_t *tn, int64_t n_test,
                        int64_t test_rows256, const float *gp, int64_t ldgp, int64_t p_cols, float *part) {
    TcState *st = (TcState *)c->tc;
    if (p_cols < 1 || p_cols > PRED_MAX_P || test_rows256 % BN != 0) {
        c->last_error = "tc_predict_t: bad shape";
        return KRR_EINVAL;
    }
    CUtensorMap t_map;
    KRR_TRY(make_map(c, &t_map, t8, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, test_rows256, c->m_pad));
    TcParams p = base_params(c);
    p.n = n_test;           // real rows of the B operand (test)
    p.n_pad = test_rows256;  // padded rows of the B operand
    p.n_test = c->n;        // real rows of the A operand (training)
    p.test_rows = c->n_pad;  // padded rows of the A operand (partial stride)
    p.norms_a = c->norms;
    p.norms_b = tn;
    p.aw = gp;
    p.ldaw = ldgp;
    p.p = p_cols;
    p.part = part;
    p.items = (c->n_pad / BM) * (test_rows256 / BN);
    return launch<KIND_F8, OP_PREDICT>(c, st->g_map, st->g_map, t_map, t_map, p);
}

// The two d K-weighted contractions of the hyperparameter gradient: one
// partial per block into part_t (test x training blocks) and part_k
// (lower-triangle training blocks).  aw = A (n_pad x ld), zw = Z, gp = G_p
// (test_rows x ld), p_cols <= 16.
krr_status tc_grad_terms(Ctx *c, const uint8_t *t8, const int32_t *tn, int64_t n_test,
                         int64_t test_rows, const float *aw, const float *zw, const float *gp,
                         int64_t ld, int64_t p_cols, double *part_t, double *part_k,
                         int64_t *items_t, int64_t *items_k) {
    TcState *st = (TcState *)c->tc;
    if (p_cols < 1 || p_cols > GRAD_MAX_P) {
        c->last_error = "tc_grad_terms: at most 16 columns per launch";
        return KRR_EINVAL;
    }
    CUtensorMap t_map;
    KRR_TRY(make_map(c, &t_map, t8, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, test_rows, c->m_pad));
    TcParams p = base_params(c);
    p.n_pad = c->n_pad;
    p.n_test = n_test;
    p.test_rows = test_rows;
    p.norms_a = tn;
    p.norms_b = c->norms;
    p.aw = aw;
    p.zw = zw;
    p.gp = gp;
    p.ldaw = ld;
    p.p = p_cols;
    p.gpart = part_t;
    p.items = (test_rows / BM) * (c->n_pad / BN);
    *items_t = p.items;
    KRR_TRY((launch<KIND_F8, OP_GRADT>(c, t_map, t_map, st->g_map, st->g_map, p)));
    TcParams q = base_params(c);
    q.norms_a = c->norms;
    q.norms_b = c->norms;
    q.aw = aw;
    q.zw = zw;
    q.ldaw = ld;
    q.p = p_cols;
    q.gpart = part_k;
    q.items = c->nt * (c->nt + 1) / 2 * (c->b / BM) * (c->b / BN);
    *items_k = q.items;
    return launch<KIND_F8, OP_GRADK>(c, st->g_map, st->g_map, st->g_map, st->g_map, q);
}

krr_status tc_predict(Ctx *c, const uint8_t *t8, const int32_t *tn, int64_t n_test,
                      int64_t rows_pad, const float *A, int64_t lda, int64_t p_cols, float *part,
                      const double *kshift, const float *tconf) {
    TcState *st = (TcState *)c->tc;
    if (p_cols < 1 || p_cols > (c->nconf ? 16 : PRED_MAX_P) || (c->nconf && !tconf)) {
        c->last_error = "tc_predict: at most 32 weight columns per launch (16 with confounders)";
        return KRR_EINVAL;
    }
    CUtensorMap t_map;
    KRR_TRY(make_map(c, &t_map, t8, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, rows_pad, c->m_pad));
    TcParams p = base_params(c);
    p.n_pad = c->n_pad;
    p.n_test = n_test;
    p.test_rows = rows_pad;
    p.norms_a = tn;
    p.norms_b = c->norms;
    p.aw = A;
    p.ldaw = lda;
    p.p = p_cols;
    p.part = part;
    p.kshift = kshift;
    p.conf_a = tconf;
    p.conf_b = c->conf;
    p.nconf = (int)c->nconf;
    p.items = (rows_pad / BM) * (c->n_pad / BN);
    return launch<KIND_F8, OP_PREDICT>(c, t_map, t_map, st->g_map, st->g_map, p);
}

}  // namespace krr
