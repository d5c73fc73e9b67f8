// Predict (Alg. 4) for callers that cannot allocate device memory.
//
// krr_predict() sizes its own working buffers with cudaMalloc on first use.
// Some callers cannot allow that: host processes whose device memory is
// reserved up front by another allocator (a pool or arena that must see
// every byte), or real-time callers that must not hit the driver's
// allocator on the hot path (cudaMalloc and cudaFree can block and
// synchronise the device).  This file gives
// them krr_predict_noalloc(), the same computation on the same kernels, with
// every working buffer carved out of one file-scope device array of fixed
// size instead of context-owned allocations.
//
// The array (about 16.8 MB) exists on every GPU
// that loads the library, from module load until process exit.  Host code
// cannot use the array's name as a device address: its device address is
// looked up with cudaGetSymbolAddress once per device, with that device
// current, on the first call made on that device.
#include <cuda_runtime.h>

#include <mutex>

#include "krr_internal.h"

namespace {

// Limits of one call (checked; larger requests get KRR_EINVAL).
constexpr int64_t NA_MAX_TEST = 256;        // held-out rows per call
constexpr int64_t NA_MAX_P = 8;             // weight columns per call
constexpr int64_t NA_MAX_NPAD = 131072;     // padded training rows
constexpr int64_t NA_MAX_MPAD = 16384;      // padded SNPs

constexpr size_t align256(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t NA_T8 = 0;                                                     // packed test rows
constexpr size_t NA_TN = NA_T8 + align256(NA_MAX_TEST * NA_MAX_MPAD);           // test norms
constexpr size_t NA_AW = NA_TN + align256(NA_MAX_TEST * 4);                     // padded weights
constexpr size_t NA_PART = NA_AW + align256(NA_MAX_NPAD * NA_MAX_P * 4);        // partial products
constexpr size_t NA_OUT = NA_PART + align256((NA_MAX_NPAD / 128) * NA_MAX_TEST * NA_MAX_P * 4);
constexpr size_t NA_CSUM = NA_OUT + align256(NA_MAX_TEST * NA_MAX_P * 4);   // FP64 column sums of the weights
constexpr size_t NA_BYTES = NA_CSUM + align256(NA_MAX_P * 8);

static __device__ __align__(256) uint8_t g_noalloc_scratch[NA_BYTES];

std::mutex g_mu;
void *g_addr[64] = {nullptr};  // device address of the array, per device ordinal

krr_status scratch_address(krr::Ctx *c, uint8_t **out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (c->device < 0 || c->device >= 64) {
        c->last_error = "krr_predict_noalloc: device ordinal out of range";
        return KRR_EINVAL;
    }
    if (!g_addr[c->device]) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != c->device) cudaSetDevice(c->device);
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (cur != c->device && cur >= 0) cudaSetDevice(cur);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            c->last_error = std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
            return KRR_ECUDA;
        }
        g_addr[c->device] = p;
    }
    *out = (uint8_t *)g_addr[c->device];
    return KRR_OK;
}

bool on_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" krr_status krr_predict_noalloc(krr_ctx *ctx, const int8_t *T, int64_t n_test,
                                          int64_t ldt, const float *A, int64_t lda, int64_t p,
                                          float *Yt, int64_t ldyt) {
    krr::Ctx *c = reinterpret_cast<krr::Ctx *>(ctx);
    if (!c) return KRR_EINVAL;
    if (!c->built) {
        c->last_error = "krr_predict_noalloc: no kernel built";
        return KRR_ESTATE;
    }
    if (c->opt.mode != KRR_MODE_MIXED || !c->tc || c->opt.kernel != KRR_KERNEL_GAUSSIAN || c->nconf > 0 || c->rr) {
        c->last_error = "krr_predict_noalloc: needs a context in KRR_MODE_MIXED with the Gaussian kernel and no "
                        "confounders";
        return KRR_EINVAL;
    }
    if (!T || !A || !Yt || n_test < 1 || n_test > NA_MAX_TEST || p < 1 || p > NA_MAX_P ||
        ldt < c->m || lda < p || ldyt < p || c->n_pad > NA_MAX_NPAD || c->m_pad > NA_MAX_MPAD) {
        c->last_error = "krr_predict_noalloc: need 1 <= n_test <= 256, 1 <= p <= 8, padded N <= 131072, "
                        "padded M <= 16384 and valid leading dimensions";
        return KRR_EINVAL;
    }
    if (!on_device(T) || !on_device(A) || !on_device(Yt)) {
        c->last_error = "krr_predict_noalloc: T, A and Yt must be device pointers";
        return KRR_EINVAL;
    }
    uint8_t *base = nullptr;
    KRR_TRY(scratch_address(c, &base));
    uint8_t *t8 = base + NA_T8;
    int32_t *tn = reinterpret_cast<int32_t *>(base + NA_TN);
    float *aw = reinterpret_cast<float *>(base + NA_AW);
    float *part = reinterpret_cast<float *>(base + NA_PART);
    float *out = reinterpret_cast<float *>(base + NA_OUT);
    double *csum = reinterpret_cast<double *>(base + NA_CSUM);
    const double *shift = c->red + krr::RED_KSHIFT;
    const int64_t rows_pad = (n_test + 127) / 128 * 128;
    // Every scratch element read below is written first in this call (the
    // packing and the weight copy zero their padding; the partials and the
    // output are written in full), so nothing needs clearing.
    krr::launch_pack_genotypes(T, n_test, c->m, ldt, rows_pad, c->m_pad, t8, nullptr, tn, c->stream);
    krr::launch_copy_rows(A, lda, aw, p, c->n, p, c->n_pad, c->stream);
    krr::launch_colsum(aw, c->n_pad, p, csum, c->stream);
    KRR_TRY(krr::tc_predict(c, t8, tn, n_test, rows_pad, aw, p, p, part, shift));
    krr::launch_predict_reduce(part, c->n_pad / 128, rows_pad, n_test, p, out, p, c->stream, shift, csum);
    krr::launch_copy_rows(out, p, Yt, ldyt, n_test, p, n_test, c->stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        c->last_error = std::string("krr_predict_noalloc: ") + cudaGetErrorString(e);
        return KRR_ECUDA;
    }
    return KRR_OK;
}
