// cf_noalloc.cu -- cf_getrf_noalloc: the FP64 LU of cf_getrf for callers that
// cannot allocate device memory.
//
// cf_getrf needs a small scratch area (the tournament's candidate lists, its
// arrival counters and the list of moved rows) and takes it from the caller
// as `work`.  Some callers have no way to provide it: code that runs while a
// stream is being captured into a CUDA graph (where cudaMalloc is not
// allowed), plugins that live inside a host framework whose allocator owns
// all device memory, or real-time code whose memory is partitioned up front.
// For them this variant keeps the scratch in a fixed array that the library
// itself places in device memory when it is loaded (kNoAllocScratchBytes on
// every GPU that loads the library, held until the process exits).  It runs
// the same kernels, in the same order, as cf_getrf.
#include <mutex>

#include "cf_common.cuh"
#include "cf_kernels.cuh"

namespace cf {

constexpr size_t kNoAllocScratchBytes = (size_t)2 << 20;   // 2 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[kMaxDevices] = {};

// The array's name in host code is only a handle; the device address that a
// kernel may use is looked up once per device, with that device current.
static int noalloc_scratch(void **out) {
    int dev = 0;
    CF_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return CF_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (g_noalloc_addr[dev] == nullptr) {
        void *p = nullptr;
        CF_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return CF_OK;
}

}  // namespace cf

using namespace cf;

extern "C" int cf_getrf_noalloc(int n, double *A, int lda, int *ipiv, int *info, const cf_options *opt,
                                cudaStream_t st) {
    if (n < 0) return -1;
    if (n > 0 && A == nullptr) return -2;
    if (lda < (n > 1 ? n : 1)) return -3;
    if (n > 0 && ipiv == nullptr) return -4;
    if (info == nullptr) return -5;
    Opts o;
    int rc = resolve_options(opt, &o);
    if (rc != CF_OK) return rc;
    if (!fp64_tourn_shape(o)) return CF_ERR_UNSUPPORTED;
    // Size check first: it needs no device and touches no memory.
    if (n > 0 && tourn_ws_bytes(n, o.leaf_h, o.arity) > kNoAllocScratchBytes) return CF_ERR_WORKSPACE;
    void *scratch = nullptr;
    if ((rc = noalloc_scratch(&scratch))) return rc;
    CF_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int), st));
    if (n == 0) return CF_OK;
    TournWS ws{};
    TournEpilogue ep{};
    if ((rc = tourn_ws_carve(scratch, n, o.leaf_h, o.arity, &ws, &ep))) return rc;
    // The array keeps whatever the previous call left: the arrival counters
    // must start at zero.
    CF_CUDA_TRY(cudaMemsetAsync(ws.counter, 0, ws.counter_bytes, st));
    const size_t ld = (size_t)lda;
    for (int k0 = 0; k0 < n; k0 += o.v) {
        const int w = o.v < n - k0 ? o.v : n - k0;
        const int m = n - k0;
        double *A00 = A + k0 + k0 * ld;
        ep.ipiv = ipiv;
        ep.k0 = k0;
        if ((rc = launch_tourn<double>(A00, lda, m, w, o.leaf_h, o.arity, ws, ep, st))) return rc;
        if ((rc = launch_apply_swaps<double>(A, lda, n, k0, ep, nullptr, st))) return rc;
        if ((rc = launch_getf2_nopiv<double>(A00, lda, w, k0, info, st))) return rc;
        if ((rc = launch_trsm_right_upper<double>(A00 + w, lda, m - w, w, A00, lda, false, nullptr, st))) return rc;
        if ((rc = launch_trsm_left_lower_unit<double>(A00 + w * ld, lda, w, n - k0 - w, A00, lda, st))) return rc;
        if ((rc = launch_gemm_f64_sub(m - w, n - k0 - w, w, A00 + w, lda, A00 + w * ld, lda, false,
                                      A00 + w + w * ld, lda, false, nullptr, st)))
            return rc;
    }
    return CF_OK;
}
