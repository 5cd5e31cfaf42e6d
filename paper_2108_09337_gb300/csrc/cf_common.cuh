// cf_common.cuh -- shared definitions of the libcf CUDA sources (sm_103a).
#pragma once

#include <atomic>

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "../../include/cf.h"

namespace cf {

// Largest block size / leaf height / candidates per tree node handled by the
// shared-memory tournament tiles.
constexpr int kMaxV = 128;

// Records the last CUDA error seen by the library (cf_last_cuda_error()).
void set_cuda_error(cudaError_t e);
// Counts enqueued kernel launches (cf_kernel_launches()).
void count_launches(long long n);

#define CF_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t cf_e_ = (expr);                         \
        if (cf_e_ != cudaSuccess) {                         \
            ::cf::set_cuda_error(cf_e_);                    \
            return CF_ERR_CUDA;                             \
        }                                                   \
    } while (0)

#define CF_LAUNCH_CHECK()              \
    do {                               \
        ::cf::count_launches(1);       \
        CF_CUDA_TRY(cudaGetLastError()); \
    } while (0)

// A CUDA event destroyed when it goes out of scope, so that every error
// return of a host routine releases it (destroying an event still pending on
// a stream is allowed: CUDA frees it once it completes).
struct ScopedEvent {
    cudaEvent_t e = nullptr;
    ScopedEvent() = default;
    ScopedEvent(const ScopedEvent &) = delete;
    ScopedEvent &operator=(const ScopedEvent &) = delete;
    ~ScopedEvent() {
        if (e) cudaEventDestroy(e);
    }
    cudaError_t create(unsigned flags = cudaEventDefault) { return cudaEventCreateWithFlags(&e, flags); }
    operator cudaEvent_t() const { return e; }
};

inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

// SM count of the current device (148 if the query fails), queried once per
// device and kept in an atomic slot, so concurrent calls from several host
// threads never race on it.
inline int device_sm_count() {
    constexpr int kDevs = 64;
    static std::atomic<int> cache[kDevs];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return 148;
    }
    int n = (dev >= 0 && dev < kDevs) ? cache[dev].load(std::memory_order_relaxed) : 0;
    if (n > 0) return n;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
        cudaGetLastError();
        n = 148;
    }
    if (dev >= 0 && dev < kDevs) cache[dev].store(n, std::memory_order_relaxed);
    return n;
}
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Carves aligned sub-buffers out of a caller-provided workspace; with a null
// base it only measures.
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *b) : base((char *)b) {}
    template <typename T>
    T *take(size_t count, size_t align = 256) {
        off = align_up(off, align);
        T *p = base ? (T *)(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
    size_t size() const { return align_up(off, 256); }
};

// Options with defaults filled in and ranges checked.
struct Opts {
    int v = 128, leaf_h = 128, arity = 8, outer_V = 0, lookahead = 1;
    double tol = 1e-14;
    int max_iter = 30, gmres_restart = 30;
    int batch_cps = 0;           // batched calls: resident CTAs per SM (0 = as many as fit)
    int fp64_residual = 0;       // mixed solvers: 1 = no pair-arithmetic residuals
    int residual_kind = 0;       // mixed solvers: 0 = tensor-core slices, 2 = pair / FP64
    // whether the caller set v, leaf_h, arity (0 selects the routine's default)
    bool v_set = false, h_set = false, ar_set = false;
};
// Returns 0 or a negative status for an out-of-range field.  Fields left 0
// take the FP64 routines' defaults (v = 128, leaf_h = 128, arity = 8).
int resolve_options(const cf_options *in, Opts *out);
// The mixed LU's defaults for the fields the caller left 0: v = 64 with the
// wide-node tournament (leaves of 512 rows, arity 8); with v > 64 given,
// leaves of 256 rows and arity 2.  Checks outer_V against the final v.
int mixed_lu_defaults(Opts *o);
// Tournament shapes of the FP64 routines: leaves of at most kMaxV rows,
// arity 2..8 (one cluster of `arity` CTAs per playoff node).
inline bool fp64_tourn_shape(const Opts &o) { return o.leaf_h <= kMaxV && o.arity <= 8; }
// Tournament shapes of the mixed-precision LU (FP32 panels): v <= 64 with
// leaves of up to 512 rows and arity up to 8 (arity * v <= 512), or
// v <= 128 with leaves of up to 256 rows and arity 2.
bool tourn32_shape_ok(int v, int h, int arity);

// Exactly rounded product and difference (no FMA contraction), so that the
// tournament, the diagonal-block factorization and the panel solves round
// exactly like the FP64 oracle.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }

}  // namespace cf
