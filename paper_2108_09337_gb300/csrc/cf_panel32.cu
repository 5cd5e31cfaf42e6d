// cf_panel32.cu -- FP32 block routines of the mixed-precision path, built for
// latency (they sit on the chain of dependent work of every step):
//
//   k_a00_lu32      LU of A00 without pivoting (S1/S2 of Fig. "prog_rep" on
//                   the rows TournPivot selected; Sec. 7.2)
//   k_a00_chol32    Cholesky of A00 (Listing "Cholesky Factorization"; CH-1)
//   k_rtrsm32       LU-3  A10 <- A10 U00^{-1}  /  CH-2  L10 <- A10 L00^{-T}
//   k_ltrsm32       LU-4  A01 <- L00^{-1} A01
//
// Each thread holds one row (or, for LU-4, one column) of its tile in
// registers and shifts it left while it eliminates, so the current column
// is always element 0; the v x v triangle is read from shared memory as
// float4 rows.  A00 kernels need one barrier per column; the panel solves
// need none.  The solve kernels also write the BF16/FP16 K-major copies
// that the tensor-core update reads.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cf_common.cuh"
#include "cf_kernels.cuh"
#include "cf_regrow.cuh"

namespace cf {

template <typename LP>
__device__ __forceinline__ LP lp_from(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 lp_from<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half lp_from<__half>(float x) { return __float2half_rn(x); }

// ---------------------------------------------------------------------------
// A00 = L00 U00, no pivoting, in place (w <= 128).  Thread r owns row r.  The
// pivot row of step k is published in shared memory (double-buffered).
// ---------------------------------------------------------------------------
struct LuStep {
    float4 (&pr)[2][kMaxV / 4];
    float (&a)[kMaxV];
    float *A00;
    int lda, w, r, kglob;
    int *info;
    template <int U>
    __device__ __forceinline__ void step(int j0) {
        const int k = j0 + U, par = k & 1;
        if (r == k) store_row4(pr[par], a);              // row k, relative to j0
        __syncthreads();
        const float *pf = reinterpret_cast<const float *>(pr[par]);
        if (r < w - k) A00[(size_t)k + (size_t)(k + r) * lda] = pf[U + r];        // U(k, k+r)
        const float piv = pf[U];
        if (r > k && r < w) {
            const float l = (piv != 0.f) ? a[U] / piv : a[U];
            A00[(size_t)r + (size_t)k * lda] = l;                                   // L(r, k)
            rank1_from<U>(a, l, pr[par], w - j0);
        }
        if (r == 0 && piv == 0.f) atomicCAS(info, 0, kglob + k + 1);
    }
};

__global__ void __launch_bounds__(kMaxV, 1) k_a00_lu32(float *A00, int lda, int w, int kglob, int *info) {
    __shared__ __align__(16) float4 pr[2][kMaxV / 4];
    const int r = threadIdx.x;
    float a[kMaxV];
#pragma unroll
    for (int k = 0; k < kMaxV; ++k) a[k] = (r < w && k < w) ? A00[(size_t)r + (size_t)k * lda] : 0.f;
    LuStep body{pr, a, A00, lda, w, r, kglob, info};
    for_blocks(a, w, body);
}

// ---------------------------------------------------------------------------
// A00 = L00 L00^T (lower), in place.  Thread r owns row r; before each
// barrier every live row publishes its current column entry, so after it
// each thread has the whole column k of the Schur complement: one barrier
// per column.  Stops at the first pivot that is not positive (info).
// ---------------------------------------------------------------------------
struct CholStep {
    float4 (&col)[2][kMaxV / 4 + 1];
    float (&a)[kMaxV];
    float *A00;
    int lda, w, r, kglob;
    int *info;
    bool failed;
    template <int U>
    __device__ __forceinline__ void step(int j0) {
        if (failed) return;                          // uniform
        const int k = j0 + U, par = k & 1;
        float *cf = reinterpret_cast<float *>(col[par]);
        if (r >= k && r < w) cf[r - j0] = a[U];      // column k by relative row
        __syncthreads();
        const float d = cf[U];
        if (!(d > 0.f)) {
            if (r == 0) atomicCAS(info, 0, kglob + k + 1);
            failed = true;                           // every thread read the same d
            return;
        }
        const float lkk = sqrtf(d);
        if (r == k) A00[(size_t)k + (size_t)k * lda] = lkk;
        if (r > k && r < w) {
            const float l = a[U] / lkk;
            A00[(size_t)r + (size_t)k * lda] = l;                               // L(r, k)
            // a(r, j0+t) -= L(r,k) L(j0+t,k) = (l / lkk) col[t], for j0+t <= r
            rank1_from<U>(a, l / lkk, col[par], r - j0 + 1);
        }
    }
};

__global__ void __launch_bounds__(kMaxV, 1) k_a00_chol32(float *A00, int lda, int w, int kglob, int *info) {
    if (*info != 0) return;
    __shared__ __align__(16) float4 col[2][kMaxV / 4 + 1];
    const int r = threadIdx.x;
    float a[kMaxV];
#pragma unroll
    for (int k = 0; k < kMaxV; ++k) a[k] = (r < w && k < w) ? A00[(size_t)r + (size_t)k * lda] : 0.f;
    CholStep body{col, a, A00, lda, w, r, kglob, info, false};
    for_blocks(a, w, body);
}

struct RtrsmStep {
    float (&a)[kMaxV];
    const float *Ms;
    float *xs;
    int w;
    template <int U>
    __device__ __forceinline__ void step(int j0) {
        const int k = j0 + U;
        const float d = Ms[k * kMaxV + k];
        const float xk = (d != 0.f) ? a[U] / d : a[U];
        xs[k] = xk;
        rank1_from<U>(a, xk, reinterpret_cast<const float4 *>(Ms + k * kMaxV + j0), w - j0);
    }
};

struct LtrsmStep {
    float (&a)[kMaxV];
    const float *Ls;
    float *xs;
    int w;
    template <int U>
    __device__ __forceinline__ void step(int j0) {
        const int k = j0 + U;
        const float xk = a[U];                       // unit diagonal
        xs[k] = xk;
        rank1_from<U>(a, xk, reinterpret_cast<const float4 *>(Ls + k * kMaxV + j0), w - j0);
    }
};

// ---------------------------------------------------------------------------
// Right solve of a panel: X (rows x w, column-major ldx) <- X M^{-1} with
// M = U00 (upper, non-unit; trans_lower = false) or M = L00^T (trans_lower).
// Thread = row; M staged row by row as Ms[k][t] = M(k, k+t).  Writes FP32
// back and lp[r*ldk + j] (j < kpad; zero for j >= w).
// ---------------------------------------------------------------------------
template <typename LP>
__global__ void __launch_bounds__(kMaxV, 1)
k_rtrsm32(float *X, int ldx, int rows, int w, const float *__restrict__ M00, int ldm, int trans_lower, LP *lp,
          int ldk, int kpad, const int *skip) {
    if (skip != nullptr && *skip != 0) return;
    extern __shared__ __align__(16) float smem[];
    float *Ms = smem;                                // [kMaxV][kMaxV]
    float *Xs = smem + kMaxV * kMaxV;                // [kMaxV][kMaxV + 4] outputs, row-major
    constexpr int XLD = kMaxV + 4;
    const int tid = threadIdx.x;
    // Ms[k][c] = M(k, c) at absolute columns, read along the stored matrix's columns
    for (int e = tid; e < kMaxV * kMaxV; e += kMaxV) {
        const int i = e % kMaxV, c = e / kMaxV;          // stored element (i, c)
        if (i < w && c < w) {
            const float v = M00[(size_t)i + (size_t)c * ldm];
            if (!trans_lower && i <= c) Ms[i * kMaxV + c] = v;          // U(i, c)
            if (trans_lower && i >= c) Ms[c * kMaxV + i] = v;           // M(c, i) = L(i, c)
        }
    }
    const int r0 = blockIdx.x * kMaxV;
    const int nr = min(kMaxV, rows - r0);
    float a[kMaxV];
    // coalesced load: for each column k, the CTA's rows are contiguous
#pragma unroll
    for (int k = 0; k < kMaxV; ++k) a[k] = (tid < nr && k < w) ? X[(size_t)(r0 + tid) + (size_t)k * ldx] : 0.f;
    __syncthreads();
    RtrsmStep body{a, Ms, Xs + tid * XLD, w};
    for_blocks(a, w, body);
    __syncthreads();
    // write back: FP32 column-major (coalesced over rows) ...
    for (int e = tid; e < kMaxV * w; e += kMaxV) {
        const int rr = e % kMaxV, k = e / kMaxV;
        if (rr < nr) X[(size_t)(r0 + rr) + (size_t)k * ldx] = Xs[rr * XLD + k];
    }
    // ... and the K-major low-precision rows (coalesced along k)
    if (lp != nullptr) {
        for (int e = tid; e < kMaxV * kpad; e += kMaxV) {
            const int k = e % kpad, rr = e / kpad;
            if (rr < nr) lp[(size_t)(r0 + rr) * ldk + k] = lp_from<LP>(k < w ? Xs[rr * XLD + k] : 0.f);
        }
    }
}

// ---------------------------------------------------------------------------
// Left solve of a row block: X (w x cols, column-major ldx) <- L00^{-1} X, L00
// unit lower.  Thread = column; L staged column by column as Ls[k][t] =
// L(k+t, k).  Writes FP32 back and lp[c*ldk + i] (i < kpad; zero for i >= w).
// ---------------------------------------------------------------------------
template <typename LP>
__global__ void __launch_bounds__(kMaxV, 1)
k_ltrsm32(float *X, int ldx, int w, int cols, const float *__restrict__ L00, int ldl, LP *lp, int ldk, int kpad) {
    extern __shared__ __align__(16) float smem[];
    float *Ls = smem;                                // [kMaxV][kMaxV]: Ls[k][t] = L(k+t, k)
    float *Xs = smem + kMaxV * kMaxV;                // [kMaxV][kMaxV + 4]: outputs by column
    constexpr int XLD = kMaxV + 4;
    const int tid = threadIdx.x;
    for (int e = tid; e < kMaxV * kMaxV; e += kMaxV) {
        const int k = e / kMaxV, i = e % kMaxV;          // Ls[k][i] = L(i, k), absolute rows
        if (k < w && i > k && i < w) Ls[e] = L00[(size_t)i + (size_t)k * ldl];
    }
    const int c0 = blockIdx.x * kMaxV;
    const int nc = min(kMaxV, cols - c0);
    const bool live = tid < nc;
    float a[kMaxV];
    const float *xc = X + (size_t)(c0 + (live ? tid : 0)) * ldx;
#pragma unroll
    for (int i = 0; i < kMaxV; ++i) a[i] = (live && i < w) ? xc[i] : 0.f;
    __syncthreads();
    LtrsmStep body{a, Ls, Xs + tid * XLD, w};
    for_blocks(a, w, body);
    __syncthreads();
    for (int e = tid; e < kMaxV * kMaxV; e += kMaxV) {
        const int i = e % kMaxV, c = e / kMaxV;
        if (c < nc) {
            if (i < w) X[(size_t)i + (size_t)(c0 + c) * ldx] = Xs[c * XLD + i];
            if (lp != nullptr && i < kpad) lp[(size_t)(c0 + c) * ldk + i] = lp_from<LP>(i < w ? Xs[c * XLD + i] : 0.f);
        }
    }
}

// ---------------------------------------------------------------------------
int launch_a00_lu32(float *A00, int lda, int w, int kglob, int *info, cudaStream_t st) {
    if (w <= 0) return CF_OK;
    k_a00_lu32<<<1, kMaxV, 0, st>>>(A00, lda, w, kglob, info);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

int launch_a00_chol32(float *A00, int lda, int w, int kglob, int *info, cudaStream_t st) {
    if (w <= 0) return CF_OK;
    k_a00_chol32<<<1, kMaxV, 0, st>>>(A00, lda, w, kglob, info);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

template <typename LP>
int launch_rtrsm32(float *X, int ldx, int rows, int w, const float *M00, int ldm, bool trans_lower, LP *lp, int ldk,
                   int kpad, const int *skip, cudaStream_t st) {
    if (rows <= 0 || w <= 0) return CF_OK;
    const size_t smem = sizeof(float) * ((size_t)kMaxV * kMaxV + (size_t)kMaxV * (kMaxV + 4));
    CF_CUDA_TRY(cudaFuncSetAttribute(k_rtrsm32<LP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_rtrsm32<LP><<<ceil_div(rows, kMaxV), kMaxV, smem, st>>>(X, ldx, rows, w, M00, ldm, trans_lower ? 1 : 0, lp, ldk,
                                                              kpad, skip);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

template <typename LP>
int launch_ltrsm32(float *X, int ldx, int w, int cols, const float *L00, int ldl, LP *lp, int ldk, int kpad,
                   cudaStream_t st) {
    if (cols <= 0 || w <= 0) return CF_OK;
    const size_t smem = sizeof(float) * ((size_t)kMaxV * kMaxV + (size_t)kMaxV * (kMaxV + 4));
    CF_CUDA_TRY(cudaFuncSetAttribute(k_ltrsm32<LP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_ltrsm32<LP><<<ceil_div(cols, kMaxV), kMaxV, smem, st>>>(X, ldx, w, cols, L00, ldl, lp, ldk, kpad);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

template int launch_rtrsm32<__nv_bfloat16>(float *, int, int, int, const float *, int, bool, __nv_bfloat16 *, int,
                                           int, const int *, cudaStream_t);
template int launch_rtrsm32<__half>(float *, int, int, int, const float *, int, bool, __half *, int, int, const int *,
                                    cudaStream_t);
template int launch_ltrsm32<__nv_bfloat16>(float *, int, int, int, const float *, int, __nv_bfloat16 *, int, int,
                                           cudaStream_t);
template int launch_ltrsm32<__half>(float *, int, int, int, const float *, int, __half *, int, int, cudaStream_t);

}  // namespace cf
