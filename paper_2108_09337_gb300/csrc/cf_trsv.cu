// cf_trsv.cu -- S-1 for the refinement loop: triangular solves with the FP32
// factors and a thin right-hand side (nrhs <= 16), one launch per solve.
//
// Block rows of 64 are processed by CTAs that take a ticket in launch order
// (atomic counter), so every block a CTA depends on belongs to a CTA that
// started earlier and never waits on a later one.  A CTA subtracts the
// contributions of the finished blocks as their flags appear, applies the
// precomputed inverse of its diagonal block, publishes its block of the
// solution and raises its flag.  The factor is read exactly once; the chain
// of dependent work is one 64 x 64 tile product per block.  Waits on flags
// are bounded: after the limit the kernel records CF_ERR_TIMEOUT and goes
// on (results are then wrong, never hung).
#include "cf_common.cuh"
#include "cf_kernels.cuh"

namespace cf {

__device__ int g_trsv_status = 0;

constexpr int kSB = 64;                // block size
constexpr long long kFlagSpin = 1ll << 22;

// Effective matrix M (n x n) seen by a solve:
//   0: M = L, unit lower (forward)       1: M = U, upper (backward)
//   2: M = L, lower (forward)            3: M = L^T (backward)
template <int MODE>
__device__ __forceinline__ float m_elem(const float *T, int ldt, int i, int k) {
    return (MODE == 3) ? T[(size_t)k + (size_t)i * ldt] : T[(size_t)i + (size_t)k * ldt];
}

// Inverse of each 64 x 64 diagonal block of M, stored block after block,
// column-major (Dinv[b*64*64 + i + 64*j]), computed in VT (float, or double
// for the FP64-arithmetic solves with the same FP32 factor).  Dynamic shared
// memory: 2 * 64 * 65 VT.
template <int MODE, typename VT>
__global__ void __launch_bounds__(256) k_diag_inverse(int n, const float *__restrict__ T, int ldt, VT *Dinv) {
    extern __shared__ __align__(16) unsigned char dsm[];
    VT (*Ms)[kSB + 1] = reinterpret_cast<VT (*)[kSB + 1]>(dsm);                               // Ms[i][k] = M(b0+i, b0+k)
    VT (*Xs)[kSB + 1] = reinterpret_cast<VT (*)[kSB + 1]>(dsm + sizeof(VT) * kSB * (kSB + 1));  // inverse
    const int b = blockIdx.x, b0 = b * kSB, nbk = min(kSB, n - b0);
    const int tid = threadIdx.x;
    for (int e = tid; e < kSB * kSB; e += 256) {
        const int i = e % kSB, k = e / kSB;
        VT v = VT(0);
        if (i < nbk && k < nbk) v = (VT)m_elem<MODE>(T, ldt, b0 + i, b0 + k);
        if (i >= nbk || k >= nbk) v = (i == k) ? VT(1) : VT(0);
        if (MODE == 0 && i == k) v = VT(1);
        Ms[i][k] = v;
        Xs[i][k] = (i == k) ? VT(1) : VT(0);
    }
    __syncthreads();
    const bool lower = (MODE != 1);
    // Solve M X = I column-parallel: thread owns column j = tid % 64 and rows
    // i = tid / 64 + 4 t.
    const int j = tid % kSB, i0 = tid / kSB;
    for (int s = 0; s < kSB; ++s) {
        const int k = lower ? s : kSB - 1 - s;
        if (MODE != 0 && i0 == 0) Xs[k][j] = Xs[k][j] / Ms[k][k];
        __syncthreads();
        const VT xk = Xs[k][j];
        for (int i = i0; i < kSB; i += 4) {
            if ((lower && i > k) || (!lower && i < k)) Xs[i][j] = fma(-Ms[i][k], xk, Xs[i][j]);
        }
        __syncthreads();
    }
    VT *D = Dinv + (size_t)b * kSB * kSB;
    for (int e = tid; e < kSB * kSB; e += 256) D[e] = Xs[e % kSB][e / kSB];
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

constexpr int kTLD = kSB + 4;          // smem leading dimension (16-byte rows)

// Stages the STORED 64 x 64 tile whose top-left element is (i0, j0) of T
// (column-major, ld ldt) into St[col * kTLD + row] with 16-byte async copies
// when the whole tile is inside the matrix and aligned; element by element
// otherwise (zero outside).
__device__ __forceinline__ void stage_tile(float *St, const float *T, int ldt, int n, int i0, int j0, bool fast) {
    const int tid = threadIdx.x;
    if (fast) {
        for (int e = tid; e < kSB * kSB / 4; e += 256) {
            const int r4 = e % (kSB / 4), c = e / (kSB / 4);
            cp_async16(St + c * kTLD + 4 * r4, T + (size_t)(i0 + 4 * r4) + (size_t)(j0 + c) * ldt);
        }
    } else {
        for (int e = tid; e < kSB * kSB; e += 256) {
            const int r = e % kSB, c = e / kSB;
            St[c * kTLD + r] = (i0 + r < n && j0 + c < n) ? T[(size_t)(i0 + r) + (size_t)(j0 + c) * ldt] : 0.f;
        }
    }
}

// VT: arithmetic and right-hand-side type (float, or double for FP64
// solves with the FP32 factor); the factor tiles stay FP32 in shared memory.
template <int MODE, int NR, typename VT>
__global__ void __launch_bounds__(256)
k_trsv_blocked(int n, int nrhs, const float *__restrict__ T, int ldt, const VT *__restrict__ Dinv, VT *X,
               int ldx, int *flags, int *ticket) {
    extern __shared__ __align__(16) float sm[];
    float *St0 = sm;                               // two tile buffers
    float *St1 = sm + kSB * kTLD;
    VT *Ds = reinterpret_cast<VT *>(sm + 2 * kSB * kTLD);   // inverse of the diagonal block
    VT *Ys = Ds + kSB * kTLD;                               // [kSB][NR + 1]
    __shared__ int s_ticket;
    constexpr bool fwd = (MODE == 0 || MODE == 2);
    constexpr int CPT = (NR + 3) / 4;              // right-hand sides per thread
    constexpr int YLD = NR + 1;
    const int nb = (n + kSB - 1) / kSB;
    const int tid = threadIdx.x;
    if (tid == 0) s_ticket = atomicAdd(ticket, 1);
    __syncthreads();
    const int s = s_ticket;
    if (s >= nb) return;
    const int b = fwd ? s : nb - 1 - s;
    const int r0 = b * kSB, rb = min(kSB, n - r0);
    const int i = tid % kSB, q = tid / kSB;        // row, rhs group
    const bool aligned = ((ldt & 3) == 0) && ((((uintptr_t)T) & 15) == 0);
    // the diagonal block's inverse does not depend on anyone: fetch it now
    {
        const VT *D = Dinv + (size_t)b * kSB * kSB;
        for (int e = tid; e < kSB * kSB; e += 256) {
            const int ii = e % kSB, kk = e / kSB;
            // MODE 3 uses (L_bb^{-1})^T
            Ds[kk * kTLD + ii] = (MODE == 3) ? D[kk + kSB * ii] : D[ii + kSB * kk];
        }
    }
    VT acc[CPT];
#pragma unroll
    for (int t = 0; t < CPT; ++t) {
        const int c = q + 4 * t;
        acc[t] = (i < rb && c < nrhs) ? X[(size_t)(r0 + i) + (size_t)c * ldx] : VT(0);
    }
    // Stored tile that holds M(block b, block cb): for MODE 3 it is L(cb, b).
    auto tile_origin = [&](int cb, int &ti, int &tj) {
        if (MODE == 3) { ti = cb * kSB; tj = r0; } else { ti = r0; tj = cb * kSB; }
    };
    if (s > 0) {
        const int cb = fwd ? 0 : nb - 1;
        int ti, tj;
        tile_origin(cb, ti, tj);
        stage_tile(St0, T, ldt, n, ti, tj, aligned && ti + kSB <= n && tj + kSB <= n);
        cp_async_commit();
    }
    for (int step = 0; step < s; ++step) {
        float *St = (step & 1) ? St1 : St0;
        if (step + 1 < s) {                        // prefetch the next tile
            const int cb = fwd ? step + 1 : nb - 2 - step;
            int ti, tj;
            tile_origin(cb, ti, tj);
            stage_tile((step & 1) ? St0 : St1, T, ldt, n, ti, tj, aligned && ti + kSB <= n && tj + kSB <= n);
        }
        cp_async_commit();
        const int cb = fwd ? step : nb - 1 - step;
        const int c0 = cb * kSB, cbk = min(kSB, n - c0);
        if (tid == 0) {
            volatile int *f = flags + cb;
            long long it = 0;
            while (*f == 0 && it < kFlagSpin) {
                ++it;
                if (it > 64) __nanosleep(20);
            }
            if (it >= kFlagSpin) atomicExch(&g_trsv_status, CF_ERR_TIMEOUT);
            __threadfence();
        }
        __syncthreads();
        for (int e = tid; e < kSB * NR; e += 256) {
            const int kk = e % kSB, c = e / kSB;
            Ys[kk * YLD + c] = (kk < cbk && c < nrhs) ? __ldcg(X + (size_t)(c0 + kk) + (size_t)c * ldx) : VT(0);
        }
        cp_async_wait<1>();                        // this step's tile has landed
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < kSB; ++kk) {
            const VT m = (VT)((MODE == 3) ? St[i * kTLD + kk] : St[kk * kTLD + i]);
#pragma unroll
            for (int t = 0; t < CPT; ++t) acc[t] = fma(-m, Ys[kk * YLD + q + 4 * t], acc[t]);
        }
        __syncthreads();
    }
    cp_async_wait<0>();
    // y_b = Dinv_b acc
#pragma unroll
    for (int t = 0; t < CPT; ++t)
        if (q + 4 * t < NR) Ys[i * YLD + q + 4 * t] = acc[t];
    __syncthreads();
    VT y[CPT];
#pragma unroll
    for (int t = 0; t < CPT; ++t) y[t] = VT(0);
#pragma unroll 8
    for (int kk = 0; kk < kSB; ++kk) {
        const VT d = Ds[kk * kTLD + i];
#pragma unroll
        for (int t = 0; t < CPT; ++t) y[t] = fma(d, Ys[kk * YLD + q + 4 * t], y[t]);
    }
#pragma unroll
    for (int t = 0; t < CPT; ++t) {
        const int c = q + 4 * t;
        if (i < rb && c < nrhs) X[(size_t)(r0 + i) + (size_t)c * ldx] = y[t];
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicExch(flags + b, 1);
}

size_t trsv_ws_bytes(int n) {
    const int nb = (n + kSB - 1) / kSB;
    return sizeof(int) * (size_t)(nb + 1);
}

size_t diag_inverse_floats(int n) {
    const int nb = (n + kSB - 1) / kSB;
    return (size_t)nb * kSB * kSB;
}

// mode: 0 unit lower, 1 upper, 2 lower, 3 lower transposed (see m_elem).
template <typename VT>
static int launch_diag_inverse_t(int mode, int n, const float *T, int ldt, VT *Dinv, cudaStream_t st) {
    if (n <= 0) return CF_OK;
    const int nb = (n + kSB - 1) / kSB;
    const size_t smem = 2 * sizeof(VT) * kSB * (kSB + 1);
    switch (mode) {
        case 0:
            CF_CUDA_TRY(cudaFuncSetAttribute(k_diag_inverse<0, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_diag_inverse<0, VT><<<nb, 256, smem, st>>>(n, T, ldt, Dinv);
            break;
        case 1:
            CF_CUDA_TRY(cudaFuncSetAttribute(k_diag_inverse<1, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_diag_inverse<1, VT><<<nb, 256, smem, st>>>(n, T, ldt, Dinv);
            break;
        case 2:
            CF_CUDA_TRY(cudaFuncSetAttribute(k_diag_inverse<2, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_diag_inverse<2, VT><<<nb, 256, smem, st>>>(n, T, ldt, Dinv);
            break;
        default: return CF_ERR_UNSUPPORTED;
    }
    CF_LAUNCH_CHECK();
    return CF_OK;
}

int launch_diag_inverse(int mode, int n, const float *T, int ldt, float *Dinv, cudaStream_t st) {
    return launch_diag_inverse_t<float>(mode, n, T, ldt, Dinv, st);
}
int launch_diag_inverse64(int mode, int n, const float *T, int ldt, double *Dinv, cudaStream_t st) {
    return launch_diag_inverse_t<double>(mode, n, T, ldt, Dinv, st);
}

template <int MODE, int NR, typename VT>
static int launch_trsv_nr(int n, int nrhs, const float *T, int ldt, const VT *Dinv, VT *X, int ldx, int *flags,
                          int *ticket, cudaStream_t st) {
    const int nb = (n + kSB - 1) / kSB;
    const size_t smem = sizeof(float) * 2 * (size_t)kSB * kTLD + sizeof(VT) * ((size_t)kSB * kTLD + (size_t)kSB * 17);
    CF_CUDA_TRY(cudaFuncSetAttribute(k_trsv_blocked<MODE, NR, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    k_trsv_blocked<MODE, NR, VT><<<nb, 256, smem, st>>>(n, nrhs, T, ldt, Dinv, X, ldx, flags, ticket);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

template <int MODE, typename VT>
static int launch_trsv_mode(int n, int nrhs, const float *T, int ldt, const VT *Dinv, VT *X, int ldx, int *sync_ws,
                            cudaStream_t st) {
    const int nb = (n + kSB - 1) / kSB;
    CF_CUDA_TRY(cudaMemsetAsync(sync_ws, 0, sizeof(int) * (size_t)(nb + 1), st));
    int *flags = sync_ws, *ticket = sync_ws + nb;
    if (nrhs <= 4) return launch_trsv_nr<MODE, 4, VT>(n, nrhs, T, ldt, Dinv, X, ldx, flags, ticket, st);
    if (nrhs <= 8) return launch_trsv_nr<MODE, 8, VT>(n, nrhs, T, ldt, Dinv, X, ldx, flags, ticket, st);
    return launch_trsv_nr<MODE, 16, VT>(n, nrhs, T, ldt, Dinv, X, ldx, flags, ticket, st);
}

template <typename VT>
static int launch_trsv_t(int mode, int n, int nrhs, const float *T, int ldt, const VT *Dinv, VT *X, int ldx,
                         int *sync_ws, cudaStream_t st) {
    if (n <= 0 || nrhs <= 0) return CF_OK;
    if (nrhs > 16) return CF_ERR_UNSUPPORTED;
    switch (mode) {
        case 0: return launch_trsv_mode<0, VT>(n, nrhs, T, ldt, Dinv, X, ldx, sync_ws, st);
        case 1: return launch_trsv_mode<1, VT>(n, nrhs, T, ldt, Dinv, X, ldx, sync_ws, st);
        case 2: return launch_trsv_mode<2, VT>(n, nrhs, T, ldt, Dinv, X, ldx, sync_ws, st);
        case 3: return launch_trsv_mode<3, VT>(n, nrhs, T, ldt, Dinv, X, ldx, sync_ws, st);
        default: return CF_ERR_UNSUPPORTED;
    }
}

// X <- M^{-1} X for nrhs <= 16 columns; sync_ws holds trsv_ws_bytes(n).
int launch_trsv_f32(int mode, int n, int nrhs, const float *T, int ldt, const float *Dinv, float *X, int ldx,
                    int *sync_ws, cudaStream_t st) {
    return launch_trsv_t<float>(mode, n, nrhs, T, ldt, Dinv, X, ldx, sync_ws, st);
}
// The same with FP64 right-hand sides and arithmetic (FP64 Dinv from
// launch_diag_inverse64); the FP32 factor is read as stored.
int launch_trsv_f64x(int mode, int n, int nrhs, const float *T, int ldt, const double *Dinv, double *X, int ldx,
                     int *sync_ws, cudaStream_t st) {
    return launch_trsv_t<double>(mode, n, nrhs, T, ldt, Dinv, X, ldx, sync_ws, st);
}

int trsv_take_status(cudaStream_t st, int *status) {
    int h = 0;
    CF_CUDA_TRY(cudaMemcpyFromSymbolAsync(&h, g_trsv_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    CF_CUDA_TRY(cudaStreamSynchronize(st));
    if (h != 0) {
        const int zero = 0;
        CF_CUDA_TRY(cudaMemcpyToSymbolAsync(g_trsv_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
    }
    *status = h;
    return CF_OK;
}

}  // namespace cf
