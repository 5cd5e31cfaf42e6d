// cf_panel.cu -- the per-step block routines around the Schur update:
//   LU-3  A10 <- A10 U00^{-1}      (Alg. 1, "Factorize A10"; Table 2)
//   LU-4  A01 <- L00^{-1} A01      (Alg. 1, "Factorize A01")
//   A00   LU without pivoting of the selected rows (Fig. "prog_rep",
//         the tournament already yields it, Sec. 7.2)
//   CH-1  potrf of A00 (Listing "Cholesky Factorization"; Table 2, v^3/6)
//   CH-2  L10 <- A10 L00^{-T}      (Table 2: costed like the LU panel solve)
//   S-1   the same triangular kernels serve the solves.
//
// The v x v triangle lives in shared memory; each CTA streams a chunk of
// rows (right solves) or columns (left solves) of the panel.  Every update
// is a separately rounded multiply and subtract in the oracle's order, so
// step 0 of a factorization reproduces the oracle's values bit for bit.
#include "cf_common.cuh"
#include "cf_kernels.cuh"

namespace cf {

constexpr int kPanelThreads = 256;
constexpr int kRB = 64;            // rows per CTA, right solves
constexpr int kCB = 64;            // columns per CTA, left solves
constexpr int kLdT = kMaxV;        // triangle tile leading dimension

// ---------------------------------------------------------------------------
// A00: LU without pivoting (w <= 128), one CTA.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kPanelThreads, 1)
k_getf2_nopiv(T *A, int lda, int w, int kglob, int *info) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *t = reinterpret_cast<T *>(smem_raw);      // t[k*kLdT + r]
    const int tid = threadIdx.x;
    for (int idx = tid; idx < w * w; idx += kPanelThreads) {
        const int k = idx / w, r = idx % w;
        t[k * kLdT + r] = A[r + (size_t)k * lda];
    }
    __syncthreads();
    const int r = tid & (kMaxV - 1), half = tid / kMaxV;
    for (int k = 0; k < w; ++k) {
        const T piv = t[k * kLdT + k];
        const bool act = (r > k && r < w);
        T l = T(0);
        if (act) l = (piv != T(0)) ? div_rn(t[k * kLdT + r], piv) : t[k * kLdT + r];
        if (piv == T(0) && tid == 0) atomicCAS(info, 0, kglob + k + 1);
        __syncthreads();
        if (act) {
            if (half == 0) t[k * kLdT + r] = l;
            for (int j = k + 1 + half; j < w; j += 2)
                t[j * kLdT + r] = sub_rn(t[j * kLdT + r], mul_rn(l, t[j * kLdT + k]));
        }
        __syncthreads();
    }
    for (int idx = tid; idx < w * w; idx += kPanelThreads) {
        const int k = idx / w, rr = idx % w;
        A[rr + (size_t)k * lda] = t[k * kLdT + rr];
    }
}

// ---------------------------------------------------------------------------
// A00: Cholesky (lower, w <= 128), one CTA.  Stops at the first pivot that is
// not positive (or NaN) and records info; later launches see info != 0.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kPanelThreads, 1)
k_potf2(T *A, int lda, int w, int kglob, int *info) {
    if (*info != 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *t = reinterpret_cast<T *>(smem_raw);
    __shared__ int fail;
    const int tid = threadIdx.x;
    for (int idx = tid; idx < w * w; idx += kPanelThreads) {
        const int k = idx / w, r = idx % w;
        if (r >= k) t[k * kLdT + r] = A[r + (size_t)k * lda];
    }
    if (tid == 0) fail = 0;
    __syncthreads();
    const int r = tid & (kMaxV - 1), half = tid / kMaxV;
    int kdone = w;
    for (int k = 0; k < w; ++k) {
        const T d = t[k * kLdT + k];
        if (!(d > T(0))) {                       // uniform: all threads read d
            if (tid == 0) atomicCAS(info, 0, kglob + k + 1);
            kdone = k;
            break;
        }
        const T lkk = sqrt(d);                                  // the pivot
        if (half == 0 && r > k && r < w) t[k * kLdT + r] = div_rn(t[k * kLdT + r], lkk);   // column scaling
        __syncthreads();
        if (tid == 0) t[k * kLdT + k] = lkk;
        if (r > k && r < w) {                                   // trailing update, j in (k, r]
            const T lik = t[k * kLdT + r];
            for (int j = k + 1 + half; j <= r; j += 2)
                t[j * kLdT + r] = sub_rn(t[j * kLdT + r], mul_rn(lik, t[k * kLdT + j]));
        }
        __syncthreads();
    }
    (void)fail;
    // Write back the lower triangle (columns past a breakdown keep their
    // partially updated values, as LAPACK leaves them).
    for (int idx = tid; idx < w * w; idx += kPanelThreads) {
        const int k = idx / w, rr = idx % w;
        if (rr >= k) A[rr + (size_t)k * lda] = t[k * kLdT + rr];
    }
    (void)kdone;
}

// ---------------------------------------------------------------------------
// Right solve X <- X M^{-1}, M upper non-unit (M(k,j) = U[k + j*ldu]) or, with
// TRANS, M = L^T for lower L (M(k,j) = L[j + k*ldu]).  X is rows x w.
// CTA: kRB rows; four lanes of one warp share a row.
// ---------------------------------------------------------------------------
template <typename T, bool TRANS>
__global__ void __launch_bounds__(kPanelThreads, 1)
k_trsm_right_upper(T *X, int ldx, int rows, int w, const T *U, int ldu, const int *skip) {
    if (skip != nullptr && *skip != 0) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Ms = reinterpret_cast<T *>(smem_raw);     // Ms[j*kLdT + k] = M(k, j)
    T *Xs = Ms + kLdT * kMaxV;                   // Xs[j*(kRB+1) + r]
    constexpr int XLD = kRB + 1;
    const int tid = threadIdx.x;
    const int r0 = blockIdx.x * kRB;
    const int nr = min(kRB, rows - r0);
    for (int idx = tid; idx < w * w; idx += kPanelThreads) {
        const int k = idx % w, j = idx / w;
        if (k <= j) Ms[j * kLdT + k] = TRANS ? U[j + (size_t)k * ldu] : U[k + (size_t)j * ldu];
    }
    for (int idx = tid; idx < kRB * w; idx += kPanelThreads) {
        const int r = idx % kRB, j = idx / kRB;
        if (r < nr) Xs[j * XLD + r] = X[(size_t)(r0 + r) + (size_t)j * ldx];
    }
    __syncthreads();
    const int r = tid >> 2, q = tid & 3;
    if (r < nr) {
        for (int k = 0; k < w; ++k) {
            if (q == 0) {
                const T ukk = Ms[k * kLdT + k];
                if (ukk != T(0)) Xs[k * XLD + r] = div_rn(Xs[k * XLD + r], ukk);
            }
            __syncwarp(0xfu << (tid & 28));
            const T xk = Xs[k * XLD + r];
            for (int j = k + 1 + q; j < w; j += 4)
                Xs[j * XLD + r] = sub_rn(Xs[j * XLD + r], mul_rn(xk, Ms[j * kLdT + k]));
            __syncwarp(0xfu << (tid & 28));
        }
    }
    __syncthreads();
    for (int idx = tid; idx < kRB * w; idx += kPanelThreads) {
        const int rr = idx % kRB, j = idx / kRB;
        if (rr < nr) X[(size_t)(r0 + rr) + (size_t)j * ldx] = Xs[j * XLD + rr];
    }
}

// ---------------------------------------------------------------------------
// Left solve X <- M^{-1} X with M = T (TRANS: M = T^T) of size w x w, lower
// (forward) or upper (backward), unit or non-unit diagonal.  X is w x cols.
// CTA: kCB columns; four lanes of one warp share a column.
// ---------------------------------------------------------------------------
template <typename T, bool LOWER, bool UNIT, bool TRANS>
__global__ void __launch_bounds__(kPanelThreads, 1)
k_trsm_left(T *X, int ldx, int w, int cols, const T *Tm, int ldt) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Ms = reinterpret_cast<T *>(smem_raw);     // Ms[k*kLdT + i] = M(i, k)
    T *Xs = Ms + kLdT * kMaxV;                   // Xs[c*XLD + i]
    constexpr int XLD = kMaxV + 1;
    const int tid = threadIdx.x;
    const int c0 = blockIdx.x * kCB;
    const int nc = min(kCB, cols - c0);
    for (int idx = tid; idx < w * w; idx += kPanelThreads) {
        const int i = idx % w, k = idx / w;
        const bool need = LOWER ? (i >= k) : (i <= k);
        if (need) Ms[k * kLdT + i] = TRANS ? Tm[k + (size_t)i * ldt] : Tm[i + (size_t)k * ldt];
    }
    for (int idx = tid; idx < kCB * w; idx += kPanelThreads) {
        const int i = idx % w, c = idx / w;
        if (c < nc) Xs[c * XLD + i] = X[(size_t)i + (size_t)(c0 + c) * ldx];
    }
    __syncthreads();
    const int c = tid >> 2, q = tid & 3;
    if (c < nc) {
        T *x = Xs + c * XLD;
        for (int s = 0; s < w; ++s) {
            const int k = LOWER ? s : (w - 1 - s);
            if (!UNIT) {
                if (q == 0) x[k] = div_rn(x[k], Ms[k * kLdT + k]);
                __syncwarp(0xfu << (tid & 28));
            }
            const T xk = x[k];
            if (LOWER) {
                for (int i = k + 1 + q; i < w; i += 4) x[i] = sub_rn(x[i], mul_rn(Ms[k * kLdT + i], xk));
            } else {
                for (int i = q; i < k; i += 4) x[i] = sub_rn(x[i], mul_rn(Ms[k * kLdT + i], xk));
            }
            __syncwarp(0xfu << (tid & 28));
        }
    }
    __syncthreads();
    for (int idx = tid; idx < kCB * w; idx += kPanelThreads) {
        const int i = idx % w, cc = idx / w;
        if (cc < nc) X[(size_t)i + (size_t)(c0 + cc) * ldx] = Xs[cc * XLD + i];
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename K>
static int set_smem(K kernel, size_t bytes) {
    CF_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return CF_OK;
}

template <typename T>
int launch_getf2_nopiv(T *A00, int lda, int w, int kglob, int *info, cudaStream_t st) {
    if (w <= 0) return CF_OK;
    const size_t smem = sizeof(T) * kLdT * kMaxV;
    int rc = set_smem(k_getf2_nopiv<T>, smem);
    if (rc) return rc;
    k_getf2_nopiv<T><<<1, kPanelThreads, smem, st>>>(A00, lda, w, kglob, info);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

template <typename T>
int launch_potf2(T *A00, int lda, int w, int kglob, int *info, cudaStream_t st) {
    if (w <= 0) return CF_OK;
    const size_t smem = sizeof(T) * kLdT * kMaxV;
    int rc = set_smem(k_potf2<T>, smem);
    if (rc) return rc;
    k_potf2<T><<<1, kPanelThreads, smem, st>>>(A00, lda, w, kglob, info);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

template <typename T>
int launch_trsm_right_upper(T *X, int ldx, int rows, int w, const T *U, int ldu, bool trans_lower,
                            const int *skip_if_nonzero, cudaStream_t st) {
    if (rows <= 0 || w <= 0) return CF_OK;
    const size_t smem = sizeof(T) * ((size_t)kLdT * kMaxV + (size_t)(kRB + 1) * kMaxV);
    const int grid = ceil_div(rows, kRB);
    if (trans_lower) {
        int rc = set_smem(k_trsm_right_upper<T, true>, smem);
        if (rc) return rc;
        k_trsm_right_upper<T, true><<<grid, kPanelThreads, smem, st>>>(X, ldx, rows, w, U, ldu, skip_if_nonzero);
    } else {
        int rc = set_smem(k_trsm_right_upper<T, false>, smem);
        if (rc) return rc;
        k_trsm_right_upper<T, false><<<grid, kPanelThreads, smem, st>>>(X, ldx, rows, w, U, ldu, skip_if_nonzero);
    }
    CF_LAUNCH_CHECK();
    return CF_OK;
}

template <typename T, bool LOWER, bool UNIT, bool TRANS>
static int launch_trsm_left_t(T *X, int ldx, int w, int cols, const T *Tm, int ldt, cudaStream_t st) {
    if (cols <= 0 || w <= 0) return CF_OK;
    const size_t smem = sizeof(T) * ((size_t)kLdT * kMaxV + (size_t)kCB * (kMaxV + 1));
    int rc = set_smem(k_trsm_left<T, LOWER, UNIT, TRANS>, smem);
    if (rc) return rc;
    k_trsm_left<T, LOWER, UNIT, TRANS><<<ceil_div(cols, kCB), kPanelThreads, smem, st>>>(X, ldx, w, cols, Tm, ldt);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

template <typename T>
int launch_trsm_left_lower_unit(T *X, int ldx, int w, int cols, const T *L, int ldl, cudaStream_t st) {
    return launch_trsm_left_t<T, true, true, false>(X, ldx, w, cols, L, ldl, st);
}

template <typename T>
int launch_trsm_left(bool lower, bool unit, bool trans, T *X, int ldx, int w, int cols, const T *Tm, int ldt,
                     cudaStream_t st) {
    if (lower && unit && !trans) return launch_trsm_left_t<T, true, true, false>(X, ldx, w, cols, Tm, ldt, st);
    if (lower && !unit && !trans) return launch_trsm_left_t<T, true, false, false>(X, ldx, w, cols, Tm, ldt, st);
    if (!lower && !unit && !trans) return launch_trsm_left_t<T, false, false, false>(X, ldx, w, cols, Tm, ldt, st);
    if (!lower && !unit && trans) return launch_trsm_left_t<T, false, false, true>(X, ldx, w, cols, Tm, ldt, st);
    return CF_ERR_UNSUPPORTED;
}
template int launch_trsm_left<double>(bool, bool, bool, double *, int, int, int, const double *, int, cudaStream_t);
template int launch_trsm_left<float>(bool, bool, bool, float *, int, int, int, const float *, int, cudaStream_t);

int launch_trsm_left_f64(bool lower, bool unit, bool trans, double *X, int ldx, int w, int cols, const double *Tm,
                         int ldt, cudaStream_t st) {
    return launch_trsm_left<double>(lower, unit, trans, X, ldx, w, cols, Tm, ldt, st);
}

template int launch_getf2_nopiv<double>(double *, int, int, int, int *, cudaStream_t);
template int launch_getf2_nopiv<float>(float *, int, int, int, int *, cudaStream_t);
template int launch_potf2<double>(double *, int, int, int, int *, cudaStream_t);
template int launch_potf2<float>(float *, int, int, int, int *, cudaStream_t);
template int launch_trsm_right_upper<double>(double *, int, int, int, const double *, int, bool, const int *,
                                             cudaStream_t);
template int launch_trsm_right_upper<float>(float *, int, int, int, const float *, int, bool, const int *,
                                            cudaStream_t);
template int launch_trsm_left_lower_unit<double>(double *, int, int, int, const double *, int, cudaStream_t);
template int launch_trsm_left_lower_unit<float>(float *, int, int, int, const float *, int, cudaStream_t);

}  // namespace cf
