// cf_batched.cu -- BAT-1: thousands of independent, uneven factorizations in
// one persistent launch (an addition of this project; the paper's small-N
// motivation is its Sec. 9.3 discussion of small matrices on many nodes).
//
// One CTA factors one matrix at a time.  CTAs pull matrix indices from an
// atomic queue ordered by decreasing n^3 (longest processing time first), so
// the few large matrices start early and the many small ones fill the tail.
// Each matrix uses the same blocked algorithm as cf_getrf / cf_potrf (Alg. 1
// with block size vb; the tournament with one leaf covering the panel, i.e.
// leaf height >= n, which is partial pivoting), run by one CTA out of L2:
// the panel copy for the pivot search and the diagonal block live in shared
// memory, the trailing update streams through registers.  Matrices up to
// n = 512 (the panel copy is 512 x vb).
//
// The mixed variant (cf_solve_batched_mixed) factors an FP32 copy held in
// the CTA's own scratch and refines each solution in FP64 to the tolerance
// (falling back to FP64 factors for a matrix the FP32 ones cannot serve),
// all inside the same launch; nothing returns to the host between matrices,
// so the whole batch can be captured in a CUDA graph.
#include <climits>
#include <cmath>
#include <vector>

#include "cf_common.cuh"
#include "cf_kernels.cuh"

namespace cf {

constexpr int kBT = 256;                // threads per CTA
constexpr int kBMaxN = 512;             // largest matrix
constexpr int kBMaxV = 32;              // largest block size

// Per-CTA shared memory: this header, then the panel copy P (kBMaxN x vb
// elements of T; its size follows the block size, which sets how many CTAs
// fit on an SM).
template <typename T>
struct BSmem {
    T D[kBMaxV * (kBMaxV + 1)];         // diagonal block
    T redv2[2][kBT / 32];               // the pivot search's warp maxima, alternating by column
    int redi2[2][kBT / 32];
    int used[kBMaxN];
    int order[kBMaxV];
    int lab[kBMaxN];
    int where_[kBMaxN];
    int fail;
};

template <typename T>
__host__ __device__ constexpr size_t bsmem_header_bytes() {
    return (sizeof(BSmem<T>) + 15) / 16 * 16;
}
template <typename T>
__host__ __device__ constexpr size_t bsmem_bytes(int vb) {
    return bsmem_header_bytes<T>() + sizeof(T) * (size_t)kBMaxN * vb;
}
template <typename T>
__device__ __forceinline__ T *bsmem_panel(BSmem<T> &s) {
    return reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(&s) + bsmem_header_bytes<T>());
}

template <typename T>
__device__ __forceinline__ T bkey(T a) {
    T x = fabs(a);
    return (x != x) ? T(-0.5) : x;
}

template <typename T>
__device__ __forceinline__ void bbetter(T &bv, int &bi, T ov, int oi) {
    if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
}

// CTA-wide argmax (value, index) with the tie rule of the tournament, one
// barrier: the warp maxima go to buffer buf (alternating from one call to
// the next, so the next call's writes never meet this call's reads) and
// every thread reduces the eight itself.
template <typename T>
__device__ __forceinline__ void cta_argmax_1bar(BSmem<T> &s, T &bv, int &bi, int buf) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        bbetter(bv, bi, ov, oi);
    }
    if (lane == 0) { s.redv2[buf][warp] = bv; s.redi2[buf][warp] = bi; }
    __syncthreads();
    bv = s.redv2[buf][0];
    bi = s.redi2[buf][0];
#pragma unroll
    for (int q = 1; q < kBT / 32; ++q) bbetter(bv, bi, s.redv2[buf][q], s.redi2[buf][q]);
}

// C (mm x nn, ldc) -= A (mm x kk, lda) * B (kk x nn, ldb), kk <= kBMaxV; if
// lower, only i >= j (relative indices, diagonal aligned).  A may be shared.
template <typename T>
__device__ void cta_gemm_sub(int mm, int nn, int kk, const T *A, int lda, const T *B, int ldb, T *C, int ldc,
                             bool lower) {
    const int tid = threadIdx.x;
    const int tr = (tid & 15) * 4, tc = (tid >> 4) * 4;      // 64 x 64 tiles, 4 x 4 per thread
    for (int j0 = 0; j0 < nn; j0 += 64) {
        for (int i0 = 0; i0 < mm; i0 += 64) {
            if (lower && j0 > i0 + 63) continue;
            T acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
            for (int p = 0; p < kk; ++p) {
                T av[4], bv[4];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int i = i0 + tr + a;
                    av[a] = i < mm ? A[(size_t)i + (size_t)p * lda] : T(0);
                }
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int j = j0 + tc + b;
                    bv[b] = j < nn ? B[(size_t)p + (size_t)j * ldb] : T(0);
                }
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
            }
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int j = j0 + tc + b;
                if (j >= nn) continue;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const int i = i0 + tr + a;
                    if (i >= mm || (lower && i < j)) continue;
                    T *c = C + (size_t)i + (size_t)j * ldc;
                    *c = *c - acc[a][b];
                }
            }
        }
    }
    __syncthreads();
}

// In-place LU of one n x n matrix (n <= kBMaxN) with the pivot rule of the
// tournament for a single leaf (partial pivoting, ties to the smallest
// position), block size vb.  Same step structure as cf_getrf.
template <typename T>
__device__ void cta_getrf(BSmem<T> &s, T *A, int n, int lda, int *ipiv, int *info, int vb) {
    const int tid = threadIdx.x;
    T *P = bsmem_panel(s);
    for (int k0 = 0; k0 < n; k0 += vb) {
        const int w = min(vb, n - k0), m = n - k0;
        T *A00 = A + k0 + (size_t)k0 * lda;
        // ---- LU-1: partial-pivoting selection on a copy of the panel
        for (int e = tid; e < m * w; e += kBT) {
            const int r = e % m, c = e / m;
            P[c * m + r] = A00[r + (size_t)c * lda];
        }
        for (int r = tid; r < m; r += kBT) s.used[r] = 0;
        __syncthreads();
        // One barrier per column: a thread reads and writes only its own
        // rows (r = tid mod kBT) and marks its own row when it wins; the
        // pivot row, final since its owner's update of the previous column,
        // is read by all after the column's barrier and written by no one.
        for (int j = 0; j < w; ++j) {
            T bv = T(-1);
            int bi = INT_MAX;
            for (int r = tid; r < m; r += kBT)
                if (!s.used[r]) bbetter(bv, bi, bkey(P[j * m + r]), r);
            cta_argmax_1bar(s, bv, bi, j & 1);
            if (tid == 0) s.order[j] = bi;
            if (bi % kBT == tid) s.used[bi] = 1;
            const T piv = P[j * m + bi];
            if (piv != T(0)) {
                for (int r = tid; r < m; r += kBT) {
                    if (s.used[r]) continue;
                    const T l = P[j * m + r] / piv;
                    for (int c = j + 1; c < w; ++c) P[c * m + r] = P[c * m + r] - l * P[c * m + bi];
                }
            }
        }
        __syncthreads();
        // ---- LU-2: interchanges (positions of the winners, as cf_getrf)
        for (int r = tid; r < m; r += kBT) { s.lab[r] = r; s.where_[r] = r; }
        __syncthreads();
        if (tid == 0) {
            for (int j = 0; j < w; ++j) {
                const int lab = s.order[j], p = s.where_[lab];
                ipiv[k0 + j] = k0 + p + 1;
                s.order[j] = p;                          // the swap partner, for the column loop
                if (p != j) {
                    const int lj = s.lab[j];
                    s.lab[j] = lab; s.where_[lab] = j;
                    s.lab[p] = lj;  s.where_[lj] = p;
                }
            }
        }
        __syncthreads();
        for (int c = tid; c < n; c += kBT) {
            T *col = A + (size_t)c * lda;
            for (int j = 0; j < w; ++j) {
                const int p = k0 + s.order[j];
                if (p != k0 + j) { const T t = col[k0 + j]; col[k0 + j] = col[p]; col[p] = t; }
            }
        }
        __syncthreads();
        // ---- A00 = L00 U00 (no pivoting) in shared memory
        for (int e = tid; e < w * w; e += kBT) {
            const int r = e % w, c = e / w;
            s.D[c * (kBMaxV + 1) + r] = A00[r + (size_t)c * lda];
        }
        __syncthreads();
        for (int k = 0; k < w; ++k) {
            const T piv = s.D[k * (kBMaxV + 1) + k];
            if (piv == T(0) && tid == 0) atomicCAS(info, 0, k0 + k + 1);
            __syncthreads();
            for (int e = tid; e < (w - k - 1); e += kBT) {
                const int r = k + 1 + e;
                if (piv != T(0)) s.D[k * (kBMaxV + 1) + r] = s.D[k * (kBMaxV + 1) + r] / piv;
            }
            __syncthreads();
            const int rem = w - k - 1;
            for (int e = tid; e < rem * rem; e += kBT) {
                const int r = k + 1 + e % rem, c = k + 1 + e / rem;
                s.D[c * (kBMaxV + 1) + r] -= s.D[k * (kBMaxV + 1) + r] * s.D[c * (kBMaxV + 1) + k];
            }
            __syncthreads();
        }
        for (int e = tid; e < w * w; e += kBT) {
            const int r = e % w, c = e / w;
            A00[r + (size_t)c * lda] = s.D[c * (kBMaxV + 1) + r];
        }
        // ---- LU-3: A10 <- A10 U00^{-1} (one row per thread, held in registers:
        // every element gets the same operations in the same order as in
        // place, without a trip through memory per multiply-add)
        for (int r = w + tid; r < m; r += kBT) {
            T *row = A00 + r;
            T v[kBMaxV];
#pragma unroll
            for (int k = 0; k < kBMaxV; ++k) v[k] = k < w ? row[(size_t)k * lda] : T(0);
#pragma unroll
            for (int k = 0; k < kBMaxV; ++k) {
                if (k < w) {
                    const T ukk = s.D[k * (kBMaxV + 1) + k];
                    T x = v[k];
                    if (ukk != T(0)) x = x / ukk;
                    v[k] = x;
#pragma unroll
                    for (int j = k + 1; j < kBMaxV; ++j)
                        if (j < w) v[j] -= x * s.D[j * (kBMaxV + 1) + k];
                }
            }
#pragma unroll
            for (int k = 0; k < kBMaxV; ++k)
                if (k < w) row[(size_t)k * lda] = v[k];
        }
        // ---- LU-4: A01 <- L00^{-1} A01 (one column per thread, in registers)
        for (int c = w + tid; c < m; c += kBT) {
            T *col = A00 + (size_t)c * lda;
            T v[kBMaxV];
#pragma unroll
            for (int i = 0; i < kBMaxV; ++i) v[i] = i < w ? col[i] : T(0);
#pragma unroll
            for (int k = 0; k < kBMaxV; ++k) {
                if (k < w) {
                    const T xk = v[k];
#pragma unroll
                    for (int i = k + 1; i < kBMaxV; ++i)
                        if (i < w) v[i] -= s.D[k * (kBMaxV + 1) + i] * xk;
                }
            }
#pragma unroll
            for (int i = 0; i < kBMaxV; ++i)
                if (i < w) col[i] = v[i];
        }
        __syncthreads();
        // ---- LU-5: A11 <- A11 - A10 A01
        if (m > w) cta_gemm_sub<T>(m - w, m - w, w, A00 + w, lda, A00 + (size_t)w * lda, lda,
                                   A00 + w + (size_t)w * lda, lda, false);
        __syncthreads();
    }
}

// In-place Cholesky (lower) of one matrix, block size vb.  Returns nonzero
// (and sets *info) on a non-positive pivot.
template <typename T>
__device__ int cta_potrf(BSmem<T> &s, T *A, int n, int lda, int *info, int vb) {
    const int tid = threadIdx.x;
    if (tid == 0) s.fail = 0;
    __syncthreads();
    for (int k0 = 0; k0 < n; k0 += vb) {
        const int w = min(vb, n - k0), m = n - k0;
        T *A00 = A + k0 + (size_t)k0 * lda;
        for (int e = tid; e < w * w; e += kBT) {
            const int r = e % w, c = e / w;
            if (r >= c) s.D[c * (kBMaxV + 1) + r] = A00[r + (size_t)c * lda];
        }
        __syncthreads();
        for (int k = 0; k < w; ++k) {
            const T d = s.D[k * (kBMaxV + 1) + k];
            if (!(d > T(0))) {
                if (tid == 0) { s.fail = 1; atomicCAS(info, 0, k0 + k + 1); }
                __syncthreads();
                return 1;
            }
            const T lkk = sqrt(d);
            __syncthreads();
            if (tid == 0) s.D[k * (kBMaxV + 1) + k] = lkk;
            for (int r = k + 1 + tid; r < w; r += kBT) s.D[k * (kBMaxV + 1) + r] /= lkk;
            __syncthreads();
            const int rem = w - k - 1;
            for (int e = tid; e < rem * rem; e += kBT) {
                const int r = k + 1 + e % rem, c = k + 1 + e / rem;
                if (r >= c) s.D[c * (kBMaxV + 1) + r] -= s.D[k * (kBMaxV + 1) + r] * s.D[k * (kBMaxV + 1) + c];
            }
            __syncthreads();
        }
        for (int e = tid; e < w * w; e += kBT) {
            const int r = e % w, c = e / w;
            if (r >= c) A00[r + (size_t)c * lda] = s.D[c * (kBMaxV + 1) + r];
        }
        // CH-2: L10 <- A10 L00^{-T} (one row per thread, held in registers)
        for (int r = w + tid; r < m; r += kBT) {
            T *row = A00 + r;
            T v[kBMaxV];
#pragma unroll
            for (int k = 0; k < kBMaxV; ++k) v[k] = k < w ? row[(size_t)k * lda] : T(0);
#pragma unroll
            for (int k = 0; k < kBMaxV; ++k) {
                if (k < w) {
                    const T x = v[k] / s.D[k * (kBMaxV + 1) + k];
                    v[k] = x;
#pragma unroll
                    for (int j = k + 1; j < kBMaxV; ++j)
                        if (j < w) v[j] -= x * s.D[k * (kBMaxV + 1) + j];
                }
            }
#pragma unroll
            for (int k = 0; k < kBMaxV; ++k)
                if (k < w) row[(size_t)k * lda] = v[k];
        }
        __syncthreads();
        // CH-3: A11 <- A11 - L10 L10^T (lower); B operand = L10^T read from A
        if (m > w) {
            // stage L10^T? read directly: B(p, j) = L10(j, p) = A00[w + j + p*lda]
            const int mm = m - w;
            T *C = A00 + w + (size_t)w * lda;
            const int tr = (tid & 15) * 4, tc = (tid >> 4) * 4;
            for (int j0 = 0; j0 < mm; j0 += 64)
                for (int i0 = j0; i0 < mm; i0 += 64) {
                    T acc[4][4];
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b] = T(0);
                    for (int p = 0; p < w; ++p) {
                        T av[4], bv[4];
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            const int i = i0 + tr + a;
                            av[a] = i < mm ? A00[w + i + (size_t)p * lda] : T(0);
                        }
#pragma unroll
                        for (int b = 0; b < 4; ++b) {
                            const int j = j0 + tc + b;
                            bv[b] = j < mm ? A00[w + j + (size_t)p * lda] : T(0);
                        }
#pragma unroll
                        for (int a = 0; a < 4; ++a)
#pragma unroll
                            for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
                    }
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int j = j0 + tc + b;
                        if (j >= mm) continue;
#pragma unroll
                        for (int a = 0; a < 4; ++a) {
                            const int i = i0 + tr + a;
                            if (i >= mm || i < j) continue;
                            C[(size_t)i + (size_t)j * lda] -= acc[a][b];
                        }
                    }
                }
        }
        __syncthreads();
    }
    return 0;
}

// Per-CTA scratch of the mixed solve: the n x n factors (FP64 room), r and
// the pivots, rounded to 1 KiB (the corrections' right-hand side lives in
// shared memory).
__host__ __device__ constexpr size_t batched_scratch_bytes_per_cta() {
    return ((sizeof(double) * ((size_t)kBMaxN * kBMaxN + kBMaxN) + sizeof(int) * kBMaxN) + 1023) / 1024 * 1024;
}

struct BatchArgs {
    int batch;
    const int *kind;          // per matrix: 0 LU, 1 Cholesky (null: all default_kind)
    int default_kind;
    const int *n;
    const int *lda;
    double *const *A;
    int *const *ipiv;         // LU only (may be null for all-Cholesky batches)
    int *info;
    const int *order;         // processing order
    int *queue;               // atomic counter, zero before the launch
    int vb;
    // mixed solve
    const double *const *B;
    double *const *X;
    int *iters;
    double *eta;
    int *solver;              // optional: 32 or 64, precision of the factors used
    double *scratch;          // per CTA: batched_scratch_bytes_per_cta()
    double tol;
    int max_iter;
};

// ---------------------------------------------------------------------------
// FP64 factorizations in place.
// ---------------------------------------------------------------------------
template <int MINB>
__global__ void __launch_bounds__(kBT, MINB) k_factor_batched(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BSmem<double> &s = *reinterpret_cast<BSmem<double> *>(smem_raw);
    __shared__ int s_idx;
    while (true) {
        if (threadIdx.x == 0) s_idx = atomicAdd(a.queue, 1);
        __syncthreads();
        const int q = s_idx;
        __syncthreads();
        if (q >= a.batch) return;
        const int i = a.order ? a.order[q] : q;
        const int n = a.n[i];
        const int kind = a.kind ? a.kind[i] : a.default_kind;
        if (threadIdx.x == 0) a.info[i] = 0;
        __syncthreads();
        if (n <= 0 || n > kBMaxN) {
            if (threadIdx.x == 0 && n > kBMaxN) a.info[i] = -1;
            continue;
        }
        if (kind == 0) cta_getrf<double>(s, a.A[i], n, a.lda[i], a.ipiv[i], a.info + i, a.vb);
        else cta_potrf<double>(s, a.A[i], n, a.lda[i], a.info + i, a.vb);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Mixed solve per matrix: FP32 factors in the CTA's scratch, FP64 refinement;
// if the FP32 factors cannot bring eta to the tolerance (factorization
// breakdown, contraction of eta slower than 1/2 per step, or max_iter), the
// matrix is refactored in FP64 in the same scratch and refinement continues
// from the current iterate (the fallback of LAPACK's dsgesv, per matrix).
// ---------------------------------------------------------------------------
__device__ double cta_max(double v, double *s_red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    v = s_red[0];
#pragma unroll
    for (int q = 1; q < kBT / 32; ++q) v = fmax(v, s_red[q]);
    __syncthreads();
    return v;
}

// r = b - A x (FP64, one row per thread); returns the componentwise-normwise
// backward error ||r||_inf / (||A||_inf ||x||_inf + ||b||_inf).
__device__ double cta_residual_eta(int n, const double *A, int lda, const double *b, const double *x, double *r,
                                   double an, double bn, double *s_red) {
    const int tid = threadIdx.x;
    double rn = 0.0, xn = 0.0;
    for (int row = tid; row < n; row += kBT) {
        double sum = 0.0;
        for (int c = 0; c < n; ++c) sum = fma(A[(size_t)row + (size_t)c * lda], x[c], sum);
        r[row] = b[row] - sum;
        rn = fmax(rn, fabs(r[row]));
    }
    for (int row = tid; row < n; row += kBT) xn = fmax(xn, fabs(x[row]));
    rn = cta_max(rn, s_red);
    xn = cta_max(xn, s_red);
    const double den = an * xn + bn;
    if (rn != rn) return rn;                       // NaN stays NaN (never converged)
    return den > 0.0 ? rn / den : (rn > 0.0 ? 1.0 : 0.0);
}

// x += (P^T L U)^{-1} r (kind 0) or (L L^T)^{-1} r (kind 1), the solve in the
// factor precision T on r scaled by 1/||r||_inf.  The right-hand side d lives
// in shared memory (sd; spiv holds the pivots for the interchanges) and the
// substitutions go by blocks of 32 rows: one warp solves the block's
// triangle with the row in a register, each column's value handed to the
// other lanes by a shuffle (no CTA barrier), then the CTA applies the
// block's columns to the rows not yet solved: two barriers per block of 32
// rows instead of two per row, and no round trip through global memory per
// row.  Every row receives the same fused multiply-adds, with the same
// operands, in the same order as in a row-by-row substitution (columns in
// increasing order for L, decreasing for U / L^T), so the result is the
// same to the bit.
template <typename T>
__device__ void cta_correct(int kind, int n, const T *W, const int *piv, const double *r, T *sd, int *spiv,
                            double *x, double *s_red) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double rn = 0.0;
    for (int row = tid; row < n; row += kBT) rn = fmax(rn, fabs(r[row]));
    rn = cta_max(rn, s_red);
    const double sc = rn > 0.0 ? rn : 1.0;
    for (int row = tid; row < n; row += kBT) sd[row] = (T)(r[row] / sc);
    if (kind == 0)
        for (int j = tid; j < n; j += kBT) spiv[j] = piv[j];
    __syncthreads();
    if (kind == 0 && tid == 0) {
        for (int j = 0; j < n; ++j) {                // row interchanges, in order
            const int p = spiv[j] - 1;
            if (p != j) { const T t = sd[j]; sd[j] = sd[p]; sd[p] = t; }
        }
    }
    __syncthreads();
    // L y = d (unit diagonal for LU), blocks from the top
    for (int b0 = 0; b0 < n; b0 += 32) {
        const int bw = min(32, n - b0);
        if (warp == 0) {
            T v = lane < bw ? sd[b0 + lane] : T(0);
            for (int k = 0; k < bw; ++k) {
                if (kind == 1 && lane == k) v = v / W[(size_t)(b0 + k) * n + b0 + k];
                const T dk = __shfl_sync(0xffffffffu, v, k);
                if (lane > k && lane < bw) v = fma(-W[(size_t)(b0 + k) * n + b0 + lane], dk, v);
            }
            if (lane < bw) sd[b0 + lane] = v;
        }
        __syncthreads();
        for (int row = b0 + bw + tid; row < n; row += kBT) {
            T acc = sd[row];
            for (int k = 0; k < bw; ++k) acc = fma(-W[(size_t)(b0 + k) * n + row], sd[b0 + k], acc);
            sd[row] = acc;
        }
        __syncthreads();
    }
    // U z = y (LU) or L^T z = y (Cholesky), blocks from the bottom
    for (int be = n; be > 0; be -= 32) {
        const int b0 = be > 32 ? be - 32 : 0, bw = be - b0;
        if (warp == 0) {
            T v = lane < bw ? sd[b0 + lane] : T(0);
            for (int k = bw - 1; k >= 0; --k) {
                if (lane == k) v = v / W[(size_t)(b0 + k) * n + b0 + k];
                const T dk = __shfl_sync(0xffffffffu, v, k);
                if (lane < k) {
                    const T u = (kind == 0) ? W[(size_t)(b0 + k) * n + b0 + lane] : W[(size_t)(b0 + lane) * n + b0 + k];
                    v = fma(-u, dk, v);
                }
            }
            if (lane < bw) sd[b0 + lane] = v;
        }
        __syncthreads();
        for (int row = tid; row < b0; row += kBT) {
            T acc = sd[row];
            for (int k = bw - 1; k >= 0; --k) {
                const T u = (kind == 0) ? W[(size_t)(b0 + k) * n + row] : W[(size_t)row * n + b0 + k];
                acc = fma(-u, sd[b0 + k], acc);
            }
            sd[row] = acc;
        }
        __syncthreads();
    }
    for (int row = tid; row < n; row += kBT) x[row] += sc * (double)sd[row];
    __syncthreads();
}

// Factors fl_T(A) into W (ld n).  Returns nonzero on breakdown; *info gets
// the first bad pivot (1-based) as the FP64 routines report it.
template <typename T>
__device__ int cta_factor_copy(unsigned char *smem_raw, int kind, int n, const double *A, int lda, T *W, int *piv,
                               int *info, int vb) {
    const int tid = threadIdx.x;
    for (int e = tid; e < n * n; e += kBT) W[e] = (T)A[(size_t)(e % n) + (size_t)(e / n) * lda];
    if (tid == 0) *info = 0;
    __syncthreads();
    BSmem<T> &s = *reinterpret_cast<BSmem<T> *>(smem_raw);
    int fail = 0;
    if (kind == 0) cta_getrf<T>(s, W, n, n, piv, info, vb);
    else fail = cta_potrf<T>(s, W, n, n, info, vb);
    __syncthreads();
    return fail || *info != 0;
}

// Refinement steps with factors W until eta <= tol (returns 0), it reaches
// it_end, or eta fails to halve in one step (returns 1).  r and eta hold the
// residual of x on entry and on exit.
template <typename T>
__device__ int cta_refine(int kind, int n, const double *A, int lda, const double *b, double *x, const T *W,
                          const int *piv, double *r, T *sd, int *spiv, double an, double bn, double tol, int &it,
                          int it_end, double &eta, double *s_red) {
    double prev = -1.0;
    while (true) {
        if (eta <= tol) return 0;
        if (it >= it_end) return 1;
        if (prev >= 0.0 && !(eta <= 0.5 * prev)) return 1;      // stalled (or NaN)
        cta_correct<T>(kind, n, W, piv, r, sd, spiv, x, s_red);
        ++it;
        prev = eta;
        eta = cta_residual_eta(n, A, lda, b, x, r, an, bn, s_red);
    }
}

template <int MINB>
__global__ void __launch_bounds__(kBT, MINB) k_solve_batched_mixed(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_idx;
    __shared__ int s_info;
    __shared__ double s_red[kBT / 32];
    unsigned char *base = reinterpret_cast<unsigned char *>(a.scratch) + batched_scratch_bytes_per_cta() * blockIdx.x;
    void *W = base;                                                          // n x n, FP32 or FP64
    double *r = reinterpret_cast<double *>(base + sizeof(double) * kBMaxN * kBMaxN);
    int *piv = reinterpret_cast<int *>(r + kBMaxN);
    const int tid = threadIdx.x;
    while (true) {
        if (tid == 0) s_idx = atomicAdd(a.queue, 1);
        __syncthreads();
        const int q = s_idx;
        __syncthreads();
        if (q >= a.batch) return;
        const int i = a.order ? a.order[q] : q;
        const int n = a.n[i], lda = a.lda[i];
        const int kind = a.kind ? a.kind[i] : a.default_kind;
        const double *A = a.A[i];
        const double *b = a.B[i];
        double *x = a.X[i];
        if (tid == 0) {
            a.info[i] = 0; a.iters[i] = 0; a.eta[i] = 0.0;
            if (a.solver) a.solver[i] = 32;
        }
        __syncthreads();
        if (n <= 0 || n > kBMaxN) {
            if (tid == 0 && n > kBMaxN) a.info[i] = -1;
            continue;
        }
        // ||A||_inf and ||b||_inf
        double an = 0.0, bn = 0.0;
        for (int row = tid; row < n; row += kBT) {
            double sum = 0.0;
            for (int c = 0; c < n; ++c) sum += fabs(A[(size_t)row + (size_t)c * lda]);
            an = fmax(an, sum);
            bn = fmax(bn, fabs(b[row]));
        }
        an = cta_max(an, s_red);
        bn = cta_max(bn, s_red);
        for (int row = tid; row < n; row += kBT) x[row] = 0.0;
        __syncthreads();
        double eta = cta_residual_eta(n, A, lda, b, x, r, an, bn, s_red);
        int it = 0;
        int bad = cta_factor_copy<float>(smem_raw, kind, n, A, lda, static_cast<float *>(W), piv, &s_info, a.vb);
        // the right-hand side of the corrections and the pivots in shared
        // memory: the panel copy and the label array of the factorization,
        // free until the next matrix
        BSmem<float> &sf = *reinterpret_cast<BSmem<float> *>(smem_raw);
        if (!bad)
            bad = cta_refine<float>(kind, n, A, lda, b, x, static_cast<const float *>(W), piv, r, bsmem_panel(sf),
                                    sf.lab, an, bn, a.tol, it, a.max_iter, eta, s_red);
        if (bad) {
            // FP64 factors; refinement resumes from the current iterate unless
            // it is not finite
            if (tid == 0 && a.solver) a.solver[i] = 64;
            if (!(eta < 1.0)) {
                for (int row = tid; row < n; row += kBT) x[row] = 0.0;
                __syncthreads();
                eta = cta_residual_eta(n, A, lda, b, x, r, an, bn, s_red);
            }
            if (cta_factor_copy<double>(smem_raw, kind, n, A, lda, static_cast<double *>(W), piv, &s_info, a.vb)) {
                if (tid == 0) a.info[i] = s_info;
            } else {
                BSmem<double> &sdb = *reinterpret_cast<BSmem<double> *>(smem_raw);
                cta_refine<double>(kind, n, A, lda, b, x, static_cast<const double *>(W), piv, r, bsmem_panel(sdb),
                                   sdb.lab, an, bn, a.tol, it, it + a.max_iter, eta, s_red);
            }
        }
        if (tid == 0) { a.iters[i] = it; a.eta[i] = eta; }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Host side: LPT order (sort by decreasing n, counting sort over n <= 512)
// ---------------------------------------------------------------------------
__global__ void k_lpt_histogram(int batch, const int *n, int *hist) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < batch; i += gridDim.x * blockDim.x) {
        int v = n[i];
        v = v < 0 ? 0 : (v > kBMaxN ? kBMaxN : v);
        atomicAdd(hist + (kBMaxN - v), 1);           // bucket 0 = largest n
    }
}

__global__ void k_lpt_scan(int *hist, int *cursor) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int sum = 0;
        for (int b = 0; b <= kBMaxN; ++b) { cursor[b] = sum; sum += hist[b]; }
    }
}

__global__ void k_lpt_scatter(int batch, const int *n, int *cursor, int *order) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < batch; i += gridDim.x * blockDim.x) {
        int v = n[i];
        v = v < 0 ? 0 : (v > kBMaxN ? kBMaxN : v);
        order[atomicAdd(cursor + (kBMaxN - v), 1)] = i;
    }
}

struct BatchWS {
    int *order, *queue, *hist, *cursor;
    double *scratch;
    size_t bytes;
};

static int sm_count_b() { return device_sm_count(); }

// Launch configuration: block size vb and resident CTAs per SM (cps).  The
// kernel variant compiled for cps resident CTAs is used; cps = 0 asks for
// the largest count the occupancy calculator grants at this vb.
struct BatchCfg {
    int vb, cps, grid;
};

template <int MINB>
static int occ_factor(size_t smem) {
    int b = 0;
    if (cudaFuncSetAttribute(k_factor_batched<MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_factor_batched<MINB>, kBT, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return b;
}
template <int MINB>
static int occ_mixed(size_t smem) {
    int b = 0;
    if (cudaFuncSetAttribute(k_solve_batched_mixed<MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_solve_batched_mixed<MINB>, kBT, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return b;
}

constexpr int kMaxCpsFactor = 3, kMaxCpsMixed = 2;

static BatchCfg resolve_cfg(const Opts &o, bool mixed) {
    BatchCfg c{};
    c.vb = o.v < kBMaxV ? o.v : kBMaxV;
    const size_t smem = bsmem_bytes<double>(c.vb);
    const int maxc = mixed ? kMaxCpsMixed : kMaxCpsFactor;
    int want = o.batch_cps > 0 ? (o.batch_cps < maxc ? o.batch_cps : maxc) : maxc;
    // largest cps <= want whose variant the hardware can hold that many times
    int cps = 1;
    for (int k = want; k >= 1; --k) {
        int occ = 0;
        if (mixed) occ = k == 2 ? occ_mixed<2>(smem) : occ_mixed<1>(smem);
        else occ = k == 3 ? occ_factor<3>(smem) : k == 2 ? occ_factor<2>(smem) : occ_factor<1>(smem);
        if (occ >= k) { cps = k; break; }
    }
    c.cps = cps;
    c.grid = sm_count_b() * cps;
    return c;
}

static int carve_batch(void *work, int batch, bool mixed, int grid, BatchWS *w) {
    Carver cv(work);
    w->order = cv.take<int>(batch > 0 ? batch : 1);
    w->queue = cv.take<int>(1);
    w->hist = cv.take<int>(kBMaxN + 1);
    w->cursor = cv.take<int>(kBMaxN + 1);
    w->scratch = mixed ? cv.take<double>(batched_scratch_bytes_per_cta() / sizeof(double) * (size_t)grid, 1024)
                       : nullptr;
    w->bytes = cv.size();
    return CF_OK;
}

static int enqueue_order(int batch, const int *n, BatchWS &w, cudaStream_t st) {
    CF_CUDA_TRY(cudaMemsetAsync(w.hist, 0, sizeof(int) * (kBMaxN + 1), st));
    CF_CUDA_TRY(cudaMemsetAsync(w.queue, 0, sizeof(int), st));
    k_lpt_histogram<<<ceil_div(batch, 256) < 1024 ? ceil_div(batch, 256) : 1024, 256, 0, st>>>(batch, n, w.hist);
    CF_LAUNCH_CHECK();
    k_lpt_scan<<<1, 32, 0, st>>>(w.hist, w.cursor);
    CF_LAUNCH_CHECK();
    k_lpt_scatter<<<ceil_div(batch, 256) < 1024 ? ceil_div(batch, 256) : 1024, 256, 0, st>>>(batch, n, w.cursor,
                                                                                          w.order);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

static int launch_factor_cfg(const BatchArgs &a, const BatchCfg &c, cudaStream_t st) {
    const size_t smem = bsmem_bytes<double>(c.vb);
    switch (c.cps) {
        case 3:
            CF_CUDA_TRY(cudaFuncSetAttribute(k_factor_batched<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_factor_batched<3><<<c.grid, kBT, smem, st>>>(a);
            break;
        case 2:
            CF_CUDA_TRY(cudaFuncSetAttribute(k_factor_batched<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_factor_batched<2><<<c.grid, kBT, smem, st>>>(a);
            break;
        default:
            CF_CUDA_TRY(cudaFuncSetAttribute(k_factor_batched<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_factor_batched<1><<<c.grid, kBT, smem, st>>>(a);
    }
    CF_LAUNCH_CHECK();
    return CF_OK;
}

static int launch_mixed_cfg(const BatchArgs &a, const BatchCfg &c, cudaStream_t st) {
    const size_t smem = bsmem_bytes<double>(c.vb);   // holds the FP32 layout too
    if (c.cps == 2) {
        CF_CUDA_TRY(cudaFuncSetAttribute(k_solve_batched_mixed<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_solve_batched_mixed<2><<<c.grid, kBT, smem, st>>>(a);
    } else {
        CF_CUDA_TRY(cudaFuncSetAttribute(k_solve_batched_mixed<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_solve_batched_mixed<1><<<c.grid, kBT, smem, st>>>(a);
    }
    CF_LAUNCH_CHECK();
    return CF_OK;
}

static size_t factor_ws_bytes(int batch, const Opts &o) {
    BatchWS w{};
    carve_batch(nullptr, batch, false, resolve_cfg(o, false).grid, &w);
    return w.bytes;
}
static size_t mixed_ws_bytes(int batch, const Opts &o) {
    BatchWS w{};
    carve_batch(nullptr, batch, true, resolve_cfg(o, true).grid, &w);
    return w.bytes;
}

// ---------------------------------------------------------------------------
// Autotuner input: synthetic matrices of the sampled sizes, diagonally
// dominant (u[-1,1] entries from a counter-based hash, n on the diagonal),
// symmetric for Cholesky entries, so every candidate factors the same bytes.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double hash_u11(unsigned long long key) {
    // SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) finaliser -> [-1, 1)
    key += 0x9E3779B97F4A7C15ull;
    key = (key ^ (key >> 30)) * 0xBF58476D1CE4E5B9ull;
    key = (key ^ (key >> 27)) * 0x94D049BB133111EBull;
    key ^= key >> 31;
    return (double)(key >> 11) * 0x1p-52 - 1.0;
}

__global__ void k_tune_fill(int cnt, const int *n, const long long *off, const long long *voff, const int *kind,
                            double *pool, double *vpool) {
    const int j = blockIdx.y;
    if (j >= cnt) return;
    const int nj = n[j];
    double *A = pool + off[j];
    const long long tot = (long long)nj * nj;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e % nj), c = (int)(e / nj);
        const int lo = (kind[j] == 1 && c < r) ? c : r, hi = (kind[j] == 1 && c < r) ? r : c;
        const unsigned long long key = ((unsigned long long)j << 40) ^ ((unsigned long long)lo << 20) ^ (unsigned long long)hi;
        A[e] = hash_u11(key) + (r == c ? (double)nj : 0.0);
    }
    if (vpool != nullptr && blockIdx.x == 0)
        for (int r = threadIdx.x; r < nj; r += blockDim.x)
            vpool[voff[j] + r] = hash_u11(0xB000000000000000ull ^ ((unsigned long long)j << 20) ^ (unsigned long long)r);
}

}  // namespace cf

using namespace cf;

extern "C" size_t cf_factor_batched_workspace_size(int batch, const cf_options *opt) {
    Opts o;
    if (resolve_options(opt, &o) != CF_OK) return 0;
    return factor_ws_bytes(batch, o);
}

extern "C" int cf_factor_batched(int batch, const int *kind, int default_kind, const int *n, double *const *A,
                                 const int *lda, int *const *ipiv, int *info, void *work, size_t lwork,
                                 const cf_options *opt, cudaStream_t st) {
    if (batch < 0) return -1;
    if (default_kind != 0 && default_kind != 1) return -3;
    if (batch > 0) {
        if (n == nullptr) return -4;
        if (A == nullptr) return -5;
        if (lda == nullptr) return -6;
        if (ipiv == nullptr && (kind != nullptr || default_kind == 0)) return -7;   // some matrix may be LU
        if (info == nullptr) return -8;
    }
    Opts o;
    int rc = resolve_options(opt, &o);
    if (rc) return rc;
    if (batch == 0) return CF_OK;
    const BatchCfg c = resolve_cfg(o, false);
    BatchWS w{};
    carve_batch(nullptr, batch, false, c.grid, &w);
    if (work == nullptr || lwork < w.bytes) return CF_ERR_WORKSPACE;
    carve_batch(work, batch, false, c.grid, &w);
    if ((rc = enqueue_order(batch, n, w, st))) return rc;
    BatchArgs a{};
    a.batch = batch; a.kind = kind; a.default_kind = default_kind; a.n = n; a.lda = lda; a.A = A;
    a.ipiv = ipiv; a.info = info; a.order = w.order; a.queue = w.queue;
    a.vb = c.vb;
    return launch_factor_cfg(a, c, st);
}

extern "C" size_t cf_getrf_batched_workspace_size(int batch, const cf_options *opt) {
    return cf_factor_batched_workspace_size(batch, opt);
}
extern "C" size_t cf_potrf_batched_workspace_size(int batch, const cf_options *opt) {
    return cf_factor_batched_workspace_size(batch, opt);
}

extern "C" int cf_getrf_batched(int batch, const int *n, double *const *A, const int *lda, int *const *ipiv,
                                int *info, void *work, size_t lwork, const cf_options *opt, cudaStream_t st) {
    if (batch < 0) return -1;
    if (batch > 0) {                 // this entry point's own argument numbers
        if (n == nullptr) return -2;
        if (A == nullptr) return -3;
        if (lda == nullptr) return -4;
        if (ipiv == nullptr) return -5;
        if (info == nullptr) return -6;
    }
    return cf_factor_batched(batch, nullptr, 0, n, A, lda, ipiv, info, work, lwork, opt, st);
}

extern "C" int cf_potrf_batched(int batch, const int *n, double *const *A, const int *lda, int *info, void *work,
                                size_t lwork, const cf_options *opt, cudaStream_t st) {
    if (batch < 0) return -1;
    if (batch > 0) {
        if (n == nullptr) return -2;
        if (A == nullptr) return -3;
        if (lda == nullptr) return -4;
        if (info == nullptr) return -5;
    }
    return cf_factor_batched(batch, nullptr, 1, n, A, lda, nullptr, info, work, lwork, opt, st);
}

extern "C" size_t cf_solve_batched_mixed_workspace_size(int batch, const cf_options *opt) {
    Opts o;
    if (resolve_options(opt, &o) != CF_OK) return 0;
    return mixed_ws_bytes(batch, o);
}

extern "C" int cf_solve_batched_mixed(int batch, const int *kind, int default_kind, const int *n,
                                      const double *const *A, const int *lda, const double *const *B,
                                      double *const *X, int *info, int *iters, double *eta, int *solver,
                                      void *work, size_t lwork, const cf_options *opt, cudaStream_t st) {
    if (batch < 0) return -1;
    if (default_kind != 0 && default_kind != 1) return -3;
    if (batch > 0) {
        if (n == nullptr) return -4;
        if (A == nullptr) return -5;
        if (lda == nullptr) return -6;
        if (B == nullptr) return -7;
        if (X == nullptr) return -8;
        if (info == nullptr) return -9;
        if (iters == nullptr) return -10;
        if (eta == nullptr) return -11;
    }
    Opts o;
    int rc = resolve_options(opt, &o);
    if (rc) return rc;
    if (batch == 0) return CF_OK;
    const BatchCfg c = resolve_cfg(o, true);
    BatchWS w{};
    carve_batch(nullptr, batch, true, c.grid, &w);
    if (work == nullptr || lwork < w.bytes) return CF_ERR_WORKSPACE;
    carve_batch(work, batch, true, c.grid, &w);
    if ((rc = enqueue_order(batch, n, w, st))) return rc;
    BatchArgs a{};
    a.batch = batch; a.kind = kind; a.default_kind = default_kind; a.n = n; a.lda = lda;
    a.A = const_cast<double *const *>(A);
    a.info = info; a.order = w.order; a.queue = w.queue;
    a.vb = c.vb;
    a.B = B; a.X = X; a.iters = iters; a.eta = eta; a.solver = solver; a.scratch = w.scratch;
    a.tol = o.tol; a.max_iter = o.max_iter;
    return launch_mixed_cfg(a, c, st);
}

// ---------------------------------------------------------------------------
// Autotuner (BAT-1): times every (block size, resident CTAs per SM) candidate
// on up to kTuneSample synthetic matrices whose sizes are an evenly spaced
// sample of the batch's, and returns the fastest in opt->v and
// opt->batch_cps.  Only the sizes and kinds of the batch are used.
// ---------------------------------------------------------------------------
namespace cf {
constexpr int kTuneSample = 512;

struct TuneLayout {
    int cnt;
    std::vector<int> n, kind, lda;
    std::vector<long long> off, voff;
    long long pool, vpool;
};

static TuneLayout tune_layout(int batch, const int *n_host, const int *kind_host, int default_kind) {
    TuneLayout L{};
    L.cnt = batch < kTuneSample ? batch : kTuneSample;
    long long acc = 0, vacc = 0;
    for (int j = 0; j < L.cnt; ++j) {
        const int i = (int)((long long)j * batch / L.cnt);
        int nj = n_host[i];
        nj = nj < 1 ? 1 : (nj > kBMaxN ? kBMaxN : nj);
        L.n.push_back(nj);
        L.kind.push_back(kind_host ? kind_host[i] : default_kind);
        L.lda.push_back(nj);
        L.off.push_back(acc);
        L.voff.push_back(vacc);
        acc += (long long)nj * nj;
        vacc += nj;
    }
    L.pool = acc;
    L.vpool = vacc;
    return L;
}

static size_t tune_ws_bytes(const TuneLayout &L, bool mixed) {
    Carver cv(nullptr);
    cv.take<double>((size_t)L.pool + 1, 256);                      // matrices
    cv.take<double>((size_t)L.vpool + 1, 256);                     // B
    cv.take<double>((size_t)L.vpool + 1, 256);                     // X
    cv.take<int>((size_t)L.vpool + 1);                             // ipiv
    cv.take<int>(4 * (size_t)L.cnt + 4);                           // n, lda, kind, info
    cv.take<int>(2 * (size_t)L.cnt + 2);                           // iters, solver
    cv.take<double>((size_t)L.cnt + 1);                            // eta
    cv.take<long long>(2 * (size_t)L.cnt + 2);                     // off, voff
    cv.take<double *>(3 * (size_t)L.cnt + 3);                      // A, B, X pointers
    cv.take<int *>((size_t)L.cnt + 1);                             // ipiv pointers
    // the batched call's own workspace at the largest candidate grid
    BatchWS w{};
    carve_batch(nullptr, L.cnt, mixed, sm_count_b() * (mixed ? kMaxCpsMixed : kMaxCpsFactor), &w);
    cv.take<unsigned char>(w.bytes, 1024);
    return cv.size();
}
}  // namespace cf

extern "C" size_t cf_batched_autotune_workspace_size(int batch, const int *n_host, const int *kind_host,
                                                     int default_kind, int mixed) {
    if (batch <= 0 || n_host == nullptr) return 0;
    return tune_ws_bytes(tune_layout(batch, n_host, kind_host, default_kind), mixed != 0);
}

extern "C" int cf_batched_autotune(int batch, const int *n_host, const int *kind_host, int default_kind, int mixed,
                                   void *work, size_t lwork, cf_options *opt, float *best_ms, cudaStream_t st) {
    if (batch <= 0) return -1;
    if (n_host == nullptr) return -2;
    if (default_kind != 0 && default_kind != 1) return -4;
    if (opt == nullptr) return -8;
    Opts o;
    int rc = resolve_options(opt, &o);
    if (rc) return rc;
    const TuneLayout L = tune_layout(batch, n_host, kind_host, default_kind);
    if (work == nullptr || lwork < tune_ws_bytes(L, mixed != 0)) return CF_ERR_WORKSPACE;
    Carver cv(work);
    double *pool = cv.take<double>((size_t)L.pool + 1, 256);
    double *vB = cv.take<double>((size_t)L.vpool + 1, 256);
    double *vX = cv.take<double>((size_t)L.vpool + 1, 256);
    int *piv = cv.take<int>((size_t)L.vpool + 1);
    int *d_n = cv.take<int>(4 * (size_t)L.cnt + 4);
    int *d_lda = d_n + L.cnt + 1, *d_kind = d_lda + L.cnt + 1, *d_info = d_kind + L.cnt + 1;
    int *d_it = cv.take<int>(2 * (size_t)L.cnt + 2);
    int *d_solver = d_it + L.cnt + 1;
    double *d_eta = cv.take<double>((size_t)L.cnt + 1);
    long long *d_off = cv.take<long long>(2 * (size_t)L.cnt + 2);
    long long *d_voff = d_off + L.cnt + 1;
    double **d_A = cv.take<double *>(3 * (size_t)L.cnt + 3);
    double **d_B = d_A + L.cnt + 1, **d_X = d_B + L.cnt + 1;
    int **d_piv = cv.take<int *>((size_t)L.cnt + 1);
    BatchWS wmax{};
    carve_batch(nullptr, L.cnt, mixed != 0, sm_count_b() * (mixed ? kMaxCpsMixed : kMaxCpsFactor), &wmax);
    unsigned char *bws = cv.take<unsigned char>(wmax.bytes, 1024);

    std::vector<double *> hA(L.cnt), hB(L.cnt), hX(L.cnt);
    std::vector<int *> hP(L.cnt);
    for (int j = 0; j < L.cnt; ++j) {
        hA[j] = pool + L.off[j];
        hB[j] = vB + L.voff[j];
        hX[j] = vX + L.voff[j];
        hP[j] = piv + L.voff[j];
    }
    CF_CUDA_TRY(cudaMemcpyAsync(d_n, L.n.data(), sizeof(int) * L.cnt, cudaMemcpyHostToDevice, st));
    CF_CUDA_TRY(cudaMemcpyAsync(d_lda, L.lda.data(), sizeof(int) * L.cnt, cudaMemcpyHostToDevice, st));
    CF_CUDA_TRY(cudaMemcpyAsync(d_kind, L.kind.data(), sizeof(int) * L.cnt, cudaMemcpyHostToDevice, st));
    CF_CUDA_TRY(cudaMemcpyAsync(d_off, L.off.data(), sizeof(long long) * L.cnt, cudaMemcpyHostToDevice, st));
    CF_CUDA_TRY(cudaMemcpyAsync(d_voff, L.voff.data(), sizeof(long long) * L.cnt, cudaMemcpyHostToDevice, st));
    CF_CUDA_TRY(cudaMemcpyAsync(d_A, hA.data(), sizeof(double *) * L.cnt, cudaMemcpyHostToDevice, st));
    CF_CUDA_TRY(cudaMemcpyAsync(d_B, hB.data(), sizeof(double *) * L.cnt, cudaMemcpyHostToDevice, st));
    CF_CUDA_TRY(cudaMemcpyAsync(d_X, hX.data(), sizeof(double *) * L.cnt, cudaMemcpyHostToDevice, st));
    CF_CUDA_TRY(cudaMemcpyAsync(d_piv, hP.data(), sizeof(int *) * L.cnt, cudaMemcpyHostToDevice, st));
    CF_CUDA_TRY(cudaStreamSynchronize(st));                      // host vectors go out of scope below

    ScopedEvent e0, e1;
    CF_CUDA_TRY(e0.create());
    CF_CUDA_TRY(e1.create());
    const int vbs[3] = {8, 16, 32};
    const int maxc = mixed ? kMaxCpsMixed : kMaxCpsFactor;
    float best = -1.f;
    int best_vb = o.v < kBMaxV ? o.v : kBMaxV, best_cps = 1;
    for (int pass = 0; pass < 2; ++pass) {                        // pass 0 warms up, pass 1 times
        for (int vi = 0; vi < 3; ++vi) {
            for (int cps = 1; cps <= maxc; ++cps) {
                Opts oc = o;
                oc.v = vbs[vi];
                oc.batch_cps = cps;
                const BatchCfg c = resolve_cfg(oc, mixed != 0);
                if (c.cps != cps) continue;                     // this many CTAs do not fit
                k_tune_fill<<<dim3(16, L.cnt), 256, 0, st>>>(L.cnt, d_n, d_off, d_voff, d_kind, pool,
                                                             mixed ? vB : nullptr);
                CF_LAUNCH_CHECK();
                BatchWS w{};
                carve_batch(bws, L.cnt, mixed != 0, c.grid, &w);
                if ((rc = enqueue_order(L.cnt, d_n, w, st))) return rc;
                BatchArgs a{};
                a.batch = L.cnt; a.kind = d_kind; a.default_kind = default_kind; a.n = d_n; a.lda = d_lda;
                a.A = d_A; a.ipiv = d_piv; a.info = d_info; a.order = w.order; a.queue = w.queue; a.vb = c.vb;
                a.B = d_B; a.X = d_X; a.iters = d_it; a.eta = d_eta; a.solver = d_solver; a.scratch = w.scratch;
                a.tol = o.tol; a.max_iter = o.max_iter;
                CF_CUDA_TRY(cudaEventRecord(e0, st));
                rc = mixed ? launch_mixed_cfg(a, c, st) : launch_factor_cfg(a, c, st);
                if (rc) return rc;
                CF_CUDA_TRY(cudaEventRecord(e1, st));
                CF_CUDA_TRY(cudaEventSynchronize(e1));
                float ms = 0.f;
                CF_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                if (pass == 1 && (best < 0.f || ms < best)) { best = ms; best_vb = c.vb; best_cps = c.cps; }
            }
        }
    }
    opt->v = best_vb;
    opt->batch_cps = best_cps;
    if (best_ms) *best_ms = best;
    return CF_OK;
}
