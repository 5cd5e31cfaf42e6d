// cf_gemm64.cu -- SIMT Schur-complement update (FP64; FP32 for the solves of
// the mixed path) and the FP64 residual.
//
//   LU-5 (FP64 path)  A11 <- A11 - A10 A01      (Alg. 1; Table 2 gemm)
//   CH-3 (FP64 path)  A11 <- A11 - L10 L10^T    (Table 2 gemmt, lower only)
//   S-1               block updates of the triangular solves
//   R-1               R = B - A X
//
// GB300 executes FP64 at about 1.2 TFLOP/s (measured: ~1.9 DFMA per clock per
// SM), two orders of magnitude below its BF16 tensor rate and far below what
// HBM could feed (the ridge is ~0.2 flop/byte).  These kernels are therefore
// DFMA-issue bound; they only need enough register blocking that shared
// memory and global loads stay off the critical path.
#include "cf_common.cuh"
#include "cf_kernels.cuh"

namespace cf {

constexpr int kBM = 64, kBN = 64, kBK = 16;
constexpr int kGemmThreads = 256;

// C[m x n] -= op(A)[m x k] * op(B)[k x n]
//   op(A)(i, p) = TA ? A[p + i*lda] : A[i + p*lda]
//   op(B)(p, j) = TB ? B[j + p*ldb] : B[p + j*ldb]
template <typename T, bool TA, bool TB, bool LOWER>
__global__ void __launch_bounds__(kGemmThreads)
k_gemm_sub(int m, int n, int k, const T *__restrict__ A, int lda, const T *__restrict__ B, int ldb,
           T *__restrict__ C, int ldc, const int *skip) {
    if (skip != nullptr && *skip != 0) return;
    const int bm = blockIdx.x * kBM, bn = blockIdx.y * kBN;
    if (LOWER && bn > bm + kBM - 1) return;      // tile strictly above the diagonal
    __shared__ __align__(16) T As[kBK][kBM + 2];
    __shared__ __align__(16) T Bs[kBK][kBN + 2];
    const int tid = threadIdx.x;
    const int tm = (tid & 15) * 4;               // 4 rows
    const int tn = (tid >> 4) * 4;               // 4 columns
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = T(0);

    for (int p0 = 0; p0 < k; p0 += kBK) {
#pragma unroll
        for (int e = 0; e < (kBM * kBK) / kGemmThreads; ++e) {
            const int idx = tid + e * kGemmThreads;
            int i, p;
            if (!TA) { i = idx % kBM; p = idx / kBM; } else { p = idx % kBK; i = idx / kBK; }
            const int gi = bm + i, gp = p0 + p;
            T v = T(0);
            if (gi < m && gp < k) v = TA ? A[(size_t)gp + (size_t)gi * lda] : A[(size_t)gi + (size_t)gp * lda];
            As[p][i] = v;
        }
#pragma unroll
        for (int e = 0; e < (kBN * kBK) / kGemmThreads; ++e) {
            const int idx = tid + e * kGemmThreads;
            int j, p;
            if (!TB) { p = idx % kBK; j = idx / kBK; } else { j = idx % kBN; p = idx / kBN; }
            const int gj = bn + j, gp = p0 + p;
            T v = T(0);
            if (gj < n && gp < k) v = TB ? B[(size_t)gj + (size_t)gp * ldb] : B[(size_t)gp + (size_t)gj * ldb];
            Bs[p][j] = v;
        }
        __syncthreads();
#pragma unroll
        for (int p = 0; p < kBK; ++p) {
            T a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[p][tm + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[p][tn + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int gj = bn + tn + j;
        if (gj >= n) continue;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int gi = bm + tm + i;
            if (gi >= m) continue;
            if (LOWER && gi < gj) continue;
            T *c = C + (size_t)gi + (size_t)gj * ldc;
            *c = *c - acc[i][j];
        }
    }
}

template <typename T>
int launch_gemm_sub_t(int m, int n, int k, const T *A, int lda, bool trans_a, const T *B, int ldb, bool trans_b,
                      T *C, int ldc, bool lower, const int *skip, cudaStream_t st) {
    if (m <= 0 || n <= 0 || k <= 0) return CF_OK;
    dim3 grid(ceil_div(m, kBM), ceil_div(n, kBN));
    if (grid.y > 65535) return CF_ERR_UNSUPPORTED;
#define CF_GEMM_CASE(TA, TB, LO)                                                                            \
    if (trans_a == TA && trans_b == TB && lower == LO) {                                                    \
        k_gemm_sub<T, TA, TB, LO><<<grid, kGemmThreads, 0, st>>>(m, n, k, A, lda, B, ldb, C, ldc, skip);   \
        CF_LAUNCH_CHECK();                                                                                  \
        return CF_OK;                                                                                       \
    }
    CF_GEMM_CASE(false, false, false)
    CF_GEMM_CASE(false, true, true)
    CF_GEMM_CASE(false, true, false)
    CF_GEMM_CASE(true, false, false)
#undef CF_GEMM_CASE
    return CF_ERR_UNSUPPORTED;
}
template int launch_gemm_sub_t<double>(int, int, int, const double *, int, bool, const double *, int, bool, double *,
                                       int, bool, const int *, cudaStream_t);
template int launch_gemm_sub_t<float>(int, int, int, const float *, int, bool, const float *, int, bool, float *, int,
                                      bool, const int *, cudaStream_t);

int launch_gemm_f64_sub_t(int m, int n, int k, const double *A, int lda, bool trans_a, const double *B, int ldb,
                          bool trans_b, double *C, int ldc, bool lower, const int *skip, cudaStream_t st) {
    return launch_gemm_sub_t<double>(m, n, k, A, lda, trans_a, B, ldb, trans_b, C, ldc, lower, skip, st);
}

int launch_gemm_f64_sub(int m, int n, int k, const double *A, int lda, const double *B, int ldb, bool trans_b,
                        double *C, int ldc, bool lower, const int *skip, cudaStream_t st) {
    return launch_gemm_f64_sub_t(m, n, k, A, lda, false, B, ldb, trans_b, C, ldc, lower, skip, st);
}

// ---------------------------------------------------------------------------
// R = B - A X (B null: R = A X), X thin (NR >= nrhs columns).  CTA: 4 RG rows;
// RG row groups of 4 rows x (256 / RG) lanes along k; the k-partial sums are
// combined in shared memory at the end in a fixed order.  Reads A once,
// coalesced along the columns.  RG = 16 (64 rows) or 8 (32 rows): the
// launcher picks the one whose grid fills the last wave of CTAs better (the
// kernel runs one CTA per SM, so a short last wave idles most SMs).
// ---------------------------------------------------------------------------
template <int NR, int RG>
__global__ void __launch_bounds__(256)
k_residual_f64(int m, int n, int nrhs, const double *__restrict__ A, int lda, const double *__restrict__ X, int ldx,
               const double *B, int ldb, double *R, int ldr) {
    constexpr int KL = 256 / RG, ROWS = 4 * RG;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double *red = reinterpret_cast<double *>(smem_raw);     // [KL][ROWS][NR]
    const int tid = threadIdx.x;
    const int rg = tid % RG, kl = tid / RG;
    const int row0 = blockIdx.x * ROWS + rg * 4;
    double acc[4][NR];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < NR; ++c) acc[i][c] = 0.0;
    for (int p = kl; p < n; p += KL) {
        double a[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = (row0 + i < m) ? A[(size_t)(row0 + i) + (size_t)p * lda] : 0.0;
        double x[NR];
#pragma unroll
        for (int c = 0; c < NR; ++c) x[c] = (c < nrhs) ? __ldg(X + (size_t)p + (size_t)c * ldx) : 0.0;
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int c = 0; c < NR; ++c) acc[i][c] = fma(a[i], x[c], acc[i][c]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int c = 0; c < NR; ++c) red[((size_t)kl * ROWS + rg * 4 + i) * NR + c] = acc[i][c];
    __syncthreads();
    for (int o = tid; o < ROWS * NR; o += 256) {
        const int rl = o / NR, c = o % NR;
        const int row = blockIdx.x * ROWS + rl;
        if (row >= m || c >= nrhs) continue;
        double sum = 0.0;
#pragma unroll 8
        for (int q = 0; q < KL; ++q) sum += red[((size_t)q * ROWS + rl) * NR + c];
        R[(size_t)row + (size_t)c * ldr] = B ? B[(size_t)row + (size_t)c * ldb] - sum : sum;   // B null: R = A X
    }
}

static int sm_count() { return device_sm_count(); }

template <int NR, int RG>
static int launch_residual_rg(int m, int n, int nrhs, const double *A, int lda, const double *X, int ldx,
                              const double *B, int ldb, double *R, int ldr, cudaStream_t st) {
    const size_t smem = sizeof(double) * 256 * 4 * NR;     // KL x ROWS x NR = 1024 NR
    CF_CUDA_TRY(cudaFuncSetAttribute(k_residual_f64<NR, RG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_residual_f64<NR, RG><<<ceil_div(m, 4 * RG), 256, smem, st>>>(m, n, nrhs, A, lda, X, ldx, B, ldb, R, ldr);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

// Fraction of the SM-slots of the last wave that a grid of c one-per-SM CTAs fills.
static double wave_fill(long long c, int sms) {
    const long long waves = (c + sms - 1) / sms;
    return waves > 0 ? (double)c / (double)(waves * sms) : 1.0;
}

template <int NR>
static int launch_residual_nr(int m, int n, int nrhs, const double *A, int lda, const double *X, int ldx,
                              const double *B, int ldb, double *R, int ldr, cudaStream_t st) {
    const int sms = sm_count();
    const bool small_rows = wave_fill(ceil_div(m, 32), sms) > wave_fill(ceil_div(m, 64), sms) + 0.02;
    if (small_rows) return launch_residual_rg<NR, 8>(m, n, nrhs, A, lda, X, ldx, B, ldb, R, ldr, st);
    return launch_residual_rg<NR, 16>(m, n, nrhs, A, lda, X, ldx, B, ldb, R, ldr, st);
}

int launch_residual_f64(int m, int n, int nrhs, const double *A, int lda, const double *X, int ldx, const double *B,
                        int ldb, double *R, int ldr, cudaStream_t st) {
    if (m <= 0 || nrhs <= 0) return CF_OK;
    for (int c0 = 0; c0 < nrhs; c0 += 16) {
        const int nc = min(16, nrhs - c0);
        const double *Xc = X + (size_t)c0 * ldx;
        const double *Bc = B ? B + (size_t)c0 * ldb : nullptr;
        double *Rc = R + (size_t)c0 * ldr;
        int rc;
        if (nc == 1) rc = launch_residual_nr<1>(m, n, nc, A, lda, Xc, ldx, Bc, ldb, Rc, ldr, st);
        else if (nc <= 2) rc = launch_residual_nr<2>(m, n, nc, A, lda, Xc, ldx, Bc, ldb, Rc, ldr, st);
        else if (nc <= 4) rc = launch_residual_nr<4>(m, n, nc, A, lda, Xc, ldx, Bc, ldb, Rc, ldr, st);
        else if (nc <= 8) rc = launch_residual_nr<8>(m, n, nc, A, lda, Xc, ldx, Bc, ldb, Rc, ldr, st);
        else rc = launch_residual_nr<16>(m, n, nc, A, lda, Xc, ldx, Bc, ldb, Rc, ldr, st);
        if (rc) return rc;
    }
    return CF_OK;
}

}  // namespace cf
