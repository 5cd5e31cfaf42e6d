// cf_mixed.cu -- mixed-precision refined solves (R-1..R-3 around LU-1..LU-5 and
// CH-1..CH-3): cf_gesv_mixed and cf_posv_mixed.
//
// Factorization.  A (FP64) is copied once into an FP32 working matrix W.  The
// factorization is COnfLUX's / COnfCHOX's blocked loop (Alg. 1; Sec. 7.5) with
// two levels of blocking: steps of width v = 128 (TournPivot, row swaps, A00,
// panel solves, all in FP32) inside slabs of width V; the Schur updates inside
// a slab use K = v, the update of the rest of the matrix is deferred to one
// K = V contraction per slab.  Every Schur update runs on the tensor cores
// (tcgen05, BF16 or FP16 operands rounded from W, FP32 accumulation into W).
// The deferral changes the order in which A11 receives its updates, not which
// updates it receives, nor the pivot rule.
//
// Refinement.  x_0 = 0; repeat r = b - A x in FP64 (the only FP64 arithmetic,
// on the untouched A), eta_j = ||r_j||_inf / (||A||_inf ||x_j||_inf +
// ||b_j||_inf), stop when max_j eta_j <= tol, else solve W d = r with the FP32
// factors and set x += d in FP64 (classical iterative refinement; Carson and
// Higham, SISC 2018, with u_f = BF16/FP16 and u = u_r = FP64).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "cf_common.cuh"
#include "cf_kernels.cuh"
#include "cf_tc.cuh"

namespace cf {

// ---------------------------------------------------------------------------
// Element-wise kernels
// ---------------------------------------------------------------------------
template <typename LP>
__device__ __forceinline__ LP to_lp(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to_lp<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half to_lp<__half>(float x) { return __float2half_rn(x); }

// dst[r*ldk + kk] = lp(src[r + kk*lds]) for kk < k, 0 for k <= kk < kpad.
template <typename LP>
__global__ void __launch_bounds__(256)
k_cvt_rows_kmajor(int rows, int k, int kpad, const float *__restrict__ src, int lds, LP *__restrict__ dst, int ldk) {
    __shared__ float t[32][33];
    const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 8 rows of threads
    for (int q = ty; q < 32; q += 8) {
        const int kk = k0 + q, r = r0 + tx;
        t[q][tx] = (r < rows && kk < k) ? src[(size_t)r + (size_t)kk * lds] : 0.f;
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
        const int r = r0 + q, kk = k0 + tx;
        if (r < rows && kk < kpad) dst[(size_t)r * ldk + kk] = to_lp<LP>(t[tx][q]);
    }
}

// dst[j*ldk + kk] = lp(src[kk + j*lds]) for kk < k, 0 for k <= kk < kpad.
template <typename LP>
__global__ void k_cvt_cols_kmajor(int k, int cols, int kpad, const float *__restrict__ src, int lds,
                                  LP *__restrict__ dst, int ldk) {
    const size_t tot = (size_t)cols * kpad;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int kk = (int)(e % kpad), j = (int)(e / kpad);
        dst[(size_t)j * ldk + kk] = to_lp<LP>(kk < k ? src[(size_t)kk + (size_t)j * lds] : 0.f);
    }
}

__global__ void k_iota(int n, int *p) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}

// Row sums of |A| (atomically accumulated over column chunks).
__global__ void __launch_bounds__(256) k_row_abssum(int n, const double *__restrict__ A, int lda, int cols_per_block,
                                                    double *rowsum) {
    const int i = blockIdx.x * 256 + threadIdx.x;
    const int j0 = blockIdx.y * cols_per_block, j1 = min(n, j0 + cols_per_block);
    if (i >= n) return;
    double s = 0.0;
#pragma unroll 8
    for (int j = j0; j < j1; ++j) s += fabs(A[(size_t)i + (size_t)j * lda]);
    atomicAdd(rowsum + i, s);
}

// out[c] = max(out[c], max_i |X[i, c]|); out must start at 0.  Non-negative
// doubles order like their bit patterns.
__global__ void k_col_absmax(int n, int ncols, const double *__restrict__ X, int ldx, unsigned long long *out) {
    const int c = blockIdx.y;
    double mx = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double v = fabs(X[(size_t)i + (size_t)c * ldx]);
        mx = (v > mx || v != v) ? v : mx;
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + c, (unsigned long long)__double_as_longlong(mx));
}

__global__ void k_diag_absmax(int n, const double *__restrict__ A, int lda, unsigned long long *out) {
    double mx = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        mx = fmax(mx, fabs(A[(size_t)i * (lda + 1)]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

__global__ void k_max_reduce(int n, const double *v, unsigned long long *out) {
    double mx = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) mx = fmax(mx, v[i]);
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(mx));
}

// Rf[i, c] = (float)(R[perm[i], c] / scale[c])   (perm == nullptr: identity)
__global__ void k_gather_scale(int n, int nrhs, const int *perm, const double *R, int ldr, const double *scale,
                               float *Rf, int ldf) {
    const size_t tot = (size_t)n * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), c = (int)(e / n);
        const int src = perm ? perm[i] : i;
        Rf[(size_t)i + (size_t)c * ldf] = (float)(R[(size_t)src + (size_t)c * ldr] / scale[c]);
    }
}

// X[:, c] += scale[c] * Df[:, c]
__global__ void k_axpy_update(int n, int nrhs, const float *Df, int ldf, const double *scale, double *X, int ldx) {
    const size_t tot = (size_t)n * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), c = (int)(e / n);
        X[(size_t)i + (size_t)c * ldx] += scale[c] * (double)Df[(size_t)i + (size_t)c * ldf];
    }
}

__global__ void k_copy_cols(int n, int nrhs, const double *S, int lds, double *D, int ldd) {
    const size_t tot = (size_t)n * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), c = (int)(e / n);
        D[(size_t)i + (size_t)c * ldd] = S[(size_t)i + (size_t)c * lds];
    }
}

// ---------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------
struct MixedWS {
    float *W = nullptr;
    int ldw = 0;
    void *Ab = nullptr, *Bb = nullptr, *Lb = nullptr, *Ub = nullptr;
    int *perm = nullptr, *ipiv = nullptr;
    TournWS tws{};
    TournEpilogue tep{};
    double *R = nullptr, *scale = nullptr, *rowsum = nullptr;
    float *Rf = nullptr;
    float *DinvL = nullptr, *DinvU = nullptr;   // inverses of the 64 x 64 diagonal blocks
    int *trsv_sync = nullptr;
    unsigned long long *norms = nullptr;   // [0..nrhs) |R|, [nrhs..2nrhs) |X|, [2nrhs..3nrhs) |B|, [3nrhs] ||A||
    size_t bytes = 0;
};

static int pick_V(int n, const Opts &o) {
    if (o.outer_V > 0) return o.outer_V;
    return n >= 8192 ? 1024 : 512;
}

static int carve_mixed(void *work, int n, int nrhs, const Opts &o, bool lu, MixedWS *w) {
    const int V = pick_V(n, o);
    const int Vp = (V + 63) / 64 * 64;
    Carver cv(work);
    w->ldw = (n + 31) / 32 * 32;
    w->W = cv.take<float>((size_t)w->ldw * (n > 0 ? n : 1), 1024);
    w->Ab = cv.take<uint16_t>((size_t)(n + 1) * kMaxV, 1024);
    w->Bb = cv.take<uint16_t>((size_t)(n + 1) * kMaxV, 1024);
    w->Lb = cv.take<uint16_t>((size_t)(n + 1) * Vp, 1024);
    w->Ub = lu ? cv.take<uint16_t>((size_t)(n + 1) * Vp, 1024) : nullptr;
    w->perm = cv.take<int>(n + 1);
    w->ipiv = cv.take<int>(n + 1);
    if (lu) {
        TournPlan p{};
        if (make_tourn_plan(n > 0 ? n : 1, 1, o.leaf_h, o.arity, &p) != CF_OK) return CF_ERR_UNSUPPORTED;
        w->tws.node_win = cv.take<int>((size_t)p.total_nodes * kMaxV);
        w->tws.node_cnt = cv.take<int>(p.total_nodes);
        w->tws.counter = cv.take<int>(p.total_nodes);
        w->tws.root_win = cv.take<int>(kMaxV);
        w->tws.counter_bytes = sizeof(int) * (size_t)p.total_nodes;
        w->tep.swap_cnt = cv.take<int>(1);
        w->tep.swap_dst = cv.take<int>(2 * kMaxV);
        w->tep.swap_src = cv.take<int>(2 * kMaxV);
    }
    w->R = cv.take<double>((size_t)n * nrhs + 1);
    w->scale = cv.take<double>(nrhs + 1);
    w->rowsum = cv.take<double>(n + 1);
    w->Rf = cv.take<float>((size_t)n * nrhs + 1);
    w->DinvL = cv.take<float>(diag_inverse_floats(n));
    w->DinvU = lu ? cv.take<float>(diag_inverse_floats(n)) : nullptr;
    w->trsv_sync = cv.take<int>(trsv_ws_bytes(n) / sizeof(int) + 1);
    w->norms = cv.take<unsigned long long>(3 * nrhs + 2);
    w->bytes = cv.size();
    return CF_OK;
}

static int grid_for(size_t tot) {
    size_t g = (tot + 255) / 256;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    return (int)g;
}

// Event pairs around selected launches on one stream; read after a sync.
struct Timer {
    std::vector<cudaEvent_t> ev;
    double flops = 0.0;
    int launches = 0;
    int begin(cudaStream_t st) {
        cudaEvent_t e;
        CF_CUDA_TRY(cudaEventCreate(&e));
        ev.push_back(e);
        CF_CUDA_TRY(cudaEventRecord(e, st));
        return CF_OK;
    }
    int end(cudaStream_t st, double fl) {
        int rc = begin(st);
        flops += fl;
        ++launches;
        return rc;
    }
    double ms() const {   // after the stream has been synchronised
        double t = 0;
        for (size_t i = 0; i + 1 < ev.size(); i += 2) {
            float x = 0;
            cudaEventElapsedTime(&x, ev[i], ev[i + 1]);
            t += x;
        }
        return t;
    }
    ~Timer() {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

template <typename LP>
static int cvt_rows(int rows, int k, int kpad, const float *src, int lds, void *dst, int ldk, cudaStream_t st) {
    if (rows <= 0) return CF_OK;
    dim3 grid(ceil_div(rows, 32), ceil_div(kpad, 32));
    k_cvt_rows_kmajor<LP><<<grid, 256, 0, st>>>(rows, k, kpad, src, lds, (LP *)dst, ldk);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

template <typename LP>
static int cvt_cols(int k, int cols, int kpad, const float *src, int lds, void *dst, int ldk, cudaStream_t st) {
    if (cols <= 0) return CF_OK;
    k_cvt_cols_kmajor<LP><<<grid_for((size_t)cols * kpad), 256, 0, st>>>(k, cols, kpad, src, lds, (LP *)dst, ldk);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

// ---------------------------------------------------------------------------
// Mixed LU of W (in place): tournament pivoting with FP32 panels, tensor-core
// Schur updates.
// ---------------------------------------------------------------------------
template <typename LP>
static int mixed_getrf(int n, MixedWS &w, int *info, const Opts &o, cudaStream_t st, Timer *tu) {
    const bool bf16 = std::is_same<LP, __nv_bfloat16>::value;
    const int v = o.v, V = pick_V(n, o);
    const size_t ld = (size_t)w.ldw;
    float *W = w.W;
    int rc;
    k_iota<<<grid_for(n), 256, 0, st>>>(n, w.perm);
    CF_LAUNCH_CHECK();
    CF_CUDA_TRY(cudaMemsetAsync(w.tws.counter, 0, w.tws.counter_bytes, st));
    for (int J0 = 0; J0 < n; J0 += V) {
        const int JE = J0 + V < n ? J0 + V : n;
        for (int k0 = J0; k0 < JE; k0 += v) {
            const int wd = v < JE - k0 ? v : JE - k0;
            const int m = n - k0;
            float *A00 = W + k0 + k0 * ld;
            w.tep.ipiv = w.ipiv;
            w.tep.k0 = k0;
            if ((rc = launch_tourn32(A00, w.ldw, m, wd, o.leaf_h, o.arity, w.tws, w.tep, st))) return rc;
            if ((rc = launch_apply_swaps<float>(W, w.ldw, n, k0, w.tep, w.perm, st))) return rc;
            if ((rc = launch_a00_lu32(A00, w.ldw, wd, k0, info, st))) return rc;
            const int below = m - wd, right = n - k0 - wd;
            // LU-3 / LU-4; they also write the K-major low-precision operands
            // of the updates.
            if ((rc = launch_rtrsm32<LP>(A00 + wd, w.ldw, below, wd, A00, w.ldw, false, (LP *)w.Ab, kMaxV, kMaxV,
                                         nullptr, st)))
                return rc;
            if ((rc = launch_ltrsm32<LP>(A00 + wd * ld, w.ldw, wd, right, A00, w.ldw, (LP *)w.Bb, kMaxV, kMaxV, st)))
                return rc;
            if (below <= 0 || right <= 0) continue;
            const int nslab = JE - (k0 + wd), nout = n - JE;
            float *C = A00 + wd + wd * ld;
            if (nslab > 0 &&
                (rc = launch_schur_tc(below, nslab, kMaxV, w.Ab, kMaxV, w.Bb, kMaxV, C, w.ldw, bf16, false, st, 0)))
                return rc;
            if (nslab > 0 && nout > 0 &&
                (rc = launch_schur_tc(nslab, nout, kMaxV, w.Ab, kMaxV, (const LP *)w.Bb + (size_t)nslab * kMaxV,
                                      kMaxV, C + (size_t)nslab * ld, w.ldw, bf16, false, st, 0)))
                return rc;
        }
        if (JE < n) {
            const int Vs = JE - J0, Vp = (Vs + 63) / 64 * 64, mr = n - JE;
            if ((rc = cvt_rows<LP>(mr, Vs, Vp, W + JE + J0 * ld, w.ldw, w.Lb, Vp, st))) return rc;
            if ((rc = cvt_cols<LP>(Vs, mr, Vp, W + J0 + JE * ld, w.ldw, w.Ub, Vp, st))) return rc;
            if (tu && (rc = tu->begin(st))) return rc;
            if ((rc = launch_schur_tc(mr, mr, Vp, w.Lb, Vp, w.Ub, Vp, W + JE + JE * ld, w.ldw, bf16, false, st, 0)))
                return rc;
            if (tu && (rc = tu->end(st, 2.0 * mr * (double)mr * Vs))) return rc;
        }
    }
    return CF_OK;
}

// ---------------------------------------------------------------------------
// Mixed Cholesky of W (lower, in place).
// ---------------------------------------------------------------------------
template <typename LP>
static int mixed_potrf(int n, MixedWS &w, int *info, const Opts &o, cudaStream_t st, Timer *tu) {
    const bool bf16 = std::is_same<LP, __nv_bfloat16>::value;
    const int v = o.v, V = pick_V(n, o);
    const size_t ld = (size_t)w.ldw;
    float *W = w.W;
    int rc;
    for (int J0 = 0; J0 < n; J0 += V) {
        const int JE = J0 + V < n ? J0 + V : n;
        for (int k0 = J0; k0 < JE; k0 += v) {
            const int wd = v < JE - k0 ? v : JE - k0;
            const int m = n - k0;
            float *A00 = W + k0 + k0 * ld;
            if ((rc = launch_a00_chol32(A00, w.ldw, wd, k0, info, st))) return rc;
            const int below = m - wd;
            if (below <= 0) continue;
            // CH-2: L10 = A10 L00^{-T}, with its K-major low-precision copy
            if ((rc = launch_rtrsm32<LP>(A00 + wd, w.ldw, below, wd, A00, w.ldw, true, (LP *)w.Ab, kMaxV, kMaxV, info,
                                         st)))
                return rc;
            const int nslab = JE - (k0 + wd);
            if (nslab <= 0) continue;
            if ((rc = launch_schur_tc(below, nslab, kMaxV, w.Ab, kMaxV, w.Ab, kMaxV, A00 + wd + wd * ld, w.ldw, bf16,
                                      true, st, 0)))
                return rc;
        }
        if (JE < n) {
            const int Vs = JE - J0, Vp = (Vs + 63) / 64 * 64, mr = n - JE;
            if ((rc = cvt_rows<LP>(mr, Vs, Vp, W + JE + J0 * ld, w.ldw, w.Lb, Vp, st))) return rc;
            if (tu && (rc = tu->begin(st))) return rc;
            if ((rc = launch_schur_tc(mr, mr, Vp, w.Lb, Vp, w.Lb, Vp, W + JE + JE * ld, w.ldw, bf16, true, st, 0)))
                return rc;
            // algorithmic flops of the triangular update: m (m + 1) K
            if (tu && (rc = tu->end(st, (double)mr * (mr + 1.0) * Vs))) return rc;
        }
    }
    return CF_OK;
}

// Correction solve with the FP32 factors: Rf <- W^{-1} P Rf, two sync-free
// blocked triangular solves.
static int solve_f32(int n, int nrhs, const MixedWS &w, bool lu, cudaStream_t st) {
    int rc;
    if ((rc = launch_trsv_f32(lu ? 0 : 2, n, nrhs, w.W, w.ldw, w.DinvL, w.Rf, n, w.trsv_sync, st))) return rc;
    return launch_trsv_f32(lu ? 1 : 3, n, nrhs, w.W, w.ldw, lu ? w.DinvU : w.DinvL, w.Rf, n, w.trsv_sync, st);
}

template <typename LP>
static int mixed_solve(int n, int nrhs, const double *A, int lda, const double *B, int ldb, double *X, int ldx,
                       int *info, cf_refine_stats *stats, void *work, size_t lwork, const Opts &o, bool lu,
                       cudaStream_t st) {
    MixedWS w;
    int rc = carve_mixed(nullptr, n, nrhs, o, lu, &w);
    if (rc) return rc;
    if (work == nullptr || lwork < w.bytes) return CF_ERR_WORKSPACE;
    if ((rc = carve_mixed(work, n, nrhs, o, lu, &w))) return rc;

    cf_refine_stats S{};
    cudaEvent_t e0, e1, e2;
    CF_CUDA_TRY(cudaEventCreate(&e0));
    CF_CUDA_TRY(cudaEventCreate(&e1));
    CF_CUDA_TRY(cudaEventCreate(&e2));
    CF_CUDA_TRY(cudaEventRecord(e0, st));
    CF_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int), st));

    // ---- factorization (Cholesky retries with a diagonal shift on breakdown)
    double shift = 0.0;
    int hinfo = 0;
    Timer tupd, tres;
    const double u_lp = std::is_same<LP, __nv_bfloat16>::value ? 0x1p-8 : 0x1p-11;
    for (int attempt = 0; attempt < 4; ++attempt) {
        // W = fl32(A) (+ shift on the diagonal)
        if ((rc = launch_split_f64(n, n, A, lda, nullptr, nullptr, w.ldw, w.W, w.ldw, shift, st))) return rc;
        CF_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int), st));
        rc = lu ? mixed_getrf<LP>(n, w, info, o, st, &tupd) : mixed_potrf<LP>(n, w, info, o, st, &tupd);
        if (rc) return rc;
        CF_CUDA_TRY(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
        CF_CUDA_TRY(cudaStreamSynchronize(st));
        if (hinfo == 0 || lu) break;
        // Cholesky broke down in low precision: refactor A + s I with
        // s = c u_lp max_i |a_ii|, c = 1, 4, 16 (diagonal shift of Higham and
        // Pranesh, SISC 2021); refinement with the unshifted A removes it.
        CF_CUDA_TRY(cudaMemsetAsync(w.norms, 0, sizeof(unsigned long long), st));
        k_diag_absmax<<<grid_for(n), 256, 0, st>>>(n, A, lda, w.norms);
        CF_LAUNCH_CHECK();
        unsigned long long dbits = 0;
        CF_CUDA_TRY(cudaMemcpyAsync(&dbits, w.norms, sizeof(dbits), cudaMemcpyDeviceToHost, st));
        CF_CUDA_TRY(cudaStreamSynchronize(st));
        double dm;
        memcpy(&dm, &dbits, sizeof(dm));
        shift = u_lp * dm * (double)(1 << (2 * attempt));
        hinfo = 0;
    }
    S.shift = shift;
    CF_CUDA_TRY(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
    CF_CUDA_TRY(cudaEventRecord(e1, st));
    int tstat = 0;
    if ((rc = tc_take_status(st, &tstat))) return rc;
    if (tstat != 0) return CF_ERR_TIMEOUT;
    S.info = hinfo;

    // ---- refinement
    const int ldr = n;
    CF_CUDA_TRY(cudaMemsetAsync(w.rowsum, 0, sizeof(double) * n, st));
    {
        const int cpb = 1024;
        dim3 g(ceil_div(n, 256), ceil_div(n, cpb));
        k_row_abssum<<<g, 256, 0, st>>>(n, A, lda, cpb, w.rowsum);
        CF_LAUNCH_CHECK();
    }
    unsigned long long *nR = w.norms, *nX = w.norms + nrhs, *nB = w.norms + 2 * nrhs, *nA = w.norms + 3 * nrhs;
    CF_CUDA_TRY(cudaMemsetAsync(w.norms, 0, sizeof(unsigned long long) * (3 * nrhs + 2), st));
    k_max_reduce<<<grid_for(n), 256, 0, st>>>(n, w.rowsum, nA);
    CF_LAUNCH_CHECK();
    k_col_absmax<<<dim3(grid_for(n), nrhs), 256, 0, st>>>(n, nrhs, B, ldb, nB);
    CF_LAUNCH_CHECK();
    // x = 0, r = b
    for (int c = 0; c < nrhs; ++c) CF_CUDA_TRY(cudaMemsetAsync(X + (size_t)c * ldx, 0, sizeof(double) * n, st));
    k_copy_cols<<<grid_for((size_t)n * nrhs), 256, 0, st>>>(n, nrhs, B, ldb, w.R, ldr);
    CF_LAUNCH_CHECK();

    if (S.info == 0) {
        if ((rc = launch_diag_inverse(lu ? 0 : 2, n, w.W, w.ldw, w.DinvL, st))) return rc;
        if (lu && (rc = launch_diag_inverse(1, n, w.W, w.ldw, w.DinvU, st))) return rc;
    }

    std::vector<unsigned long long> hn(3 * nrhs + 2);
    std::vector<double> hscale(nrhs);
    double eta_prev = HUGE_VAL, eta = HUGE_VAL;
    int it = 0, stall = 0;
    bool converged = false;
    for (;; ++it) {
        if (it > 0) {
            if ((rc = tres.begin(st))) return rc;
            if ((rc = launch_residual_f64(n, n, nrhs, A, lda, X, ldx, B, ldb, w.R, ldr, st))) return rc;
            if ((rc = tres.end(st, 2.0 * n * (double)n * nrhs))) return rc;
        }
        CF_CUDA_TRY(cudaMemsetAsync(w.norms, 0, sizeof(unsigned long long) * 2 * nrhs, st));
        k_col_absmax<<<dim3(grid_for(n), nrhs), 256, 0, st>>>(n, nrhs, w.R, ldr, nR);
        CF_LAUNCH_CHECK();
        k_col_absmax<<<dim3(grid_for(n), nrhs), 256, 0, st>>>(n, nrhs, X, ldx, nX);
        CF_LAUNCH_CHECK();
        CF_CUDA_TRY(cudaMemcpyAsync(hn.data(), w.norms, sizeof(unsigned long long) * (3 * nrhs + 1),
                                    cudaMemcpyDeviceToHost, st));
        CF_CUDA_TRY(cudaStreamSynchronize(st));
        double anorm;
        memcpy(&anorm, &hn[3 * nrhs], sizeof(double));
        eta = 0.0;
        for (int c = 0; c < nrhs; ++c) {
            double r, x, b;
            memcpy(&r, &hn[c], 8);
            memcpy(&x, &hn[nrhs + c], 8);
            memcpy(&b, &hn[2 * nrhs + c], 8);
            const double den = anorm * x + b;
            const double e = den > 0 ? r / den : (r > 0 ? HUGE_VAL : 0.0);
            eta = (e > eta || e != e) ? e : eta;
            hscale[c] = r > 0 ? r : 1.0;
        }
        if (it == 1) S.eta0 = eta;
        if (eta <= o.tol) { converged = true; break; }
        if (it >= o.max_iter || S.info != 0) break;
        if (it >= 2 && eta > 0.5 * eta_prev) {
            if (++stall >= 2) break;
        } else {
            stall = 0;
        }
        eta_prev = eta < eta_prev ? eta : eta_prev;
        CF_CUDA_TRY(cudaMemcpyAsync(w.scale, hscale.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
        k_gather_scale<<<grid_for((size_t)n * nrhs), 256, 0, st>>>(n, nrhs, lu ? w.perm : nullptr, w.R, ldr, w.scale,
                                                                  w.Rf, n);
        CF_LAUNCH_CHECK();
        if ((rc = solve_f32(n, nrhs, w, lu, st))) return rc;
        k_axpy_update<<<grid_for((size_t)n * nrhs), 256, 0, st>>>(n, nrhs, w.Rf, n, w.scale, X, ldx);
        CF_LAUNCH_CHECK();
    }
    CF_CUDA_TRY(cudaEventRecord(e2, st));
    CF_CUDA_TRY(cudaEventSynchronize(e2));
    if ((rc = trsv_take_status(st, &tstat))) return rc;
    if (tstat != 0) return CF_ERR_TIMEOUT;
    float f_ms = 0, r_ms = 0;
    cudaEventElapsedTime(&f_ms, e0, e1);
    cudaEventElapsedTime(&r_ms, e1, e2);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    S.iterations = it;
    S.solver = 0;
    S.converged = converged ? 1 : 0;
    S.eta = eta;
    S.factor_ms = f_ms;
    S.refine_ms = r_ms;
    S.residual_ms = tres.ms();
    S.residual_launches = tres.launches;
    S.update_ms = tupd.ms();
    S.update_flops = tupd.flops;
    S.update_launches = tupd.launches;
    if (stats) *stats = S;
    return converged ? CF_OK : CF_ERR_NOT_CONVERGED;
}

static int check_mixed_args(int n, int nrhs, const double *A, int lda, const double *B, int ldb, double *X, int ldx,
                            cf_prec prec, int *info) {
    if (n < 0) return -1;
    if (nrhs < 0) return -2;
    if (n > 0 && A == nullptr) return -3;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (n > 0 && nrhs > 0 && B == nullptr) return -5;
    if (ldb < (n > 1 ? n : 1)) return -6;
    if (n > 0 && nrhs > 0 && X == nullptr) return -7;
    if (ldx < (n > 1 ? n : 1)) return -8;
    if (prec != CF_BF16 && prec != CF_F16) return -9;
    if (info == nullptr) return -10;
    return CF_OK;
}

}  // namespace cf

using namespace cf;

static size_t mixed_ws_size(int n, int nrhs, cf_prec prec, const cf_options *opt, bool lu) {
    (void)prec;
    Opts o;
    if (resolve_options(opt, &o) != CF_OK) return 0;
    MixedWS w;
    if (carve_mixed(nullptr, n > 0 ? n : 1, nrhs > 0 ? nrhs : 1, o, lu, &w) != CF_OK) return 0;
    return w.bytes;
}

static int mixed_entry(int n, int nrhs, const double *A, int lda, const double *B, int ldb, double *X, int ldx,
                       cf_prec prec, int *info, cf_refine_stats *stats, void *work, size_t lwork,
                       const cf_options *opt, cudaStream_t st, bool lu) {
    int rc = check_mixed_args(n, nrhs, A, lda, B, ldb, X, ldx, prec, info);
    if (rc) return rc;
    Opts o;
    if ((rc = resolve_options(opt, &o))) return rc;
    if (n == 0 || nrhs == 0) {
        if (stats) { memset(stats, 0, sizeof(*stats)); stats->converged = 1; }
        return CF_OK;
    }
    if (prec == CF_BF16)
        return mixed_solve<__nv_bfloat16>(n, nrhs, A, lda, B, ldb, X, ldx, info, stats, work, lwork, o, lu, st);
    return mixed_solve<__half>(n, nrhs, A, lda, B, ldb, X, ldx, info, stats, work, lwork, o, lu, st);
}

extern "C" size_t cf_gesv_mixed_workspace_size(int n, int nrhs, cf_prec prec, const cf_options *opt) {
    return mixed_ws_size(n, nrhs, prec, opt, true);
}

extern "C" int cf_gesv_mixed(int n, int nrhs, const double *A, int lda, const double *B, int ldb, double *X, int ldx,
                             cf_prec prec, int *info, cf_refine_stats *stats, void *work, size_t lwork,
                             const cf_options *opt, cudaStream_t st) {
    return mixed_entry(n, nrhs, A, lda, B, ldb, X, ldx, prec, info, stats, work, lwork, opt, st, true);
}

extern "C" size_t cf_posv_mixed_workspace_size(int n, int nrhs, cf_prec prec, const cf_options *opt) {
    return mixed_ws_size(n, nrhs, prec, opt, false);
}

extern "C" int cf_posv_mixed(int n, int nrhs, const double *A, int lda, const double *B, int ldb, double *X, int ldx,
                             cf_prec prec, int *info, cf_refine_stats *stats, void *work, size_t lwork,
                             const cf_options *opt, cudaStream_t st) {
    return mixed_entry(n, nrhs, A, lda, B, ldb, X, ldx, prec, info, stats, work, lwork, opt, st, false);
}
