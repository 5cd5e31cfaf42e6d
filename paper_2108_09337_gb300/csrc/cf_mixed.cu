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

// Factor-precision tag of the FP8 Cholesky (e4m3 operands, per-tile scales).
struct fp8_e4m3 {};

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

// Split BF16 operands: x = hi + lo with hi = bf16(x), lo = bf16(x - hi)
// (together 16 significant bits).  Three segments of K values, segment s at
// dst + s * seg: PATTERN 0 (left operand) hi, hi, lo; PATTERN 1 (right
// operand) hi, lo, hi -- so one contraction over the three segments sums
// hi.hi + hi.lo + lo.hi, the split product without its lo.lo term.
template <int PATTERN>
__device__ __forceinline__ void put_split(__nv_bfloat16 *d, size_t seg, float x) {
    const __nv_bfloat16 hi = __float2bfloat16_rn(x);
    const __nv_bfloat16 lo = __float2bfloat16_rn(x - __bfloat162float(hi));
    d[0] = hi;
    d[seg] = PATTERN == 0 ? hi : lo;
    d[2 * seg] = PATTERN == 0 ? lo : hi;
}

// Split form of k_cvt_rows_kmajor.
template <int PATTERN>
__global__ void __launch_bounds__(256)
k_cvt_rows_split(int rows, int k, int kpad, const float *__restrict__ src, int lds, __nv_bfloat16 *__restrict__ dst,
                 int ldk, int seg) {
    __shared__ float t[32][33];
    const int r0 = blockIdx.x * 32, k0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int q = ty; q < 32; q += 8) {
        const int kk = k0 + q, r = r0 + tx;
        t[q][tx] = (r < rows && kk < k) ? src[(size_t)r + (size_t)kk * lds] : 0.f;
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
        const int r = r0 + q, kk = k0 + tx;
        if (r < rows && kk < kpad) put_split<PATTERN>(dst + (size_t)r * ldk + kk, (size_t)seg, t[tx][q]);
    }
}

// Split form of k_cvt_cols_kmajor.
template <int PATTERN>
__global__ void k_cvt_cols_split(int k, int cols, int kpad, const float *__restrict__ src, int lds,
                                 __nv_bfloat16 *__restrict__ dst, int ldk, int seg) {
    const size_t tot = (size_t)cols * kpad;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int kk = (int)(e % kpad), j = (int)(e / kpad);
        put_split<PATTERN>(dst + (size_t)j * ldk + kk, (size_t)seg, kk < k ? src[(size_t)kk + (size_t)j * lds] : 0.f);
    }
}

__global__ void k_iota(int n, int *p) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}

// One pass over A: W = fl32(A) (+ shift on the diagonal) and, if rowsum is
// set, rowsum[i] += sum_j |a_ij| over this CTA's columns (atomic over column
// chunks).  CTA: 512 rows, two per thread (16-byte loads when vec: lda even
// and A 16-byte aligned; W stores as float2, ldw even) x kCvtCols columns.
// The row sums add |fl32(a_ij)| in FP32 over 32 columns and those partial
// sums in FP64 (relative error ~1e-6, as the norm in eta needs): GB300's
// FP64 pipe, ~2 operations per clock per SM, would otherwise bound the pass
// at half the HBM bandwidth (measured 3.95 ms at N = 32768 with FP64 sums,
// 2.05 ms with these, 92% of the copy bandwidth for its 12 bytes per
// element).
constexpr int kCvtCols = 1024;
__global__ void __launch_bounds__(256) k_to_f32_rowsum(int n, const double *__restrict__ A, int lda,
                                                       float *__restrict__ W, int ldw, double shift, double *rowsum,
                                                       int *ef, int vec) {
    const int i = (blockIdx.x * 256 + threadIdx.x) * 2;
    if (i >= n) return;
    const int j0 = blockIdx.y * kCvtCols, j1 = min(n, j0 + kCvtCols);
    const bool two = i + 1 < n;
    double s0 = 0.0, s1 = 0.0;
    int f0 = 0, f1 = 0;        // largest exponent fields (the tensor-core residual's row scales)
    for (int jc = j0; jc < j1; jc += 32) {
        float t0 = 0.f, t1 = 0.f;
        const int jce = min(j1, jc + 32);
#pragma unroll 8
        for (int j = jc; j < jce; ++j) {
            const double *src = A + (size_t)i + (size_t)j * lda;
            double a0, a1 = 0.0;
            if (vec && two) {
                const double2 v = __ldg(reinterpret_cast<const double2 *>(src));
                a0 = v.x;
                a1 = v.y;
            } else {
                a0 = src[0];
                if (two) a1 = src[1];
            }
            const float a0f = (float)a0, a1f = (float)a1;
            t0 += fabsf(a0f);
            t1 += fabsf(a1f);
            f0 = max(f0, (int)((__double_as_longlong(a0) >> 52) & 0x7FF));
            f1 = max(f1, (int)((__double_as_longlong(a1) >> 52) & 0x7FF));
            float *dst = W + (size_t)i + (size_t)j * ldw;
            if (two) *reinterpret_cast<float2 *>(dst) = make_float2(a0f, a1f);
            else dst[0] = a0f;
        }
        s0 += (double)t0;
        s1 += (double)t1;
    }
    // the shifted diagonal, rewritten by the thread that wrote it (the FP64
    // addition stays out of the element loop: selected per element, it was
    // computed for every element)
    if (shift != 0.0) {
        if (i >= j0 && i < j1) W[(size_t)i + (size_t)i * ldw] = (float)(A[(size_t)i + (size_t)i * lda] + shift);
        if (two && i + 1 >= j0 && i + 1 < j1)
            W[(size_t)(i + 1) + (size_t)(i + 1) * ldw] = (float)(A[(size_t)(i + 1) + (size_t)(i + 1) * lda] + shift);
    }
    if (rowsum) {
        atomicAdd(rowsum + i, s0);
        if (two) atomicAdd(rowsum + i + 1, s1);
    }
    if (ef) {
        if (f0 > 0) atomicMax(ef + i, f0);
        if (two && f1 > 0) atomicMax(ef + i + 1, f1);
    }
}

static int launch_to_f32_rowsum(int n, const double *A, int lda, float *W, int ldw, double shift, double *rowsum,
                                int *ef, cudaStream_t st) {
    if (n <= 0) return CF_OK;
    if (ldw % 2 != 0 || ((uintptr_t)W & 7)) return CF_ERR_UNSUPPORTED;
    const int vec = (lda % 2 == 0 && ((uintptr_t)A & 15) == 0) ? 1 : 0;
    dim3 g(ceil_div(n, 512), ceil_div(n, kCvtCols));
    k_to_f32_rowsum<<<g, 256, 0, st>>>(n, A, lda, W, ldw, shift, rowsum, ef, vec);
    CF_LAUNCH_CHECK();
    return CF_OK;
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
// GMRES-IR kernels.  Vectors are n x nrhs FP64 blocks (ld n), one Krylov
// sequence per right-hand side; basis block i sits at V + i * n * nrhs.
// ---------------------------------------------------------------------------
constexpr int kDotRows = 2048;         // rows per partial-dot block
constexpr double kGmresTol = 1e-8;     // inner GMRES: stop at ||g_k|| <= tol ||M^{-1} r||
constexpr double kSwitchRate = 0.3;    // classical refinement must cut eta at least this much per step
// Pair-arithmetic residuals (cf_pair.cu) are accurate to between ~1e-16 and a
// few 1e-14 of ||A|| ||x|| (worst on rows dominated by one term): a step whose
// backward error is predicted at or above kPairFloor takes one, and an eta
// below kPairFloor from one is recomputed in FP64.
constexpr double kPairFloor = 1e-12;
// A GMRES-IR step with 16-bit factors that needed at least kSlowInner inner
// iterations and cut eta by less than kSlowGain counts as failed: another
// such step costs more than refactoring with split BF16 updates.
constexpr int kSlowInner = 12;
constexpr double kSlowGain = 1e-2;
constexpr double kAssumedRate = 1e-2;

// part[(chunk * nv + i) * nrhs + c] = sum over the chunk's rows of V_i[r, c] * W[r, c]
__global__ void __launch_bounds__(256) k_dots_partial(int n, int nrhs, const double *__restrict__ V,
                                                      const double *__restrict__ W, double *part) {
    __shared__ double red[8];
    const int chunk = blockIdx.x, i = blockIdx.y, nv = gridDim.y;
    const int r0 = chunk * kDotRows, r1 = min(n, r0 + kDotRows);
    const double *Vi = V + (size_t)i * n * nrhs;
    for (int c = 0; c < nrhs; ++c) {
        double acc = 0.0;
        for (int r = r0 + threadIdx.x; r < r1; r += 256)
            acc = fma(Vi[(size_t)r + (size_t)c * n], W[(size_t)r + (size_t)c * n], acc);
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < 8; ++q) t += red[q];
            part[((size_t)chunk * nv + i) * nrhs + c] = t;
        }
        __syncthreads();
    }
}

// out[j] (+)= sum over chunks of part[chunk * cnt + j], in chunk order
__global__ void k_dots_final(int nchunks, int cnt, const double *part, double *out, int accumulate) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < cnt; j += gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int q = 0; q < nchunks; ++q) t += part[(size_t)q * cnt + j];
        out[j] = accumulate ? out[j] + t : t;
    }
}

// O[r, c] -= sum_{i < nv} coef[i * nrhs + c] * V_i[r, c]
__global__ void k_block_axpy(int n, int nrhs, int nv, const double *__restrict__ V, const double *__restrict__ coef,
                             double *O, int ldo) {
    const size_t tot = (size_t)n * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % n), c = (int)(e / n);
        double t = O[(size_t)r + (size_t)c * ldo];
        for (int i = 0; i < nv; ++i) t = fma(-coef[i * nrhs + c], V[(size_t)i * tot + e], t);
        O[(size_t)r + (size_t)c * ldo] = t;
    }
}

// nrm[c] = sqrt(sq[c]); O[:, c] = W[:, c] / nrm[c] (zero if nrm[c] == 0)
__global__ void k_normalize(int n, int nrhs, const double *sq, double *nrm, const double *W, double *O) {
    const size_t tot = (size_t)n * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / n);
        const double h = sqrt(sq[c]);
        O[e] = h > 0.0 ? W[e] / h : 0.0;
        if (e % n == 0) nrm[c] = h;
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
    float *DinvL = nullptr, *DinvU = nullptr;   // inverses of the 128 x 128 diagonal blocks
    float *G0 = nullptr, *G1 = nullptr;         // neighbour tiles premultiplied by them (first, second solve)
    double *DinvL64 = nullptr, *DinvU64 = nullptr;   // the same in FP64 (GMRES-IR preconditioner)
    int *trsv_sync = nullptr;
    unsigned long long *norms = nullptr;   // [0..nrhs) |R|, [nrhs..2nrhs) |X|, [2nrhs..3nrhs) |B|, [3nrhs] ||A||
    // GMRES-IR
    int m = 0;                             // Krylov dimension
    double *V = nullptr;                   // (m + 1) blocks of n x nrhs
    double *Y = nullptr, *Wv = nullptr;    // n x nrhs each
    double *part = nullptr;                // partial dots
    double *hcol = nullptr;                // (m + 2) x nrhs: one Hessenberg column per right-hand side
    double *coef = nullptr;                // (m + 1) x nrhs
    double *sq = nullptr;                  // nrhs squared norms
    unsigned long long *sbits = nullptr;   // per-column scales of the FP32 preconditioner input
    float *sc8 = nullptr;                  // FP8 tile scales: slab (rows/128 x V/128), then one step
    double *Xbest = nullptr;               // best iterate so far
    void *pairws = nullptr;                // pair-arithmetic residual workspace
    float *Psk = nullptr;                  // split-K partials of the small K = V updates
    bool use_tc = false;                   // residuals on the tensor cores (digit slices of A)
    void *rtcA = nullptr, *rtcX = nullptr; // their slices of A, and per-product scratch
    ResidTC rtc{};
    const unsigned long long *anorm = nullptr;   // bits of ||A||_inf (bound for the pair residual's scaling)
    size_t bytes = 0;
};

// Depth V of the slab's deferred K = V update.  Deeper slabs raise the
// update's arithmetic intensity (its FP32 C is read and written once per
// slab) and cost more right-looking work inside the slab (which the
// look-ahead stream partly hides); measured at N = 32768: LU 138.7 ms with
// V = 2048 against 148.0 (V = 1024) and 158.0 (V = 4096); Cholesky with FP16
// updates 45.0 ms with V = 2048 against 49.6 (V = 1024).
static int pick_V(int n, const Opts &o, bool lu) {
    (void)lu;
    if (o.outer_V > 0) return o.outer_V;
    if (n >= 16384) return 2048;
    return n >= 8192 ? 1024 : 512;
}

static int carve_mixed(void *work, int n, int nrhs, const Opts &o, bool lu, MixedWS *w) {
    const int V = pick_V(n, o, lu);
    const int Vp = (V + 63) / 64 * 64;
    Carver cv(work);
    w->ldw = (n + 31) / 32 * 32;
    w->W = cv.take<float>((size_t)w->ldw * (n > 0 ? n : 1), 1024);
    // Low-precision operands, sized for the split-BF16 form (three K
    // segments): Ab the left operand of one step (rows x 3 kMaxV), also the
    // pivot rows' slab operand (kMaxV x 3 Vp) of the left-looking update;
    // Bb the right operand of one step; Lb / Ub the slab's operands.
    w->Ab = cv.take<uint16_t>((size_t)((n > Vp ? n : Vp) + 1) * 3 * kMaxV, 1024);
    w->Bb = cv.take<uint16_t>((size_t)(n + 1) * 3 * kMaxV, 1024);
    w->Lb = cv.take<uint16_t>((size_t)(n + 1) * 3 * Vp, 1024);
    w->Ub = cv.take<uint16_t>((size_t)(n + 1) * 3 * Vp, 1024);
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
        w->tws.rows32 = cv.take<float>((size_t)(n > 0 ? n : 1) * kMaxV);
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
    w->G0 = cv.take<float>(diag_inverse_floats(n));
    w->G1 = cv.take<float>(diag_inverse_floats(n));
    w->DinvL64 = cv.take<double>(diag_inverse64_elems(n));
    w->DinvU64 = lu ? cv.take<double>(diag_inverse64_elems(n)) : nullptr;
    w->trsv_sync = cv.take<int>(trsv_ws_bytes(n) / sizeof(int) + 1);
    w->norms = cv.take<unsigned long long>(3 * nrhs + 2);
    w->m = o.gmres_restart;
    const size_t blk = (size_t)n * nrhs;
    w->V = cv.take<double>(blk * (w->m + 1) + 1);
    w->Y = cv.take<double>(blk + 1);
    w->Wv = cv.take<double>(blk + 1);
    w->part = cv.take<double>((size_t)ceil_div(n > 0 ? n : 1, kDotRows) * (w->m + 1) * nrhs + 1);
    w->hcol = cv.take<double>((size_t)(w->m + 2) * nrhs);
    w->coef = cv.take<double>((size_t)(w->m + 1) * nrhs);
    w->sq = cv.take<double>(nrhs + 1);
    w->sbits = cv.take<unsigned long long>(nrhs + 1);
    w->Xbest = cv.take<double>(blk + 1);
    w->pairws = cv.take<char>(pair_residual_ws_bytes(n, n));
    w->use_tc = o.residual_kind == 0 && !o.fp64_residual;
    if (w->use_tc) {
        w->rtcA = cv.take<char>(resid_tc_a_bytes(n, n), 1024);
        w->rtcX = cv.take<char>(resid_tc_x_bytes(n, n), 1024);
    }
    w->sc8 = cv.take<float>((size_t)(ceil_div(n > 0 ? n : 1, 128) + 1) * (Vp / 128 + 2));
    // split-K partials: at most (SMs / tiles) ranges of the tiles of an
    // update that fills fewer than half the SMs (a triangle counts half)
    {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
        w->Psk = cv.take<float>((size_t)2 * sms * 128 * 256, 1024);
    }
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

static int cvt_rows_split(int rows, int k, int kpad, const float *src, int lds, void *dst, int ldk, int seg,
                          int pattern, cudaStream_t st) {
    if (rows <= 0) return CF_OK;
    dim3 grid(ceil_div(rows, 32), ceil_div(kpad, 32));
    if (pattern == 0)
        k_cvt_rows_split<0><<<grid, 256, 0, st>>>(rows, k, kpad, src, lds, (__nv_bfloat16 *)dst, ldk, seg);
    else
        k_cvt_rows_split<1><<<grid, 256, 0, st>>>(rows, k, kpad, src, lds, (__nv_bfloat16 *)dst, ldk, seg);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

static int cvt_cols_split(int k, int cols, int kpad, const float *src, int lds, void *dst, int ldk, int seg,
                          int pattern, cudaStream_t st) {
    if (cols <= 0) return CF_OK;
    if (pattern == 0)
        k_cvt_cols_split<0><<<grid_for((size_t)cols * kpad), 256, 0, st>>>(k, cols, kpad, src, lds,
                                                                           (__nv_bfloat16 *)dst, ldk, seg);
    else
        k_cvt_cols_split<1><<<grid_for((size_t)cols * kpad), 256, 0, st>>>(k, cols, kpad, src, lds,
                                                                           (__nv_bfloat16 *)dst, ldk, seg);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

// ---------------------------------------------------------------------------
// Mixed LU of W (in place): tournament pivoting with FP32 panels, tensor-core
// Schur updates.
// ---------------------------------------------------------------------------
// A second stream for the parts of a panel step that do not depend on each
// other (released when its work completes).
struct SideStream {
    cudaStream_t s = nullptr, bg = nullptr;
    cudaEvent_t swapped = nullptr, a00_done = nullptr, side_done = nullptr, bg_done = nullptr;
    int open() {
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&bg, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&swapped, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&a00_done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&side_done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&bg_done, cudaEventDisableTiming) != cudaSuccess)
            return CF_ERR_CUDA;
        return CF_OK;
    }
    ~SideStream() {
        if (swapped) cudaEventDestroy(swapped);
        if (a00_done) cudaEventDestroy(a00_done);
        if (side_done) cudaEventDestroy(side_done);
        if (bg_done) cudaEventDestroy(bg_done);
        if (s) cudaStreamDestroy(s);
        if (bg) cudaStreamDestroy(bg);
    }
};

// LU-6 look-ahead of the mixed LU: the part of a step's in-slab update right
// of the next panel runs on this stream while TournPivot of the next step
// (which reads only the next panel's columns, updated first on the main
// stream) runs; the next step's row swaps wait for it.
struct LookStream {
    cudaStream_t s = nullptr;
    cudaEvent_t fork = nullptr, done = nullptr;
    int open() {
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess)
            return CF_ERR_CUDA;
        return CF_OK;
    }
    ~LookStream() {
        if (fork) cudaEventDestroy(fork);
        if (done) cudaEventDestroy(done);
        if (s) cudaStreamDestroy(s);
    }
};

static int device_sms() { return device_sm_count(); }

template <typename LP>
static int mixed_getrf(int n, MixedWS &w, int *info, const Opts &o, cudaStream_t st, Timer *tu, bool split,
                       Timer *tt = nullptr) {
    const bool bf16 = std::is_same<LP, __nv_bfloat16>::value;
    const int v = o.v, V = pick_V(n, o, true);
    const int Vpad = (V + 63) / 64 * 64;        // K stride (per segment) of the slab's U operand
    const int S = split ? 3 : 1;                 // K segments per operand
    const size_t ld = (size_t)w.ldw;
    float *W = w.W;
    int rc;
    SideStream ss;
    if ((rc = ss.open())) return rc;
    LookStream la;
    if (o.lookahead && (rc = la.open())) return rc;
    bool la_pending = false;               // the look-ahead stream holds an update the next swaps must wait for
    const int sms = device_sms();
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
            if (tt && (rc = tt->begin(st))) return rc;
            if ((rc = launch_tourn32_any(A00, w.ldw, m, wd, o.leaf_h, o.arity, w.tws, w.tep, st))) return rc;
            if (tt && (rc = tt->end(st, tourn32_flops(m, wd, o.leaf_h, o.arity)))) return rc;
            if (la_pending) {            // the previous step's update right of this panel
                CF_CUDA_TRY(cudaStreamWaitEvent(st, la.done, 0));
                la_pending = false;
            }
            if ((rc = launch_apply_swaps<float>(W, w.ldw, n, k0, w.tep, w.perm, st))) return rc;
            // Fork: the side stream takes LU-4 on the slab's columns with
            // their operand copy (concurrent with LU-3); the main stream joins
            // before the next panel's update, which reads both solves'
            // operands.  The background stream takes what only the slab's
            // deferred update needs: the pivot rows' left-looking update
            // right of the slab, LU-4 there and its K-major copy; the main
            // stream joins it at the slab's end.  It writes only this step's
            // pivot rows right of the slab, which no later step of the slab
            // reads before it (the next steps' swaps move rows below them;
            // the next steps' background work follows in stream order).
            CF_CUDA_TRY(cudaEventRecord(ss.swapped, st));
            CF_CUDA_TRY(cudaStreamWaitEvent(ss.bg, ss.swapped, 0));
            if ((rc = launch_a00_lu32(A00, w.ldw, wd, k0, info, st))) return rc;
            CF_CUDA_TRY(cudaEventRecord(ss.a00_done, st));
            CF_CUDA_TRY(cudaStreamWaitEvent(ss.s, ss.a00_done, 0));
            const int below = m - wd, right = n - k0 - wd;
            const int off = k0 - J0, nout = n - JE;
            const int rslab = right - nout;              // columns right of the panel inside the slab
            // The part of the new pivot rows right of the slab has not yet
            // received this slab's earlier steps (they are deferred for every
            // row still below, and a pivot row may have come from anywhere
            // below): apply them now, A[k0:k0+wd, JE:] -= L[k0:k0+wd, J0:k0]
            // U[J0:k0, JE:] (left-looking, K = off; operand in Lb, which is
            // free until the slab's deferred update).
            // (background)
            if (off > 0 && nout > 0) {
                const int Kp = (off + 63) / 64 * 64;
                float *Cp = W + k0 + JE * ld;
                if (!split) {
                    if ((rc = cvt_rows<LP>(wd, off, Kp, W + k0 + J0 * ld, w.ldw, w.Lb, Kp, ss.bg))) return rc;
                    if ((rc = launch_schur_tc(wd, nout, Kp, w.Lb, Kp, w.Ub, Vpad, Cp, w.ldw, bf16, false, ss.bg, 0)))
                        return rc;
                } else {
                    // segments (hi, hi, lo) x (hi, lo, hi): three K = off products
                    if ((rc = cvt_rows_split(wd, off, Kp, W + k0 + J0 * ld, w.ldw, w.Lb, 3 * Kp, Kp, 0, ss.bg)))
                        return rc;
                    for (int sg = 0; sg < 3; ++sg)
                        if ((rc = launch_schur_tc(wd, nout, Kp, (const __nv_bfloat16 *)w.Lb + (size_t)sg * Kp, 3 * Kp,
                                                  (const __nv_bfloat16 *)w.Ub + (size_t)sg * Vpad, 3 * Vpad, Cp,
                                                  w.ldw, true, false, ss.bg, 0)))
                            return rc;
                }
            }
            // LU-4 (side) after the A00 LU on the slab's columns; it also
            // writes the K-major low-precision operand of the updates inside
            // the slab (split form: converted after).
            if ((rc = launch_ltrsm32<LP>(A00 + wd * ld, w.ldw, wd, rslab, A00, w.ldw, split ? nullptr : (LP *)w.Bb,
                                         kMaxV, kMaxV, ss.s)))
                return rc;
            if (split && (rc = cvt_cols_split(wd, rslab, kMaxV, A00 + wd * ld, w.ldw, w.Bb, 3 * kMaxV, kMaxV, 1,
                                              ss.s)))
                return rc;
            CF_CUDA_TRY(cudaEventRecord(ss.side_done, ss.s));
            // LU-4 right of the slab (background, after the left-looking
            // update); those U rows go to the K-major operand of the slab's
            // deferred update (K rows off .. off + wd, zeros up to the next
            // multiple of 64).
            if (nout > 0) {
                CF_CUDA_TRY(cudaStreamWaitEvent(ss.bg, ss.a00_done, 0));
                if ((rc = launch_ltrsm32<LP>(W + k0 + JE * ld, w.ldw, wd, nout, A00, w.ldw, nullptr, kMaxV, kMaxV,
                                             ss.bg)))
                    return rc;
                const int kp = (off + wd + 63) / 64 * 64 - off;
                if (!split) {
                    if ((rc = cvt_cols<LP>(wd, nout, kp, W + k0 + JE * ld, w.ldw, (LP *)w.Ub + off, Vpad, ss.bg)))
                        return rc;
                } else if ((rc = cvt_cols_split(wd, nout, kp, W + k0 + JE * ld, w.ldw,
                                                (__nv_bfloat16 *)w.Ub + off, 3 * Vpad, Vpad, 1, ss.bg))) {
                    return rc;
                }
            }
            CF_CUDA_TRY(cudaEventRecord(ss.bg_done, ss.bg));
            // LU-3 (main)
            if ((rc = launch_rtrsm32<LP>(A00 + wd, w.ldw, below, wd, A00, w.ldw, false,
                                         split ? nullptr : (LP *)w.Ab, kMaxV, kMaxV, nullptr, st)))
                return rc;
            if (split && (rc = cvt_rows_split(below, wd, kMaxV, A00 + wd, w.ldw, w.Ab, 3 * kMaxV, kMaxV, 0, st)))
                return rc;
            CF_CUDA_TRY(cudaStreamWaitEvent(st, ss.side_done, 0));
            if (below <= 0 || right <= 0) continue;
            // A11 restricted to the slab's remaining columns (every row below)
            const int nslab = JE - (k0 + wd);
            float *C = A00 + wd + wd * ld;
            // depth: the step's columns rounded up to 64 (the operands are
            // zero past wd); the split form's three segments sit kMaxV apart
            const int Kin = split ? S * kMaxV : (wd + 63) / 64 * 64;
            if (nslab <= 0) continue;
            const int wn = v < nslab ? v : nslab;        // the next panel's columns
            const bool split_la = o.lookahead && nslab > wn;
            if (split_la) CF_CUDA_TRY(cudaEventRecord(la.fork, st));
            if ((rc = launch_schur_tc(below, split_la ? wn : nslab, Kin, w.Ab, S * kMaxV, w.Bb, S * kMaxV, C, w.ldw,
                                      bf16, false, st, 0)))
                return rc;
            if (split_la) {
                // the rest of the slab's columns beside the next TournPivot,
                // on the SMs its leaves leave free
                CF_CUDA_TRY(cudaStreamWaitEvent(la.s, la.fork, 0));
                int cap = sms - ceil_div(below, o.leaf_h);
                if (cap < sms / 4) cap = sms / 4;
                if ((rc = launch_schur_tc(below, nslab - wn, Kin, w.Ab, S * kMaxV,
                                          (const uint16_t *)w.Bb + (size_t)wn * S * kMaxV, S * kMaxV,
                                          C + (size_t)wn * ld, w.ldw, bf16, false, la.s, cap)))
                    return rc;
                CF_CUDA_TRY(cudaEventRecord(la.done, la.s));
                la_pending = true;
            }
        }
        if (la_pending) {
            CF_CUDA_TRY(cudaStreamWaitEvent(st, la.done, 0));
            la_pending = false;
        }
        CF_CUDA_TRY(cudaStreamWaitEvent(st, ss.bg_done, 0));    // the slab's pivot rows right of it
        if (JE < n) {
            // deferred update of everything right of and below the slab
            const int Vs = JE - J0, Vp = (Vs + 63) / 64 * 64, mr = n - JE;
            if (!split) {
                if ((rc = cvt_rows<LP>(mr, Vs, Vp, W + JE + J0 * ld, w.ldw, w.Lb, Vp, st))) return rc;
            } else if ((rc = cvt_rows_split(mr, Vs, Vp, W + JE + J0 * ld, w.ldw, w.Lb, 3 * Vp, Vp, 0, st))) {
                return rc;
            }
            if (tu && (rc = tu->begin(st))) return rc;
            // the last slabs' updates have few tiles: split K over the SMs
            const int ks = schur_tc_splitk(mr, mr, S * Vp, false);
            if ((rc = launch_schur_tc_splitk(mr, mr, S * Vp, w.Lb, S * Vp, w.Ub, S * Vpad, W + JE + JE * ld, w.ldw,
                                             bf16, false, ks, w.Psk, st, 0)))
                return rc;
            if (tu && (rc = tu->end(st, 2.0 * mr * (double)mr * Vs))) return rc;
        }
    }
    return CF_OK;
}

// ---------------------------------------------------------------------------
// Mixed Cholesky with FP8 e4m3 updates: the same two-level loop as below,
// with every trailing update's operand (the FP32 L10 block) quantized to e4m3
// with one FP32 scale per 128 x 128 tile, and the updates run by the FP8
// tensor-core kernel, which applies the tile scales per K-block of 128.
// Requires V to be a multiple of 128.
// ---------------------------------------------------------------------------
static int mixed_potrf_fp8(int n, MixedWS &w, int *info, const Opts &o, cudaStream_t st, Timer *tu) {
    const int v = o.v, V = pick_V(n, o, false);
    if (V % 128 != 0) return CF_ERR_UNSUPPORTED;
    const size_t ld = (size_t)w.ldw;
    float *W = w.W;
    const int nrb = ceil_div(n, 128);
    float *sc_slab = w.sc8;                                  // nrb x (V / 128)
    float *sc_step = w.sc8 + (size_t)nrb * (V / 128);        // nrb x 1
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
            // CH-2 in FP32 (no low-precision copy: the FP8 operand needs the
            // whole tile's amax first)
            if ((rc = launch_rtrsm32<__nv_bfloat16>(A00 + wd, w.ldw, below, wd, A00, w.ldw, true, nullptr, kMaxV,
                                                    kMaxV, info, st)))
                return rc;
            const int nslab = JE - (k0 + wd);
            if (nslab <= 0) continue;
            if ((rc = launch_quant_e4m3(below, wd, 128, A00 + wd, w.ldw, w.Ab, 128, sc_step, 1, st))) return rc;
            if ((rc = launch_schur_fp8(below, nslab, 128, w.Ab, 128, sc_step, 1, w.Ab, 128, sc_step, 1,
                                       A00 + wd + wd * ld, w.ldw, true, st)))
                return rc;
        }
        if (JE < n) {
            const int Vs = JE - J0, Vp8 = (Vs + 127) / 128 * 128, mr = n - JE;
            if ((rc = launch_quant_e4m3(mr, Vs, Vp8, W + JE + J0 * ld, w.ldw, w.Lb, Vp8, sc_slab, Vp8 / 128, st)))
                return rc;
            if (tu && (rc = tu->begin(st))) return rc;
            if ((rc = launch_schur_fp8(mr, mr, Vp8, w.Lb, Vp8, sc_slab, Vp8 / 128, w.Lb, Vp8, sc_slab, Vp8 / 128,
                                       W + JE + JE * ld, w.ldw, true, st)))
                return rc;
            if (tu && (rc = tu->end(st, (double)mr * (mr + 1.0) * Vs))) return rc;
        }
    }
    return CF_OK;
}

// ---------------------------------------------------------------------------
// Mixed Cholesky of W (lower, in place).
// ---------------------------------------------------------------------------
template <typename LP>
static int mixed_potrf(int n, MixedWS &w, int *info, const Opts &o, cudaStream_t st, Timer *tu, bool split) {
    const bool bf16 = std::is_same<LP, __nv_bfloat16>::value;
    const int v = o.v, V = pick_V(n, o, false);
    const int S = split ? 3 : 1;
    const size_t ld = (size_t)w.ldw;
    float *W = w.W;
    int rc;
    // LU-6 for the Cholesky: the in-slab update of the next panel's columns
    // first, the rest on the look-ahead stream beside the next A00 Cholesky;
    // the next panel solve (which rewrites the operand buffers) waits for it
    LookStream la;
    if (o.lookahead && (rc = la.open())) return rc;
    bool la_pending = false;
    const int sms = device_sms();
    for (int J0 = 0; J0 < n; J0 += V) {
        const int JE = J0 + V < n ? J0 + V : n;
        for (int k0 = J0; k0 < JE; k0 += v) {
            const int wd = v < JE - k0 ? v : JE - k0;
            const int m = n - k0;
            float *A00 = W + k0 + k0 * ld;
            if ((rc = launch_a00_chol32(A00, w.ldw, wd, k0, info, st))) return rc;
            if (la_pending) {
                CF_CUDA_TRY(cudaStreamWaitEvent(st, la.done, 0));
                la_pending = false;
            }
            const int below = m - wd;
            if (below <= 0) continue;
            // CH-2: L10 = A10 L00^{-T}, with its K-major low-precision copy
            if ((rc = launch_rtrsm32<LP>(A00 + wd, w.ldw, below, wd, A00, w.ldw, true, split ? nullptr : (LP *)w.Ab,
                                         kMaxV, kMaxV, info, st)))
                return rc;
            const int nslab = JE - (k0 + wd);
            if (nslab <= 0) continue;
            const void *Bop = w.Ab;
            if (split) {   // left (hi, hi, lo) and right (hi, lo, hi) forms of L10
                if ((rc = cvt_rows_split(below, wd, kMaxV, A00 + wd, w.ldw, w.Ab, 3 * kMaxV, kMaxV, 0, st))) return rc;
                if ((rc = cvt_rows_split(below, wd, kMaxV, A00 + wd, w.ldw, w.Bb, 3 * kMaxV, kMaxV, 1, st))) return rc;
                Bop = w.Bb;
            }
            const int Kin = split ? S * kMaxV : (wd + 63) / 64 * 64;   // as in the LU
            const int wn = v < nslab ? v : nslab;                         // the next panel's columns
            const bool split_la = o.lookahead && nslab > wn;
            if (split_la) CF_CUDA_TRY(cudaEventRecord(la.fork, st));
            float *C = A00 + wd + wd * ld;
            if ((rc = launch_schur_tc(below, split_la ? wn : nslab, Kin, w.Ab, S * kMaxV, Bop, S * kMaxV, C, w.ldw,
                                      bf16, true, st, 0)))
                return rc;
            if (split_la) {
                // rows and columns from wn on (the lower triangle keeps its diagonal)
                CF_CUDA_TRY(cudaStreamWaitEvent(la.s, la.fork, 0));
                const size_t off = (size_t)wn * S * kMaxV;
                if ((rc = launch_schur_tc(below - wn, nslab - wn, Kin, (const uint16_t *)w.Ab + off, S * kMaxV,
                                          (const uint16_t *)Bop + off, S * kMaxV, C + wn + (size_t)wn * ld, w.ldw,
                                          bf16, true, la.s, sms - 1)))
                    return rc;
                CF_CUDA_TRY(cudaEventRecord(la.done, la.s));
                la_pending = true;
            }
        }
        if (la_pending) {
            CF_CUDA_TRY(cudaStreamWaitEvent(st, la.done, 0));
            la_pending = false;
        }
        if (JE < n) {
            const int Vs = JE - J0, Vp = (Vs + 63) / 64 * 64, mr = n - JE;
            const void *Bop = w.Lb;
            if (!split) {
                if ((rc = cvt_rows<LP>(mr, Vs, Vp, W + JE + J0 * ld, w.ldw, w.Lb, Vp, st))) return rc;
            } else {
                if ((rc = cvt_rows_split(mr, Vs, Vp, W + JE + J0 * ld, w.ldw, w.Lb, 3 * Vp, Vp, 0, st))) return rc;
                if ((rc = cvt_rows_split(mr, Vs, Vp, W + JE + J0 * ld, w.ldw, w.Ub, 3 * Vp, Vp, 1, st))) return rc;
                Bop = w.Ub;
            }
            if (tu && (rc = tu->begin(st))) return rc;
            const int ks = schur_tc_splitk(mr, mr, S * Vp, true);
            if ((rc = launch_schur_tc_splitk(mr, mr, S * Vp, w.Lb, S * Vp, Bop, S * Vp, W + JE + JE * ld, w.ldw, bf16,
                                             true, ks, w.Psk, st, 0)))
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
    if ((rc = launch_trsv_f32(lu ? 0 : 2, n, nrhs, w.W, w.ldw, w.DinvL, w.G0, w.Rf, n, w.trsv_sync, st))) return rc;
    return launch_trsv_f32(lu ? 1 : 3, n, nrhs, w.W, w.ldw, lu ? w.DinvU : w.DinvL, w.G1, w.Rf, n, w.trsv_sync, st);
}

// ---------------------------------------------------------------------------
// GMRES-IR correction (Carson and Higham, SISC 2017/2018; the preconditioner
// applied in FP32 as in the multi-precision GMRES-IR analysis of Amestoy et
// al., 2021): for every column of r = w.R, left-preconditioned restarted
// GMRES on M^{-1} A d = M^{-1} r with M = the low-precision factors, the
// products with A in FP64 on the untouched A, classical Gram-Schmidt with one
// reorthogonalisation, Givens rotations of the small Hessenberg systems on
// the host; then X += d.  All right-hand sides advance together (one FP64
// product A [v_1 .. v_nrhs] per step).
// ---------------------------------------------------------------------------
// Z[i, c] = Y[perm[i], c] (perm == nullptr: copy)
__global__ void k_gather_rows(int n, int nrhs, const int *perm, const double *Y, double *Z) {
    const size_t tot = (size_t)n * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), c = (int)(e / n);
        Z[e] = Y[(size_t)(perm ? perm[i] : i) + (size_t)c * n];
    }
}

// Rf[:, c] = (float)(Z[:, c] / s_c), s_c = max_i |Z[i, c]| read from the bit
// patterns k_col_absmax leaves (1 if 0); and back, Z[:, c] = s_c Rf[:, c].
__global__ void k_to_f32_scaled(int n, int nrhs, const double *Z, const unsigned long long *sbits, float *Rf) {
    const size_t tot = (size_t)n * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const double sc = __longlong_as_double((long long)sbits[e / n]);
        Rf[e] = (float)(Z[e] / (sc > 0.0 ? sc : 1.0));
    }
}
__global__ void k_from_f32_scaled(int n, int nrhs, const float *Rf, const unsigned long long *sbits, double *Z) {
    const size_t tot = (size_t)n * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const double sc = __longlong_as_double((long long)sbits[e / n]);
        Z[e] = (sc > 0.0 ? sc : 1.0) * (double)Rf[e];
    }
}

// Z = M^{-1} Y with the FP32-stored factors.  Applied in FP64 arithmetic by
// default: in FP32 the Krylov relations are polluted at the FP32 level times
// the factors' condition, and GMRES stalls on the hard cases (e.g. unshifted
// uniform LU at N = 32768).  With FP8 factors (unit roundoff 2^-4) the
// factorization error dominates that level, and the FP32 solves (memory-
// bound, a fraction of the FP64 ones' time) are used.
static int apply_precond(int n, int nrhs, const double *Yin, double *Z, MixedWS &w, bool lu, bool f32,
                         cudaStream_t st) {
    const size_t blk = (size_t)n * nrhs;
    k_gather_rows<<<grid_for(blk), 256, 0, st>>>(n, nrhs, lu ? w.perm : nullptr, Yin, Z);
    CF_LAUNCH_CHECK();
    int rc;
    if (f32) {
        CF_CUDA_TRY(cudaMemsetAsync(w.sbits, 0, sizeof(unsigned long long) * nrhs, st));
        k_col_absmax<<<dim3(grid_for(n), nrhs), 256, 0, st>>>(n, nrhs, Z, n, w.sbits);
        CF_LAUNCH_CHECK();
        k_to_f32_scaled<<<grid_for(blk), 256, 0, st>>>(n, nrhs, Z, w.sbits, w.Rf);
        CF_LAUNCH_CHECK();
        if ((rc = solve_f32(n, nrhs, w, lu, st))) return rc;
        k_from_f32_scaled<<<grid_for(blk), 256, 0, st>>>(n, nrhs, w.Rf, w.sbits, Z);
        CF_LAUNCH_CHECK();
        return CF_OK;
    }
    if ((rc = launch_trsv_f64x(lu ? 0 : 2, n, nrhs, w.W, w.ldw, w.DinvL64, Z, n, w.trsv_sync, st))) return rc;
    return launch_trsv_f64x(lu ? 1 : 3, n, nrhs, w.W, w.ldw, lu ? w.DinvU64 : w.DinvL64, Z, n, w.trsv_sync, st);
}

// out[i * nrhs + c] (+)= <V_i[:, c], W[:, c]> for i < nv, fixed summation order.
static int block_dots(int n, int nrhs, const double *V, int nv, const double *W, double *out, int accumulate,
                      MixedWS &w, cudaStream_t st) {
    const int nch = ceil_div(n, kDotRows);
    k_dots_partial<<<dim3(nch, nv), 256, 0, st>>>(n, nrhs, V, W, w.part);
    CF_LAUNCH_CHECK();
    const int cnt = nv * nrhs;
    k_dots_final<<<ceil_div(cnt, 256), 256, 0, st>>>(nch, cnt, w.part, out, accumulate);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

static int gmres_correct(int n, int nrhs, const double *A, int lda, double *X, int ldx, MixedWS &w, bool lu,
                         bool prec_f32, bool pair, double tau, cudaStream_t st, Timer &tres, int *inner) {
    // products with A: tensor-core slices (w.use_tc), pair arithmetic or FP64
    const size_t blk = (size_t)n * nrhs;
    const int m = w.m;
    int rc;
    *inner = 0;
    // z0 = M^{-1} r, beta = ||z0||_2, v_0 = z0 / beta
    if ((rc = apply_precond(n, nrhs, w.R, w.Wv, w, lu, prec_f32, st))) return rc;
    if ((rc = block_dots(n, nrhs, w.Wv, 1, w.Wv, w.sq, 0, w, st))) return rc;
    k_normalize<<<grid_for(blk), 256, 0, st>>>(n, nrhs, w.sq, w.hcol, w.Wv, w.V);
    CF_LAUNCH_CHECK();
    std::vector<double> beta(nrhs);
    CF_CUDA_TRY(cudaMemcpyAsync(beta.data(), w.hcol, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, st));
    CF_CUDA_TRY(cudaStreamSynchronize(st));

    // per column: R (upper triangle of the rotated Hessenberg, column-major
    // (m+1) x m), rotations, rotated right-hand side g
    const int ldh = m + 1;
    std::vector<double> R((size_t)nrhs * ldh * m, 0.0), cs((size_t)nrhs * m, 1.0), sn((size_t)nrhs * m, 0.0);
    std::vector<double> g((size_t)nrhs * ldh, 0.0);
    std::vector<int> kdim(nrhs, 0);
    std::vector<char> done(nrhs, 0);
    for (int c = 0; c < nrhs; ++c) {
        g[(size_t)c * ldh] = beta[c];
        done[c] = !(beta[c] > 0.0);
    }
    std::vector<double> h1((size_t)(m + 2) * nrhs), h2((size_t)(m + 1) * nrhs);
    int k = 0;
    for (; k < m; ++k) {
        bool all = true;
        for (int c = 0; c < nrhs; ++c) all = all && done[c];
        if (all) break;
        const double *Vk = w.V + (size_t)k * blk;
        if ((rc = tres.begin(st))) return rc;
        rc = w.use_tc ? resid_tc_apply(w.rtc, nrhs, Vk, n, nullptr, 0, w.Y, n, w.rtcX, st)   // Y = A v_k
             : pair   ? launch_residual_pair(n, n, nrhs, A, lda, w.anorm, Vk, n, nullptr, 0, w.Y, n, w.pairws, st)
                      : launch_residual_f64(n, n, nrhs, A, lda, Vk, n, nullptr, 0, w.Y, n, st);
        if (rc) return rc;
        if ((rc = tres.end(st, 2.0 * n * (double)n * nrhs))) return rc;
        if ((rc = apply_precond(n, nrhs, w.Y, w.Wv, w, lu, prec_f32, st))) return rc;                // w = M^{-1} Y
        if ((rc = block_dots(n, nrhs, w.V, k + 1, w.Wv, w.hcol, 0, w, st))) return rc;               // CGS pass 1
        k_block_axpy<<<grid_for(blk), 256, 0, st>>>(n, nrhs, k + 1, w.V, w.hcol, w.Wv, n);
        CF_LAUNCH_CHECK();
        if ((rc = block_dots(n, nrhs, w.V, k + 1, w.Wv, w.coef, 0, w, st))) return rc;               // CGS pass 2
        k_block_axpy<<<grid_for(blk), 256, 0, st>>>(n, nrhs, k + 1, w.V, w.coef, w.Wv, n);
        CF_LAUNCH_CHECK();
        if ((rc = block_dots(n, nrhs, w.Wv, 1, w.Wv, w.sq, 0, w, st))) return rc;
        k_normalize<<<grid_for(blk), 256, 0, st>>>(n, nrhs, w.sq, w.hcol + (size_t)(k + 1) * nrhs, w.Wv,
                                                   w.V + (size_t)(k + 1) * blk);
        CF_LAUNCH_CHECK();
        CF_CUDA_TRY(cudaMemcpyAsync(h1.data(), w.hcol, sizeof(double) * (k + 2) * nrhs, cudaMemcpyDeviceToHost, st));
        CF_CUDA_TRY(cudaMemcpyAsync(h2.data(), w.coef, sizeof(double) * (k + 1) * nrhs, cudaMemcpyDeviceToHost, st));
        CF_CUDA_TRY(cudaStreamSynchronize(st));
        for (int c = 0; c < nrhs; ++c) {
            if (done[c]) continue;
            double *col = &R[((size_t)c * m + k) * ldh];
            for (int i = 0; i <= k; ++i) col[i] = h1[(size_t)i * nrhs + c] + h2[(size_t)i * nrhs + c];
            col[k + 1] = h1[(size_t)(k + 1) * nrhs + c];
            const bool breakdown = !(col[k + 1] > 0.0);
            double *csc = &cs[(size_t)c * m], *snc = &sn[(size_t)c * m], *gc = &g[(size_t)c * ldh];
            for (int i = 0; i < k; ++i) {
                const double t = csc[i] * col[i] + snc[i] * col[i + 1];
                col[i + 1] = -snc[i] * col[i] + csc[i] * col[i + 1];
                col[i] = t;
            }
            const double rr = std::hypot(col[k], col[k + 1]);
            csc[k] = rr > 0.0 ? col[k] / rr : 1.0;
            snc[k] = rr > 0.0 ? col[k + 1] / rr : 0.0;
            col[k] = rr;
            col[k + 1] = 0.0;
            gc[k + 1] = -snc[k] * gc[k];
            gc[k] = csc[k] * gc[k];
            kdim[c] = k + 1;
            if (breakdown || std::fabs(gc[k + 1]) <= tau * beta[c]) done[c] = 1;
        }
    }
    *inner = k;
    // y = R^{-1} g per column; X += V y
    int nv = 0;
    std::vector<double> cy((size_t)(m + 1) * nrhs, 0.0);
    for (int c = 0; c < nrhs; ++c) {
        const int kc = kdim[c];
        nv = kc > nv ? kc : nv;
        std::vector<double> y(kc > 0 ? kc : 1);
        for (int i = kc - 1; i >= 0; --i) {
            double t = g[(size_t)c * ldh + i];
            for (int q = i + 1; q < kc; ++q) t -= R[((size_t)c * m + q) * ldh + i] * y[q];
            const double d = R[((size_t)c * m + i) * ldh + i];
            y[i] = d != 0.0 ? t / d : 0.0;
        }
        for (int i = 0; i < kc; ++i) cy[(size_t)i * nrhs + c] = -y[i];
    }
    if (nv > 0) {
        CF_CUDA_TRY(cudaMemcpyAsync(w.coef, cy.data(), sizeof(double) * nv * nrhs, cudaMemcpyHostToDevice, st));
        k_block_axpy<<<grid_for(blk), 256, 0, st>>>(n, nrhs, nv, w.V, w.coef, X, ldx);
        CF_LAUNCH_CHECK();
        CF_CUDA_TRY(cudaStreamSynchronize(st));    // cy is host memory that goes out of scope
    }
    return CF_OK;
}

template <typename LP>
static int mixed_solve(int n, int nrhs, const double *A, int lda, const double *B, int ldb, double *X, int ldx,
                       int *info, cf_refine_stats *stats, void *work, size_t lwork, const Opts &o, bool lu,
                       bool split0, cudaStream_t st) {
    MixedWS w;
    int rc = carve_mixed(nullptr, n, nrhs, o, lu, &w);
    if (rc) return rc;
    if (work == nullptr || lwork < w.bytes) return CF_ERR_WORKSPACE;
    if ((rc = carve_mixed(work, n, nrhs, o, lu, &w))) return rc;
    if (w.use_tc) {
        w.rtc = resid_tc_layout(n, n);
        resid_tc_carve(&w.rtc, w.rtcA);
    }

    cf_refine_stats S{};
    ScopedEvent e0, e1, e2;
    CF_CUDA_TRY(e0.create());
    CF_CUDA_TRY(e1.create());
    CF_CUDA_TRY(e2.create());
    CF_CUDA_TRY(cudaEventRecord(e0, st));
    CF_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int), st));

    // ---- factorization (Cholesky retries with a diagonal shift on breakdown)
    Timer tupd, tres, tpair, ttourn, ttc, tprep;
    double shift = 0.0;
    int hinfo = 0;
    bool need_rowsum = true;     // row sums of |A| come with the first W = fl32(A)
    // one factorization of fl32(A) into w.W: split = BF16 hi + lo operands
    auto factorize = [&](bool split) -> int {
        const double u_lp = split                                  ? 0x1p-16
                            : std::is_same<LP, __nv_bfloat16>::value ? 0x1p-8
                            : std::is_same<LP, fp8_e4m3>::value    ? 0x1p-4
                                                                   : 0x1p-11;
        shift = 0.0;
        int rc2 = CF_OK;
        for (int attempt = 0; attempt < 4; ++attempt) {
            // W = fl32(A) (+ shift on the diagonal)
            if (need_rowsum) CF_CUDA_TRY(cudaMemsetAsync(w.rowsum, 0, sizeof(double) * (n > 0 ? n : 1), st));
            if (need_rowsum && w.use_tc) CF_CUDA_TRY(cudaMemsetAsync(w.rtc.Ef, 0, sizeof(int) * (size_t)w.rtc.mpad, st));
            rc2 = launch_to_f32_rowsum(n, A, lda, w.W, w.ldw, shift, need_rowsum ? w.rowsum : nullptr,
                                       need_rowsum && w.use_tc ? w.rtc.Ef : nullptr, st);
            if (rc2) return rc2;
            need_rowsum = false;
            CF_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int), st));
            if (split)
                rc2 = lu ? mixed_getrf<__nv_bfloat16>(n, w, info, o, st, &tupd, true, &ttourn)
                         : mixed_potrf<__nv_bfloat16>(n, w, info, o, st, &tupd, true);
            else if constexpr (std::is_same<LP, fp8_e4m3>::value)
                rc2 = lu ? CF_ERR_UNSUPPORTED : mixed_potrf_fp8(n, w, info, o, st, &tupd);
            else
                rc2 = lu ? mixed_getrf<LP>(n, w, info, o, st, &tupd, false, &ttourn)
                         : mixed_potrf<LP>(n, w, info, o, st, &tupd, false);
            if (rc2) return rc2;
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
        CF_CUDA_TRY(cudaMemcpyAsync(&hinfo, info, sizeof(int), cudaMemcpyDeviceToHost, st));
        int tstat = 0;
        if ((rc2 = tc_take_status(st, &tstat))) return rc2;
        if (tstat != 0) return CF_ERR_TIMEOUT;
        if ((rc2 = fp8_take_status(st, &tstat))) return rc2;
        if (tstat != 0) return CF_ERR_TIMEOUT;
        return CF_OK;
    };
    bool split = split0;
    if ((rc = factorize(split))) return rc;
    S.shift = shift;
    CF_CUDA_TRY(cudaEventRecord(e1, st));
    S.info = hinfo;

    // ---- refinement
    const int ldr = n;
    unsigned long long *nR = w.norms, *nX = w.norms + nrhs, *nB = w.norms + 2 * nrhs, *nA = w.norms + 3 * nrhs;
    CF_CUDA_TRY(cudaMemsetAsync(w.norms, 0, sizeof(unsigned long long) * (3 * nrhs + 2), st));
    k_max_reduce<<<grid_for(n), 256, 0, st>>>(n, w.rowsum, nA);
    CF_LAUNCH_CHECK();
    w.anorm = nA;
    k_col_absmax<<<dim3(grid_for(n), nrhs), 256, 0, st>>>(n, nrhs, B, ldb, nB);
    CF_LAUNCH_CHECK();
    // x = 0, r = b
    for (int c = 0; c < nrhs; ++c) CF_CUDA_TRY(cudaMemsetAsync(X + (size_t)c * ldx, 0, sizeof(double) * n, st));
    k_copy_cols<<<grid_for((size_t)n * nrhs), 256, 0, st>>>(n, nrhs, B, ldb, w.R, ldr);
    CF_LAUNCH_CHECK();

    auto diag_inverses = [&]() -> int {
        int rc2 = launch_diag_inverse(lu ? 0 : 2, n, w.W, w.ldw, w.DinvL, st);
        if (rc2 == CF_OK && lu) rc2 = launch_diag_inverse(1, n, w.W, w.ldw, w.DinvU, st);
        if (rc2 == CF_OK) rc2 = launch_neighbor_premul(lu ? 0 : 2, n, w.W, w.ldw, w.DinvL, w.G0, st);
        if (rc2 == CF_OK) rc2 = launch_neighbor_premul(lu ? 1 : 3, n, w.W, w.ldw, lu ? w.DinvU : w.DinvL, w.G1, st);
        return rc2;
    };
    if (S.info == 0 && (rc = diag_inverses())) return rc;

    std::vector<unsigned long long> hn(3 * nrhs + 2);
    std::vector<double> hscale(nrhs);
    double eta_prev = HUGE_VAL, eta_pp = HUGE_VAL, eta = HUGE_VAL, eta_best = HUGE_VAL;
    int it = 0, stall = 0, solver = 0, it_limit = o.max_iter, last_inner = 0;
    bool used_gmres = false;
    bool converged = false, escalated = false;
    // the digit slices of A for the tensor-core residuals, cut once per solve
    // (the row exponent fields came with the first W = fl32(A))
    if (w.use_tc) {
        if ((rc = tprep.begin(st))) return rc;
        if ((rc = resid_tc_prepare(&w.rtc, A, lda, true, st))) return rc;
        if ((rc = tprep.end(st, 0.0))) return rc;
    }
    // R = B - A X on the tensor cores, in pair arithmetic or in FP64
    auto residual = [&](bool pair) -> int {
        Timer &t = w.use_tc ? ttc : pair ? tpair : tres;
        int rc2 = t.begin(st);
        if (rc2) return rc2;
        rc2 = w.use_tc ? resid_tc_apply(w.rtc, nrhs, X, ldx, B, ldb, w.R, ldr, w.rtcX, st)
              : pair   ? launch_residual_pair(n, n, nrhs, A, lda, w.anorm, X, ldx, B, ldb, w.R, ldr, w.pairws, st)
                       : launch_residual_f64(n, n, nrhs, A, lda, X, ldx, B, ldb, w.R, ldr, st);
        if (rc2) return rc2;
        return t.end(st, 2.0 * n * (double)n * nrhs);
    };
    // eta = max_c ||r_c|| / (||A|| ||x_c|| + ||b_c||) and the per-column
    // scales of the next correction's right-hand side (one synchronisation)
    auto measure = [&]() -> int {
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
        return CF_OK;
    };
    for (;; ++it) {
        bool pair = false;
        if (it > 0) {
            // backward error this residual should show: the last one times
            // the last step's contraction; before two refinement residuals
            // exist (the first eta is that of x = 0) a contraction of
            // kAssumedRate is assumed: erring high costs at most a pair
            // residual that is then redone in FP64
            const double rate = (it >= 3 && eta_pp < HUGE_VAL && eta_pp > 0.0) ? std::fmin(1.0, eta_prev / eta_pp)
                                                                              : kAssumedRate;
            const double pred = eta_prev < HUGE_VAL ? eta_prev * rate : HUGE_VAL;
            pair = !w.use_tc && !o.fp64_residual && !(pred < kPairFloor);
            if ((rc = residual(pair))) return rc;
        }
        if ((rc = measure())) return rc;
        if (pair && eta < kPairFloor) {   // too close to the pair residual's accuracy: redo in FP64
            if ((rc = residual(false))) return rc;
            if ((rc = measure())) return rc;
        }
        if (it == 1) S.eta0 = eta;
        if (eta <= o.tol) { converged = true; break; }
        if (eta < eta_best) {          // keep the best iterate
            eta_best = eta;
            k_copy_cols<<<grid_for((size_t)n * nrhs), 256, 0, st>>>(n, nrhs, X, ldx, w.Xbest, n);
            CF_LAUNCH_CHECK();
        }
        // Classical refinement that fails to cut eta by kSwitchRate in one
        // step hands over to GMRES-IR (at that rate the remaining classical
        // steps would each cost as much as an inner GMRES step and converge
        // slower); GMRES-IR that fails to halve eta twice in a row, the step
        // budget, or a breakdown of the low-precision factorization ends the
        // attempt.
        bool give_up = it >= it_limit || S.info != 0;
        if (!give_up && solver == 0 && it >= 1 && !(eta <= kSwitchRate * eta_prev)) {
            solver = 1;
            if ((rc = launch_diag_inverse64(lu ? 0 : 2, n, w.W, w.ldw, w.DinvL64, st))) return rc;
            if (lu && (rc = launch_diag_inverse64(1, n, w.W, w.ldw, w.DinvU64, st))) return rc;
        } else if (!give_up && solver == 1 &&
                   (!(eta <= 0.5 * eta_prev) ||
                    (!split && !std::is_same<LP, fp8_e4m3>::value && last_inner >= kSlowInner &&
                     !(eta <= kSlowGain * eta_prev)))) {
            // before escalating one failed (or slow) GMRES-IR step is enough
            // (refactoring costs about one step); after it, two failed in a row
            give_up = ++stall >= (split ? 2 : 1);
        } else {
            stall = 0;
        }
        if (give_up) {
            if (split) break;
            // Escalate once: refactor with split BF16 updates (hi + lo
            // operands, 16 significant bits) and refine on from the best
            // iterate with a fresh step budget.
            split = escalated = true;
            if ((rc = factorize(true))) return rc;
            S.info = hinfo;
            S.shift = shift;
            if (S.info != 0) break;
            if ((rc = diag_inverses())) return rc;
            if (eta_best < eta) {
                k_copy_cols<<<grid_for((size_t)n * nrhs), 256, 0, st>>>(n, nrhs, w.Xbest, n, X, ldx);
                CF_LAUNCH_CHECK();
            }
            solver = 0;
            stall = 0;
            last_inner = 0;
            eta_prev = eta_pp = HUGE_VAL;
            it_limit = it + o.max_iter;
            continue;
        }
        eta_pp = eta_prev;
        eta_prev = eta;
        if (solver == 0) {
            CF_CUDA_TRY(cudaMemcpyAsync(w.scale, hscale.data(), sizeof(double) * nrhs, cudaMemcpyHostToDevice, st));
            k_gather_scale<<<grid_for((size_t)n * nrhs), 256, 0, st>>>(n, nrhs, lu ? w.perm : nullptr, w.R, ldr,
                                                                      w.scale, w.Rf, n);
            CF_LAUNCH_CHECK();
            if ((rc = solve_f32(n, nrhs, w, lu, st))) return rc;
            k_axpy_update<<<grid_for((size_t)n * nrhs), 256, 0, st>>>(n, nrhs, w.Rf, n, w.scale, X, ldx);
            CF_LAUNCH_CHECK();
        } else {
            int inner = 0;
            used_gmres = true;
            const bool prec_f32 = std::is_same<LP, fp8_e4m3>::value && !split;
            const bool gpair = !o.fp64_residual;
            if ((rc = gmres_correct(n, nrhs, A, lda, X, ldx, w, lu, prec_f32, gpair, kGmresTol, st,
                                    w.use_tc ? ttc : gpair ? tpair : tres, &inner)))
                return rc;
            S.gmres_iterations += inner;
            last_inner = inner;
        }
    }
    if (!converged && eta_best < eta) {   // hand back the best iterate
        k_copy_cols<<<grid_for((size_t)n * nrhs), 256, 0, st>>>(n, nrhs, w.Xbest, n, X, ldx);
        CF_LAUNCH_CHECK();
        eta = eta_best;
    }
    CF_CUDA_TRY(cudaEventRecord(e2, st));
    CF_CUDA_TRY(cudaEventSynchronize(e2));
    int tstat = 0;
    if ((rc = trsv_take_status(st, &tstat))) return rc;
    if (tstat != 0) return CF_ERR_TIMEOUT;
    if ((rc = rtc_take_status(st, &tstat))) return rc;
    if (tstat != 0) return CF_ERR_TIMEOUT;
    float f_ms = 0, r_ms = 0;
    cudaEventElapsedTime(&f_ms, e0, e1);
    cudaEventElapsedTime(&r_ms, e1, e2);
    S.iterations = it;
    S.solver = used_gmres ? 1 : 0;
    S.escalated = escalated ? 1 : 0;
    S.converged = converged ? 1 : 0;
    S.eta = eta;
    S.factor_ms = f_ms;
    S.refine_ms = r_ms;
    S.residual_ms = tres.ms();
    S.residual_launches = tres.launches;
    S.pair_ms = tpair.ms();
    S.pair_launches = tpair.launches;
    S.tc_ms = ttc.ms();
    S.tc_launches = ttc.launches;
    S.tc_prep_ms = tprep.ms();
    S.tourn_ms = ttourn.ms();
    S.tourn_launches = ttourn.launches;
    S.tourn_flops = ttourn.flops;
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
    if (prec != CF_BF16 && prec != CF_F16 && prec != CF_FP8E4M3 && prec != CF_BF16X3) return -9;
    if (info == nullptr) return -10;
    return CF_OK;
}

}  // namespace cf

using namespace cf;

static size_t mixed_ws_size(int n, int nrhs, cf_prec prec, const cf_options *opt, bool lu) {
    (void)prec;
    Opts o;
    if (resolve_options(opt, &o) != CF_OK) return 0;
    if (lu && mixed_lu_defaults(&o) != CF_OK) return 0;
    if (!lu && (o.outer_V % o.v) != 0) return 0;
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
    if (lu && (rc = mixed_lu_defaults(&o))) return rc;
    if (!lu && (o.outer_V % o.v) != 0) return CF_ERR_UNSUPPORTED;
    if (n == 0 || nrhs == 0) {
        if (stats) { memset(stats, 0, sizeof(*stats)); stats->converged = 1; }
        return CF_OK;
    }
    if (prec == CF_BF16 || prec == CF_BF16X3)
        return mixed_solve<__nv_bfloat16>(n, nrhs, A, lda, B, ldb, X, ldx, info, stats, work, lwork, o, lu,
                                          prec == CF_BF16X3, st);
    if (prec == CF_FP8E4M3) {
        if (lu) return -9;                     // FP8 updates: Cholesky only
        if (pick_V(n, o, false) % 128 != 0) return CF_ERR_UNSUPPORTED;
        return mixed_solve<fp8_e4m3>(n, nrhs, A, lda, B, ldb, X, ldx, info, stats, work, lwork, o, lu, false, st);
    }
    return mixed_solve<__half>(n, nrhs, A, lda, B, ldb, X, ldx, info, stats, work, lwork, o, lu, false, st);
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
