// cf_pair.cu -- R-1 on the FP32 pipes: R = B - A X with FP64 operands,
// computed in pairs of FP32 numbers ("double-float" arithmetic).
//
// GB300 runs FP64 at ~2 operations per clock per SM and FP32 at 128, so the
// FP64 residual (cf_gemm64.cu) is bound by the FP64 pipe while HBM idles.
// This kernel forms every term a_ij x_j as an FP32 pair instead:
//
//   * A is read in FP64 once and split on the fly, with integer operations
//     only, into ah (the leading 24 bits of a 2^-ea, truncated) and al (the
//     remaining 29 bits rounded to 24), so ah + al = a 2^-ea to 2^-47
//     relative.  2^ea is a power of two above max |a_ij| (the caller's bound),
//     which keeps every scaled element below 2 and every product in FP32
//     range; elements below 2^-74 of the bound are dropped (at most n 2^-74 of
//     ||A|| ||x|| in all).
//   * X is split once per call (k_pair_split_x) into xh = fl32(x 2^-sx),
//     xl = fl32(x 2^-sx - xh) with 2^sx a power of two per column.
//   * Per term: the exact product ah xh = p + e (FMA), the cross products
//     ah xl + al xh, and Knuth's TwoSum of p into the running pair (hi, lo):
//     twelve FP32 operations, issued as packed f32x2 instructions over two
//     right-hand sides.
//   * Every kTile (16) terms the pair is added into an FP64 accumulator
//     and restarted, so the pair's 48 bits are relative to the partial sum of
//     one chunk, not of the whole row.
//
// Accuracy: about 2^-48 sqrt(kTile) of the largest partial sums of a chunk
// (the running pair's low word collects the rounding errors of the chunk and
// itself rounds at 2^-24 of its size): from ~1e-16 of ||A||_inf ||x||_inf
// on dense rows to a few 1e-14 on rows dominated by one term (the FP64 kernel
// reaches ~1e-16).  That is ample for the residual of a refinement step whose
// backward error is above ~1e-12 and for the matrix-vector products of
// GMRES; the mixed solvers take their last, certifying residual in FP64.
#include "cf_common.cuh"
#include "cf_kernels.cuh"

namespace cf {

namespace {
constexpr int kPairThreads = 256;  // rows per CTA (one per thread)
constexpr int kTile = 16;          // terms per stage, and between FP64 restarts
constexpr int kStages = 3;         // stages in shared memory
constexpr int kPairMaxSplit = 8;   // split of the k range over CTAs (partial sums in the workspace)
constexpr int kPairGroup = 16;     // right-hand sides per pass
}  // namespace

// Power-of-two exponent of a positive bound given by its FP64 bit pattern (0
// for zero, subnormal or non-finite bounds).
__device__ __forceinline__ int pair_scale_exp(unsigned long long bits) {
    const int e = (int)((bits >> 52) & 0x7ff);
    return (e == 0 || e == 0x7ff) ? 0 : e - 1023;
}

// a 2^-ea = ah + al (see the file comment).  Subnormal a counts as zero;
// |a| 2^-ea >= 2^128 (a bound that was too small) and inf / NaN give NaN.
__device__ __forceinline__ void pair_split_a(double a, int ea, float &ah, float &al) {
    const unsigned hw = (unsigned)__double2hiint(a), lw = (unsigned)__double2loint(a);
    const int e = (int)((hw >> 20) & 0x7ffu);
    const int d = e - ea;                                   // biased exponent of a 2^-ea
    const unsigned sgn = hw & 0x80000000u;
    const unsigned t = (hw & 0x7fffffffu) - ((unsigned)(896 + ea) << 20);   // rebias 1023 -> 127, scale
    const float h = __uint_as_float(__funnelshift_l(lw, t, 3) | sgn);        // 8 exponent + 23 mantissa bits
    const float r = __uint2float_rn(lw & 0x1fffffffu);                       // the 29 bits below
    const float sc = __uint_as_float(((unsigned)(d - 948) << 23) | sgn);     // +-2^(d - 1075)
    const float l = __fmul_rn(r, sc);
    const bool special = e == 0x7ff || d > 1150;
    const bool fast = (unsigned)(d - 949) <= 201u && e != 0 && !special;     // 2^-74 <= |a 2^-ea| < 2^128
    ah = fast ? h : (special ? __uint_as_float(0x7fc00000u) : 0.f);
    al = fast ? l : 0.f;
}

// Exact FP32 -> FP64 from the bit pattern (subnormal -> 0, inf / NaN -> NaN).
__device__ __forceinline__ double pair_f2d(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned mag = u & 0x7fffffffu;
    double d = __hiloint2double((int)((u & 0x80000000u) | ((mag >> 3) + 0x38000000u)), (int)(u << 29));
    d = mag < 0x00800000u ? 0.0 : d;
    return mag >= 0x7f800000u ? __longlong_as_double(0x7ff8000000000000LL) : d;
}

// (hi, lo) += (ah + al)(xh + xl) for two right-hand sides at once.  nah = -ah.
// Every operation is explicitly rounded; subtractions are FMAs with -1.
__device__ __forceinline__ void pair_term(float2 &hi, float2 &lo, float2 ah, float2 al, float2 nah, float2 xh,
                                          float2 xl) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 np = __fmul2_rn(nah, xh);                 // -p, p = fl(ah xh)
    const float2 e = __ffma2_rn(ah, xh, np);               // ah xh - p, exact
    float2 l = __ffma2_rn(ah, xl, lo);
    l = __ffma2_rn(al, xh, l);
    l = __fadd2_rn(l, e);
    const float2 s = __ffma2_rn(np, m1, hi);               // s = fl(hi + p)
    const float2 bb = __ffma2_rn(hi, m1, s);               // s - hi
    const float2 t2 = __ffma2_rn(__ffma2_rn(bb, m1, s), m1, hi);   // hi - (s - bb)
    const float2 t3n = __fadd2_rn(np, bb);                 // -(p - bb)
    lo = __fadd2_rn(l, __ffma2_rn(t3n, m1, t2));           // TwoSum error of hi + p
    hi = s;
}

// Split one group of NR right-hand sides (columns c0 .. c0+NR-1 of X, zeros
// past nrhs): one CTA per column.  Xs holds, per term p, NR/2 float4
// {xh_c, xh_c+1, xl_c, xl_c+1}; sx[c] the column's scale exponent.
template <int NR>
__global__ void __launch_bounds__(256) k_pair_split_x(int n, int nrhs, const double *__restrict__ X, int ldx,
                                                      float *__restrict__ Xs, int *__restrict__ sx) {
    constexpr int NQ = NR / 2;
    const int c = blockIdx.x;
    const bool live = c < nrhs;
    __shared__ double wmax[8];
    double mx = 0.0;
    if (live)
        for (int i = threadIdx.x; i < n; i += 256) {
            const double v = fabs(X[(size_t)i + (size_t)c * ldx]);
            mx = (v > mx || v != v) ? v : mx;
        }
    for (int o = 16; o > 0; o >>= 1) {
        const double t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = (t > mx || t != t) ? t : mx;
    }
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = mx;
    __syncthreads();
    mx = wmax[0];
    for (int w = 1; w < 8; ++w) mx = (wmax[w] > mx || wmax[w] != wmax[w]) ? wmax[w] : mx;
    const int s = (mx > 0.0 && mx <= 1.7976931348623157e308) ? ilogb(mx) : 0;
    if (threadIdx.x == 0) sx[c] = s;
    const int q = c >> 1, half = c & 1;
    for (int i = threadIdx.x; i < n; i += 256) {
        float h = 0.f, l = 0.f;
        if (live) {
            const double v = ldexp(X[(size_t)i + (size_t)c * ldx], -s);
            h = __double2float_rn(v);
            l = __double2float_rn(v - (double)h);
        }
        float *dst = Xs + ((size_t)i * NQ + q) * 4;
        dst[half] = h;
        dst[2 + half] = l;
    }
}

__device__ __forceinline__ void pair_cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void pair_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void pair_cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void pair_cp_async8(void *dst, const void *src, unsigned src_bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(src_bytes)
                 : "memory");
}

// Shared memory of k_residual_pair<NR>: kStages stages of kTile terms, the A
// elements of the CTA's 256 rows and the split X values.
template <int NR>
constexpr size_t pair_smem_bytes() {
    return (size_t)kStages * kTile * kPairThreads * sizeof(double) + (size_t)kStages * kTile * (NR / 2) * 16;
}

// Partial sums of A X over the k range of blockIdx.y for 256 rows (one per
// thread) x NR right-hand sides.  All warps walk the same k sequence in
// stages of kTile terms: the stage's A elements (one 8-byte copy per thread
// and term: coalesced 2 KB column segments) and split X values go to shared
// memory by cp.async, kStages - 1 stages ahead of the one being summed, so
// that ~100 KB per SM are in flight without holding registers.
// P == nullptr: R = B - 2^(ea + sx) S directly (B null: R = A X); else the
// unscaled partials go to P[ks][c][m].
template <int NR>
__global__ void __launch_bounds__(kPairThreads, 2)
k_residual_pair(int m, int n, int kspan, const double *__restrict__ A, int lda, const unsigned long long *amax,
                const float4 *__restrict__ Xs, const int *__restrict__ sx, const double *B, int ldb, double *R,
                int ldr, double *P) {
    constexpr int NQ = NR / 2;
    constexpr int XT = kTile * NQ;                          // float4 per X stage
    extern __shared__ __align__(16) unsigned char pair_smem[];
    double *as = reinterpret_cast<double *>(pair_smem);     // [kStages][kTile][kPairThreads]
    float4 *xs = reinterpret_cast<float4 *>(as + (size_t)kStages * kTile * kPairThreads);   // [kStages][XT]
    const int row = blockIdx.x * kPairThreads + threadIdx.x;
    const bool okr = row < m;
    const int k0 = blockIdx.y * kspan, k1 = min(n, k0 + kspan);
    const int ntile = k1 > k0 ? (k1 - k0 + kTile - 1) / kTile : 0;
    const int ea = pair_scale_exp(*amax);

    // stage t -> buffer t % kStages; rows past m and terms past k1 are zero
    // (zero-filled copies: a = 0 and x = 0 add nothing)
    auto issue = [&](int t) {
        const int base = k0 + t * kTile, b = t % kStages;
        double *ad = as + (size_t)b * kTile * kPairThreads + threadIdx.x;
#pragma unroll
        for (int tt = 0; tt < kTile; ++tt) {
            const bool ok = okr && base + tt < k1;
            const double *src = ok ? A + (size_t)row + (size_t)(base + tt) * lda : A;
            pair_cp_async8(ad + tt * kPairThreads, src, ok ? 8u : 0u);
        }
        float4 *xd = xs + (size_t)b * XT;
        for (int i = threadIdx.x; i < XT; i += kPairThreads) {
            if (base + i / NQ < k1) pair_cp_async16(xd + i, Xs + (size_t)base * NQ + i);
            else xd[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
#pragma unroll
    for (int t = 0; t < kStages - 1; ++t) {
        if (t < ntile) issue(t);
        pair_cp_commit();
    }

    float2 hi[NQ], lo[NQ];
    double acc[NR];
#pragma unroll
    for (int q = 0; q < NQ; ++q) hi[q] = lo[q] = make_float2(0.f, 0.f);
#pragma unroll
    for (int c = 0; c < NR; ++c) acc[c] = 0.0;
    // Restart: both words of the running pairs go into the FP64
    // accumulators.  (An FP32 accumulator for the low words would round at
    // 2^-24 of the largest chunk's low word on every later add, which on
    // rows with one dominant term is as large as the error the restarts
    // avoid.)
    auto flush = [&]() {
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            acc[2 * q] += pair_f2d(hi[q].x) + pair_f2d(lo[q].x);
            acc[2 * q + 1] += pair_f2d(hi[q].y) + pair_f2d(lo[q].y);
            hi[q] = lo[q] = make_float2(0.f, 0.f);
        }
    };

    for (int t = 0; t < ntile; ++t) {
        pair_cp_wait<kStages - 2>();                        // stage t has landed
        __syncthreads();                                    // ... for every thread; stage t - 1 is free
        if (t + kStages - 1 < ntile) issue(t + kStages - 1);
        pair_cp_commit();
        const double *at = as + (size_t)(t % kStages) * kTile * kPairThreads + threadIdx.x;
        const float4 *xt = xs + (size_t)(t % kStages) * XT;
#pragma unroll 4
        for (int tt = 0; tt < kTile; ++tt) {
            float ah, al;
            pair_split_a(at[tt * kPairThreads], ea, ah, al);
            const float2 AH = make_float2(ah, ah), AL = make_float2(al, al), NAH = make_float2(-ah, -ah);
            const float4 *xp = xt + tt * NQ;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const float4 xv = xp[q];
                pair_term(hi[q], lo[q], AH, AL, NAH, make_float2(xv.x, xv.y), make_float2(xv.z, xv.w));
            }
        }
        flush();                                            // every kTile = 16 terms
    }
    pair_cp_wait<0>();
    if (!okr) return;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = 2 * q + h;
            const double s = acc[c] + (pair_f2d(h ? hi[q].y : hi[q].x) + pair_f2d(h ? lo[q].y : lo[q].x));
            if (P) {
                P[((size_t)blockIdx.y * NR + c) * m + row] = s;
            } else {
                const double ax = ldexp(s, ea + sx[c]);
                R[(size_t)row + (size_t)c * ldr] = B ? B[(size_t)row + (size_t)c * ldb] - ax : ax;
            }
        }
    }
}

// R = B - 2^(ea + sx) sum_ks P[ks]  (fixed order over ks)
__global__ void k_pair_finish(int m, int nc, int NR, int ks, const double *__restrict__ P,
                              const unsigned long long *amax, const int *__restrict__ sx, const double *B, int ldb,
                              double *R, int ldr) {
    const int ea = pair_scale_exp(*amax);
    const size_t tot = (size_t)m * nc;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int r = (int)(e % m), c = (int)(e / m);
        double s = 0.0;
        for (int k = 0; k < ks; ++k) s += P[((size_t)k * NR + c) * m + r];
        const double ax = ldexp(s, ea + sx[c]);
        R[(size_t)r + (size_t)c * ldr] = B ? B[(size_t)r + (size_t)c * ldb] - ax : ax;
    }
}

// max |a_ij| as FP64 bits (out must start at 0); 256 threads per CTA.
__global__ void __launch_bounds__(256) k_mat_absmax(int m, int n, const double *__restrict__ A, int lda, unsigned long long *out) {
    const size_t tot = (size_t)m * n;
    double mx = 0.0;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const double v = fabs(A[(e % m) + (e / m) * (size_t)lda]);
        mx = (v > mx || v != v) ? v : mx;
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double t = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = (t > mx || t != t) ? t : mx;
    }
    __shared__ double wm[8];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) mx = (wm[w] > mx || wm[w] != wm[w]) ? wm[w] : mx;
        atomicMax(out, (unsigned long long)__double_as_longlong(mx));   // one atomic per CTA
    }
}

namespace {

int sm_count_pair() { return device_sm_count(); }

template <int NR>
int resident_ctas() {
    static const int occ = [] {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, k_residual_pair<NR>, kPairThreads,
                                                          pair_smem_bytes<NR>()) != cudaSuccess ||
            o <= 0) {
            cudaGetLastError();
            o = 1;
        }
        return o;
    }();
    return occ;
}

// Split of the k range over CTAs: the smallest split whose grid fills the
// last wave of CTA slots within 2% of the best one.
int pick_split(int row_blocks, int n, int slots) {
    double best = 0.0;
    double fill[kPairMaxSplit + 1] = {};
    for (int ks = 1; ks <= kPairMaxSplit; ++ks) {
        if (ks > 1 && n / ks < 256) break;
        const long long c = (long long)row_blocks * ks;
        const long long waves = (c + slots - 1) / slots;
        fill[ks] = (double)c / (double)(waves * slots);
        best = fill[ks] > best ? fill[ks] : best;
    }
    for (int ks = 1; ks <= kPairMaxSplit; ++ks)
        if (fill[ks] >= best - 0.02) return ks;
    return 1;
}

template <int NR>
int launch_group(int m, int n, int nc, const double *A, int lda, const unsigned long long *amax, const double *X,
                 int ldx, const double *B, int ldb, double *R, int ldr, float *Xs, int *sx, double *P,
                 cudaStream_t st) {
    k_pair_split_x<NR><<<NR, 256, 0, st>>>(n, nc, X, ldx, Xs, sx);
    CF_LAUNCH_CHECK();
    CF_CUDA_TRY(cudaFuncSetAttribute(k_residual_pair<NR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)pair_smem_bytes<NR>()));   // per device: set on every call
    const int rb = ceil_div(m, kPairThreads);
    const int ks = pick_split(rb, n, sm_count_pair() * resident_ctas<NR>());
    const int kspan = ceil_div(ceil_div(n, ks), kTile) * kTile;
    dim3 grid(rb, ks);
    k_residual_pair<NR><<<grid, kPairThreads, pair_smem_bytes<NR>(), st>>>(m, n, kspan, A, lda, amax,
                                                          reinterpret_cast<const float4 *>(Xs), sx, B, ldb, R, ldr,
                                                          ks > 1 ? P : nullptr);
    CF_LAUNCH_CHECK();
    if (ks > 1) {
        size_t g = ((size_t)m * nc + 255) / 256;
        if (g > 4096) g = 4096;
        k_pair_finish<<<(int)g, 256, 0, st>>>(m, nc, NR, ks, P, amax, sx, B, ldb, R, ldr);
        CF_LAUNCH_CHECK();
    }
    return CF_OK;
}

}  // namespace

size_t pair_residual_ws_bytes(int m, int n) {
    Carver cv(nullptr);
    const size_t mm = m > 0 ? m : 1, nn = n > 0 ? n : 1;
    cv.take<float>(nn * kPairGroup * 2);                       // Xs
    cv.take<int>(kPairGroup);                                  // sx
    cv.take<double>((size_t)kPairMaxSplit * kPairGroup * mm);  // P
    cv.take<unsigned long long>(1);                            // max |a| (standalone entry point)
    return cv.size();
}

int launch_residual_pair(int m, int n, int nrhs, const double *A, int lda, const unsigned long long *amax,
                         const double *X, int ldx, const double *B, int ldb, double *R, int ldr, void *ws,
                         cudaStream_t st) {
    if (m <= 0 || nrhs <= 0) return CF_OK;
    Carver cv(ws);
    const size_t nn = n > 0 ? n : 1;
    float *Xs = cv.take<float>(nn * kPairGroup * 2);
    int *sx = cv.take<int>(kPairGroup);
    double *P = cv.take<double>((size_t)kPairMaxSplit * kPairGroup * m);
    if (n <= 0) {   // R = B (or 0)
        for (int c = 0; c < nrhs; ++c) {
            if (B)
                CF_CUDA_TRY(cudaMemcpyAsync(R + (size_t)c * ldr, B + (size_t)c * ldb, sizeof(double) * m,
                                            cudaMemcpyDeviceToDevice, st));
            else
                CF_CUDA_TRY(cudaMemsetAsync(R + (size_t)c * ldr, 0, sizeof(double) * m, st));
        }
        return CF_OK;
    }
    for (int c0 = 0; c0 < nrhs; c0 += kPairGroup) {
        const int nc = min(kPairGroup, nrhs - c0);
        const double *Xc = X + (size_t)c0 * ldx;
        const double *Bc = B ? B + (size_t)c0 * ldb : nullptr;
        double *Rc = R + (size_t)c0 * ldr;
        int rc;
        if (nc <= 2) rc = launch_group<2>(m, n, nc, A, lda, amax, Xc, ldx, Bc, ldb, Rc, ldr, Xs, sx, P, st);
        else if (nc <= 4) rc = launch_group<4>(m, n, nc, A, lda, amax, Xc, ldx, Bc, ldb, Rc, ldr, Xs, sx, P, st);
        else if (nc <= 8) rc = launch_group<8>(m, n, nc, A, lda, amax, Xc, ldx, Bc, ldb, Rc, ldr, Xs, sx, P, st);
        else rc = launch_group<16>(m, n, nc, A, lda, amax, Xc, ldx, Bc, ldb, Rc, ldr, Xs, sx, P, st);
        if (rc) return rc;
    }
    return CF_OK;
}

// Standalone form: the bound is max |a_ij|, computed here.
int launch_residual_pair_auto(int m, int n, int nrhs, const double *A, int lda, const double *X, int ldx,
                              const double *B, int ldb, double *R, int ldr, void *ws, cudaStream_t st) {
    if (m <= 0 || nrhs <= 0) return CF_OK;
    Carver cv(ws);
    const size_t mm = m > 0 ? m : 1, nn = n > 0 ? n : 1;
    cv.take<float>(nn * kPairGroup * 2);
    cv.take<int>(kPairGroup);
    cv.take<double>((size_t)kPairMaxSplit * kPairGroup * mm);
    unsigned long long *amax = cv.take<unsigned long long>(1);
    CF_CUDA_TRY(cudaMemsetAsync(amax, 0, sizeof(unsigned long long), st));
    if (n > 0) {
        size_t g = ((size_t)m * n + 255) / 256;
        if (g > 4096) g = 4096;
        k_mat_absmax<<<(int)g, 256, 0, st>>>(m, n, A, lda, amax);
        CF_LAUNCH_CHECK();
    }
    return launch_residual_pair(m, n, nrhs, A, lda, amax, X, ldx, B, ldb, R, ldr, ws, st);
}

}  // namespace cf
