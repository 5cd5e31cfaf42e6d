// cf_resid_tc.cu -- R-1 at FP64 accuracy on the tensor cores:
//     R = B - A X     (A m x n FP64, X n x nrhs FP64, column-major)
//
// GB300 runs FP64 at ~2 operations per clock per SM, so an FP64 residual at
// N = 32768 with 16 right-hand sides costs ~29 ms even at 95% of that pipe,
// while the BF16 tensor cores run ~500x faster.  The product is therefore
// formed exactly from small integers:
//   * per row i of A, E_i is the exponent with max_j |a_ij| < 2^E_i, and
//     q_ij = round(a_ij 2^(62 - E_i)) (to nearest, ties away from zero) is an
//     integer of at most 62 bits; X is cut the same way per column (F_k, p_jk);
//   * q = sum_s d_s 256^(7-s) in eight balanced base-256 digits (the top one
//     in [-64, 64], the others in [-128, 127]), each exact in BF16;
//   * Q_d = sum_{s+t=d} sum_j d_s(q_ij) e_t(p_jk), d = 0..7 (the digit pairs
//     below 2^-64 of the leading one are dropped): one tcgen05.mma chain per
//     128-row tile accumulates, for every A digit s, the products with the X
//     digits t = 0..7-s into the accumulator columns of diagonal s + t, so a
//     single FP32 accumulator of 8 x 16 columns holds all eight diagonals.
//     A product is at most 2^14 (2^13 with a top digit) and a chunk of 128
//     consecutive j adds at most 128 products of each of 8 digit pairs, two
//     of them with a top digit: at most 7 x 2^21 < 2^24, so the FP32
//     accumulation of a chunk is exact in any order; chunks are added in int64
//     registers and K ranges in int64 with atomics (integers: exact and
//     order-independent);
//   * R = B - 2^(E_i + F_k - 68) sum_d Q_d 256^(7-d), combined in
//     double-double.
// The error is a few 2^-63 of max_j |a_ij| ||x_k|| per term (the rounding of
// q and p and the dropped pairs), below the FP64 product's own.  The A slices
// (8 m n BF16) are cut once and reused for every residual with the same A.
// Rows (columns of X) with a non-finite entry give NaN.
//
// Kernel layout (sm_103a): persistent CTAs over (128-row tile, K range)
// units; warp 0 issues TMA loads (128-byte swizzle) of the X digits (128 x 64
// per K block) and bulk copies of the eight A digit tiles (128 x 64 each,
// stored tile after tile already in the 128-byte-swizzled shared-memory
// image, so each is one contiguous 16 KB read of HBM), warp 1 issues
// the MMAs (M = 128, N = 128 - 16 s, K = 16) into one of two TMEM
// accumulators, warps 2-9 read the other accumulator back after each chunk of
// 128 K and add it to int64 registers.  Every mbarrier wait is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "cf_common.cuh"
#include "cf_kernels.cuh"
#include "cf_tc.cuh"
#include "cf_umma.cuh"

namespace cf {

__device__ int g_rtc_status = 0;       // 0 or CF_ERR_TIMEOUT

namespace rtc {

using namespace umma;

constexpr int ND = 8;                 // digits per element
constexpr int QBITS = 8 * ND - 2;     // fixed-point bits of q (top digit <= 64)
constexpr int NR = 16;                // right-hand sides per launch (zero padded)
constexpr int NCOL = ND * NR;         // accumulator columns: diagonal d, rhs k at d * NR + k
constexpr int BM = 128, BK = 64, KC = 128;
constexpr int XST = 2, AST = 12;      // pipeline depths (X tiles, A digit tiles: 1.5 K blocks in flight)
constexpr int UMMA_K = 16;
constexpr int EPI = 8;                // epilogue warps
constexpr int kThreads = 64 + 32 * EPI;
constexpr uint32_t kXBytes = NCOL * BK * 2;   // 16384
constexpr uint32_t kABytes = BM * BK * 2;     // 16384
constexpr uint32_t kAccStride = 128;          // TMEM columns per accumulator
constexpr uint32_t kTmemCols = 256;

struct Smem {
    uint64_t xfull[XST], xempty[XST];
    uint64_t afull[AST], aempty[AST];
    uint64_t acc_full[2], acc_empty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort_flag;
};

struct Problem {
    int m, n, mpad;
    int nkb;              // K blocks of 64
    int tiles_m;
    int kranges;          // K ranges per tile
    int kb_per_range;     // K blocks per range (even)
    int nunits;
    unsigned long long *Q;   // [NCOL][mpad] int64 sums (two's complement)
    const uint8_t *S;        // A digit tiles (a_tile_offset), 16 KB each
};

// Byte offset of the digit-d tile of row tile rt and K block kb in the A
// slices: tiles of one (rt, kb) are consecutive (eight digits, 128 KB), K
// blocks of a row tile follow each other.
__host__ __device__ __forceinline__ size_t a_tile_offset(int rt, int kb, int d, int nkb) {
    return (((size_t)rt * nkb + kb) * ND + d) * (size_t)(BM * BK * 2);
}

__device__ __forceinline__ void unit_coords(const Problem &p, int u, int &m0, int &kb0, int &kb1) {
    const int tile = u % p.tiles_m, kr = u / p.tiles_m;
    m0 = tile * BM;
    kb0 = kr * p.kb_per_range;
    kb1 = min(p.nkb, kb0 + p.kb_per_range);
}

__global__ void __launch_bounds__(kThreads, 1)
k_resid_tc(const __grid_constant__ CUtensorMap tmX, Problem p) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *stageX = base;
    uint8_t *stageA = base + XST * kXBytes;
    Smem &s = *reinterpret_cast<Smem *>(stageA + AST * kABytes);
    volatile int *abort_flag = &s.abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < XST; ++i) { mbar_init(&s.xfull[i], 1); mbar_init(&s.xempty[i], 1); }
        for (int i = 0; i < AST; ++i) { mbar_init(&s.afull[i], 1); mbar_init(&s.aempty[i], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&s.acc_full[i], 1); mbar_init(&s.acc_empty[i], EPI); }
        mbar_init(&s.drain, 1);
        s.abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = s.tmem_base;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            int ix = 0, ia = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < p.nunits && ok; u += gridDim.x) {
                int m0, kb0, kb1;
                unit_coords(p, u, m0, kb0, kb1);
                for (int kb = kb0; kb < kb1 && ok; ++kb) {
                    {
                        const int st = ix % XST;
                        const uint32_t ph = (uint32_t)(ix / XST) & 1u;
                        if (!wait_bounded(&s.xempty[st], ph ^ 1u, abort_flag, &g_rtc_status)) { ok = false; break; }
                        mbar_arrive_expect_tx(&s.xfull[st], kXBytes);
                        tma_load_2d(stageX + st * kXBytes, &tmX, &s.xfull[st], kb * BK, 0);
                        ++ix;
                    }
                    for (int d = 0; d < ND; ++d) {
                        const int st = ia % AST;
                        const uint32_t ph = (uint32_t)(ia / AST) & 1u;
                        if (!wait_bounded(&s.aempty[st], ph ^ 1u, abort_flag, &g_rtc_status)) { ok = false; break; }
                        mbar_arrive_expect_tx(&s.afull[st], kABytes);
                        bulk_load_stream(stageA + st * kABytes, p.S + a_tile_offset(m0 / BM, kb, d, p.nkb), kABytes,
                                         &s.afull[st]);
                        ++ia;
                    }
                }
            }
            if (!ok) {
                // every issued copy must land before the CTA exits
                for (int j = (ix > XST ? ix - XST : 0); j < ix; ++j) {
                    const uint32_t ph = (uint32_t)(j / XST) & 1u;
                    for (long long i = 0; i < kSpinLimit && !mbar_try_wait(&s.xfull[j % XST], ph); ++i)
                        __nanosleep(64);
                }
                for (int j = (ia > AST ? ia - AST : 0); j < ia; ++j) {
                    const uint32_t ph = (uint32_t)(j / AST) & 1u;
                    for (long long i = 0; i < kSpinLimit && !mbar_try_wait(&s.afull[j % AST], ph); ++i)
                        __nanosleep(64);
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            int ix = 0, ia = 0, nacc = 0;
            bool ok = true, issued = false;
            for (int u = blockIdx.x; u < p.nunits && ok; u += gridDim.x) {
                int m0, kb0, kb1;
                unit_coords(p, u, m0, kb0, kb1);
                for (int c0 = kb0; c0 < kb1 && ok; c0 += KC / BK) {
                    const int b = nacc & 1;
                    const uint32_t aph = (uint32_t)(nacc >> 1) & 1u;
                    if (!wait_bounded(&s.acc_empty[b], aph ^ 1u, abort_flag, &g_rtc_status)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t dacc = tmem_base + (uint32_t)b * kAccStride;
                    const int c1 = min(kb1, c0 + KC / BK);
                    for (int kb = c0; kb < c1 && ok; ++kb) {
                        const int xs = ix % XST;
                        if (!wait_bounded(&s.xfull[xs], (uint32_t)(ix / XST) & 1u, abort_flag, &g_rtc_status)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t bd = make_sw128_desc(smem_u32(stageX + xs * kXBytes));
                        for (int d = 0; d < ND; ++d) {
                            const int as = ia % AST;
                            if (!wait_bounded(&s.afull[as], (uint32_t)(ia / AST) & 1u, abort_flag, &g_rtc_status)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
                            const uint64_t ad = make_sw128_desc(smem_u32(stageA + as * kABytes));
                            // A digit d times X digits t = 0..6-d into the columns of diagonals d..6
                            const uint32_t idesc = make_idesc(true, BM, NCOL - NR * d);
#pragma unroll
                            for (int kk = 0; kk < BK / UMMA_K; ++kk)
                                umma_f16(dacc + (uint32_t)(NR * d), ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2),
                                         idesc, (kb > c0 || d > 0 || kk > 0) ? 1u : 0u);
                            issued = true;
                            umma_commit(&s.aempty[as]);
                            ++ia;
                        }
                        if (!ok) break;
                        umma_commit(&s.xempty[xs]);
                        ++ix;
                    }
                    if (!ok) break;
                    umma_commit(&s.acc_full[b]);
                    ++nacc;
                }
            }
            if (issued) {
                umma_commit(&s.drain);
                for (long long i = 0; i < kSpinLimit && !mbar_try_wait(&s.drain, 0); ++i) __nanosleep(64);
            }
        }
    } else {
        // ------------------------------------------------ epilogue (warps 2..9)
        const int e = warp - 2;
        const int quarter = warp & 3;             // TMEM lanes 32 * quarter ..
        const int half = e >> 2;                  // columns 0..63 or 64..127
        long long acc[64];
#pragma unroll
        for (int j = 0; j < 64; ++j) acc[j] = 0;
        int nacc = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < p.nunits && ok; u += gridDim.x) {
            int m0, kb0, kb1;
            unit_coords(p, u, m0, kb0, kb1);
            for (int c0 = kb0; c0 < kb1; c0 += KC / BK) {
                const int b = nacc & 1;
                const uint32_t aph = (uint32_t)(nacc >> 1) & 1u;
                if (lane == 0) ok = wait_bounded(&s.acc_full[b], aph, abort_flag, &g_rtc_status);
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok) break;
                tc_fence_after();
                const uint32_t taddr =
                    tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)b * kAccStride + (uint32_t)(64 * half);
                uint32_t r[32];
                TMEM_LD32(taddr, r);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[j] += (long long)__float2int_rn(__uint_as_float(r[j]));
                TMEM_LD32(taddr + 32, r);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 32; ++j) acc[32 + j] += (long long)__float2int_rn(__uint_as_float(r[j]));
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&s.acc_empty[b]);
                ++nacc;
            }
            if (!ok) break;
            const int row = m0 + quarter * 32 + lane;
            if (row < p.m) {
#pragma unroll
                for (int j = 0; j < 64; ++j)
                    if (acc[j] != 0)
                        atomicAdd(p.Q + (size_t)(64 * half + j) * p.mpad + row, (unsigned long long)acc[j]);
            }
#pragma unroll
            for (int j = 0; j < 64; ++j) acc[j] = 0;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kTmemCols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Digit slicing
// ---------------------------------------------------------------------------
// Biased exponent field of |x| (0x7FF for inf / NaN).
__device__ __forceinline__ int exp_field(double x) {
    return (int)((__double_as_longlong(x) >> 52) & 0x7FF);
}

// Row maxima of the exponent field of A (column-major): rows along threads,
// columns split over blockIdx.y; Ef must be zero before.
__global__ void __launch_bounds__(256) k_row_expmax(int m, int n, const double *__restrict__ A, int lda, int cols_per,
                                                    int *Ef) {
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= m) return;
    const int j0 = blockIdx.y * cols_per, j1 = min(n, j0 + cols_per);
    int f = 0;
    for (int j = j0; j < j1; ++j) f = max(f, exp_field(A[(size_t)i + (size_t)j * lda]));
    if (f > 0) atomicMax(Ef + i, f);
}

// Column maxima of the exponent field of X (n x nrhs, column-major); Gf
// must be zero before.
__global__ void __launch_bounds__(256) k_col_expmax(int n, int nrhs, const double *__restrict__ X, int ldx,
                                                    int *Gf) {
    const int k = blockIdx.y;
    int f = 0;
    for (int j = blockIdx.x * 256 + threadIdx.x; j < n; j += gridDim.x * 256)
        f = max(f, exp_field(X[(size_t)j + (size_t)k * ldx]));
    f = __reduce_max_sync(0xffffffffu, (unsigned)f);
    if ((threadIdx.x & 31) == 0 && f > 0) atomicMax(Gf + k, f);
}

// q = round(x 2^(62 - E)), E = max(F, 1) - 1022 for the row's (column's)
// largest exponent field F, as an integer of at most 62 bits, from the
// bits of x (ties away from zero); then its eight balanced base-256 digits,
// most significant first.
__device__ __forceinline__ void digits8(double x, int F, float (&dg)[ND]) {
    const long long bits = __double_as_longlong(x);
    const int f = (int)((bits >> 52) & 0x7FF);
    const long long mant = bits & ((1ll << 52) - 1);
    const long long m53 = f == 0 ? mant : (mant | (1ll << 52));
    // x 2^(62 - E) = m53 2^sh with sh = f - F + (62 - 53): at most 9 (f <= F)
    const int sh = (f == 0 ? 1 : f) - (F > 0 ? F : 1) + (QBITS - 53);
    long long q;
    if (sh >= 0) q = m53 << (sh > QBITS - 53 ? QBITS - 53 : sh);
    else if (-sh >= 60) q = 0;
    else q = (m53 + (1ll << (-sh - 1))) >> (-sh);
    if (bits < 0) q = -q;
    // the seven low digits are the bytes of q + 128 (1 + 256 + ... + 256^6)
    // less 128 each, the top one what is left above them (|top| <= 64)
    const long long t = q + 0x0080808080808080ll;
    const unsigned lo = (unsigned)t, hi = (unsigned)(t >> 32);
#pragma unroll
    for (int b = 0; b < 4; ++b) dg[ND - 1 - b] = (float)((lo >> (8 * b)) & 255u) - 128.f;
#pragma unroll
    for (int b = 0; b < 3; ++b) dg[ND - 5 - b] = (float)((hi >> (8 * b)) & 255u) - 128.f;
    dg[0] = (float)(t >> 56);
}

// A (m x n FP64, column-major) -> eight BF16 digit slices in 128 x 64
// tiles (a_tile_offset), each the image the MMA reads from shared memory:
// row r of a tile is 128 bytes at r * 128, its 16-byte chunk c (columns
// 8c .. 8c + 7 of the K block) at chunk position c ^ (r mod 8) (the 128-byte
// swizzle).  Columns n .. ldk - 1 are zero.  CTA: 32 rows x 128 columns
// (two K blocks); thread: row i (lane, so that the loads are coalesced), 16
// consecutive j (warp).  Each slice goes through shared memory and out as
// whole 128-byte tile rows (16-byte stores scattered over tile rows, without
// the staging, measured 2.4x slower: 12.9 against 5.4 ms at N = 32768).
constexpr int kSliceRows = 32, kSliceCols = 128;
constexpr int kSlicePitch = kSliceCols + 8;      // BF16 per staged row: 272 bytes, fewer bank conflicts

__global__ void __launch_bounds__(256) k_slice_a(int m, int n, const double *__restrict__ A, int lda, const int *Ef,
                                                 uint8_t *S, int nkb) {
    __shared__ __align__(16) __nv_bfloat16 tile[kSliceRows * kSlicePitch];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i0 = blockIdx.x * kSliceRows, jt = blockIdx.y * kSliceCols;
    const int i = i0 + lane;
    const int j0 = jt + warp * 16;
    const bool valid = i < m && j0 < n;
    const int F = valid ? Ef[i] : 0;
    uint32_t pk[ND][8];                                // the 16 digits of each slice, as BF16 pairs
#pragma unroll
    for (int c = 0; c < 16; c += 2) {
        float d0[ND], d1[ND];
        const double x0 = (valid && j0 + c < n) ? A[(size_t)i + (size_t)(j0 + c) * lda] : 0.0;
        const double x1 = (valid && j0 + c + 1 < n) ? A[(size_t)i + (size_t)(j0 + c + 1) * lda] : 0.0;
        digits8(x0, F, d0);
        digits8(x1, F, d1);
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(d0[d], d1[d]);
            pk[d][c / 2] = *reinterpret_cast<const uint32_t *>(&h);
        }
    }
    const int rows = min(kSliceRows, m - i0);
#pragma unroll
    for (int d = 0; d < ND; ++d) {
        uint4 *sdst = reinterpret_cast<uint4 *>(tile + lane * kSlicePitch + warp * 16);
        sdst[0] = make_uint4(pk[d][0], pk[d][1], pk[d][2], pk[d][3]);
        sdst[1] = make_uint4(pk[d][4], pk[d][5], pk[d][6], pk[d][7]);
        __syncthreads();
        // 32 rows x 16 chunks of 8 BF16 (two K blocks): two rows per warp store
#pragma unroll
        for (int it = 0; it < 2; ++it) {
            const int c = threadIdx.x + 256 * it;
            const int r = c >> 4, q = c & 15;
            const int kb = (jt >> 6) + (q >> 3), ch = q & 7;
            const int gi = i0 + r, rl = gi & (BM - 1);
            if (r < rows && kb < nkb) {
                const uint4 v = *reinterpret_cast<const uint4 *>(tile + r * kSlicePitch + q * 8);
                *reinterpret_cast<uint4 *>(S + a_tile_offset(gi / BM, kb, d, nkb) + (size_t)rl * 128 +
                                           (size_t)((ch ^ (rl & 7)) * 16)) = v;
            }
        }
        __syncthreads();
    }
}

// X (n x nrhs FP64) -> digits Xs[(d * NR + k) * ldk + j] for k < nrhs, zero
// rows for nrhs <= k < NR.
__global__ void __launch_bounds__(256) k_slice_x(int n, int nrhs, const double *__restrict__ X, int ldx,
                                                 const int *Gf, __nv_bfloat16 *Xs, int ldk) {
    const int j = blockIdx.x * 256 + threadIdx.x;
    const int k = blockIdx.y;
    if (j >= n) return;
    float dg[ND];
    if (k < nrhs) {
        digits8(X[(size_t)j + (size_t)k * ldx], Gf[k], dg);
    } else {
#pragma unroll
        for (int d = 0; d < ND; ++d) dg[d] = 0.f;
    }
#pragma unroll
    for (int d = 0; d < ND; ++d) Xs[(size_t)(d * NR + k) * ldk + j] = __float2bfloat16_rn(dg[d]);
}

__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
    s = a + b;
    const double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// R = B - 2^(E_i + F_k - 68) sum_d Q_d 256^(7-d) in double-double; with B
// null, R = A X (the product alone).
__global__ void __launch_bounds__(256) k_resid_combine(int m, int nrhs, const unsigned long long *Q, int mpad,
                                                       const int *Ef, const int *Gf, const double *B, int ldb,
                                                       double *R, int ldr) {
    const int i = blockIdx.x * 256 + threadIdx.x;
    const int k = blockIdx.y;
    if (i >= m || k >= nrhs) return;
    const int F = Ef[i], G = Gf[k];
    const double b = B ? B[(size_t)i + (size_t)k * ldb] : 0.0;
    double out;
    if (F == 0x7FF || G == 0x7FF) {
        out = __longlong_as_double(0x7FF8000000000000ll);   // NaN: a non-finite entry in the row or column
    } else {
        double hi = 0.0, lo = 0.0;
#pragma unroll
        for (int d = 0; d < ND; ++d) {
            const long long q = (long long)Q[(size_t)(d * NR + k) * mpad + i];
            const double t = ldexp((double)q, 8 * (ND - 1 - d));   // exact: |q| < 2^53
            double s, e;
            two_sum(hi, t, s, e);
            hi = s;
            lo += e;
        }
        // q p = 2^(2 QBITS - E - F) a x and sum_d Q_d 256^(7-d) = q p / 256^(ND - 1)
        const int sc = ((F > 0 ? F : 1) - 1022) + ((G > 0 ? G : 1) - 1022) - 2 * QBITS + 8 * (ND - 1);
        hi = ldexp(hi, sc);
        lo = ldexp(lo, sc);
        double s, e;
        two_sum(b, -hi, s, e);
        out = s + (e - lo);
        if (!B) out = hi + lo;
    }
    R[(size_t)i + (size_t)k * ldr] = out;
}

}  // namespace rtc

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static int make_bf16_map(CUtensorMap *map, const void *ptr, long long rows, int k, int ld, int box_rows) {
    cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)rtc::BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? CF_OK : CF_ERR_CUDA;
}

static int rtc_num_sms() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 148;
}

ResidTC resid_tc_layout(int m, int n) {
    ResidTC L{};
    L.m = m;
    L.n = n;
    L.mpad = (m + rtc::BM - 1) / rtc::BM * rtc::BM;
    L.ldk = (n + 63) / 64 * 64;
    return L;
}

size_t resid_tc_a_bytes(int m, int n) {
    const ResidTC L = resid_tc_layout(m > 0 ? m : 1, n > 0 ? n : 1);
    Carver cv(nullptr);
    cv.take<__nv_bfloat16>((size_t)rtc::ND * L.mpad * L.ldk, 1024);
    cv.take<int>(L.mpad);
    return cv.size();
}

size_t resid_tc_x_bytes(int m, int n) {
    const ResidTC L = resid_tc_layout(m > 0 ? m : 1, n > 0 ? n : 1);
    Carver cv(nullptr);
    cv.take<__nv_bfloat16>((size_t)rtc::NCOL * L.ldk, 1024);
    cv.take<unsigned long long>((size_t)rtc::NCOL * L.mpad);
    cv.take<int>(rtc::NR);
    return cv.size();
}

void resid_tc_carve(ResidTC *L, void *wsA) {
    Carver cv(wsA);
    L->S = cv.take<__nv_bfloat16>((size_t)rtc::ND * L->mpad * L->ldk, 1024);
    L->Ef = cv.take<int>(L->mpad);
}

int resid_tc_prepare(ResidTC *L, const double *A, int lda, bool ef_ready, cudaStream_t st) {
    const int m = L->m, n = L->n;
    if (m <= 0 || n <= 0) return CF_OK;
    if (!ef_ready) {
        CF_CUDA_TRY(cudaMemsetAsync(L->Ef, 0, sizeof(int) * (size_t)L->mpad, st));
        const int cols_per = 256;
        rtc::k_row_expmax<<<dim3(ceil_div(m, 256), ceil_div(n, cols_per)), 256, 0, st>>>(m, n, A, lda, cols_per,
                                                                                        L->Ef);
        CF_LAUNCH_CHECK();
    }
    rtc::k_slice_a<<<dim3(ceil_div(m, rtc::kSliceRows), ceil_div(n, rtc::kSliceCols)), 256, 0, st>>>(
        m, n, A, lda, L->Ef, reinterpret_cast<uint8_t *>(L->S), L->ldk / rtc::BK);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

int resid_tc_apply(const ResidTC &L, int nrhs, const double *X, int ldx, const double *B, int ldb, double *R, int ldr,
                   void *wsX, cudaStream_t st) {
    using namespace rtc;
    const int m = L.m, n = L.n;
    if (m <= 0 || nrhs <= 0) return CF_OK;
    Carver cv(wsX);
    __nv_bfloat16 *Xs = cv.take<__nv_bfloat16>((size_t)NCOL * L.ldk, 1024);
    unsigned long long *Q = cv.take<unsigned long long>((size_t)NCOL * L.mpad);
    int *Gf = cv.take<int>(NR);
    int rc = get_encoder();
    if (rc) return rc;
    CUtensorMap tx;
    if ((rc = make_bf16_map(&tx, Xs, NCOL, n, L.ldk, NCOL))) return rc;
    Problem p{};
    p.m = m;
    p.n = n;
    p.mpad = L.mpad;
    p.nkb = ceil_div(n, BK);
    p.tiles_m = ceil_div(m, BM);
    p.S = reinterpret_cast<const uint8_t *>(L.S);
    const int sms = rtc_num_sms();
    // K ranges: enough units for several waves, each range whole chunks
    const int nchunks = ceil_div(p.nkb, KC / BK);
    int kr = ceil_div(8 * sms, p.tiles_m);
    if (kr > nchunks) kr = nchunks;
    if (kr < 1) kr = 1;
    p.kb_per_range = ceil_div(nchunks, kr) * (KC / BK);
    p.kranges = ceil_div(p.nkb, p.kb_per_range);
    p.nunits = p.tiles_m * p.kranges;
    p.Q = Q;
    const size_t smem = 1024 + XST * kXBytes + AST * kABytes + sizeof(Smem);
    CF_CUDA_TRY(cudaFuncSetAttribute(k_resid_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    for (int k0 = 0; k0 < nrhs; k0 += NR) {
        const int nk = nrhs - k0 < NR ? nrhs - k0 : NR;
        CF_CUDA_TRY(cudaMemsetAsync(Gf, 0, sizeof(int) * NR, st));
        CF_CUDA_TRY(cudaMemsetAsync(Q, 0, sizeof(unsigned long long) * (size_t)NCOL * L.mpad, st));
        k_col_expmax<<<dim3(ceil_div(n, 256) < 64 ? ceil_div(n, 256) : 64, nk), 256, 0, st>>>(
            n, nk, X + (size_t)k0 * ldx, ldx, Gf);
        CF_LAUNCH_CHECK();
        k_slice_x<<<dim3(ceil_div(n, 256), NR), 256, 0, st>>>(n, nk, X + (size_t)k0 * ldx, ldx, Gf, Xs, L.ldk);
        CF_LAUNCH_CHECK();
        const int grid = p.nunits < sms ? p.nunits : sms;
        k_resid_tc<<<grid, kThreads, smem, st>>>(tx, p);
        CF_LAUNCH_CHECK();
        k_resid_combine<<<dim3(ceil_div(m, 256), nk), 256, 0, st>>>(m, nk, Q, L.mpad, L.Ef, Gf,
                                                                     B ? B + (size_t)k0 * ldb : nullptr, ldb,
                                                                     R + (size_t)k0 * ldr, ldr);
        CF_LAUNCH_CHECK();
    }
    return CF_OK;
}

int rtc_take_status(cudaStream_t st, int *status) {
    int h = 0;
    CF_CUDA_TRY(cudaMemcpyFromSymbolAsync(&h, g_rtc_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    CF_CUDA_TRY(cudaStreamSynchronize(st));
    if (h != 0) {
        const int zero = 0;
        CF_CUDA_TRY(cudaMemcpyToSymbolAsync(g_rtc_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
        CF_CUDA_TRY(cudaStreamSynchronize(st));
    }
    *status = h;
    return CF_OK;
}

}  // namespace cf

extern "C" size_t cf_residual_tc_workspace_size(int m, int n, int nrhs) {
    (void)nrhs;
    cf::Carver cv(nullptr);
    cv.take<char>(cf::resid_tc_a_bytes(m, n), 1024);
    cv.take<char>(cf::resid_tc_x_bytes(m, n), 1024);
    return cv.size();
}

extern "C" int cf_residual_tc(int m, int n, int nrhs, const double *A, int lda, const double *X, int ldx,
                              const double *B, int ldb, double *R, int ldr, void *work, size_t lwork,
                              cudaStream_t stream) {
    using namespace cf;
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (nrhs < 0) return -3;
    if (m > 0 && n > 0 && A == nullptr) return -4;
    if (lda < (m > 1 ? m : 1)) return -5;
    if (n > 0 && nrhs > 0 && X == nullptr) return -6;
    if (ldx < (n > 1 ? n : 1)) return -7;
    if (m > 0 && nrhs > 0 && B == nullptr) return -8;
    if (ldb < (m > 1 ? m : 1)) return -9;
    if (m > 0 && nrhs > 0 && R == nullptr) return -10;
    if (ldr < (m > 1 ? m : 1)) return -11;
    if (m == 0 || nrhs == 0) return CF_OK;
    if (work == nullptr || lwork < cf_residual_tc_workspace_size(m, n, nrhs)) return CF_ERR_WORKSPACE;
    if (n == 0) {
        if (R != B || ldr != ldb)
            for (int k = 0; k < nrhs; ++k)
                CF_CUDA_TRY(cudaMemcpyAsync(R + (size_t)k * ldr, B + (size_t)k * ldb, sizeof(double) * (size_t)m,
                                            cudaMemcpyDeviceToDevice, stream));
        return CF_OK;
    }
    Carver cv(work);
    void *wa = cv.take<char>(resid_tc_a_bytes(m, n), 1024);
    void *wx = cv.take<char>(resid_tc_x_bytes(m, n), 1024);
    ResidTC L = resid_tc_layout(m, n);
    resid_tc_carve(&L, wa);
    int rc = resid_tc_prepare(&L, A, lda, false, stream);
    if (rc != CF_OK) return rc;
    return resid_tc_apply(L, nrhs, X, ldx, B, ldb, R, ldr, wx, stream);
}
