// cf_fp8.cu -- CH-3 (and LU-5) with FP8 e4m3 operands and per-128 x 128-tile
// FP32 scales on the 5th-generation tensor cores:
//     C[m x n] -= sum_kb sA(i, kb) sB(j, kb) (qA qB^T)_kb      (FP32 C)
// where kb runs over K-blocks of 128 and sA(i, kb) is the scale of the
// 128 x 128 tile of A holding row i in K-block kb (the paper's Table 2
// gemmt / gemm with FP8 operands and tile scales, an addition of this
// project: the paper has no low-precision update).
//
// A tile scale changes from one K-block to the next, so the K sum cannot run
// in one tensor-memory accumulator.  Per output tile (128 x 256) and K-block:
//   * warp 1 (one lane) issues four tcgen05.mma kind::f8f6f4 (M=128, N=256,
//     K=32) into one of two TMEM accumulators (double-buffered across
//     K-blocks), warp 0 feeds a 4-stage TMA ring (128-byte swizzle, one
//     K-block of A and B per stage);
//   * eight epilogue warps (two per TMEM lane quadrant, one per 128-column
//     half) read the K-block's accumulator with tcgen05.ld and add it, times
//     the scalar sA sB of that tile pair, into FP32 registers (one row x 128
//     columns per thread), then release the accumulator;
//   * after the last K-block they apply C -= sum with coalesced column
//     accesses (lower: only i >= j).
// Every mbarrier wait is bounded (CF_ERR_TIMEOUT in g_fp8_status, drain, free
// TMEM, return).
#include <cuda.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include "cf_common.cuh"
#include "cf_kernels.cuh"
#include "cf_tc.cuh"
#include "cf_umma.cuh"

namespace cf {

__device__ int g_fp8_status = 0;      // 0 or CF_ERR_TIMEOUT

namespace f8 {

using namespace umma;

constexpr int BM = 128, BN = 256, BK = 128, STAGES = 4;   // BK: bytes = elements
constexpr int UMMA_K = 32;
constexpr int kEpiWarps = 8;
constexpr int kThreads = 64 + 32 * kEpiWarps;              // 10 warps
constexpr uint32_t kStageA = BM * BK;                      // 16 KB
constexpr uint32_t kStageB = BN * BK;                      // 32 KB
constexpr uint32_t kStageBytes = kStageA + kStageB;
constexpr uint32_t kTmemCols = 2 * BN;                     // two accumulators

struct Smem {
    uint64_t full[STAGES];
    uint64_t empty[STAGES];
    uint64_t acc_full[2];
    uint64_t acc_empty[2];
    uint64_t drain;
    uint32_t tmem_base;
    int abort_flag;
};

struct Problem {
    int m, n, k;
    float *C;
    int ldc;
    int lower;
    int tiles_m, tiles_n, ntiles;
    const float *sA;
    int ldsa;
    const float *sB;
    int ldsb;
};

// Instruction descriptor, kind::f8f6f4: D = F32 (bit 4), A = B = E4M3 (format
// 0 at bits 7 and 10), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t make_idesc_e4m3(int M, int N) {
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}

#define TMEM_LD16(taddr, r)                                                                                   \
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];" \
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),    \
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),            \
                   "=r"(r[15])                                                                                         \
                 : "r"(taddr))

__device__ __forceinline__ bool tile_coords(const Problem &p, int t, int &m0, int &n0) {
    m0 = (t % p.tiles_m) * BM;
    n0 = (t / p.tiles_m) * BN;
    if (p.lower && n0 > m0 + BM - 1) return false;   // strictly above the diagonal
    return true;
}

__global__ void __launch_bounds__(kThreads, 1)
k_schur_fp8(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, Problem p,
            uint32_t idesc) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *stageA = base;
    uint8_t *stageB = base + STAGES * kStageA;
    Smem &s = *reinterpret_cast<Smem *>(base + STAGES * kStageBytes);
    volatile int *abort_flag = &s.abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkb = p.k / BK;

    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) { mbar_init(&s.full[i], 1); mbar_init(&s.empty[i], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&s.acc_full[i], 1); mbar_init(&s.acc_empty[i], kEpiWarps); }
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
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
                int m0, n0;
                if (!tile_coords(p, t, m0, n0)) continue;
                for (int kb = 0; kb < nkb; ++kb, ++it) {
                    const int st = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!wait_bounded(&s.empty[st], ph ^ 1u, abort_flag, &g_fp8_status)) { ok = false; break; }
                    mbar_arrive_expect_tx(&s.full[st], kStageBytes);
                    tma_load_2d(stageA + st * kStageA, &tmA, &s.full[st], kb * BK, m0);
                    tma_load_2d(stageB + st * kStageB, &tmB, &s.full[st], kb * BK, n0);
                }
            }
            if (!ok) {
                for (int j = (it > STAGES ? it - STAGES : 0); j < it; ++j) {
                    const int st = j % STAGES;
                    const uint32_t ph = (uint32_t)(j / STAGES) & 1u;
                    for (long long i = 0; i < kSpinLimit && !mbar_try_wait(&s.full[st], ph); ++i) __nanosleep(64);
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer: one accumulator per K-block
        if (lane == 0) {
            int it = 0, kc = 0;
            bool ok = true, issued = false;
            for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
                int m0, n0;
                if (!tile_coords(p, t, m0, n0)) continue;
                for (int kb = 0; kb < nkb; ++kb, ++it, ++kc) {
                    const int b = kc & 1;
                    const uint32_t aph = (uint32_t)(kc >> 1) & 1u;
                    if (!wait_bounded(&s.acc_empty[b], aph ^ 1u, abort_flag, &g_fp8_status)) { ok = false; break; }
                    const int st = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!wait_bounded(&s.full[st], ph, abort_flag, &g_fp8_status)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t d_tmem = tmem_base + (uint32_t)(b * BN);
                    const uint64_t ad = make_sw128_desc(smem_u32(stageA + st * kStageA));
                    const uint64_t bd = make_sw128_desc(smem_u32(stageB + st * kStageB));
#pragma unroll
                    for (int kk = 0; kk < BK / UMMA_K; ++kk)   // 32 bytes per step inside the swizzled row
                        umma_f8(d_tmem, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc, kk > 0 ? 1u : 0u);
                    issued = true;
                    umma_commit(&s.empty[st]);
                    umma_commit(&s.acc_full[b]);
                }
            }
            if (issued) {
                umma_commit(&s.drain);
                for (long long i = 0; i < kSpinLimit && !mbar_try_wait(&s.drain, 0); ++i) __nanosleep(64);
            }
        }
    } else {
        // ------------------------------------------------ promotion + epilogue (warps 2..9)
        const int quarter = warp & 3;                 // TMEM lanes 32*quarter ..
        const int half = (warp - 2) >> 2;             // columns half*128 .. of the tile
        int kc = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
            int m0, n0;
            if (!tile_coords(p, t, m0, n0)) continue;
            const int row = m0 + quarter * 32 + lane;
            const int cb = n0 / 128 + half;           // column block of the scales
            const bool half_live = n0 + half * 128 < p.n;
            float sum[128];
#pragma unroll
            for (int j = 0; j < 128; ++j) sum[j] = 0.f;
            for (int kb = 0; kb < nkb; ++kb, ++kc) {
                const int b = kc & 1;
                const uint32_t aph = (uint32_t)(kc >> 1) & 1u;
                if (lane == 0) ok = wait_bounded(&s.acc_full[b], aph, abort_flag, &g_fp8_status);
                ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
                if (!ok) break;
                tc_fence_after();
                const float sc = half_live ? p.sA[(size_t)(m0 / 128) * p.ldsa + kb] * p.sB[(size_t)cb * p.ldsb + kb]
                                           : 0.f;
#pragma unroll
                for (int c0 = 0; c0 < 128; c0 += 16) {
                    uint32_t r[16];
                    const uint32_t taddr =
                        tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * BN + half * 128 + c0);
                    TMEM_LD16(taddr, r);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < 16; ++j) sum[c0 + j] = fmaf(sc, __uint_as_float(r[j]), sum[c0 + j]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&s.acc_empty[b]);
            }
            if (!ok) break;
            if (row < p.m && half_live) {
                float *crow = p.C + row;
#pragma unroll
                for (int j = 0; j < 128; ++j) {
                    const int col = n0 + half * 128 + j;
                    if (col < p.n && (!p.lower || row >= col)) crow[(size_t)col * p.ldc] -= sum[j];
                }
            }
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
// Quantization of an FP32 column-major block to K-major e4m3 with one FP32
// scale per 128 x 128 tile.  CTA = one tile: stage it in shared memory
// (coalesced along rows), reduce amax, write 4 codes per thread per word
// (coalesced along K).
// ---------------------------------------------------------------------------
constexpr int kQT = 128, kQLD = kQT + 1;

__global__ void __launch_bounds__(256) k_quant_e4m3(int rows, int k, const float *__restrict__ src, int lds_src,
                                                    uint8_t *__restrict__ q, int ldq, float *scales, int lds) {
    extern __shared__ float tile[];                 // [kQT][kQLD]: tile[kk * kQLD + r]
    __shared__ float red[8];
    const int rb = blockIdx.x, kb = blockIdx.y;
    const int r0 = rb * kQT, k0 = kb * kQT;
    const int tid = threadIdx.x;
    float amax = 0.f;
    for (int e = tid; e < kQT * kQT; e += 256) {
        const int r = e % kQT, kk = e / kQT;
        const float x = (r0 + r < rows && k0 + kk < k) ? src[(size_t)(r0 + r) + (size_t)(k0 + kk) * lds_src] : 0.f;
        tile[kk * kQLD + r] = x;
        amax = fmaxf(amax, fabsf(x));
    }
    for (int o = 16; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
    if ((tid & 31) == 0) red[tid >> 5] = amax;
    __syncthreads();
    amax = red[0];
#pragma unroll
    for (int w = 1; w < 8; ++w) amax = fmaxf(amax, red[w]);
    const float inv = amax > 0.f ? 448.f / amax : 1.f;
    if (tid == 0) scales[(size_t)rb * lds + kb] = amax > 0.f ? amax / 448.f : 1.f;
    // 128 rows x 32 words of 4 codes
    for (int e = tid; e < kQT * (kQT / 4); e += 256) {
        const int r = e / (kQT / 4), w4 = e % (kQT / 4);
        if (r0 + r >= rows) continue;
        uint32_t word = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float x = tile[(w4 * 4 + i) * kQLD + r] * inv;
            const uint32_t c = (uint32_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
            word |= c << (8 * i);
        }
        *reinterpret_cast<uint32_t *>(q + (size_t)(r0 + r) * ldq + k0 + w4 * 4) = word;
    }
}

}  // namespace f8

// 2-D K-major byte operand: rows x k bytes, row pitch ld bytes.
static int make_map_u8(CUtensorMap *map, const void *ptr, int rows, int k, int ld, int box_rows) {
    cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld};
    cuuint32_t box[2] = {(cuuint32_t)f8::BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? CF_OK : CF_ERR_CUDA;
}

static int num_sms_fp8() { return device_sm_count(); }

int launch_schur_fp8(int m, int n, int k, const void *qA, int ldqa, const float *sA, int ldsa, const void *qB,
                     int ldqb, const float *sB, int ldsb, float *C, int ldc, bool lower, cudaStream_t st) {
    if (m <= 0 || n <= 0 || k <= 0) return CF_OK;
    if (k % f8::BK != 0 || ldqa % 16 != 0 || ldqb % 16 != 0 || ldqa < k || ldqb < k) return CF_ERR_UNSUPPORTED;
    if (((uintptr_t)qA & 15) || ((uintptr_t)qB & 15) || sA == nullptr || sB == nullptr) return CF_ERR_UNSUPPORTED;
    int rc = get_encoder();
    if (rc) return rc;
    CUtensorMap ta, tb;
    if ((rc = make_map_u8(&ta, qA, m, k, ldqa, f8::BM))) return rc;
    if ((rc = make_map_u8(&tb, qB, n, k, ldqb, f8::BN))) return rc;
    f8::Problem p;
    p.m = m; p.n = n; p.k = k; p.C = C; p.ldc = ldc; p.lower = lower ? 1 : 0;
    p.tiles_m = ceil_div(m, f8::BM);
    p.tiles_n = ceil_div(n, f8::BN);
    p.ntiles = p.tiles_m * p.tiles_n;
    p.sA = sA; p.ldsa = ldsa; p.sB = sB; p.ldsb = ldsb;
    const size_t smem = 1024 + f8::STAGES * f8::kStageBytes + sizeof(f8::Smem);
    CF_CUDA_TRY(cudaFuncSetAttribute(f8::k_schur_fp8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int grid = num_sms_fp8();
    if (grid > p.ntiles) grid = p.ntiles;
    f8::k_schur_fp8<<<grid, f8::kThreads, smem, st>>>(ta, tb, p, f8::make_idesc_e4m3(f8::BM, f8::BN));
    CF_LAUNCH_CHECK();
    return CF_OK;
}

int launch_quant_e4m3(int rows, int k, int kpad, const float *src, int lds_src, void *q, int ldq, float *scales,
                      int lds, cudaStream_t st) {
    if (rows <= 0 || kpad <= 0) return CF_OK;
    if (kpad % f8::kQT != 0 || k > kpad || ldq < kpad || ldq % 4 != 0 || ((uintptr_t)q & 3)) return CF_ERR_UNSUPPORTED;
    const size_t smem = sizeof(float) * f8::kQT * f8::kQLD;
    CF_CUDA_TRY(cudaFuncSetAttribute(f8::k_quant_e4m3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(ceil_div(rows, f8::kQT), kpad / f8::kQT);
    f8::k_quant_e4m3<<<grid, 256, smem, st>>>(rows, k, src, lds_src, (uint8_t *)q, ldq, scales, lds);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

int fp8_take_status(cudaStream_t st, int *status) {
    int h = 0;
    CF_CUDA_TRY(cudaMemcpyFromSymbolAsync(&h, g_fp8_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    CF_CUDA_TRY(cudaStreamSynchronize(st));
    if (h != 0) {
        const int zero = 0;
        CF_CUDA_TRY(cudaMemcpyToSymbolAsync(g_fp8_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
        CF_CUDA_TRY(cudaStreamSynchronize(st));
    }
    *status = h;
    return CF_OK;
}

}  // namespace cf

extern "C" int cf_quantize_e4m3(int rows, int k, const float *src, int lds, void *q, int ldq, float *scales,
                                int ld_scales, cudaStream_t stream) {
    if (rows < 0) return -1;
    if (k < 0) return -2;
    if (rows > 0 && k > 0 && src == nullptr) return -3;
    if (lds < (rows > 1 ? rows : 1)) return -4;
    const int kpad = (k + 127) / 128 * 128;
    if (rows > 0 && k > 0 && q == nullptr) return -5;
    if (ldq < kpad || ldq % 16 != 0) return -6;
    if (rows > 0 && k > 0 && scales == nullptr) return -7;
    if (ld_scales < kpad / 128) return -8;
    if (rows == 0 || k == 0) return CF_OK;
    return cf::launch_quant_e4m3(rows, k, kpad, src, lds, q, ldq, scales, ld_scales, stream);
}

extern "C" int cf_schur_update_fp8(int m, int n, int k, const void *qA, int ldqa, const float *sA, int ldsa,
                                   const void *qB, int ldqb, const float *sB, int ldsb, float *C, int ldc, int lower,
                                   cudaStream_t stream) {
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (k < 0 || k % 128 != 0) return -3;
    if (m > 0 && k > 0 && qA == nullptr) return -4;
    if (ldqa < k || ldqa % 16 != 0) return -5;
    if (m > 0 && k > 0 && sA == nullptr) return -6;
    if (ldsa < k / 128) return -7;
    if (n > 0 && k > 0 && qB == nullptr) return -8;
    if (ldqb < k || ldqb % 16 != 0) return -9;
    if (n > 0 && k > 0 && sB == nullptr) return -10;
    if (ldsb < k / 128) return -11;
    if (m > 0 && n > 0 && C == nullptr) return -12;
    if (ldc < (m > 1 ? m : 1)) return -13;
    return cf::launch_schur_fp8(m, n, k, qA, ldqa, sA, ldsa, qB, ldqb, sB, ldsb, C, ldc, lower != 0, stream);
}
