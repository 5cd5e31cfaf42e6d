// cf_tc.cu -- LU-5 / CH-3 on the 5th-generation tensor cores:
//     C[m x n] -= A[m x k] * B[n x k]^T     (FP32 C, column-major)
// with A and B in BF16 or FP16, K-major (row i of A holds its k values
// contiguously), FP32 accumulation in tensor memory.
//
// This is Alg. 1 ("Factorize A11", Table 2's local gemm) and, with
// `lower`, COnfCHOX's triangular gemmt -- where most of both methods' work lies
// (Sec. 7.5).  Design for sm_103a:
//   * persistent CTAs, one per SM, walking 128 x 256 output tiles;
//   * warp 0 issues TMA loads (128-byte swizzle) into a 4-stage ring of
//     shared-memory stages, warp 1 (one elected lane) issues tcgen05.mma
//     (kind::f16, M=128, N=256, K=16) into one of two TMEM accumulators,
//     warps 2-5 drain the other accumulator with tcgen05.ld and apply
//     C -= acc with coalesced column accesses, so the epilogue of tile i
//     overlaps the MMAs of tile i+1;
//   * every mbarrier wait is bounded; on expiry the kernel records
//     CF_ERR_TIMEOUT in a device status word, drains its own copies and
//     MMAs (again bounded), frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "cf_common.cuh"
#include "cf_kernels.cuh"
#include "cf_tc.cuh"
#include "cf_umma.cuh"

namespace cf {

__device__ int g_tc_status = 0;       // 0 or CF_ERR_TIMEOUT

namespace tc {

using namespace umma;

constexpr int BM = 128, BN = 256, BK = 64, STAGES = 4;
constexpr int UMMA_K = 16;
constexpr int kThreads = 192;         // 6 warps
constexpr uint32_t kStageA = BM * BK * 2;     // 16 KB
constexpr uint32_t kStageB = BN * BK * 2;     // 32 KB
constexpr uint32_t kStageBytes = kStageA + kStageB;
constexpr uint32_t kTmemCols = 2 * BN;        // two accumulators

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
    // split-K: work unit u is tile u % ntiles over K blocks
    // [s kps, (s + 1) kps), s = u / ntiles; with P set, each unit writes its
    // accumulator to P[(s ntiles + tile) BM BN + col BM + row] instead of
    // updating C (k_splitk_reduce then subtracts the partials in order)
    int ksplit, kps, nunits;
    float *P;
    // MMA width: 64 or 128 when the whole output is that narrow (the B
    // box, the MMA and the epilogue cover only those columns), else BN
    int nmma;
    uint32_t bbytes;       // bytes of one B stage as loaded: nmma x BK x 2
};

// Tile t -> (bm, bn), M fastest so consecutive CTAs share a B tile in L2.
__device__ __forceinline__ bool tile_coords(const Problem &p, int t, int &m0, int &n0) {
    m0 = (t % p.tiles_m) * BM;
    n0 = (t / p.tiles_m) * BN;
    if (p.lower && n0 > m0 + BM - 1) return false;   // strictly above the diagonal
    return true;
}

// NARROW: outputs of at most 128 columns (p.nmma = 64 or 128: the B box, the
// MMA and the epilogue cover only those); the wide form keeps compile-time
// 256-column loops (measured 7-20% faster for wide outputs than the same
// loops with run-time bounds).
template <bool NARROW>
__global__ void __launch_bounds__(kThreads, 1)
k_schur_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, Problem p,
           uint32_t idesc) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *stageA = base;
    uint8_t *stageB = base + STAGES * kStageA;
    Smem &s = *reinterpret_cast<Smem *>(base + STAGES * kStageBytes);
    volatile int *abort_flag = &s.abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nkb = p.k / BK;
    auto unit_k = [&](int u, int &t, int &kb0, int &kb1) {
        t = u % p.ntiles;
        const int sp = u / p.ntiles;
        kb0 = sp * p.kps;
        kb1 = min(nkb, kb0 + p.kps);
    };

    if (threadIdx.x == 0) {
        for (int i = 0; i < STAGES; ++i) { mbar_init(&s.full[i], 1); mbar_init(&s.empty[i], 1); }
        for (int i = 0; i < 2; ++i) { mbar_init(&s.acc_full[i], 1); mbar_init(&s.acc_empty[i], 4); }
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
            for (int u = blockIdx.x; u < p.nunits && ok; u += gridDim.x) {
                int t, kb0, kb1, m0, n0;
                unit_k(u, t, kb0, kb1);
                if (!tile_coords(p, t, m0, n0)) continue;
                for (int kb = kb0; kb < kb1; ++kb, ++it) {
                    const int st = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!wait_bounded(&s.empty[st], ph ^ 1u, abort_flag, &g_tc_status)) { ok = false; break; }
                    mbar_arrive_expect_tx(&s.full[st], NARROW ? kStageA + p.bbytes : kStageBytes);
                    tma_load_2d(stageA + st * kStageA, &tmA, &s.full[st], kb * BK, m0);
                    tma_load_2d(stageB + st * kStageB, &tmB, &s.full[st], kb * BK, n0);
                }
            }
            if (!ok) {
                // Drain: every issued stage's copy must land before the CTA exits.
                for (int j = (it > STAGES ? it - STAGES : 0); j < it; ++j) {
                    const int st = j % STAGES;
                    const uint32_t ph = (uint32_t)(j / STAGES) & 1u;
                    for (long long i = 0; i < kSpinLimit && !mbar_try_wait(&s.full[st], ph); ++i) __nanosleep(64);
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        if (lane == 0) {
            int it = 0, tcount = 0;
            bool ok = true, issued = false;
            for (int u = blockIdx.x; u < p.nunits && ok; u += gridDim.x) {
                int t, kb0, kb1, m0, n0;
                unit_k(u, t, kb0, kb1);
                if (!tile_coords(p, t, m0, n0)) continue;
                const int b = tcount & 1;
                const uint32_t aph = (uint32_t)(tcount >> 1) & 1u;
                if (!wait_bounded(&s.acc_empty[b], aph ^ 1u, abort_flag, &g_tc_status)) { ok = false; break; }
                tc_fence_after();
                const uint32_t d_tmem = tmem_base + (uint32_t)(b * BN);
                for (int kb = kb0; kb < kb1; ++kb, ++it) {
                    const int st = it % STAGES;
                    const uint32_t ph = (uint32_t)(it / STAGES) & 1u;
                    if (!wait_bounded(&s.full[st], ph, abort_flag, &g_tc_status)) { ok = false; break; }
                    tc_fence_after();
                    const uint64_t ad = make_sw128_desc(smem_u32(stageA + st * kStageA));
                    const uint64_t bd = make_sw128_desc(smem_u32(stageB + st * kStageB));
#pragma unroll
                    for (int kk = 0; kk < BK / UMMA_K; ++kk) {
                        // advance 16 elements = 32 bytes inside the swizzled row
                        umma_f16(d_tmem, ad + (uint64_t)(kk * 2), bd + (uint64_t)(kk * 2), idesc,
                                 (kb > kb0 || kk > 0) ? 1u : 0u);
                    }
                    issued = true;
                    umma_commit(&s.empty[st]);
                }
                if (!ok) break;
                umma_commit(&s.acc_full[b]);
                ++tcount;
            }
            if (issued) {
                // Let every MMA this CTA issued finish before TMEM is freed.
                umma_commit(&s.drain);
                for (long long i = 0; i < kSpinLimit && !mbar_try_wait(&s.drain, 0); ++i) __nanosleep(64);
            }
        }
    } else {
        // ------------------------------------------------ epilogue (warps 2..5)
        const int quarter = warp & 3;                 // TMEM lanes 32*quarter ..
        int tcount = 0;
        for (int u = blockIdx.x; u < p.nunits; u += gridDim.x) {
            int t, kb0, kb1, m0, n0;
            unit_k(u, t, kb0, kb1);
            if (!tile_coords(p, t, m0, n0)) continue;
            const int b = tcount & 1;
            const uint32_t aph = (uint32_t)(tcount >> 1) & 1u;
            bool ok = true;
            if (lane == 0) ok = wait_bounded(&s.acc_full[b], aph, abort_flag, &g_tc_status);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) break;
            tc_fence_after();
            // narrow outputs: the columns of this tile that exist (and, for the
            // lower form, reach the diagonal of the tile's last row)
            int cmax = BN;
            if constexpr (NARROW) {
                cmax = min(p.nmma, p.n - n0);
                if (p.lower) cmax = min(cmax, m0 + BM - n0);
            }
            if (p.P != nullptr) {
                // split-K partial: the accumulator's live columns, column-major
                float *dst = p.P + ((size_t)(u / p.ntiles) * p.ntiles + t) * (BM * BN) + quarter * 32 + lane;
#pragma unroll 1
                for (int c0 = 0; c0 < (NARROW ? cmax : BN); c0 += 32) {
                    uint32_t r[32];
                    const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * BN + c0);
                    TMEM_LD32(taddr, r);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < 32; ++j) dst[(size_t)(c0 + j) * BM] = __uint_as_float(r[j]);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&s.acc_empty[b]);
                ++tcount;
                continue;
            }
            const int row = m0 + quarter * 32 + lane;
            const bool row_ok = row < p.m;
            float *crow = p.C + row;
#pragma unroll 1
            for (int c0 = 0; c0 < (NARROW ? cmax : BN); c0 += 32) {
                const int colbase = n0 + c0;
                float cv[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = colbase + j;
                    const bool ok2 = row_ok && col < p.n && (!p.lower || row >= col);
                    cv[j] = ok2 ? crow[(size_t)col * p.ldc] : 0.f;
                }
                uint32_t r[32];
                const uint32_t taddr = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * BN + c0);
                TMEM_LD32(taddr, r);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = colbase + j;
                    const bool ok2 = row_ok && col < p.n && (!p.lower || row >= col);
                    if (ok2) crow[(size_t)col * p.ldc] = cv[j] - __uint_as_float(r[j]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&s.acc_empty[b]);
            ++tcount;
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

// C -= sum_s P_s over the split-K partials of every tile, in the order
// s = 0, 1, ...: a deterministic sum, whatever order the units ran in.
__global__ void __launch_bounds__(256) k_splitk_reduce(Problem p) {
    const int t = blockIdx.y;
    const int m0 = (t % p.tiles_m) * BM, n0 = (t / p.tiles_m) * BN;
    if (p.lower && n0 > m0 + BM - 1) return;
    for (int e = blockIdx.x * 256 + threadIdx.x; e < BM * BN; e += gridDim.x * 256) {
        const int row = m0 + e % BM, col = n0 + e / BM;
        if (row >= p.m || col >= p.n || (p.lower && row < col)) continue;
        float acc = 0.f;
        for (int sp = 0; sp < p.ksplit; ++sp) acc += p.P[((size_t)sp * p.ntiles + t) * (BM * BN) + e];
        float *c = p.C + row + (size_t)col * p.ldc;
        *c = *c - acc;
    }
}

}  // namespace tc

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
static std::once_flag g_encode_once;

int get_encoder() {
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
    });
    return g_encode ? CF_OK : CF_ERR_CUDA;
}

// 2-D K-major operand: rows x k elements of 2 bytes, row pitch ld elements.
static int make_operand_map(CUtensorMap *map, const void *ptr, int rows, int k, int ld, int box_rows) {
    cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? CF_OK : CF_ERR_CUDA;
}

static int num_sms() { return device_sm_count(); }

int schur_tc_splitk(int m, int n, int k, bool lower) {
    // Only outputs with too few tiles to occupy half the SMs, and only ranges
    // at least 2048 deep, at most 4 of them.  Measured on GB300 (FP16, one
    // launch): M = 512..1024 at K = 8192 and M = 256..1024 at K = 16384 run
    // 1.5-2.3x faster in 4 ranges; every shape at K <= 2048 runs slower split
    // (the partial-sum round trip and the second launch cost more than the
    // idle SMs), so the mixed solvers' K = V <= 2048 updates never split.
    const int tiles = ceil_div(m, tc::BM) * ceil_div(n, tc::BN);
    const int eff = lower ? (tiles + ceil_div(m, tc::BM)) / 2 : tiles;     // about half the tiles of a triangle
    const int sms = num_sms();
    if (m <= 0 || n <= 0 || eff * 2 > sms) return 1;
    int ks = sms / (eff > 0 ? eff : 1);
    if (ks > k / 2048) ks = k / 2048;
    if (ks > 4) ks = 4;
    return ks < 2 ? 1 : ks;
}

size_t schur_tc_splitk_bytes(int m, int n, int ksplit) {
    if (ksplit <= 1 || m <= 0 || n <= 0) return 0;
    return sizeof(float) * (size_t)ksplit * ceil_div(m, tc::BM) * ceil_div(n, tc::BN) * tc::BM * tc::BN;
}

int launch_schur_tc(int m, int n, int k, const void *A, int lda_k, const void *B, int ldb_k, float *C, int ldc,
                    bool bf16, bool lower, cudaStream_t st, int max_ctas) {
    return launch_schur_tc_splitk(m, n, k, A, lda_k, B, ldb_k, C, ldc, bf16, lower, 1, nullptr, st, max_ctas);
}

int launch_schur_tc_splitk(int m, int n, int k, const void *A, int lda_k, const void *B, int ldb_k, float *C, int ldc,
                           bool bf16, bool lower, int ksplit, float *P, cudaStream_t st, int max_ctas) {
    if (m <= 0 || n <= 0 || k <= 0) return CF_OK;
    if (k % tc::BK != 0 || lda_k % 8 != 0 || ldb_k % 8 != 0 || lda_k < k || ldb_k < k) return CF_ERR_UNSUPPORTED;
    if (((uintptr_t)A & 15) || ((uintptr_t)B & 15)) return CF_ERR_UNSUPPORTED;
    int rc = get_encoder();
    if (rc) return rc;
    // narrow outputs (a panel's next columns): the MMA, the B box and the
    // epilogue cover only 64 or 128 columns instead of 256
    const int nmma = n <= 64 ? 64 : n <= 128 ? 128 : tc::BN;
    CUtensorMap ta, tb;
    if ((rc = make_operand_map(&ta, A, m, k, lda_k, tc::BM))) return rc;
    if ((rc = make_operand_map(&tb, B, n, k, ldb_k, nmma))) return rc;
    tc::Problem p;
    p.nmma = nmma;
    p.bbytes = (uint32_t)nmma * tc::BK * 2;
    p.m = m; p.n = n; p.k = k; p.C = C; p.ldc = ldc; p.lower = lower ? 1 : 0;
    p.tiles_m = ceil_div(m, tc::BM);
    p.tiles_n = ceil_div(n, tc::BN);
    p.ntiles = p.tiles_m * p.tiles_n;
    const int nkb = k / tc::BK;
    if (ksplit < 1 || P == nullptr) ksplit = 1;
    if (ksplit > nkb) ksplit = nkb;
    p.kps = ceil_div(nkb, ksplit);
    p.ksplit = ceil_div(nkb, p.kps);          // every range non-empty
    p.nunits = p.ntiles * p.ksplit;
    p.P = p.ksplit > 1 ? P : nullptr;
    const size_t smem = 1024 + tc::STAGES * tc::kStageBytes + sizeof(tc::Smem);
    int grid = num_sms();
    if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
    if (grid > p.nunits) grid = p.nunits;
    if (nmma < tc::BN) {
        CF_CUDA_TRY(cudaFuncSetAttribute(tc::k_schur_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        tc::k_schur_tc<true><<<grid, tc::kThreads, smem, st>>>(ta, tb, p, tc::make_idesc(bf16, tc::BM, nmma));
    } else {
        CF_CUDA_TRY(cudaFuncSetAttribute(tc::k_schur_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        tc::k_schur_tc<false><<<grid, tc::kThreads, smem, st>>>(ta, tb, p, tc::make_idesc(bf16, tc::BM, nmma));
    }
    CF_LAUNCH_CHECK();
    if (p.P != nullptr) {
        tc::k_splitk_reduce<<<dim3(8, p.ntiles), 256, 0, st>>>(p);
        CF_LAUNCH_CHECK();
    }
    return CF_OK;
}

int tc_take_status(cudaStream_t st, int *status) {
    int h = 0;
    CF_CUDA_TRY(cudaMemcpyFromSymbolAsync(&h, g_tc_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    CF_CUDA_TRY(cudaStreamSynchronize(st));
    if (h != 0) {
        const int zero = 0;
        CF_CUDA_TRY(cudaMemcpyToSymbolAsync(g_tc_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
        CF_CUDA_TRY(cudaStreamSynchronize(st));
    }
    *status = h;
    return CF_OK;
}

}  // namespace cf

extern "C" int cf_schur_update_lp(int m, int n, int k, const void *A_lp, int lda_k, const void *B_lp, int ldb_k,
                                  float *C, int ldc, cf_prec prec, int lower, cudaStream_t stream) {
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (k < 0 || k % 64 != 0) return -3;
    if (m > 0 && k > 0 && A_lp == nullptr) return -4;
    if (lda_k < k || lda_k % 8 != 0) return -5;
    if (n > 0 && k > 0 && B_lp == nullptr) return -6;
    if (ldb_k < k || ldb_k % 8 != 0) return -7;
    if (m > 0 && n > 0 && C == nullptr) return -8;
    if (ldc < (m > 1 ? m : 1)) return -9;
    if (prec != CF_BF16 && prec != CF_F16) return -10;
    return cf::launch_schur_tc(m, n, k, A_lp, lda_k, B_lp, ldb_k, C, ldc, prec == CF_BF16, lower != 0, stream, 0);
}

extern "C" size_t cf_schur_update_lp_splitk_workspace_size(int m, int n, int k, int ksplit) {
    (void)k;
    return cf::schur_tc_splitk_bytes(m, n, ksplit);
}

extern "C" int cf_schur_update_lp_splitk(int m, int n, int k, const void *A_lp, int lda_k, const void *B_lp, int ldb_k,
                                         float *C, int ldc, cf_prec prec, int lower, int ksplit, void *work,
                                         size_t lwork, cudaStream_t stream) {
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (k < 0 || k % 64 != 0) return -3;
    if (m > 0 && k > 0 && A_lp == nullptr) return -4;
    if (lda_k < k || lda_k % 8 != 0) return -5;
    if (n > 0 && k > 0 && B_lp == nullptr) return -6;
    if (ldb_k < k || ldb_k % 8 != 0) return -7;
    if (m > 0 && n > 0 && C == nullptr) return -8;
    if (ldc < (m > 1 ? m : 1)) return -9;
    if (prec != CF_BF16 && prec != CF_F16) return -10;
    if (ksplit < 1 || ksplit > 64) return -12;
    if (m == 0 || n == 0 || k == 0) return CF_OK;
    if (ksplit > 1 && (work == nullptr || lwork < cf::schur_tc_splitk_bytes(m, n, ksplit))) return CF_ERR_WORKSPACE;
    return cf::launch_schur_tc_splitk(m, n, k, A_lp, lda_k, B_lp, ldb_k, C, ldc, prec == CF_BF16, lower != 0, ksplit,
                                      (float *)work, stream, 0);
}

extern "C" int cf_device_status(cudaStream_t stream) {
    int s = 0, s8 = 0, st = 0, sr = 0;
    int rc = cf::tc_take_status(stream, &s);
    if (rc != CF_OK) return rc;
    if ((rc = cf::fp8_take_status(stream, &s8)) != CF_OK) return rc;
    if ((rc = cf::trsv_take_status(stream, &st)) != CF_OK) return rc;
    if ((rc = cf::rtc_take_status(stream, &sr)) != CF_OK) return rc;
    return s != 0 ? s : (s8 != 0 ? s8 : (st != 0 ? st : sr));
}
