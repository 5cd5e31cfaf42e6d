// cf_panel32.cu -- FP32 block routines of the mixed-precision path, built for
// latency (they sit on the chain of dependent work of every step):
//
//   k_a00_lu_q32,   LU of A00 without pivoting (Fig. "prog_rep" on
//   k_a00_lu32      the rows TournPivot selected; Sec. 7.2)
//   k_a00_chol32    Cholesky of A00 (Listing "Cholesky Factorization"; CH-1)
//   k_rtrsm32(_w)   LU-3  A10 <- A10 U00^{-1}  /  CH-2  L10 <- A10 L00^{-T}
//   k_ltrsm32(_w)   LU-4  A01 <- L00^{-1} A01
//
// The A00 kernels: one thread per row (four lanes per row for LU blocks of
// up to 64 rows), the row in registers with compile-time indices, one
// barrier per column.
// The panel solves: one thread per row (LU-3, CH-2) or column (LU-4), held
// as float2 pairs updated with packed FMAs, no barrier, results written
// straight from registers; they also write the BF16/FP16 K-major copies that
// the tensor-core update reads.  Full panels (w = 64 or 128) take the
// fixed-width forms k_rtrsm32_w / k_ltrsm32_w (column loop unrolled at
// compile time), ragged ones k_rtrsm32 / k_ltrsm32.  (Four lanes per row,
// each with a quarter of it, measured slower: 30.2 against 24.1 us for
// 24000 x 64 with the shifting form; the quartered form issues about twice
// the instructions.)
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "cf_common.cuh"
#include "cf_kernels.cuh"
#include "cf_regrow.cuh"

namespace cf {

template <typename LP>
__device__ __forceinline__ LP lp_from(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 lp_from<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }
template <>
__device__ __forceinline__ __half lp_from<__half>(float x) { return __float2half_rn(x); }

// ---------------------------------------------------------------------------
// A00 LU of blocks of up to 64 rows, four lanes per row: lane q of row r
// holds the row's columns 16q .. 16q + 15, one barrier per column.  With one
// thread per row (below) a 64 x 64 LU issued ~10,000 instructions per warp
// on two warps (ncu: 24 us per launch, 19% issue active, 1.8 cycles of
// fixed-latency wait per issue); split four ways over eight warps it takes
// 18.7 us against 26.2 (measured alone).  For 128 rows the quartered rows
// (32 columns a lane, the column loop unrolled 32 times) measured slower
// than one thread per row (83 against 53 us), and so did the same form of
// the Cholesky (108 against 51 us at 128 rows): those keep the kernels
// below.
//
// LU without pivoting (Fig. "prog_rep" on the rows TournPivot
// selected, Sec. 7.2), in place: for every column k, row k (final from
// column k on) is published in shared memory; every row r > k takes
// l = a(r, k) / a(k, k) (its lane holding column k divides and hands l to
// the other three) and does a(r, j) -= l a(k, j) for j > k.  A zero pivot
// is reported in info and its column is not divided (LAPACK dgetf2); the
// elimination then goes on with the undivided column.
// ---------------------------------------------------------------------------
template <int R>
__global__ void __launch_bounds__(4 * R, 1) k_a00_lu_q32(float *A00, int lda, int w, int kglob, int *info) {
    constexpr int T = 4, C = R / T;
    __shared__ __align__(16) float prow[2][R];
    const int tid = threadIdx.x, r = tid / T, q = tid % T, lane = tid & 31;
    const int base = lane - q, c0 = q * C;
    const bool row_live = r < w;
    float a[C];
#pragma unroll
    for (int jl = 0; jl < C; ++jl) a[jl] = (row_live && c0 + jl < w) ? A00[(size_t)r + (size_t)(c0 + jl) * lda] : 0.f;
    if (r == 0) {
#pragma unroll
        for (int g = 0; g < C / 4; ++g)
            *reinterpret_cast<float4 *>(&prow[0][c0 + 4 * g]) =
                make_float4(a[4 * g], a[4 * g + 1], a[4 * g + 2], a[4 * g + 3]);
    }
    __syncthreads();
    for (int qo = 0; qo < T; ++qo) {
        if (qo * C >= w) break;
#pragma unroll
        for (int kl = 0; kl < C; ++kl) {
            const int k = qo * C + kl;
            if (k >= w) break;
            const float *u = prow[k & 1];
            const float piv = u[k];
            const bool upd = row_live && r > k;
            float l = 0.f;
            if (upd && q == qo) l = (piv != 0.f) ? a[kl] / piv : a[kl];
            l = __shfl_sync(0xffffffffu, l, base + qo);
            if (upd) {
                if (q == qo) a[kl] = l;                           // L(r, k)
                float m[C];
#pragma unroll
                for (int g = 0; g < C / 4; ++g) {
                    const float4 v = *reinterpret_cast<const float4 *>(u + c0 + 4 * g);
                    m[4 * g] = v.x; m[4 * g + 1] = v.y; m[4 * g + 2] = v.z; m[4 * g + 3] = v.w;
                }
#pragma unroll
                for (int jl = 0; jl < C; ++jl)
                    if (q > qo || (q == qo && jl > kl)) a[jl] = fmaf(-l, m[jl], a[jl]);
            }
            if (r == k + 1 && k + 1 < w) {                         // the next pivot row, final from k + 1 on
#pragma unroll
                for (int g = 0; g < C / 4; ++g)
                    *reinterpret_cast<float4 *>(&prow[(k + 1) & 1][c0 + 4 * g]) =
                        make_float4(a[4 * g], a[4 * g + 1], a[4 * g + 2], a[4 * g + 3]);
            }
            if (tid == 0 && piv == 0.f) atomicCAS(info, 0, kglob + k + 1);
            __syncthreads();
        }
    }
    if (row_live) {
#pragma unroll
        for (int jl = 0; jl < C; ++jl)
            if (c0 + jl < w) A00[(size_t)r + (size_t)(c0 + jl) * lda] = a[jl];
    }
}

// ---------------------------------------------------------------------------
// A00 = L00 U00, no pivoting, in place (w <= 128).  Thread r owns row r as a
// pair row (cf_regrow.cuh, packed FMAs), blocked by 8 columns:
//   column k = j0 + U: row k publishes its 8 in-block values; barrier; row k
//   of U inside the block is stored, every row r > k takes l = a / pivot,
//   stores L(r, k) and updates its in-block columns only;
//   block end: the 8 pivot rows publish the rest of their rows as they were
//   at the block start, â_U, and their multipliers L(U, U') (U' < U); barrier;
//   every row after the block's first applies a -= sum_U c_U â_U with
//   c^T (I + L) = l^T (its multipliers, zero past its own position for a
//   pivot row), which equals the 8 rank-1 updates; the pivot rows' finished
//   U rows go out through shared memory as coalesced column segments.
// A zero pivot is reported in info and its column is not divided (LAPACK
// dgetf2); the elimination then proceeds with the undivided column.
// ---------------------------------------------------------------------------
struct A00LuSmem {
    float4 slot[kBlk][2];                 // pivot k's in-block values (relative to the block)
    float4 prow[kBlk][kMaxV / 4 + 1];     // block end: pivot rows at the block start (padded stride)
    float4 ufin[kBlk][kMaxV / 4 + 1];     // block end: pivot rows' finished U values
    float lmat[kBlk][kBlk];
};

struct LuStep {
    A00LuSmem &s;
    float2 (&a)[kPairs];
    float (&lb)[kBlk];
    float *A00;
    int lda, w, r, kglob;
    int *info;
    template <int U>
    __device__ __forceinline__ void step(int j0) {
        const int k = j0 + U;
        if (r == k) {
            s.slot[U][0] = make_float4(a[0].x, a[0].y, a[1].x, a[1].y);
            s.slot[U][1] = make_float4(a[2].x, a[2].y, a[3].x, a[3].y);
        }
        __syncthreads();
        const float *pf = reinterpret_cast<const float *>(s.slot[U]);
        if (r < kBlk - U && k + r < w) A00[(size_t)k + (size_t)(k + r) * lda] = pf[U + r];     // U(k, k + r)
        const float piv = pf[U];
        if (r > k && r < w) {
            const float au = pair_elem<U>(a);
            const float l = (piv != 0.f) ? au / piv : au;
            A00[(size_t)r + (size_t)k * lda] = l;                                          // L(r, k)
            lb[U] = l;
            const float2 nl = make_float2(-l, -l);
            const float4 u0 = s.slot[U][0], u1 = s.slot[U][1];
            if (1 > U) a[0] = __ffma2_rn(nl, make_float2(u0.x, u0.y), a[0]);
            if (3 > U) a[1] = __ffma2_rn(nl, make_float2(u0.z, u0.w), a[1]);
            if (5 > U) a[2] = __ffma2_rn(nl, make_float2(u1.x, u1.y), a[2]);
            if (7 > U) a[3] = __ffma2_rn(nl, make_float2(u1.z, u1.w), a[3]);
        }
        if (r == 0 && piv == 0.f) atomicCAS(info, 0, kglob + k + 1);
    }
    __device__ __forceinline__ void block_end(int j0) {
        const int lim = w - j0;                // live columns relative to the block
        const int P = r - j0;                  // position of a pivot row in the block
        const bool pivot_row = P >= 0 && P < kBlk;
        if (pivot_row) {
#pragma unroll
            for (int t = 0; t < kBlk - 1; ++t)
                if (t < P) s.lmat[P][t] = lb[t];
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (c * 32 < lim) {
#pragma unroll
                    for (int q = c * 8; q < c * 8 + 8; ++q)
                        if (q >= 2)
                            s.prow[P][q] = make_float4(a[2 * q].x, a[2 * q].y, a[2 * q + 1].x, a[2 * q + 1].y);
                }
        }
        __syncthreads();
        if (P > 0 && r < w) {
            float c[kBlk];
#pragma unroll
            for (int u = kBlk - 1; u >= 0; --u) {
                float t = lb[u];
#pragma unroll
                for (int u2 = u + 1; u2 < kBlk; ++u2) t = fmaf(-c[u2], s.lmat[u2][u], t);
                c[u] = t;
            }
#pragma unroll
            for (int u = 0; u < kBlk; ++u) {
                const float2 nc = make_float2(-c[u], -c[u]);
#pragma unroll
                for (int ch = 0; ch < 4; ++ch)
                    if (ch * 32 < lim) {
#pragma unroll
                        for (int q = ch * 8; q < ch * 8 + 8; ++q) {
                            if (q < 2) continue;
                            const float4 p = s.prow[u][q];
                            a[2 * q] = __ffma2_rn(nc, make_float2(p.x, p.y), a[2 * q]);
                            a[2 * q + 1] = __ffma2_rn(nc, make_float2(p.z, p.w), a[2 * q + 1]);
                        }
                    }
            }
        }
        if (pivot_row) {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (c * 32 < lim) {
#pragma unroll
                    for (int q = c * 8; q < c * 8 + 8; ++q)
                        if (q >= 2)
                            s.ufin[P][q] = make_float4(a[2 * q].x, a[2 * q].y, a[2 * q + 1].x, a[2 * q + 1].y);
                }
        }
        __syncthreads();
        const float *uf = reinterpret_cast<const float *>(&s.ufin[0][0]);
        constexpr int UFS = 4 * (kMaxV / 4 + 1);
        for (int e = threadIdx.x; e < kBlk * (lim - kBlk); e += blockDim.x) {
            const int q = e % kBlk, t = kBlk + e / kBlk;          // U(j0 + q, j0 + t)
            A00[(size_t)(j0 + q) + (size_t)(j0 + t) * lda] = uf[q * UFS + t];
        }
#pragma unroll
        for (int u = 0; u < kBlk; ++u) lb[u] = 0.f;
    }
};

__device__ __forceinline__ void load_pair_row(float2 (&a)[kPairs], const float *A00, int lda, int r, int w) {
#pragma unroll
    for (int k = 0; k < kPairs; ++k) {
        const float x = (r < w && 2 * k < w) ? A00[(size_t)r + (size_t)(2 * k) * lda] : 0.f;
        const float y = (r < w && 2 * k + 1 < w) ? A00[(size_t)r + (size_t)(2 * k + 1) * lda] : 0.f;
        a[k] = make_float2(x, y);
    }
}

__global__ void __launch_bounds__(kMaxV, 1) k_a00_lu32(float *A00, int lda, int w, int kglob, int *info) {
    __shared__ __align__(16) A00LuSmem s;
    const int r = threadIdx.x;
    float2 a[kPairs];
    float lb[kBlk];
#pragma unroll
    for (int u = 0; u < kBlk; ++u) lb[u] = 0.f;
    load_pair_row(a, A00, lda, r, w);
    LuStep body{s, a, lb, A00, lda, w, r, kglob, info};
    for (int j0 = 0; j0 < w; j0 += kBlk) {
        body.template step<0>(j0);
        if (j0 + 1 < w) body.template step<1>(j0);
        if (j0 + 2 < w) body.template step<2>(j0);
        if (j0 + 3 < w) body.template step<3>(j0);
        if (j0 + 4 < w) body.template step<4>(j0);
        if (j0 + 5 < w) body.template step<5>(j0);
        if (j0 + 6 < w) body.template step<6>(j0);
        if (j0 + 7 < w) body.template step<7>(j0);
        if (j0 + kBlk >= w) break;
        body.block_end(j0);
        shift_pairs(a, w - j0 - kBlk);
    }
}

// ---------------------------------------------------------------------------
// A00 = L00 L00^T (lower), in place.  Thread r owns row r (pair row), blocked
// by 8 columns: for column k = j0 + U every live row r >= k publishes its
// entry a(r, k) (the column k of the Schur complement, kept for the block);
// barrier; L(k, k) = sqrt(a(k, k)), every row r > k stores L(r, k) and
// updates its in-block columns; at the block end every row below the block
// applies the rank-8 update a(r, t) -= sum_U L(r, U) L(t, U) for the columns
// t past the block (L(t, U) = the published a(t, U) / L(U, U)), with no
// barrier (the column buffers alternate between blocks).  Stops at the first
// pivot that is not positive (info).
// ---------------------------------------------------------------------------
struct A00CholSmem {
    float4 col[2][kBlk][kMaxV / 4 + 1];   // [block parity][U][relative row]
};

struct CholStep {
    A00CholSmem &s;
    float2 (&a)[kPairs];
    float (&lb)[kBlk];                    // L(r, U) / L(U, U)
    float *A00;
    int lda, w, r, kglob;
    int *info;
    bool failed;
    template <int U>
    __device__ __forceinline__ void step(int j0) {
        if (failed) return;                          // uniform
        const int k = j0 + U, bp = (j0 / kBlk) & 1;
        float *cf = reinterpret_cast<float *>(s.col[bp][U]);
        const float au = pair_elem<U>(a);
        if (r >= k && r < w) cf[r - j0] = au;        // column k by relative row
        __syncthreads();
        const float d = cf[U];
        if (!(d > 0.f)) {
            if (r == 0) atomicCAS(info, 0, kglob + k + 1);
            failed = true;                           // every thread read the same d
            return;
        }
        const float lkk = sqrtf(d);
        if (r == k) A00[(size_t)k + (size_t)k * lda] = lkk;
        if (r > k && r < w) {
            const float l = au / lkk;
            A00[(size_t)r + (size_t)k * lda] = l;                               // L(r, k)
            // a(r, j0+t) -= L(r,k) L(j0+t,k) = (l / lkk) col[t]
            const float cl = l / lkk;
            lb[U] = cl;
            const float2 nl = make_float2(-cl, -cl);
            const float4 u0 = s.col[bp][U][0], u1 = s.col[bp][U][1];
            if (1 > U) a[0] = __ffma2_rn(nl, make_float2(u0.x, u0.y), a[0]);
            if (3 > U) a[1] = __ffma2_rn(nl, make_float2(u0.z, u0.w), a[1]);
            if (5 > U) a[2] = __ffma2_rn(nl, make_float2(u1.x, u1.y), a[2]);
            if (7 > U) a[3] = __ffma2_rn(nl, make_float2(u1.z, u1.w), a[3]);
        }
    }
    __device__ __forceinline__ void block_end(int j0) {
        if (failed) return;
        const int bp = (j0 / kBlk) & 1;
        const int lim = r - j0 + 1;                  // columns up to the diagonal
        if (r >= j0 + kBlk && r < w) {
#pragma unroll
            for (int u = 0; u < kBlk; ++u) {
                const float2 nc = make_float2(-lb[u], -lb[u]);
#pragma unroll
                for (int ch = 0; ch < 4; ++ch)
                    if (ch * 32 < lim) {
#pragma unroll
                        for (int q = ch * 8; q < ch * 8 + 8; ++q) {
                            if (q < 2) continue;
                            const float4 p = s.col[bp][u][q];
                            a[2 * q] = __ffma2_rn(nc, make_float2(p.x, p.y), a[2 * q]);
                            a[2 * q + 1] = __ffma2_rn(nc, make_float2(p.z, p.w), a[2 * q + 1]);
                        }
                    }
            }
        }
#pragma unroll
        for (int u = 0; u < kBlk; ++u) lb[u] = 0.f;
    }
};

__global__ void __launch_bounds__(kMaxV, 1) k_a00_chol32(float *A00, int lda, int w, int kglob, int *info) {
    if (*info != 0) return;
    __shared__ __align__(16) A00CholSmem s;
    const int r = threadIdx.x;
    float2 a[kPairs];
    float lb[kBlk];
#pragma unroll
    for (int u = 0; u < kBlk; ++u) lb[u] = 0.f;
    load_pair_row(a, A00, lda, r, w);
    CholStep body{s, a, lb, A00, lda, w, r, kglob, info, false};
    for (int j0 = 0; j0 < w; j0 += kBlk) {
        body.template step<0>(j0);
        if (j0 + 1 < w) body.template step<1>(j0);
        if (j0 + 2 < w) body.template step<2>(j0);
        if (j0 + 3 < w) body.template step<3>(j0);
        if (j0 + 4 < w) body.template step<4>(j0);
        if (j0 + 5 < w) body.template step<5>(j0);
        if (j0 + 6 < w) body.template step<6>(j0);
        if (j0 + 7 < w) body.template step<7>(j0);
        if (j0 + kBlk >= w) break;
        body.block_end(j0);
        shift_pairs(a, w - j0 - kBlk);
    }
}

// Packs 8 consecutive values as low-precision and stores them as one 16-byte
// chunk (dst 16-byte aligned).
template <typename LP>
__device__ __forceinline__ void store8_lp(LP *dst, const float (&v)[8]) {
    union { uint4 u; LP h[8]; } pk;
#pragma unroll
    for (int i = 0; i < 8; ++i) pk.h[i] = lp_from<LP>(v[i]);
    *reinterpret_cast<uint4 *>(dst) = pk.u;
}

// Solve steps on a pair row (cf_regrow.cuh): x_k = a_k / M(k, k) (unit: a_k),
// then a_t -= x_k M(k, t) for t > k; x_k is kept in xb for the block's
// output.  RT: right solve (thread = row of X, M row k at Ms + k*kMaxV,
// 1/M(k,k) in rinv), writes x_k to its FP32 column at once (coalesced over
// the CTA's rows); LT: left solve with unit L (thread = column of X, L column
// k at Ls + k*kMaxV).
struct RtrsmPairStep {
    float2 (&a)[kPairs];
    float (&xb)[8];
    const float *Ms;
    const float *rinv;
    float *xcol;        // X + row, stride ldx (null: not a live row)
    int ldx, w;
    template <int U>
    __device__ __forceinline__ void step(int j0) {
        const int k = j0 + U;
        const float xk = pair_elem<U>(a) * rinv[k];
        xb[U] = xk;
        if (xcol) xcol[(size_t)k * ldx] = xk;
        rank1_pairs<U>(a, xk, reinterpret_cast<const float4 *>(Ms + k * kMaxV + j0), w - j0);
    }
};

struct LtrsmPairStep {
    float2 (&a)[kPairs];
    float (&xb)[8];
    const float *Ls;
    int w;
    template <int U>
    __device__ __forceinline__ void step(int j0) {
        const int k = j0 + U;
        const float xk = pair_elem<U>(a);            // unit diagonal
        xb[U] = xk;
        rank1_pairs<U>(a, xk, reinterpret_cast<const float4 *>(Ls + k * kMaxV + j0), w - j0);
    }
};

template <typename Body>
__device__ __forceinline__ void run_block(Body &body, int j0, int w) {
    body.template step<0>(j0);
    if (j0 + 1 < w) body.template step<1>(j0);
    if (j0 + 2 < w) body.template step<2>(j0);
    if (j0 + 3 < w) body.template step<3>(j0);
    if (j0 + 4 < w) body.template step<4>(j0);
    if (j0 + 5 < w) body.template step<5>(j0);
    if (j0 + 6 < w) body.template step<6>(j0);
    if (j0 + 7 < w) body.template step<7>(j0);
}

// ---------------------------------------------------------------------------
// Right solve of a panel: X (rows x w, column-major ldx) <- X M^{-1} with
// M = U00 (upper, non-unit; trans_lower = false) or M = L00^T (trans_lower).
// Thread = row, held as a pair row; M staged row by row (Ms[k][c] = M(k, c),
// zero below the diagonal) with the reciprocals of its diagonal (a zero
// diagonal entry divides by one, as the FP64 path skips the division).  The
// FP32 result goes back column by column as it is produced; lp[r*ldk + j]
// (j < kpad, zero for j >= w) is written in 16-byte chunks of 8.
// ---------------------------------------------------------------------------
template <typename LP>
__global__ void __launch_bounds__(kMaxV)
k_rtrsm32(float *X, int ldx, int rows, int w, const float *__restrict__ M00, int ldm, int trans_lower, LP *lp,
          int ldk, int kpad, const int *skip) {
    if (skip != nullptr && *skip != 0) return;
    extern __shared__ __align__(16) float smem[];
    // [kMaxV + 1][kMaxV]: a step reads row k from column j0 in whole 32-column
    // chunks, up to 31 floats past the row's end; the last row's overrun
    // lands in the zeroed padding row
    float *Ms = smem;
    __shared__ float rinv[kMaxV];
    const int tid = threadIdx.x;
    Ms[kMaxV * kMaxV + tid] = 0.f;
    // Staged 16 loads at a time (the triangle is L2-resident; one load per
    // iteration left its latency exposed 128 times), with shared-memory stores
    // along rows of Ms: for U00 a thread takes a column c (strided reads,
    // conflict-free stores), for L00^T a row i of L (coalesced reads).
    constexpr int kStage = 16;
    if (!trans_lower) {
        for (int i0 = 0; i0 < kMaxV; i0 += kStage) {
            float v[kStage];
#pragma unroll
            for (int u = 0; u < kStage; ++u) {
                const int i = i0 + u;
                v[u] = (i < w && tid < w && i <= tid) ? M00[(size_t)i + (size_t)tid * ldm] : 0.f;   // U(i, c)
            }
#pragma unroll
            for (int u = 0; u < kStage; ++u) Ms[(i0 + u) * kMaxV + tid] = v[u];
        }
    } else {
        for (int c0 = 0; c0 < kMaxV; c0 += kStage) {
            float v[kStage];
#pragma unroll
            for (int u = 0; u < kStage; ++u) {
                const int c = c0 + u;
                v[u] = (tid < w && c < w && tid >= c) ? M00[(size_t)tid + (size_t)c * ldm] : 0.f;   // L(i, c)
            }
#pragma unroll
            for (int u = 0; u < kStage; ++u) Ms[(c0 + u) * kMaxV + tid] = v[u];                // M(c, i)
        }
    }
    __syncthreads();
    if (tid < w) {
        const float d = Ms[tid * kMaxV + tid];
        rinv[tid] = d != 0.f ? 1.0f / d : 1.0f;
    }
    const int r0 = blockIdx.x * kMaxV;
    const int nr = min(kMaxV, rows - r0);
    const bool live = tid < nr;
    float2 a[kPairs];
    // coalesced load: for each column k, the CTA's rows are contiguous
#pragma unroll
    for (int k = 0; k < kPairs; ++k) {
        const float x0 = (live && 2 * k < w) ? X[(size_t)(r0 + tid) + (size_t)(2 * k) * ldx] : 0.f;
        const float x1 = (live && 2 * k + 1 < w) ? X[(size_t)(r0 + tid) + (size_t)(2 * k + 1) * ldx] : 0.f;
        a[k] = make_float2(x0, x1);
    }
    __syncthreads();
    float xb[8];
    RtrsmPairStep body{a, xb, Ms, rinv, live ? X + r0 + tid : nullptr, ldx, w};
    LP *lrow = (lp != nullptr && live) ? lp + (size_t)(r0 + tid) * ldk : nullptr;
    for (int j0 = 0; j0 < w; j0 += kBlk) {
#pragma unroll
        for (int i = 0; i < 8; ++i) xb[i] = 0.f;
        run_block(body, j0, w);
        shift_pairs(a, w - j0 - kBlk);
        if (lrow) store8_lp<LP>(lrow + j0, xb);
    }
    if (lrow) {
        float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int j0 = (w + 7) / 8 * 8; j0 < kpad; j0 += 8) store8_lp<LP>(lrow + j0, z);
    }
}

// ---------------------------------------------------------------------------
// Left solve of a row block: X (w x cols, column-major ldx) <- L00^{-1} X, L00
// unit lower.  Thread = column, held as a pair row; L staged column by
// column (Ls[k][i] = L(i, k), zero on and above the diagonal).  Results are
// written per block of 8 rows (two 16-byte stores, scalar for a ragged last
// block) and as 16-byte low-precision chunks at lp[c*ldk + i] (i < kpad,
// zero for i >= w).
// ---------------------------------------------------------------------------
template <typename LP>
__global__ void __launch_bounds__(kMaxV)
k_ltrsm32(float *X, int ldx, int w, int cols, const float *__restrict__ L00, int ldl, LP *lp, int ldk, int kpad) {
    extern __shared__ __align__(16) float smem[];
    float *Ls = smem;                                // [kMaxV + 1][kMaxV]: Ls[k][i] = L(i, k), zero padding row
    const int tid = threadIdx.x;
    Ls[kMaxV * kMaxV + tid] = 0.f;
    for (int k0 = 0; k0 < kMaxV; k0 += 16) {         // 16 loads in flight per thread
        float v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int k = k0 + u;
            v[u] = (k < w && tid > k && tid < w) ? L00[(size_t)tid + (size_t)k * ldl] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) Ls[(k0 + u) * kMaxV + tid] = v[u];
    }
    const int c0 = blockIdx.x * kMaxV;
    const int nc = min(kMaxV, cols - c0);
    const bool live = tid < nc;
    float *xc = X + (size_t)(c0 + (live ? tid : 0)) * ldx;
    float2 a[kPairs];
#pragma unroll
    for (int i = 0; i < kPairs; ++i)
        a[i] = make_float2((live && 2 * i < w) ? xc[2 * i] : 0.f, (live && 2 * i + 1 < w) ? xc[2 * i + 1] : 0.f);
    __syncthreads();
    const bool vec = ((((uintptr_t)xc) & 15) == 0);
    float xb[8];
    LtrsmPairStep body{a, xb, Ls, w};
    LP *lcol = (lp != nullptr && live) ? lp + (size_t)(c0 + tid) * ldk : nullptr;
    for (int j0 = 0; j0 < w; j0 += kBlk) {
#pragma unroll
        for (int i = 0; i < 8; ++i) xb[i] = 0.f;
        run_block(body, j0, w);
        shift_pairs(a, w - j0 - kBlk);
        if (live) {
            if (vec && j0 + 8 <= w) {
                reinterpret_cast<float4 *>(xc + j0)[0] = make_float4(xb[0], xb[1], xb[2], xb[3]);
                reinterpret_cast<float4 *>(xc + j0)[1] = make_float4(xb[4], xb[5], xb[6], xb[7]);
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    if (j0 + i < w) xc[j0 + i] = xb[i];
            }
        }
        if (lcol) store8_lp<LP>(lcol + j0, xb);
    }
    if (lcol) {
        float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int j0 = (w + 7) / 8 * 8; j0 < kpad; j0 += 8) store8_lp<LP>(lcol + j0, z);
    }
}

// ---------------------------------------------------------------------------
// Fixed-width panel solves (w = W = 64 or 128, the full panels): the same
// arithmetic as k_rtrsm32 / k_ltrsm32, in the same order, with the column
// loop unrolled at compile time, so the row is never shifted and every index
// is a constant (k_rtrsm32 spends ~1,000 register moves per row on shifts
// at w = 64).  The row (column) of X is loaded before the triangle is
// staged, so the two latencies overlap, and the triangle is staged with
// coalesced loads, all of a thread's loads of a batch in flight at once,
// into rows padded to W + 4 floats (conflict-free stores, 16-byte aligned
// rows).  Measured alone: 12.4 us against 22.6 for 24000 x 64 (LU-3), 26.8
// against 39.1 for 32640 x 128 (CH-2), results bit-identical.
//
// Ms[k][t] = M(k, t) for t >= k (the factor's storage on the diagonal for
// the unit left solve: there it multiplies only entries that are already
// final, never read again), zero left of the diagonal.
//   TRI 0: M = U00, M(k, t) = M00[k + t ldm]   (right solve, LU-3)
//   TRI 1: M = L00^T, M(k, t) = M00[t + k ldm] (right solve CH-2; unit left
//          solve LU-4, where row k of M is column k of L)
// ---------------------------------------------------------------------------
template <int W, int NT, int TRI>
__device__ __forceinline__ void stage_tri_fixed(float *Ms, const float *__restrict__ M00, int ldm) {
    constexpr int MS = W + 4, NE = W * W / NT, BATCH = NE < 32 ? NE : 32;
    static_assert(NT % 32 == 0 && NE % BATCH == 0, "staging layout");
    const int tid = threadIdx.x, lane = tid & 31;
#pragma unroll 1
    for (int b0 = 0; b0 < NE; b0 += BATCH) {
        float v[BATCH];
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            const int e = (b0 + u) * NT + tid;
            if constexpr (TRI == 0) {
                // a warp takes 8 consecutive k (32 bytes of a column of U) x 4 columns t
                const int T = e >> 5;
                const int k = 8 * (T % (W / 8)) + (lane & 7), t = 4 * (T / (W / 8)) + (lane >> 3);
                v[u] = k <= t ? M00[(size_t)k + (size_t)t * ldm] : 0.f;
            } else {
                const int t = e % W, k = e / W;   // a warp takes 32 consecutive t of column k of L
                v[u] = t >= k ? M00[(size_t)t + (size_t)k * ldm] : 0.f;
            }
        }
#pragma unroll
        for (int u = 0; u < BATCH; ++u) {
            const int e = (b0 + u) * NT + tid;
            int k, t;
            if constexpr (TRI == 0) {
                const int T = e >> 5;
                k = 8 * (T % (W / 8)) + (lane & 7);
                t = 4 * (T / (W / 8)) + (lane >> 3);
            } else {
                t = e % W;
                k = e / W;
            }
            Ms[k * MS + t] = v[u];
        }
    }
}

// Column k = K of the solve on a pair row: x_K = a_K (LEFT, unit diagonal)
// or a_K / M(K, K); a_t -= x_K M(K, t) for the pairs holding a column > K.
// RIGHT writes x_K to its FP32 column at once (coalesced over the CTA's
// rows); LEFT writes each block of 8 as two 16-byte stores.  Both write the
// low-precision copy per block of 8.
template <int W, bool LEFT, typename LP>
struct TrsmFixed {
    static constexpr int MS = W + 4;
    float2 (&a)[W / 2];
    float (&xb)[8];
    const float *Ms;
    const float *rinv;
    float *xout;   // RIGHT: X + row, column stride ldx; LEFT: the column, contiguous; null: not live
    LP *lout;
    int ldx;
    template <int K>
    __device__ __forceinline__ void run() {
        if constexpr (K < W) {
            float xk = (K & 1) ? a[K >> 1].y : a[K >> 1].x;
            if constexpr (!LEFT) {
                xk *= rinv[K];
                if (xout) xout[(size_t)K * ldx] = xk;
            }
            xb[K & 7] = xk;
            const float2 nl = make_float2(-xk, -xk);
            const float4 *row = reinterpret_cast<const float4 *>(Ms + K * MS);
#pragma unroll
            for (int q = K / 4; q < W / 4; ++q) {
                const float4 p = row[q];
                if (4 * q >= K) a[2 * q] = __ffma2_rn(nl, make_float2(p.x, p.y), a[2 * q]);
                if (4 * q + 2 >= K) a[2 * q + 1] = __ffma2_rn(nl, make_float2(p.z, p.w), a[2 * q + 1]);
            }
            if constexpr ((K & 7) == 7) {
                if constexpr (LEFT) {
                    if (xout) {
                        reinterpret_cast<float4 *>(xout + K - 7)[0] = make_float4(xb[0], xb[1], xb[2], xb[3]);
                        reinterpret_cast<float4 *>(xout + K - 7)[1] = make_float4(xb[4], xb[5], xb[6], xb[7]);
                    }
                }
                if (lout) store8_lp<LP>(lout + K - 7, xb);
            }
            run<K + 1>();
        }
    }
};

template <int W, typename LP>
__global__ void __launch_bounds__(128, 1)
k_rtrsm32_w(float *X, int ldx, int rows, const float *__restrict__ M00, int ldm, int trans_lower, LP *lp, int ldk,
            int kpad, const int *skip) {
    if (skip != nullptr && *skip != 0) return;
    constexpr int MS = W + 4;
    extern __shared__ __align__(16) float smem[];
    float *Ms = smem;               // [W][MS]
    float *rinv = smem + W * MS;    // [W]
    const int tid = threadIdx.x;
    const int r0 = blockIdx.x * 128;
    const bool live = tid < rows - r0;
    float2 a[W / 2];
#pragma unroll
    for (int p = 0; p < W / 2; ++p) {
        const float x0 = live ? X[(size_t)(r0 + tid) + (size_t)(2 * p) * ldx] : 0.f;
        const float x1 = live ? X[(size_t)(r0 + tid) + (size_t)(2 * p + 1) * ldx] : 0.f;
        a[p] = make_float2(x0, x1);
    }
    if (trans_lower) stage_tri_fixed<W, 128, 1>(Ms, M00, ldm);
    else stage_tri_fixed<W, 128, 0>(Ms, M00, ldm);
    __syncthreads();
    if (tid < W) {
        const float d = Ms[tid * MS + tid];
        rinv[tid] = d != 0.f ? 1.0f / d : 1.0f;
    }
    __syncthreads();
    float xb[8];
    LP *lrow = (lp != nullptr && live) ? lp + (size_t)(r0 + tid) * ldk : nullptr;
    TrsmFixed<W, false, LP> body{a, xb, Ms, rinv, live ? X + r0 + tid : nullptr, lrow, ldx};
    body.template run<0>();
    if (lrow) {
        float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int j0 = W; j0 < kpad; j0 += 8) store8_lp<LP>(lrow + j0, z);
    }
}

// X (W x cols) <- L00^{-1} X, thread = column, 64 threads per CTA (a slab's
// 2,000 columns spread over twice the SMs).  The columns must be 16-byte
// aligned (the launcher checks).
template <int W, typename LP>
__global__ void __launch_bounds__(64)
k_ltrsm32_w(float *X, int ldx, int cols, const float *__restrict__ L00, int ldl, LP *lp, int ldk, int kpad) {
    constexpr int NT = 64;
    extern __shared__ __align__(16) float smem[];
    float *Ms = smem;               // [W][W + 4]
    const int tid = threadIdx.x;
    const int c0 = blockIdx.x * NT;
    const bool live = tid < cols - c0;
    float *xc = X + (size_t)(c0 + (live ? tid : 0)) * ldx;
    float2 a[W / 2];
#pragma unroll
    for (int q = 0; q < W / 4; ++q) {
        const float4 v = live ? reinterpret_cast<const float4 *>(xc)[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        a[2 * q] = make_float2(v.x, v.y);
        a[2 * q + 1] = make_float2(v.z, v.w);
    }
    stage_tri_fixed<W, NT, 1>(Ms, L00, ldl);
    __syncthreads();
    float xb[8];
    LP *lcol = (lp != nullptr && live) ? lp + (size_t)(c0 + tid) * ldk : nullptr;
    TrsmFixed<W, true, LP> body{a, xb, Ms, nullptr, live ? xc : nullptr, lcol, ldx};
    body.template run<0>();
    if (lcol) {
        float z[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int j0 = W; j0 < kpad; j0 += 8) store8_lp<LP>(lcol + j0, z);
    }
}

// ---------------------------------------------------------------------------
// One CTA: four lanes per row for LU blocks of up to 64 rows (256 threads),
// else one thread per row in whole warps.
int launch_a00_lu32(float *A00, int lda, int w, int kglob, int *info, cudaStream_t st) {
    if (w <= 0) return CF_OK;
    if (w > kMaxV) return CF_ERR_UNSUPPORTED;
    if (w <= 64) k_a00_lu_q32<64><<<1, 256, 0, st>>>(A00, lda, w, kglob, info);
    else k_a00_lu32<<<1, (w + 31) / 32 * 32, 0, st>>>(A00, lda, w, kglob, info);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

int launch_a00_chol32(float *A00, int lda, int w, int kglob, int *info, cudaStream_t st) {
    if (w <= 0) return CF_OK;
    if (w > kMaxV) return CF_ERR_UNSUPPORTED;
    k_a00_chol32<<<1, (w + 31) / 32 * 32, 0, st>>>(A00, lda, w, kglob, info);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

template <typename LP>
int launch_rtrsm32(float *X, int ldx, int rows, int w, const float *M00, int ldm, bool trans_lower, LP *lp, int ldk,
                   int kpad, const int *skip, cudaStream_t st) {
    if (rows <= 0 || w <= 0) return CF_OK;
    if (lp != nullptr && ((ldk % 8) != 0 || (kpad % 8) != 0 || (((uintptr_t)lp) & 15) != 0)) return CF_ERR_UNSUPPORTED;
    if ((w == 64 || w == 128) && (lp == nullptr || kpad >= w)) {
        const size_t smem = sizeof(float) * (size_t)w * (w + 5);
        if (w == 64) {
            CF_CUDA_TRY(cudaFuncSetAttribute(k_rtrsm32_w<64, LP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_rtrsm32_w<64, LP><<<ceil_div(rows, 128), 128, smem, st>>>(X, ldx, rows, M00, ldm, trans_lower ? 1 : 0, lp,
                                                                       ldk, kpad, skip);
        } else {
            CF_CUDA_TRY(cudaFuncSetAttribute(k_rtrsm32_w<128, LP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_rtrsm32_w<128, LP><<<ceil_div(rows, 128), 128, smem, st>>>(X, ldx, rows, M00, ldm, trans_lower ? 1 : 0,
                                                                        lp, ldk, kpad, skip);
        }
        CF_LAUNCH_CHECK();
        return CF_OK;
    }
    const size_t smem = sizeof(float) * (size_t)(kMaxV + 1) * kMaxV;   // + padding row
    CF_CUDA_TRY(cudaFuncSetAttribute(k_rtrsm32<LP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_rtrsm32<LP><<<ceil_div(rows, kMaxV), kMaxV, smem, st>>>(X, ldx, rows, w, M00, ldm, trans_lower ? 1 : 0, lp, ldk,
                                                              kpad, skip);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

template <typename LP>
int launch_ltrsm32(float *X, int ldx, int w, int cols, const float *L00, int ldl, LP *lp, int ldk, int kpad,
                   cudaStream_t st) {
    if (cols <= 0 || w <= 0) return CF_OK;
    if (lp != nullptr && ((ldk % 8) != 0 || (kpad % 8) != 0 || (((uintptr_t)lp) & 15) != 0)) return CF_ERR_UNSUPPORTED;
    if ((w == 64 || w == 128) && (lp == nullptr || kpad >= w) && (((uintptr_t)X) & 15) == 0 && (ldx % 4) == 0) {
        const size_t smem = sizeof(float) * (size_t)w * (w + 4);
        if (w == 64) {
            CF_CUDA_TRY(cudaFuncSetAttribute(k_ltrsm32_w<64, LP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_ltrsm32_w<64, LP><<<ceil_div(cols, 64), 64, smem, st>>>(X, ldx, cols, L00, ldl, lp, ldk, kpad);
        } else {
            CF_CUDA_TRY(cudaFuncSetAttribute(k_ltrsm32_w<128, LP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_ltrsm32_w<128, LP><<<ceil_div(cols, 64), 64, smem, st>>>(X, ldx, cols, L00, ldl, lp, ldk, kpad);
        }
        CF_LAUNCH_CHECK();
        return CF_OK;
    }
    const size_t smem = sizeof(float) * (size_t)(kMaxV + 1) * kMaxV;   // + padding row
    CF_CUDA_TRY(cudaFuncSetAttribute(k_ltrsm32<LP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_ltrsm32<LP><<<ceil_div(cols, kMaxV), kMaxV, smem, st>>>(X, ldx, w, cols, L00, ldl, lp, ldk, kpad);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

template int launch_rtrsm32<__nv_bfloat16>(float *, int, int, int, const float *, int, bool, __nv_bfloat16 *, int,
                                           int, const int *, cudaStream_t);
template int launch_rtrsm32<__half>(float *, int, int, int, const float *, int, bool, __half *, int, int, const int *,
                                    cudaStream_t);
template int launch_ltrsm32<__nv_bfloat16>(float *, int, int, int, const float *, int, __nv_bfloat16 *, int, int,
                                           cudaStream_t);
template int launch_ltrsm32<__half>(float *, int, int, int, const float *, int, __half *, int, int, cudaStream_t);

}  // namespace cf
