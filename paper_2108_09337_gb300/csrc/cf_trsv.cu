// cf_trsv.cu -- S-1 for the refinement loop: triangular solves with the FP32
// factors and a thin right-hand side (nrhs <= 16), one launch per solve.
//
// Block rows (128 for FP32, 64 for FP64 arithmetic) are processed by CTAs
// that take a ticket in launch order
// (atomic counter), so every block a CTA depends on belongs to a CTA that
// started earlier and never waits on a later one.  A CTA subtracts the
// contributions of the finished blocks as their flags appear, applies the
// precomputed inverse of its diagonal block, publishes its block of the
// solution and raises its flag.  The factor is read exactly once; with the
// neighbour tiles premultiplied by the diagonal inverses (FP32 solves), the
// chain of dependent work is one tile product per block.  Waits on flags
// are bounded: after the limit the kernel records CF_ERR_TIMEOUT and goes
// on (results are then wrong, never hung).
#include "cf_common.cuh"
#include "cf_kernels.cuh"

namespace cf {

__device__ int g_trsv_status = 0;

// Block sizes: the FP32 solves use 128-row blocks (half the chain of
// dependent blocks of 64-row ones; their shared memory fits one CTA per SM);
// the FP64-arithmetic solves keep 64-row blocks (FP64 tiles of 128 would not
// fit).
constexpr int kSB32 = 128, kSB64 = 64;
constexpr long long kFlagSpin = 1ll << 22;

// Effective matrix M (n x n) seen by a solve:
//   0: M = L, unit lower (forward)       1: M = U, upper (backward)
//   2: M = L, lower (forward)            3: M = L^T (backward)
template <int MODE>
__device__ __forceinline__ float m_elem(const float *T, int ldt, int i, int k) {
    return (MODE == 3) ? T[(size_t)k + (size_t)i * ldt] : T[(size_t)i + (size_t)k * ldt];
}

// Inverse of each SB x SB diagonal block of M, stored block after block,
// column-major (Dinv[b*SB*SB + i + SB*j]), computed in VT (float, or double
// for the FP64-arithmetic solves with the same FP32 factor).  Dynamic shared
// memory: 2 * SB * (SB + 1) VT.
template <int SB, int MODE, typename VT>
__global__ void __launch_bounds__(256) k_diag_inverse(int n, const float *__restrict__ T, int ldt, VT *Dinv) {
    extern __shared__ __align__(16) unsigned char dsm[];
    VT (*Ms)[SB + 1] = reinterpret_cast<VT (*)[SB + 1]>(dsm);                             // Ms[i][k] = M(b0+i, b0+k)
    VT (*Xs)[SB + 1] = reinterpret_cast<VT (*)[SB + 1]>(dsm + sizeof(VT) * SB * (SB + 1));  // inverse
    constexpr int G = 256 / SB;                      // row groups of the column-parallel solve
    const int b = blockIdx.x, b0 = b * SB, nbk = min(SB, n - b0);
    const int tid = threadIdx.x;
    for (int e = tid; e < SB * SB; e += 256) {
        const int i = e % SB, k = e / SB;
        VT v = VT(0);
        if (i < nbk && k < nbk) v = (VT)m_elem<MODE>(T, ldt, b0 + i, b0 + k);
        if (i >= nbk || k >= nbk) v = (i == k) ? VT(1) : VT(0);
        if (MODE == 0 && i == k) v = VT(1);
        Ms[i][k] = v;
        Xs[i][k] = (i == k) ? VT(1) : VT(0);
    }
    __syncthreads();
    const bool lower = (MODE != 1);
    // Solve M X = I column-parallel: thread owns column j = tid % SB and rows
    // i = tid / SB + G t.
    const int j = tid % SB, i0 = tid / SB;
    for (int s = 0; s < SB; ++s) {
        const int k = lower ? s : SB - 1 - s;
        if (MODE != 0 && i0 == 0) Xs[k][j] = Xs[k][j] / Ms[k][k];
        __syncthreads();
        const VT xk = Xs[k][j];
        for (int i = i0; i < SB; i += G) {
            if ((lower && i > k) || (!lower && i < k)) Xs[i][j] = fma(-Ms[i][k], xk, Xs[i][j]);
        }
        __syncthreads();
    }
    VT *D = Dinv + (size_t)b * SB * SB;
    for (int e = tid; e < SB * SB; e += 256) D[e] = Xs[e % SB][e / SB];
}

// G_b = Dinv_b M(b, b - 1) (forward modes) or Dinv_b M(b, b + 1) (backward),
// the neighbour block of M premultiplied by the inverse of the diagonal
// block as the solve applies it (MODE 3: (L_bb^-1)^T), stored like Dinv
// (column-major SB x SB per block); blocks without a neighbour are skipped.
// Dynamic shared memory: 2 SB (SB + 1) floats.
template <int SB, int MODE>
__global__ void __launch_bounds__(256) k_neighbor_premul(int n, const float *__restrict__ T, int ldt,
                                                         const float *__restrict__ Dinv, float *Gout) {
    extern __shared__ __align__(16) float gsm[];
    float (*Dm)[SB + 1] = reinterpret_cast<float (*)[SB + 1]>(gsm);                // Dm[i][k]
    float (*Mm)[SB + 1] = reinterpret_cast<float (*)[SB + 1]>(gsm + SB * (SB + 1));  // Mm[k][j]
    const int nb = (n + SB - 1) / SB, b = blockIdx.x;
    constexpr bool fwd = (MODE == 0 || MODE == 2);
    const int nbk = fwd ? b - 1 : b + 1;
    if (nbk < 0 || nbk >= nb) return;
    const int b0 = b * SB, c0 = nbk * SB, tid = threadIdx.x;
    const float *D = Dinv + (size_t)b * SB * SB;
    for (int e = tid; e < SB * SB; e += 256) {
        const int i = e % SB, k = e / SB;
        Dm[i][k] = (MODE == 3) ? D[k + SB * i] : D[i + SB * k];
        // e as (row k, column j) of the neighbour tile
        const int kr = e % SB, j = e / SB;
        Mm[kr][j] = (b0 + kr < n && c0 + j < n) ? m_elem<MODE>(T, ldt, b0 + kr, c0 + j) : 0.f;
    }
    __syncthreads();
    // thread: column j, rows i0, i0 + 2, ...
    const int j = tid % SB, i0 = tid / SB;
    constexpr int R = SB / 2;
    float g[R];
#pragma unroll
    for (int t = 0; t < R; ++t) g[t] = 0.f;
    for (int k = 0; k < SB; ++k) {
        const float mk = Mm[k][j];
#pragma unroll
        for (int t = 0; t < R; ++t) g[t] = fmaf(Dm[i0 + 2 * t][k], mk, g[t]);
    }
    float *G = Gout + (size_t)b * SB * SB;
#pragma unroll
    for (int t = 0; t < R; ++t) G[(i0 + 2 * t) + SB * j] = g[t];
}

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(int *p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Stages the STORED SB x SB tile whose top-left element is (i0, j0) of T
// (column-major, ld ldt) into St[col * (SB + 4) + row] with 16-byte async
// copies when the whole tile is inside the matrix and aligned; element by
// element otherwise (zero outside).
template <int SB>
__device__ __forceinline__ void stage_tile(float *St, const float *T, int ldt, int n, int i0, int j0, bool fast) {
    constexpr int TLD = SB + 4;
    const int tid = threadIdx.x;
    if (fast) {
        for (int e = tid; e < SB * SB / 4; e += 256) {
            const int r4 = e % (SB / 4), c = e / (SB / 4);
            cp_async16(St + c * TLD + 4 * r4, T + (size_t)(i0 + 4 * r4) + (size_t)(j0 + c) * ldt);
        }
    } else {
        for (int e = tid; e < SB * SB; e += 256) {
            const int r = e % SB, c = e / SB;
            St[c * TLD + r] = (i0 + r < n && j0 + c < n) ? T[(size_t)(i0 + r) + (size_t)(j0 + c) * ldt] : 0.f;
        }
    }
}

// Thread layout of the blocked solves (256 threads, 8 warps).  A thread
// holds 4 rows x C right-hand sides of its block's accumulator (C = 8 where
// the block allows).  The lanes of a warp cover LR row quads and LC = NR / C
// column groups; WR warps cover the block's rows and the KS = 8 / WR warp
// groups split k of every tile product (partial sums, added through shared
// memory once per product that has to be complete).  Per k a warp issues one
// 16-byte tile load and C / 4 16-byte Y loads for 4 C FMAs: measured alone,
// a 128 x 128 x 16 product takes 1.46 us this way (4 x 8 per thread)
// against 2.59 us with 4 x 2 per thread and all 128 k in every warp.
template <int SB, int NR>
struct TrsvMap {
    static constexpr int C0 = NR < 8 ? NR : 8;
    static constexpr int LR0 = 32 / (NR / C0);
    static constexpr int LR = 4 * LR0 <= SB ? LR0 : SB / 4;   // lanes along rows (row quads)
    static constexpr int LC = 32 / LR;                         // lanes along columns
    static constexpr int C = NR / LC;                          // right-hand sides per thread
    static constexpr int RW = 4 * LR;                          // rows per warp
    static constexpr int WR = SB / RW;                         // warps over the rows
    static constexpr int KS = 8 / WR;                          // k split
    static constexpr int KW = SB / KS;                         // k per split
    static constexpr int YLD = NR + 4;                         // staged Y row: 16-byte aligned rows
    static_assert(NR == 4 || NR == 8 || NR == 16, "right-hand-side classes");
    static_assert(C == 2 || C == 4 || C == 8, "whole Y vectors per thread");
    static_assert(LR * LC == 32 && WR >= 1 && WR * RW == SB && KS * WR == 8, "thread layout");
    static_assert(KW % 4 == 0, "k per split: whole vectors");
    // the k parts' partial sums [KS][NR][SB] fit the tile buffer that is free
    // at the end of a block (else they get their own region)
    static constexpr bool RED_IN_TILE = (size_t)KS * NR * SB * 8 <= (size_t)SB * (SB + 4) * 4;
};

template <int SB, typename VT, int NR>
__host__ __device__ constexpr size_t trsv_smem_bytes() {
    using M = TrsvMap<SB, NR>;
    return sizeof(float) * 2 * (size_t)SB * (SB + 4) +                 // two tile buffers
           sizeof(VT) * ((size_t)SB * (SB + 4) +                       // inverse of the diagonal block
                         (size_t)SB * M::YLD +                         // staged Y
                         (M::RED_IN_TILE ? 0 : (size_t)M::KS * SB * NR));   // partial sums of the k split
}

// Four consecutive 16-byte-aligned shared-memory values as VT.
template <typename VT>
__device__ __forceinline__ void load4(VT (&m)[4], const float *p) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    m[0] = (VT)v.x; m[1] = (VT)v.y; m[2] = (VT)v.z; m[3] = (VT)v.w;
}
__device__ __forceinline__ void load4(double (&m)[4], const double *p) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    m[0] = a.x; m[1] = a.y; m[2] = b.x; m[3] = b.y;
}
__device__ __forceinline__ void load4(float (&m)[4], const float *p) {
    const float4 v = *reinterpret_cast<const float4 *>(p);
    m[0] = v.x; m[1] = v.y; m[2] = v.z; m[3] = v.w;
}
__device__ __forceinline__ void load2(float (&y)[2], const float *p) {
    const float2 v = *reinterpret_cast<const float2 *>(p);
    y[0] = v.x; y[1] = v.y;
}
__device__ __forceinline__ void load2(double (&y)[2], const double *p) {
    const double2 v = *reinterpret_cast<const double2 *>(p);
    y[0] = v.x; y[1] = v.y;
}

// Row r (0..3) of a thread: rb + r (consecutive; column-major tiles are
// read as one vector per k), or rb + LR r (strided: the transposed solve,
// whose row-major tiles are read as one vector per four k, so that the
// lanes of a warp read consecutive rows without bank conflicts), where rb
// is the thread's base row.
template <bool STRIDED, int LR>
__device__ __forceinline__ int trow(int rbase, int r) { return STRIDED ? rbase + LR * r : rbase + r; }

// acc[r][t] += sign * sum_{k0 <= kk < k1} Mt(row(r), kk) * Ys[kk * YLD + c + t]
// for one staged tile, t < C; Mt(i, kk) = Tt[kk * LD + i] (COLMAJ) or
// Tt[i * LD + kk].  The C Y values of a k are C / 2 or C / 4 vectors.
template <typename VT, int C>
__device__ __forceinline__ void loady(VT (&y)[C], const VT *p) {
    if constexpr (C == 2) {
        load2(y, p);
    } else {
#pragma unroll
        for (int q = 0; q < C; q += 4) {
            VT v[4];
            load4(v, p + q);
            y[q] = v[0]; y[q + 1] = v[1]; y[q + 2] = v[2]; y[q + 3] = v[3];
        }
    }
}

template <int LR, int C, bool COLMAJ, bool STRIDED, typename MT, typename VT>
__device__ __forceinline__ void tile_mac(VT (&acc)[4][C], const MT *Tt, int LD, const VT *Ys, int YLD, int rbase,
                                         int c, int k0, int k1, VT sign) {
    if (COLMAJ) {
#pragma unroll 4
        for (int kk = k0; kk < k1; ++kk) {
            VT m[4];
            if (!STRIDED) {
                load4(m, Tt + kk * LD + rbase);
            } else {
#pragma unroll
                for (int r = 0; r < 4; ++r) m[r] = (VT)Tt[kk * LD + trow<true, LR>(rbase, r)];
            }
            VT y[C];
            loady<VT, C>(y, Ys + kk * YLD + c);
#pragma unroll
            for (int t = 0; t < C; ++t)
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[r][t] = fma(sign * m[r], y[t], acc[r][t]);
        }
    } else {
#pragma unroll 1
        for (int k4 = k0; k4 < k1; k4 += 4) {
            VT m[4][4];
#pragma unroll
            for (int r = 0; r < 4; ++r) load4(m[r], Tt + trow<STRIDED, LR>(rbase, r) * LD + k4);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                VT y[C];
                loady<VT, C>(y, Ys + (k4 + u) * YLD + c);
#pragma unroll
                for (int t = 0; t < C; ++t)
#pragma unroll
                    for (int r = 0; r < 4; ++r) acc[r][t] = fma(sign * m[r][u], y[t], acc[r][t]);
            }
        }
    }
}

// Stages the tile of one step of block r0 / SB: the stored tile of M's block
// (r0, column block of the step), or G_b for the last step when pre.
template <int SB, int MODE>
__device__ __forceinline__ void trsv_stage_step(float *dst, int step, int s, bool pre, const float *Gb,
                                                const float *T, int ldt, int n, int nb, int r0, bool aligned) {
    constexpr bool fwd = (MODE == 0 || MODE == 2);
    if (pre && step == s - 1) {
        stage_tile<SB>(dst, Gb, SB, SB, 0, 0, (((uintptr_t)Gb) & 15) == 0);
        return;
    }
    const int cb = fwd ? step : nb - 1 - step;
    const int ti = (MODE == 3) ? cb * SB : r0, tj = (MODE == 3) ? r0 : cb * SB;
    stage_tile<SB>(dst, T, ldt, n, ti, tj, aligned && ti + SB <= n && tj + SB <= n);
}
// Block solve of one ticket.  VT: arithmetic and right-hand-side type
// (float, or double for FP64 solves with the FP32 factor); the factor tiles
// stay FP32 in shared memory.
//
// Per step (one finished block's tile): the tile of the next step is
// prefetched with cp.async; the flags of later blocks are polled a warp at
// a time (up to 64 per poll), so for blocks that finished long ago neither
// the flag nor the data costs a dependent round trip: the Y block of the
// next step is loaded into registers while this step's tile product runs.
// Only the first unfinished block is waited for (bounded).  The k parts'
// partial sums meet in shared memory once per block before the diagonal
// inverse is applied (and once more for its product).
template <int SB, int MODE, int NR, typename VT>
__global__ void __launch_bounds__(256, 1)        // one CTA per SM (shared memory)
k_trsv_blocked(int n, int nrhs, const float *__restrict__ T, int ldt, const VT *__restrict__ Dinv,
               const float *__restrict__ Gn, VT *X, int ldx, int *flags, int *ticket, long long spin_limit) {
    using Map = TrsvMap<SB, NR>;
    constexpr int TLD = SB + 4;
    constexpr int LR = Map::LR, C = Map::C, RW = Map::RW, WR = Map::WR, KS = Map::KS, KW = Map::KW;
    constexpr int YLD = Map::YLD;
    constexpr int YPT = SB * NR / 256;             // Y values per thread of one block
    static_assert(SB * NR % 256 == 0, "Y block: whole values per thread");
    constexpr bool STR = (MODE == 3);              // strided rows (see trow)
    extern __shared__ __align__(16) float sm[];
    float *St0 = sm;                               // two tile buffers
    float *St1 = sm + SB * TLD;
    VT *Ds = reinterpret_cast<VT *>(sm + 2 * SB * TLD);     // inverse of the diagonal block
    VT *Ys = Ds + SB * TLD;                                 // [SB][YLD]
    VT *RedOwn = Ys + SB * YLD;                             // [KS][NR][SB] unless in a free tile buffer
    __shared__ int s_ticket, s_upto;
    constexpr bool fwd = (MODE == 0 || MODE == 2);
    const int nb = (n + SB - 1) / SB;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) s_ticket = atomicAdd(ticket, 1);
    __syncthreads();
    const int s = s_ticket;
    if (s >= nb) return;
    const int b = fwd ? s : nb - 1 - s;
    const int r0 = b * SB, rb = min(SB, n - r0);
    const int wr = warp % WR, kp = warp / WR;      // row warp, k part
    const int lr = lane % LR, lc = lane / LR;
    const int rbase = wr * RW + (STR ? lr : 4 * lr);
    const int c = C * lc;                          // first of the thread's right-hand sides
    const int k0 = kp * KW, k1 = k0 + KW;
    const bool aligned = ((ldt & 3) == 0) && ((((uintptr_t)T) & 15) == 0);
    // the diagonal block's inverse does not depend on anyone: fetch it now
    // (Ds[kk * TLD + ii] = (Dinv_b)(ii, kk); MODE 3 uses (L_bb^{-1})^T)
    {
        const VT *D = Dinv + (size_t)b * SB * SB;
        for (int e = tid; e < SB * SB; e += 256) {
            const int ii = e % SB, kk = e / SB;
            Ds[kk * TLD + ii] = (MODE == 3) ? D[kk + SB * ii] : D[ii + SB * kk];
        }
    }
    // the right-hand side lives in the k-part-0 threads; the others sum from 0
    VT acc[4][C];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int t = 0; t < C; ++t) {
            const int i = trow<STR, LR>(rbase, r);
            acc[r][t] = (kp == 0 && i < rb && c + t < nrhs) ? X[(size_t)(r0 + i) + (size_t)(c + t) * ldx] : VT(0);
        }
    // With Gn (the neighbour block's tile premultiplied by this block's
    // diagonal inverse, G_b = Dinv_b M(b, b -+ 1)), the last step, which waits
    // for the neighbour, is one tile product: y = Dinv_b acc - G_b x_nb, with
    // Dinv_b acc formed before the wait.
    const bool pre = (Gn != nullptr) && s > 0;
    const float *Gb = pre ? Gn + (size_t)b * SB * SB : nullptr;
    if (s > 0) {
        trsv_stage_step<SB, MODE>(St0, 0, s, pre, Gb, T, ldt, n, nb, r0, aligned);
        cp_async_commit();
    }
    // Partial sums of the k parts: Red[kp][col][row] in the tile buffer that
    // is free when they meet (the other one holds the last step's tile, or
    // nothing), else in their own region.
    auto red_at = [&](int last_buf) -> VT * {
        if constexpr (Map::RED_IN_TILE) return reinterpret_cast<VT *>(last_buf ? St0 : St1);
        else return RedOwn;
    };
    auto put_partial = [&](VT *Red, const VT (&v)[4][C]) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int t = 0; t < C; ++t) Red[((size_t)kp * NR + c + t) * SB + trow<STR, LR>(rbase, r)] = v[r][t];
    };
    // element e = tid + 256 j of the block (row e % SB, column e / SB): the
    // sum of the KS partial sums, in k-part order
    auto sum_partial = [&](const VT *Red, int e) -> VT {
        VT v = Red[e];
#pragma unroll
        for (int q = 1; q < KS; ++q) v += Red[(size_t)q * NR * SB + e];
        return v;
    };
    // Y block of a step: value e = tid + 256 j is (row e % SB, column e / SB)
    auto load_y = [&](VT (&v)[YPT], int step) {
        const int cb = fwd ? step : nb - 1 - step;
        const int c0 = cb * SB, cbk = min(SB, n - c0);
#pragma unroll
        for (int j = 0; j < YPT; ++j) {
            const int e = tid + 256 * j, kk = e % SB, cc = e / SB;
            v[j] = (kk < cbk && cc < nrhs) ? __ldcg(X + (size_t)(c0 + kk) + (size_t)cc * ldx) : VT(0);
        }
    };
    auto store_y = [&](const VT (&v)[YPT]) {
#pragma unroll
        for (int j = 0; j < YPT; ++j) {
            const int e = tid + 256 * j;
            Ys[(e % SB) * YLD + e / SB] = v[j];
        }
    };
    // Warp 0: waits (bounded) for the flag of step `from`, then extends the
    // run of finished steps as far as the next unset flag (at most 64
    // more); s_upto = the first step past the run.  The flags are read with
    // acquire semantics (GPU scope): with the barrier that follows, every
    // later read of those blocks' solutions by any thread of the CTA sees
    // them (the producer publishes with a release store).
    auto poll = [&](int from) {
        if (warp == 0) {
            if (lane == 0) {
                const int *f = flags + (fwd ? from : nb - 1 - from);
                long long it = 0;
                while (ld_acquire_gpu(f) == 0 && it < spin_limit) {
                    ++it;
                    if (it > 64) __nanosleep(20);
                }
                if (it >= spin_limit) atomicExch(&g_trsv_status, CF_ERR_TIMEOUT);
            }
            __syncwarp();
            int u = from + 1;
#pragma unroll 1
            for (int chunk = 0; chunk < 2 && u < s; ++chunk) {
                const int idx = u + lane;
                const int fl = (idx < s) ? ld_acquire_gpu(flags + (fwd ? idx : nb - 1 - idx)) : 1;
                const unsigned unset = ~__ballot_sync(0xffffffffu, fl != 0);
                if (unset == 0u) {
                    u = min(s, u + 32);
                } else {
                    u = min(s, u + __ffs(unset) - 1);
                    break;
                }
            }
            if (lane == 0) s_upto = u;
        }
    };
    int upto = 0;                                  // steps [0, upto) are known finished
    bool have = false;                             // this step's Y block is in yv
    VT yv[YPT];
    for (int step = 0; step < s; ++step) {
        float *St = (step & 1) ? St1 : St0;
        if (step + 1 < s)                          // prefetch the next tile
            trsv_stage_step<SB, MODE>((step & 1) ? St0 : St1, step + 1, s, pre, Gb, T, ldt, n, nb, r0, aligned);
        cp_async_commit();
        const bool last = (step == s - 1);
        if (last && pre) {
            // acc <- Dinv_b acc before the neighbour's wait: the partial sums
            // meet in Ys, then every k part takes its share of the product
            VT *Red = red_at(step & 1);
            put_partial(Red, acc);
            __syncthreads();
#pragma unroll
            for (int j = 0; j < YPT; ++j) {
                const int e = tid + 256 * j;
                Ys[(e % SB) * YLD + e / SB] = sum_partial(Red, e);
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int t = 0; t < C; ++t) acc[r][t] = VT(0);
            tile_mac<LR, C, true, STR>(acc, Ds, TLD, Ys, YLD, rbase, c, k0, k1, VT(1));
            __syncthreads();
        }
        // this step's Y block
        if (have) {
            store_y(yv);
        } else {
            if (step >= upto) poll(step);
            __syncthreads();
            upto = s_upto;
            VT v[YPT];
            load_y(v, step);
            store_y(v);
        }
        // the next step's Y block into registers while this step computes
        have = (step + 1 < upto);
        if (have) load_y(yv, step + 1);
        cp_async_wait<1>();                        // this step's tile has landed
        __syncthreads();
        // M(i, kk) = St[kk * TLD + i], or St[i * TLD + kk] for MODE 3; G_b
        // is staged column-major in every mode
        if (last && pre) tile_mac<LR, C, true, STR>(acc, St, TLD, Ys, YLD, rbase, c, k0, k1, VT(-1));
        else tile_mac<LR, C, MODE != 3, STR>(acc, St, TLD, Ys, YLD, rbase, c, k0, k1, VT(-1));
        __syncthreads();
    }
    cp_async_wait<0>();
    VT *Red = red_at(s > 0 ? ((s - 1) & 1) : 1);
    if (!pre) {
        // y_b = Dinv_b acc: the partial sums meet in Ys, then the k parts
        // share the product
        put_partial(Red, acc);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < YPT; ++j) {
            const int e = tid + 256 * j;
            Ys[(e % SB) * YLD + e / SB] = sum_partial(Red, e);
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int t = 0; t < C; ++t) acc[r][t] = VT(0);
        tile_mac<LR, C, true, STR>(acc, Ds, TLD, Ys, YLD, rbase, c, k0, k1, VT(1));
        __syncthreads();
    }
    // y_b: the sum of the k parts, stored by all threads (coalesced)
    put_partial(Red, acc);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < YPT; ++j) {
        const int e = tid + 256 * j, i = e % SB, cc = e / SB;
        const VT v = sum_partial(Red, e);
        if (i < rb && cc < nrhs) X[(size_t)(r0 + i) + (size_t)cc * ldx] = v;
    }
    // publish: the barrier orders every thread's stores of the block before
    // thread 0's release store of the flag (release is cumulative)
    __syncthreads();
    if (tid == 0) st_release_gpu(flags + b, 1);
}

// Flags for the smaller block size (the larger needs fewer).
size_t trsv_ws_bytes(int n) {
    const int nb = (n + kSB64 - 1) / kSB64;
    return sizeof(int) * (size_t)(nb + 1);
}

// Elements of the FP32 (128-row blocks) and FP64 (64-row blocks) inverse sets.
size_t diag_inverse_floats(int n) {
    const int nb = (n + kSB32 - 1) / kSB32;
    return (size_t)nb * kSB32 * kSB32;
}
size_t diag_inverse64_elems(int n) {
    const int nb = (n + kSB64 - 1) / kSB64;
    return (size_t)nb * kSB64 * kSB64;
}

template <int SB, int MODE, typename VT>
static int launch_diag_inverse_m(int n, const float *T, int ldt, VT *Dinv, cudaStream_t st) {
    const int nb = (n + SB - 1) / SB;
    const size_t smem = 2 * sizeof(VT) * SB * (SB + 1);
    CF_CUDA_TRY(cudaFuncSetAttribute(k_diag_inverse<SB, MODE, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    k_diag_inverse<SB, MODE, VT><<<nb, 256, smem, st>>>(n, T, ldt, Dinv);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

// mode: 0 unit lower, 1 upper, 2 lower, 3 lower transposed (see m_elem).
template <int SB, typename VT>
static int launch_diag_inverse_t(int mode, int n, const float *T, int ldt, VT *Dinv, cudaStream_t st) {
    if (n <= 0) return CF_OK;
    switch (mode) {
        case 0: return launch_diag_inverse_m<SB, 0, VT>(n, T, ldt, Dinv, st);
        case 1: return launch_diag_inverse_m<SB, 1, VT>(n, T, ldt, Dinv, st);
        case 2: return launch_diag_inverse_m<SB, 2, VT>(n, T, ldt, Dinv, st);
        default: return CF_ERR_UNSUPPORTED;
    }
}

int launch_diag_inverse(int mode, int n, const float *T, int ldt, float *Dinv, cudaStream_t st) {
    return launch_diag_inverse_t<kSB32, float>(mode, n, T, ldt, Dinv, st);
}
int launch_diag_inverse64(int mode, int n, const float *T, int ldt, double *Dinv, cudaStream_t st) {
    return launch_diag_inverse_t<kSB64, double>(mode, n, T, ldt, Dinv, st);
}

template <int SB, int MODE, int NR, typename VT>
static int launch_trsv_nr(int n, int nrhs, const float *T, int ldt, const VT *Dinv, const float *Gn, VT *X, int ldx,
                          int *flags, int *ticket, long long spin, cudaStream_t st) {
    const int nb = (n + SB - 1) / SB;
    const size_t smem = trsv_smem_bytes<SB, VT, NR>();
    CF_CUDA_TRY(cudaFuncSetAttribute(k_trsv_blocked<SB, MODE, NR, VT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    k_trsv_blocked<SB, MODE, NR, VT><<<nb, 256, smem, st>>>(n, nrhs, T, ldt, Dinv, Gn, X, ldx, flags, ticket, spin);
    CF_LAUNCH_CHECK();
    return CF_OK;
}

// withhold: the first ticket is taken before the launch (failure-detection
// test: the first block is never solved and every wait for it runs out).
template <int SB, int MODE, typename VT>
static int launch_trsv_mode(int n, int nrhs, const float *T, int ldt, const VT *Dinv, const float *Gn, VT *X, int ldx,
                            int *sync_ws, bool withhold, long long spin, cudaStream_t st) {
    const int nb = (n + SB - 1) / SB;
    CF_CUDA_TRY(cudaMemsetAsync(sync_ws, 0, sizeof(int) * (size_t)(nb + 1), st));
    int *flags = sync_ws, *ticket = sync_ws + nb;
    if (withhold) CF_CUDA_TRY(cudaMemsetAsync(ticket, 1, 1, st));     // ticket = 1 (little-endian low byte)
    if (nrhs <= 4) return launch_trsv_nr<SB, MODE, 4, VT>(n, nrhs, T, ldt, Dinv, Gn, X, ldx, flags, ticket, spin, st);
    if (nrhs <= 8) return launch_trsv_nr<SB, MODE, 8, VT>(n, nrhs, T, ldt, Dinv, Gn, X, ldx, flags, ticket, spin, st);
    return launch_trsv_nr<SB, MODE, 16, VT>(n, nrhs, T, ldt, Dinv, Gn, X, ldx, flags, ticket, spin, st);
}

template <int SB, typename VT>
static int launch_trsv_t(int mode, int n, int nrhs, const float *T, int ldt, const VT *Dinv, const float *Gn, VT *X,
                         int ldx, int *sync_ws, cudaStream_t st, bool withhold = false,
                         long long spin = kFlagSpin) {
    if (n <= 0 || nrhs <= 0) return CF_OK;
    if (nrhs > 16) return CF_ERR_UNSUPPORTED;
    switch (mode) {
        case 0: return launch_trsv_mode<SB, 0, VT>(n, nrhs, T, ldt, Dinv, Gn, X, ldx, sync_ws, withhold, spin, st);
        case 1: return launch_trsv_mode<SB, 1, VT>(n, nrhs, T, ldt, Dinv, Gn, X, ldx, sync_ws, withhold, spin, st);
        case 2: return launch_trsv_mode<SB, 2, VT>(n, nrhs, T, ldt, Dinv, Gn, X, ldx, sync_ws, withhold, spin, st);
        case 3: return launch_trsv_mode<SB, 3, VT>(n, nrhs, T, ldt, Dinv, Gn, X, ldx, sync_ws, withhold, spin, st);
        default: return CF_ERR_UNSUPPORTED;
    }
}

// X <- M^{-1} X for nrhs <= 16 columns; sync_ws holds trsv_ws_bytes(n).
// Gn (may be null): the premultiplied neighbour tiles of launch_neighbor_premul
// for the same mode and Dinv.
int launch_trsv_f32(int mode, int n, int nrhs, const float *T, int ldt, const float *Dinv, const float *Gn, float *X,
                    int ldx, int *sync_ws, cudaStream_t st) {
    return launch_trsv_t<kSB32, float>(mode, n, nrhs, T, ldt, Dinv, Gn, X, ldx, sync_ws, st);
}
// The same with FP64 right-hand sides and arithmetic (FP64 Dinv from
// launch_diag_inverse64); the FP32 factor is read as stored.
int launch_trsv_f64x(int mode, int n, int nrhs, const float *T, int ldt, const double *Dinv, double *X, int ldx,
                     int *sync_ws, cudaStream_t st) {
    return launch_trsv_t<kSB64, double>(mode, n, nrhs, T, ldt, Dinv, nullptr, X, ldx, sync_ws, st);
}

// G_b for every block of an FP32 solve (k_neighbor_premul); Gout holds
// diag_inverse_floats(n) floats.
int launch_neighbor_premul(int mode, int n, const float *T, int ldt, const float *Dinv, float *Gout,
                           cudaStream_t st) {
    if (n <= 0) return CF_OK;
    constexpr int SB = kSB32;
    const int nb = (n + SB - 1) / SB;
    const size_t smem = sizeof(float) * 2 * SB * (SB + 1);
#define CF_PREMUL(M)                                                                                            \
    case M:                                                                                                     \
        CF_CUDA_TRY(cudaFuncSetAttribute(k_neighbor_premul<SB, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)smem));                                                           \
        k_neighbor_premul<SB, M><<<nb, 256, smem, st>>>(n, T, ldt, Dinv, Gout);                                \
        break;
    switch (mode) {
        CF_PREMUL(0)
        CF_PREMUL(1)
        CF_PREMUL(2)
        CF_PREMUL(3)
        default: return CF_ERR_UNSUPPORTED;
    }
#undef CF_PREMUL
    CF_LAUNCH_CHECK();
    return CF_OK;
}

// The C-ABI solve and its failure-detection variant: Dinv in work, then the
// blocked solve (no premultiplied neighbour tiles).
static size_t trsv_api_ws(int n) {
    Carver cv(nullptr);
    cv.take<float>(diag_inverse_floats(n > 0 ? n : 1));
    cv.take<int>(trsv_ws_bytes(n > 0 ? n : 1) / sizeof(int) + 1);
    return cv.size();
}

static int trsv_api(int mode, int n, int nrhs, const float *T, int ldt, float *X, int ldx, bool withhold,
                    long long spin, void *work, size_t lwork, cudaStream_t st) {
    if (mode < 0 || mode > 3) return -1;
    if (n < 0) return -2;
    if (nrhs < 0 || nrhs > 16) return -3;
    if (n > 0 && T == nullptr) return -4;
    if (ldt < (n > 1 ? n : 1)) return -5;
    if (n > 0 && nrhs > 0 && X == nullptr) return -6;
    if (ldx < (n > 1 ? n : 1)) return -7;
    if (n == 0 || nrhs == 0) return CF_OK;
    if (work == nullptr || lwork < trsv_api_ws(n)) return CF_ERR_WORKSPACE;
    Carver cv(work);
    float *Dinv = cv.take<float>(diag_inverse_floats(n));
    int *sync = cv.take<int>(trsv_ws_bytes(n) / sizeof(int) + 1);
    // mode 3 (L^T) reads the inverses of L's diagonal blocks transposed
    int rc = launch_diag_inverse(mode == 3 ? 2 : mode, n, T, ldt, Dinv, st);
    if (rc != CF_OK) return rc;
    return launch_trsv_t<kSB32, float>(mode, n, nrhs, T, ldt, Dinv, nullptr, X, ldx, sync, st, withhold, spin);
}

int trsv_take_status(cudaStream_t st, int *status) {
    int h = 0;
    CF_CUDA_TRY(cudaMemcpyFromSymbolAsync(&h, g_trsv_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    CF_CUDA_TRY(cudaStreamSynchronize(st));
    if (h != 0) {
        const int zero = 0;
        CF_CUDA_TRY(cudaMemcpyToSymbolAsync(g_trsv_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
    }
    *status = h;
    return CF_OK;
}

}  // namespace cf

extern "C" size_t cf_trsv_f32_workspace_size(int n) { return cf::trsv_api_ws(n); }

extern "C" int cf_trsv_f32(int mode, int n, int nrhs, const float *T, int ldt, float *X, int ldx, void *work,
                           size_t lwork, cudaStream_t stream) {
    return cf::trsv_api(mode, n, nrhs, T, ldt, X, ldx, false, cf::kFlagSpin, work, lwork, stream);
}

extern "C" int cf_trsv_f32_withheld(int mode, int n, int nrhs, const float *T, int ldt, float *X, int ldx,
                                    long long spin_limit, void *work, size_t lwork, cudaStream_t stream) {
    if (spin_limit < 0) return -8;
    return cf::trsv_api(mode, n, nrhs, T, ldt, X, ldx, true, spin_limit > 0 ? spin_limit : cf::kFlagSpin, work,
                        lwork, stream);
}

