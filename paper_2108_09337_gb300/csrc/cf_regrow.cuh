// cf_regrow.cuh -- register-row elimination shared by the FP32 panel kernels.
//
// A thread holds one row (or column) of a tile of width <= 128 in a register
// array a[128], indexed RELATIVE to the start j0 of the current block of 8
// columns: a[t] is column j0 + t.  Inside a block the eight columns are
// unrolled, so every index is a compile-time constant; after the block the
// row shifts left by 8 (120 register moves per 8 columns instead of 127 per
// column).  Pivot rows / columns are read from shared memory at their
// absolute column positions, 32-byte aligned because j0 is a multiple of 8.
#pragma once

#include "cf_common.cuh"

namespace cf {

constexpr int kBlk = 8;

// a[t] -= l * p[t] for U < t < 128 (U compile-time), p4 = &p[j0] as float4;
// 32-column chunks at or beyond the live width `lim` (relative) are skipped.
template <int U>
__device__ __forceinline__ void rank1_from(float (&a)[kMaxV], float l, const float4 *p4, int lim) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if ((c + 1) * 32 - 1 > U) {
            if (c * 32 < lim) {
#pragma unroll
                for (int q = c * 8; q < c * 8 + 8; ++q) {
                    if (4 * q + 3 > U) {
                        const float4 p = p4[q];
                        if (4 * q + 0 > U) a[4 * q + 0] = fmaf(-l, p.x, a[4 * q + 0]);
                        if (4 * q + 1 > U) a[4 * q + 1] = fmaf(-l, p.y, a[4 * q + 1]);
                        if (4 * q + 2 > U) a[4 * q + 2] = fmaf(-l, p.z, a[4 * q + 2]);
                        a[4 * q + 3] = fmaf(-l, p.w, a[4 * q + 3]);
                    }
                }
            }
        }
    }
}

__device__ __forceinline__ void shift_block(float (&a)[kMaxV]) {
#pragma unroll
    for (int t = kBlk; t < kMaxV; ++t) a[t - kBlk] = a[t];
}

// Stores a[0..127] as 32 float4 (dst 16-byte aligned).
__device__ __forceinline__ void store_row4(float4 *dst, const float (&a)[kMaxV]) {
#pragma unroll
    for (int q = 0; q < kMaxV / 4; ++q) dst[q] = make_float4(a[4 * q], a[4 * q + 1], a[4 * q + 2], a[4 * q + 3]);
}

// Runs body.template operator()<U>(j) for U = 0..7, j = j0 + U < n, over
// blocks j0 = 0, 8, ..., shifting `a` by 8 after each block.
template <typename Body>
__device__ __forceinline__ void for_blocks(float (&a)[kMaxV], int n, Body &body) {
    for (int j0 = 0; j0 < n; j0 += kBlk) {
        body.template step<0>(j0);
        if (j0 + 1 < n) body.template step<1>(j0);
        if (j0 + 2 < n) body.template step<2>(j0);
        if (j0 + 3 < n) body.template step<3>(j0);
        if (j0 + 4 < n) body.template step<4>(j0);
        if (j0 + 5 < n) body.template step<5>(j0);
        if (j0 + 6 < n) body.template step<6>(j0);
        if (j0 + 7 < n) body.template step<7>(j0);
        shift_block(a);
    }
}

}  // namespace cf

// ---------------------------------------------------------------------------
// Pair form: the row as float2 a[64] (a[p] = columns j0 + 2p, j0 + 2p + 1),
// updated with packed FP32 FMAs (__ffma2_rn, sm_100 and later: two
// correctly rounded fmaf per instruction).  Elements at or left of the
// current column are dead once its multiplier is taken, so a pair holding
// the current column and the next one is updated whole.
// ---------------------------------------------------------------------------
namespace cf {

constexpr int kPairs = kMaxV / 2;

template <int U>
__device__ __forceinline__ float pair_elem(const float2 (&a)[kPairs]) {
    return (U & 1) ? a[U >> 1].y : a[U >> 1].x;
}

// a[t] -= l * p[t] for U < t < 128 (pair granularity), p4 = &p[j0] as float4;
// 32-column chunks at or beyond the live width `lim` (relative) are skipped.
template <int U>
__device__ __forceinline__ void rank1_pairs(float2 (&a)[kPairs], float l, const float4 *p4, int lim) {
    const float2 nl = make_float2(-l, -l);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if ((c + 1) * 32 - 1 > U) {
            if (c * 32 < lim) {
#pragma unroll
                for (int q = c * 8; q < c * 8 + 8; ++q) {
                    if (4 * q + 3 > U) {
                        const float4 p = p4[q];
                        if (4 * q + 1 > U) a[2 * q] = __ffma2_rn(nl, make_float2(p.x, p.y), a[2 * q]);
                        a[2 * q + 1] = __ffma2_rn(nl, make_float2(p.z, p.w), a[2 * q + 1]);
                    }
                }
            }
        }
    }
}

// Shift left by one block of 8 columns; chunks beyond the live width `lim`
// (relative to the new block start) hold nothing live and are left alone.
__device__ __forceinline__ void shift_pairs(float2 (&a)[kPairs], int lim) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if (c * 32 < lim) {
#pragma unroll
            for (int p = c * 16; p < c * 16 + 16; ++p)
                if (p + kBlk / 2 < kPairs) a[p] = a[p + kBlk / 2];
        }
    }
}

// Stores float4 q with 4q + 3 >= U (the element U on) inside the 32-column
// chunks below `lim`.
template <int U>
__device__ __forceinline__ void store_live_pairs(float4 *dst, const float2 (&a)[kPairs], int lim) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        if ((c + 1) * 32 - 1 >= U && c * 32 < lim) {
#pragma unroll
            for (int q = c * 8; q < c * 8 + 8; ++q)
                if (4 * q + 3 >= U) dst[q] = make_float4(a[2 * q].x, a[2 * q].y, a[2 * q + 1].x, a[2 * q + 1].y);
        }
    }
}

// Runs body.template step<U>(j0) for U = 0..7, j0 + U < n, over blocks
// j0 = 0, 8, ..., shifting the pair row after each block.
template <typename Body>
__device__ __forceinline__ void for_blocks_pairs(float2 (&a)[kPairs], int n, int w, Body &body) {
    for (int j0 = 0; j0 < n; j0 += kBlk) {
        body.template step<0>(j0);
        if (j0 + 1 < n) body.template step<1>(j0);
        if (j0 + 2 < n) body.template step<2>(j0);
        if (j0 + 3 < n) body.template step<3>(j0);
        if (j0 + 4 < n) body.template step<4>(j0);
        if (j0 + 5 < n) body.template step<5>(j0);
        if (j0 + 6 < n) body.template step<6>(j0);
        if (j0 + 7 < n) body.template step<7>(j0);
        shift_pairs(a, w - j0 - kBlk);
    }
}

}  // namespace cf
