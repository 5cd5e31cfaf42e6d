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
