// cf_tc.cuh -- tensor-core Schur update (cf_tc.cu).
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include "cf_common.cuh"

namespace cf {

// cuTensorMapEncodeTiled, looked up once through the runtime (no -lcuda):
// get_encoder() returns CF_OK once g_encode is set.
extern PFN_cuTensorMapEncodeTiled_v12000 g_encode;
int get_encoder();

// C[m x n] -= A[m x k] * B[n x k]^T; A, B K-major BF16 (bf16) or FP16, C FP32
// column-major.  lower: only i >= j.  max_ctas > 0 caps the persistent grid.
int launch_schur_tc(int m, int n, int k, const void *A, int lda_k, const void *B, int ldb_k, float *C, int ldc,
                    bool bf16, bool lower, cudaStream_t st, int max_ctas);
// Split-K form (the paper's split of the reduction dimension, Sec. 7.1-7.2,
// for outputs with too few tiles to fill the SMs): ksplit K ranges run as
// separate work units that write their FP32 partials to P
// (schur_tc_splitk_bytes), then C -= sum of the partials in range order
// (deterministic).  ksplit <= 1 or P null: the plain update.
int launch_schur_tc_splitk(int m, int n, int k, const void *A, int lda_k, const void *B, int ldb_k, float *C, int ldc,
                           bool bf16, bool lower, int ksplit, float *P, cudaStream_t st, int max_ctas);
// The number of K ranges the mixed solvers use for an update (1: none).
int schur_tc_splitk(int m, int n, int k, bool lower);
size_t schur_tc_splitk_bytes(int m, int n, int ksplit);

// Synchronises st, returns (and clears) the device status word of the
// BF16/FP16 tensor-core kernel: 0 or CF_ERR_TIMEOUT (fp8_take_status: the
// same for the FP8 kernel).
int tc_take_status(cudaStream_t st, int *status);

// FP8 e4m3 operands with per-128 x 128-tile FP32 scales (cf_fp8.cu):
//   C[m x n] -= sum_kb sA[i / 128, kb] sB[j / 128, kb] (qA qB^T)_kb
// qA (m x k) and qB (n x k) K-major bytes, row pitch ldqa / ldqb bytes
// (multiples of 16), k a multiple of 128; sA[rb * ldsa + kb] is the scale of
// rows rb*128.. and K-block kb.  lower: only i >= j.
int launch_schur_fp8(int m, int n, int k, const void *qA, int ldqa, const float *sA, int ldsa, const void *qB,
                     int ldqb, const float *sB, int ldsb, float *C, int ldc, bool lower, cudaStream_t st);
// q (rows x kpad bytes, pitch ldq) and scales (ceil(rows/128) x kpad/128,
// pitch lds) from the FP32 column-major rows x k block src (ld lds_src):
// per 128 x 128 tile, scale = amax / 448 (1 if the tile is zero) and
// q = e4m3(x / scale) saturated to +-448; zeros for k <= kk < kpad.
int launch_quant_e4m3(int rows, int k, int kpad, const float *src, int lds_src, void *q, int ldq, float *scales,
                      int lds, cudaStream_t st);
int fp8_take_status(cudaStream_t st, int *status);

}  // namespace cf
