// cf_tc.cuh -- tensor-core Schur update (cf_tc.cu).
#pragma once

#include "cf_common.cuh"

namespace cf {

// C[m x n] -= A[m x k] * B[n x k]^T; A, B K-major BF16 (bf16) or FP16, C FP32
// column-major.  lower: only i >= j.  max_ctas > 0 caps the persistent grid.
int launch_schur_tc(int m, int n, int k, const void *A, int lda_k, const void *B, int ldb_k, float *C, int ldc,
                    bool bf16, bool lower, cudaStream_t st, int max_ctas);

// Synchronises st, returns (and clears) the device status word of the
// tensor-core kernels: 0 or CF_ERR_TIMEOUT.
int tc_take_status(cudaStream_t st, int *status);

}  // namespace cf
