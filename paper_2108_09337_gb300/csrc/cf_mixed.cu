// cf_mixed.cu -- mixed-precision refined solves (placeholder until the
// tensor-core update lands).
#include "cf_common.cuh"
#include "cf_kernels.cuh"

extern "C" size_t cf_gesv_mixed_workspace_size(int, int, cf_prec, const cf_options *) { return 0; }
extern "C" int cf_gesv_mixed(int, int, const double *, int, const double *, int, double *, int, cf_prec, int *,
                             cf_refine_stats *, void *, size_t, const cf_options *, cudaStream_t) {
    return CF_ERR_UNSUPPORTED;
}
extern "C" size_t cf_posv_mixed_workspace_size(int, int, cf_prec, const cf_options *) { return 0; }
extern "C" int cf_posv_mixed(int, int, const double *, int, const double *, int, double *, int, cf_prec, int *,
                             cf_refine_stats *, void *, size_t, const cf_options *, cudaStream_t) {
    return CF_ERR_UNSUPPORTED;
}
