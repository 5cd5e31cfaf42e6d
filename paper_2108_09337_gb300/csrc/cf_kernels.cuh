// cf_kernels.cuh -- launchers shared between the libcf translation units.
#pragma once

#include "cf_common.cuh"

namespace cf {

constexpr int kMaxLevels = 32;

// Shape of one tournament: levels of the reduction tree.
struct TournPlan {
    int m, w, h, arity;
    int nleaves;
    int nlevels;              // including the leaf level
    int cnt[kMaxLevels];      // nodes per level
    int off[kMaxLevels];      // first node index of each level
    int total_nodes;
};

// Device scratch of a tournament.
struct TournWS {
    int *node_win;            // [total_nodes][kMaxV] panel rows chosen by each node
    int *node_cnt;            // [total_nodes]
    int *counter;             // [total_nodes] arrivals; zero before and after
    int *root_win;            // [kMaxV] winners in pivot order
    size_t counter_bytes;
    // FP32 tournament, optional: [m][kMaxV] row-major copy of the panel's
    // original rows, written by the leaves, read by the playoff nodes
    float *rows32 = nullptr;
};

// Root-node outputs used by the LU driver (ipiv == nullptr: none).
struct TournEpilogue {
    int *ipiv;
    int k0;
    int *swap_cnt;            // [1] number of moved rows
    int *swap_dst;            // [2*kMaxV] destination positions (relative to k0)
    int *swap_src;            // [2*kMaxV] source positions (relative to k0)
};

int make_tourn_plan(int m, int w, int h, int arity, TournPlan *plan);
size_t tourn_ws_bytes(int m, int h, int arity);
int tourn_ws_carve(void *work, int m, int h, int arity, TournWS *ws, TournEpilogue *ep);

template <typename T>
int launch_tourn(const T *P, int ldp, int m, int w, int h, int arity, const TournWS &ws, const TournEpilogue &ep,
                 cudaStream_t st);
template <typename T>
int launch_apply_swaps(T *A, int lda, int ncols, int k0, const TournEpilogue &ep, int *perm, cudaStream_t st);

// ---- panel kernels (cf_panel.cu)
// LU of the w x w diagonal block without pivoting (Fig. "prog_rep").
template <typename T>
int launch_getf2_nopiv(T *A00, int lda, int w, int kglob, int *info, cudaStream_t st);
// A10 <- A10 * U^{-1}: rows x w block X, U upper non-unit w x w (or, with
// trans_lower, U = L^T for a lower L).  Optional low-precision copy of the
// result, K-major: lp[(r) * ldlp + c].
template <typename T>
int launch_trsm_right_upper(T *X, int ldx, int rows, int w, const T *U, int ldu, bool trans_lower,
                            const int *skip_if_nonzero, cudaStream_t st);
// A01 <- L^{-1} * A01: w x cols block X, L unit lower w x w.
template <typename T>
int launch_trsm_left_lower_unit(T *X, int ldx, int w, int cols, const T *L, int ldl, cudaStream_t st);
// Cholesky of the w x w diagonal block (lower), Listing "Cholesky".
template <typename T>
int launch_potf2(T *A00, int lda, int w, int kglob, int *info, cudaStream_t st);

// ---- FP64 GEMM / SYRK (cf_gemm64.cu)
// C -= A * op(B); op(B)(p, j) = trans_b ? B[j + p*ldb] : B[p + j*ldb].
// lower: only entries with i >= j are touched.  skip_if_nonzero: device int
// whose nonzero value turns the launch into a no-op (Cholesky breakdown).
int launch_gemm_f64_sub(int m, int n, int k, const double *A, int lda, const double *B, int ldb, bool trans_b,
                        double *C, int ldc, bool lower, const int *skip_if_nonzero, cudaStream_t st);
// Generic SIMT form: C -= op(A) op(B) for T = double or float.
template <typename T>
int launch_gemm_sub_t(int m, int n, int k, const T *A, int lda, bool trans_a, const T *B, int ldb, bool trans_b,
                      T *C, int ldc, bool lower, const int *skip, cudaStream_t st);
// Left triangular solve X <- M^{-1} X (w <= 128) for the solves.
template <typename T>
int launch_trsm_left(bool lower, bool unit, bool trans, T *X, int ldx, int w, int cols, const T *Tm, int ldt,
                     cudaStream_t st);
// ---- FP32 panel kernels of the mixed path (cf_tourn32.cu, cf_panel32.cu)
int launch_tourn32(const float *P, int ldp, int m, int w, int h, int arity, const TournWS &ws, const TournEpilogue &ep,
                   cudaStream_t st);
// The same rule for panels of w <= 64 columns: leaves of up to 512 rows,
// arity up to 8 (cf_tourn32w.cu).
bool tourn32w_supported(int w, int h, int arity);
int launch_tourn32w(const float *P, int ldp, int m, int w, int h, int arity, const TournWS &ws,
                    const TournEpilogue &ep, cudaStream_t st);
// Either FP32 tournament: the wide-node kernel for panels of <= 64 columns
// when it takes (h, arity), else the v <= 128 kernel (h <= 256, arity 2).
int launch_tourn32_any(const float *P, int ldp, int m, int w, int h, int arity, const TournWS &ws,
                       const TournEpilogue &ep, cudaStream_t st);
int launch_a00_lu32(float *A00, int lda, int w, int kglob, int *info, cudaStream_t st);
int launch_a00_chol32(float *A00, int lda, int w, int kglob, int *info, cudaStream_t st);
template <typename LP>
int launch_rtrsm32(float *X, int ldx, int rows, int w, const float *M00, int ldm, bool trans_lower, LP *lp, int ldk,
                   int kpad, const int *skip, cudaStream_t st);
template <typename LP>
int launch_ltrsm32(float *X, int ldx, int w, int cols, const float *L00, int ldl, LP *lp, int ldk, int kpad,
                   cudaStream_t st);

// ---- thin triangular solves with FP32 factors (cf_trsv.cu)
// mode: 0 unit lower (L of LU), 1 upper (U), 2 lower (Cholesky L), 3 L^T.
size_t trsv_ws_bytes(int n);
size_t diag_inverse_floats(int n);      // FP32 inverses (128-row blocks)
size_t diag_inverse64_elems(int n);     // FP64 inverses (64-row blocks)
int launch_diag_inverse(int mode, int n, const float *T, int ldt, float *Dinv, cudaStream_t st);
int launch_diag_inverse64(int mode, int n, const float *T, int ldt, double *Dinv, cudaStream_t st);
int launch_trsv_f64x(int mode, int n, int nrhs, const float *T, int ldt, const double *Dinv, double *X, int ldx,
                     int *sync_ws, cudaStream_t st);
int launch_neighbor_premul(int mode, int n, const float *T, int ldt, const float *Dinv, float *Gout, cudaStream_t st);
int launch_trsv_f32(int mode, int n, int nrhs, const float *T, int ldt, const float *Dinv, const float *Gn, float *X,
                    int ldx,
                    int *sync_ws, cudaStream_t st);
int trsv_take_status(cudaStream_t st, int *status);
// R = B - A X (B null: R = A X) in FP32-pair arithmetic (cf_pair.cu).  amax:
// device pointer to the FP64 bits of a bound >= max |a_ij| (e.g. ||A||_inf);
// ws: pair_residual_ws_bytes(m, n) bytes.  The _auto form computes max |a_ij|
// itself into the workspace.
size_t pair_residual_ws_bytes(int m, int n);
// Elimination flops of one FP32 tournament (cf_tourn32.cu).
double tourn32_flops(int m, int w, int h, int arity = 2);
int launch_residual_pair(int m, int n, int nrhs, const double *A, int lda, const unsigned long long *amax,
                         const double *X, int ldx, const double *B, int ldb, double *R, int ldr, void *ws,
                         cudaStream_t st);
int launch_residual_pair_auto(int m, int n, int nrhs, const double *A, int lda, const double *X, int ldx,
                              const double *B, int ldb, double *R, int ldr, void *ws, cudaStream_t st);
// R = B - A X at FP64 accuracy on the tensor cores from BF16 digit slices
// (cf_resid_tc.cu).  resid_tc_carve places the slices and the row exponent
// fields in wsA (resid_tc_a_bytes, kept while the slices are used);
// resid_tc_prepare cuts A (after computing Ef unless ef_ready: the caller
// filled Ef with the row maxima of the exponent fields); resid_tc_apply forms
// R for any X (resid_tc_x_bytes of scratch; B null: R = A X).
struct ResidTC {
    int m, n, mpad, ldk;
    void *S;          // 8 digit slices of A in 128 x 64 BF16 tiles (tile-major, swizzled): mpad x ldk per digit
    int *Ef;          // per-row largest exponent field of A
};
ResidTC resid_tc_layout(int m, int n);
size_t resid_tc_a_bytes(int m, int n);
size_t resid_tc_x_bytes(int m, int n);
void resid_tc_carve(ResidTC *L, void *wsA);
int resid_tc_prepare(ResidTC *L, const double *A, int lda, bool ef_ready, cudaStream_t st);
int resid_tc_apply(const ResidTC &L, int nrhs, const double *X, int ldx, const double *B, int ldb, double *R, int ldr,
                   void *wsX, cudaStream_t st);
int rtc_take_status(cudaStream_t st, int *status);
// R = B - A X for a thin X (nrhs columns).
int launch_residual_f64(int m, int n, int nrhs, const double *A, int lda, const double *X, int ldx, const double *B,
                        int ldb, double *R, int ldr, cudaStream_t st);

}  // namespace cf
