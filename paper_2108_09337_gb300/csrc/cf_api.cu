// cf_api.cu -- C ABI of the FP64 path: cf_getrf, cf_potrf, cf_getrs, cf_potrs,
// cf_residual, options and status strings.
//
// The host loop of cf_getrf follows COnfLUX's outer loop (Alg. 1) on one
// GPU: per step t of width v, TournPivot on the current panel (LU-1), the row
// interchanges (LU-2; the paper masks rows instead because its matrix is
// replicated over c layers -- a single copy swaps in O(vN) per step), the LU
// of the selected rows A00, the two triangular solves (LU-3, LU-4) and the
// Schur update of A11 (LU-5).  The paper's scatters, broadcasts and
// reductions between ranks have no counterpart on one device.
#include <atomic>
#include <cstring>

#include "cf_common.cuh"
#include "cf_kernels.cuh"

namespace cf {

static std::atomic<int> g_last_cuda_error{0};
static std::atomic<long long> g_launches{0};
void set_cuda_error(cudaError_t e) { g_last_cuda_error.store((int)e); }
void count_launches(long long n) { g_launches.fetch_add(n); }

int launch_trsm_left_f64(bool lower, bool unit, bool trans, double *X, int ldx, int w, int cols, const double *Tm,
                         int ldt, cudaStream_t st);
int launch_gemm_f64_sub_t(int m, int n, int k, const double *A, int lda, bool trans_a, const double *B, int ldb,
                          bool trans_b, double *C, int ldc, bool lower, const int *skip, cudaStream_t st);

int resolve_options(const cf_options *in, Opts *o) {
    *o = Opts();
    if (in == nullptr) return CF_OK;
    if (in->v != 0) { o->v = in->v; o->v_set = true; }
    if (in->leaf_h != 0) { o->leaf_h = in->leaf_h; o->h_set = true; }
    if (in->arity != 0) { o->arity = in->arity; o->ar_set = true; }
    o->outer_V = in->outer_V;
    o->lookahead = in->lookahead;
    if (in->tol > 0) o->tol = in->tol;
    if (in->max_iter > 0) o->max_iter = in->max_iter;
    if (in->gmres_restart > 0) o->gmres_restart = in->gmres_restart;
    o->batch_cps = in->batch_cps;
    o->fp64_residual = in->fp64_residual;
    if (o->fp64_residual < 0 || o->fp64_residual > 1) return CF_ERR_UNSUPPORTED;
    o->residual_kind = in->residual_kind;
    if (o->residual_kind != 0 && o->residual_kind != 2) return CF_ERR_UNSUPPORTED;
    if (o->v < 1 || o->v > kMaxV) return CF_ERR_UNSUPPORTED;
    // the widest shapes any routine takes (FP32 tournament at v <= 64); each
    // routine checks its own narrower limits (FP64: leaf_h <= kMaxV, arity <= 4)
    if (o->leaf_h < 1 || o->leaf_h > 4 * kMaxV) return CF_ERR_UNSUPPORTED;
    if (o->arity < 2 || o->arity > 8) return CF_ERR_UNSUPPORTED;
    // outer_V: a multiple of v (of 64, the smallest default v, when v is left
    // to the routine; the mixed solvers check it again against their v)
    if (o->outer_V < 0 || (o->outer_V % (o->v_set ? o->v : 64)) != 0) return CF_ERR_UNSUPPORTED;
    if (o->gmres_restart < 1 || o->gmres_restart > 256) return CF_ERR_UNSUPPORTED;
    if (o->batch_cps < 0 || o->batch_cps > 8) return CF_ERR_UNSUPPORTED;
    return CF_OK;
}

// ipiv (1-based interchanges) -> row order: perm[i] = original row now at i.
__global__ void k_ipiv_to_perm(int n, const int *ipiv, int *perm) {
    extern __shared__ int sp[];
    const bool use_smem = (size_t)n * sizeof(int) <= 200 * 1024;
    int *p = use_smem ? sp : perm;
    for (int i = threadIdx.x; i < n; i += blockDim.x) p[i] = i;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < n; ++i) {
            const int j = ipiv[i] - 1;
            if (j != i) { const int t = p[i]; p[i] = p[j]; p[j] = t; }
        }
    }
    __syncthreads();
    if (use_smem)
        for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = p[i];
}

// Out[i, c] = In[perm[i], c]
__global__ void k_gather_rows(int n, int nrhs, const int *perm, const double *In, int ldi, double *Out, int ldo) {
    const size_t tot = (size_t)n * nrhs;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < tot; e += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(e % n), c = (int)(e / n);
        Out[(size_t)i + (size_t)c * ldo] = In[(size_t)perm[i] + (size_t)c * ldi];
    }
}

}  // namespace cf

using namespace cf;

int cf::mixed_lu_defaults(Opts *o) {
    if (!o->v_set) o->v = 64;
    if (!o->h_set) o->leaf_h = o->v <= 64 ? 512 : 256;
    if (!o->ar_set) o->arity = o->v <= 64 ? (8 * o->v <= 512 ? 8 : 512 / o->v) : 2;
    if ((o->outer_V % o->v) != 0) return CF_ERR_UNSUPPORTED;
    return tourn32_shape_ok(o->v, o->leaf_h, o->arity) ? CF_OK : CF_ERR_UNSUPPORTED;
}

extern "C" void cf_default_options(cf_options *opt) {
    if (opt == nullptr) return;
    Opts o;
    opt->v = 0;          // each routine's default (FP64: 128 / 128 / 2; mixed LU: 64 / 512 / 8)
    opt->leaf_h = 0;
    opt->arity = 0;
    opt->outer_V = o.outer_V;
    opt->lookahead = o.lookahead;
    opt->tol = o.tol;
    opt->max_iter = o.max_iter;
    opt->gmres_restart = o.gmres_restart;
    opt->batch_cps = o.batch_cps;
    opt->fp64_residual = o.fp64_residual;
    opt->residual_kind = o.residual_kind;
}

extern "C" const char *cf_status_string(int s) {
    switch (s) {
        case CF_OK: return "ok";
        case CF_ERR_CUDA: return "CUDA error";
        case CF_ERR_WORKSPACE: return "workspace too small";
        case CF_ERR_NOT_CONVERGED: return "refinement did not reach the tolerance";
        case CF_ERR_TIMEOUT: return "bounded device wait timed out";
        case CF_ERR_UNSUPPORTED: return "unsupported configuration";
        default: return s < 0 ? "invalid argument" : "unknown status";
    }
}

extern "C" int cf_last_cuda_error(void) { return g_last_cuda_error.load(); }

extern "C" long long cf_kernel_launches(void) { return g_launches.load(); }

// ------------------------------------------------------------------- getrf
extern "C" size_t cf_workspace_size(int op, int n, int nrhs, cf_prec prec, const cf_options *opt) {
    if (n < 0 || nrhs < 0) return 0;
    Opts o;
    if (resolve_options(opt, &o) != CF_OK) return 0;
    switch (op) {
        case CF_OP_GETRF: return cf_getrf_workspace_size(n, opt);
        case CF_OP_POTRF: return cf_potrf_workspace_size(n, opt);
        case CF_OP_GETRS: return cf_getrs_workspace_size(n, nrhs);
        case CF_OP_POTRS: return 0;
        case CF_OP_GESV_MIXED: return cf_gesv_mixed_workspace_size(n, nrhs, prec, opt);
        case CF_OP_POSV_MIXED: return cf_posv_mixed_workspace_size(n, nrhs, prec, opt);
        case CF_OP_GETRF_BATCHED: return cf_getrf_batched_workspace_size(n, opt);
        case CF_OP_POTRF_BATCHED: return cf_potrf_batched_workspace_size(n, opt);
        case CF_OP_FACTOR_BATCHED: return cf_factor_batched_workspace_size(n, opt);
        case CF_OP_SOLVE_BATCHED_MIXED: return cf_solve_batched_mixed_workspace_size(n, opt);
        case CF_OP_RESIDUAL_PAIR: return cf_residual_pair_workspace_size(n, n, nrhs);
        case CF_OP_TOURN_SELECT: return cf_tourn_workspace_size(n, nrhs, o.leaf_h, o.arity);
        default: return 0;
    }
}

extern "C" size_t cf_getrf_workspace_size(int n, const cf_options *opt) {
    Opts o;
    if (resolve_options(opt, &o) != CF_OK || !fp64_tourn_shape(o)) return 0;
    return tourn_ws_bytes(n > 0 ? n : 1, o.leaf_h, o.arity);
}

// LU-6 look-ahead (FP64 path).  Step t runs its panel chain (TournPivot,
// swaps, A00, both panel solves) and the update of only the next panel's
// columns on a high-priority stream, and the update of the remaining columns
// on a low-priority stream.  TournPivot of step t+1 reads only the next
// panel's columns, so it runs while the wide update of step t is still in
// flight (latency-bound selection next to an FP64-ALU-bound GEMM); the swaps
// of step t+1 wait for that update.  Both streams fork from and join back to
// the caller's stream, so the call stays stream-ordered (and capturable).
namespace cf {
// The two streams of a look-ahead factorization, forked from and joined back
// to the caller's stream.
struct LookaheadStreams {
    cudaStream_t sp = nullptr, su = nullptr;   // panel chain (high priority), wide updates (low)
    cudaEvent_t ev[5] = {};                    // fork, panel ready, rest done, join panel, join update
    int open(cudaStream_t st) {
        int lo = 0, hi = 0;
        if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
            cudaStreamCreateWithPriority(&sp, cudaStreamNonBlocking, hi) != cudaSuccess ||
            cudaStreamCreateWithPriority(&su, cudaStreamNonBlocking, lo) != cudaSuccess)
            return CF_ERR_CUDA;
        for (auto &e : ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return CF_ERR_CUDA;
        if (cudaEventRecord(ev[0], st) != cudaSuccess || cudaStreamWaitEvent(sp, ev[0], 0) != cudaSuccess ||
            cudaStreamWaitEvent(su, ev[0], 0) != cudaSuccess)
            return CF_ERR_CUDA;
        return CF_OK;
    }
    int panel_to_update() {      // the wide update may start once the panel is ready
        return (cudaEventRecord(ev[1], sp) == cudaSuccess && cudaStreamWaitEvent(su, ev[1], 0) == cudaSuccess)
                   ? CF_OK : CF_ERR_CUDA;
    }
    int update_done() { return cudaEventRecord(ev[2], su) == cudaSuccess ? CF_OK : CF_ERR_CUDA; }
    int wait_update() { return cudaStreamWaitEvent(sp, ev[2], 0) == cudaSuccess ? CF_OK : CF_ERR_CUDA; }
    int join(cudaStream_t st) {
        return (cudaEventRecord(ev[3], sp) == cudaSuccess && cudaEventRecord(ev[4], su) == cudaSuccess &&
                cudaStreamWaitEvent(st, ev[3], 0) == cudaSuccess && cudaStreamWaitEvent(st, ev[4], 0) == cudaSuccess)
                   ? CF_OK : CF_ERR_CUDA;
    }
    ~LookaheadStreams() {        // safe with work in flight: released on completion
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        if (sp) cudaStreamDestroy(sp);
        if (su) cudaStreamDestroy(su);
    }
};

static int getrf_lookahead(int n, double *A, int lda, int *ipiv, int *info, const Opts &o, TournWS &ws,
                           TournEpilogue &ep, cudaStream_t st) {
    LookaheadStreams L;
    int rc = L.open(st);
    if (rc) return rc;
    cudaStream_t sp = L.sp, su = L.su;
    auto fail = [](int r) { return r; };
    const size_t ld = (size_t)lda;
    bool rest_pending = false;
    for (int k0 = 0; k0 < n; k0 += o.v) {
        const int w = o.v < n - k0 ? o.v : n - k0;
        const int m = n - k0;
        double *A00 = A + k0 + k0 * ld;
        ep.ipiv = ipiv;
        ep.k0 = k0;
        if ((rc = launch_tourn<double>(A00, lda, m, w, o.leaf_h, o.arity, ws, ep, sp))) return fail(rc);
        if (rest_pending && (rc = L.wait_update())) return fail(rc);
        if ((rc = launch_apply_swaps<double>(A, lda, n, k0, ep, nullptr, sp))) return fail(rc);
        if ((rc = launch_getf2_nopiv<double>(A00, lda, w, k0, info, sp))) return fail(rc);
        if ((rc = launch_trsm_right_upper<double>(A00 + w, lda, m - w, w, A00, lda, false, nullptr, sp)))
            return fail(rc);
        if ((rc = launch_trsm_left_lower_unit<double>(A00 + w * ld, lda, w, n - k0 - w, A00, lda, sp)))
            return fail(rc);
        rest_pending = false;
        const int right = n - k0 - w;
        if (m - w <= 0 || right <= 0) continue;
        const int w1 = o.v < right ? o.v : right;       // the next panel's columns
        if ((rc = launch_gemm_f64_sub(m - w, w1, w, A00 + w, lda, A00 + w * ld, lda, false, A00 + w + w * ld, lda,
                                      false, nullptr, sp)))
            return fail(rc);
        if (right > w1) {
            if ((rc = L.panel_to_update())) return fail(rc);
            if ((rc = launch_gemm_f64_sub(m - w, right - w1, w, A00 + w, lda, A00 + (w + w1) * ld, lda, false,
                                          A00 + w + (w + w1) * ld, lda, false, nullptr, su)))
                return fail(rc);
            if ((rc = L.update_done())) return fail(rc);
            rest_pending = true;
        }
    }
    return L.join(st);
}

// The same for Cholesky: step t's diagonal factorization and panel solve,
// then the update of the next panel's columns (every row below) on the
// high-priority stream; the lower update of the rest on the low-priority
// one.  Step t+1's panel work overlaps that rest; its own update of the next
// columns waits for it (same columns).
static int potrf_lookahead(int n, double *A, int lda, int *info, const Opts &o, cudaStream_t st) {
    LookaheadStreams L;
    int rc = L.open(st);
    if (rc) return rc;
    cudaStream_t sp = L.sp, su = L.su;
    const size_t ld = (size_t)lda;
    bool rest_pending = false;
    for (int k0 = 0; k0 < n; k0 += o.v) {
        const int w = o.v < n - k0 ? o.v : n - k0;
        const int m = n - k0;
        double *A00 = A + k0 + k0 * ld;
        if ((rc = launch_potf2<double>(A00, lda, w, k0, info, sp))) return rc;
        if ((rc = launch_trsm_right_upper<double>(A00 + w, lda, m - w, w, A00, lda, true, info, sp))) return rc;
        const int rest = m - w;
        if (rest <= 0) continue;
        if (rest_pending && (rc = L.wait_update())) return rc;
        rest_pending = false;
        const int w1 = o.v < rest ? o.v : rest;
        if ((rc = launch_gemm_f64_sub(rest, w1, w, A00 + w, lda, A00 + w, lda, true, A00 + w + w * ld, lda, true,
                                      info, sp)))
            return rc;
        if (rest > w1) {
            if ((rc = L.panel_to_update())) return rc;
            if ((rc = launch_gemm_f64_sub(rest - w1, rest - w1, w, A00 + w + w1, lda, A00 + w + w1, lda, true,
                                          A00 + (w + w1) + (w + w1) * ld, lda, true, info, su)))
                return rc;
            if ((rc = L.update_done())) return rc;
            rest_pending = true;
        }
    }
    return L.join(st);
}
}  // namespace cf

extern "C" int cf_getrf(int n, double *A, int lda, int *ipiv, int *info, void *work, size_t lwork,
                        const cf_options *opt, cudaStream_t st) {
    if (n < 0) return -1;
    if (n > 0 && A == nullptr) return -2;
    if (lda < (n > 1 ? n : 1)) return -3;
    if (n > 0 && ipiv == nullptr) return -4;
    if (info == nullptr) return -5;
    Opts o;
    int rc = resolve_options(opt, &o);
    if (rc != CF_OK) return rc;
    if (!fp64_tourn_shape(o)) return CF_ERR_UNSUPPORTED;
    CF_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int), st));
    if (n == 0) return CF_OK;
    if (work == nullptr || lwork < cf_getrf_workspace_size(n, opt)) return CF_ERR_WORKSPACE;
    TournWS ws{};
    TournEpilogue ep{};
    rc = tourn_ws_carve(work, n, o.leaf_h, o.arity, &ws, &ep);
    if (rc != CF_OK) return rc;
    CF_CUDA_TRY(cudaMemsetAsync(ws.counter, 0, ws.counter_bytes, st));
    if (o.lookahead) return getrf_lookahead(n, A, lda, ipiv, info, o, ws, ep, st);
    const size_t ld = (size_t)lda;
    for (int k0 = 0; k0 < n; k0 += o.v) {
        const int w = o.v < n - k0 ? o.v : n - k0;
        const int m = n - k0;
        double *A00 = A + k0 + k0 * ld;
        ep.ipiv = ipiv;
        ep.k0 = k0;
        // LU-1 TournPivot on A[k0:n, k0:k0+w]
        if ((rc = launch_tourn<double>(A00, lda, m, w, o.leaf_h, o.arity, ws, ep, st))) return rc;
        // LU-2 interchanges on all n columns
        if ((rc = launch_apply_swaps<double>(A, lda, n, k0, ep, nullptr, st))) return rc;
        // A00 = L00 U00 (no further pivoting)
        if ((rc = launch_getf2_nopiv<double>(A00, lda, w, k0, info, st))) return rc;
        // LU-3 A10 <- A10 U00^{-1}
        if ((rc = launch_trsm_right_upper<double>(A00 + w, lda, m - w, w, A00, lda, false, nullptr, st))) return rc;
        // LU-4 A01 <- L00^{-1} A01
        if ((rc = launch_trsm_left_lower_unit<double>(A00 + w * ld, lda, w, n - k0 - w, A00, lda, st))) return rc;
        // LU-5 A11 <- A11 - A10 A01
        if ((rc = launch_gemm_f64_sub(m - w, n - k0 - w, w, A00 + w, lda, A00 + w * ld, lda, false,
                                      A00 + w + w * ld, lda, false, nullptr, st)))
            return rc;
    }
    return CF_OK;
}

// ------------------------------------------------------------------- potrf
extern "C" size_t cf_potrf_workspace_size(int n, const cf_options *opt) {
    (void)n;
    (void)opt;
    return 0;
}

extern "C" int cf_potrf(int n, double *A, int lda, int *info, void *work, size_t lwork, const cf_options *opt,
                        cudaStream_t st) {
    (void)work;
    (void)lwork;
    if (n < 0) return -1;
    if (n > 0 && A == nullptr) return -2;
    if (lda < (n > 1 ? n : 1)) return -3;
    if (info == nullptr) return -4;
    Opts o;
    int rc = resolve_options(opt, &o);
    if (rc != CF_OK) return rc;
    CF_CUDA_TRY(cudaMemsetAsync(info, 0, sizeof(int), st));
    if (o.lookahead && n > 0) return potrf_lookahead(n, A, lda, info, o, st);
    const size_t ld = (size_t)lda;
    for (int k0 = 0; k0 < n; k0 += o.v) {
        const int w = o.v < n - k0 ? o.v : n - k0;
        const int m = n - k0;
        double *A00 = A + k0 + k0 * ld;
        // CH-1 L00 = chol(A00)
        if ((rc = launch_potf2<double>(A00, lda, w, k0, info, st))) return rc;
        // CH-2 L10 <- A10 L00^{-T}
        if ((rc = launch_trsm_right_upper<double>(A00 + w, lda, m - w, w, A00, lda, true, info, st))) return rc;
        // CH-3 A11 <- A11 - L10 L10^T (lower)
        if ((rc = launch_gemm_f64_sub(m - w, m - w, w, A00 + w, lda, A00 + w, lda, true, A00 + w + w * ld, lda,
                                      true, info, st)))
            return rc;
    }
    return CF_OK;
}

// ------------------------------------------------------------------- solves
extern "C" size_t cf_getrs_workspace_size(int n, int nrhs) {
    Carver cv(nullptr);
    cv.take<int>(n > 0 ? n : 1);
    cv.take<double>((size_t)(n > 0 ? n : 1) * (nrhs > 0 ? nrhs : 1));
    return cv.size();
}

extern "C" int cf_getrs(int n, int nrhs, const double *LU, int lda, const int *ipiv, double *B, int ldb, void *work,
                        size_t lwork, cudaStream_t st) {
    if (n < 0) return -1;
    if (nrhs < 0) return -2;
    if (n > 0 && LU == nullptr) return -3;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (n > 0 && ipiv == nullptr) return -5;
    if (n > 0 && nrhs > 0 && B == nullptr) return -6;
    if (ldb < (n > 1 ? n : 1)) return -7;
    if (n == 0 || nrhs == 0) return CF_OK;
    if (work == nullptr || lwork < cf_getrs_workspace_size(n, nrhs)) return CF_ERR_WORKSPACE;
    Carver cv(work);
    int *perm = cv.take<int>(n);
    double *T = cv.take<double>((size_t)n * nrhs);
    const size_t smem = (size_t)n * sizeof(int) <= 200 * 1024 ? (size_t)n * sizeof(int) : 0;
    if (smem > 48 * 1024) CF_CUDA_TRY(cudaFuncSetAttribute(k_ipiv_to_perm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_ipiv_to_perm<<<1, 1024, smem, st>>>(n, ipiv, perm);
    CF_LAUNCH_CHECK();
    k_gather_rows<<<1024, 256, 0, st>>>(n, nrhs, perm, B, ldb, T, n);
    CF_LAUNCH_CHECK();
    int rc;
    const size_t ld = (size_t)lda;
    const int v = kMaxV;
    for (int k0 = 0; k0 < n; k0 += v) {                 // L y = P b
        const int w = v < n - k0 ? v : n - k0;
        if ((rc = launch_trsm_left_f64(true, true, false, T + k0, n, w, nrhs, LU + k0 + k0 * ld, lda, st))) return rc;
        if ((rc = launch_gemm_f64_sub_t(n - k0 - w, nrhs, w, LU + (k0 + w) + k0 * ld, lda, false, T + k0, n, false,
                                        T + k0 + w, n, false, nullptr, st)))
            return rc;
    }
    const int nb = (n + v - 1) / v;
    for (int b = nb - 1; b >= 0; --b) {                 // U x = y
        const int k0 = b * v;
        const int w = v < n - k0 ? v : n - k0;
        if ((rc = launch_trsm_left_f64(false, false, false, T + k0, n, w, nrhs, LU + k0 + k0 * ld, lda, st))) return rc;
        if ((rc = launch_gemm_f64_sub_t(k0, nrhs, w, LU + k0 * ld, lda, false, T + k0, n, false, T, n, false, nullptr,
                                        st)))
            return rc;
    }
    CF_CUDA_TRY(cudaMemcpy2DAsync(B, sizeof(double) * ldb, T, sizeof(double) * n, sizeof(double) * n, nrhs,
                                  cudaMemcpyDeviceToDevice, st));
    return CF_OK;
}

extern "C" int cf_potrs(int n, int nrhs, const double *L, int lda, double *B, int ldb, cudaStream_t st) {
    if (n < 0) return -1;
    if (nrhs < 0) return -2;
    if (n > 0 && L == nullptr) return -3;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (n > 0 && nrhs > 0 && B == nullptr) return -5;
    if (ldb < (n > 1 ? n : 1)) return -6;
    if (n == 0 || nrhs == 0) return CF_OK;
    int rc;
    const size_t ld = (size_t)lda, lb = (size_t)ldb;
    const int v = kMaxV;
    for (int k0 = 0; k0 < n; k0 += v) {                 // L y = b
        const int w = v < n - k0 ? v : n - k0;
        if ((rc = launch_trsm_left_f64(true, false, false, B + k0, ldb, w, nrhs, L + k0 + k0 * ld, lda, st))) return rc;
        if ((rc = launch_gemm_f64_sub_t(n - k0 - w, nrhs, w, L + (k0 + w) + k0 * ld, lda, false, B + k0, ldb, false,
                                        B + k0 + w, ldb, false, nullptr, st)))
            return rc;
    }
    const int nb = (n + v - 1) / v;
    for (int b = nb - 1; b >= 0; --b) {                 // L^T x = y
        const int k0 = b * v;
        const int w = v < n - k0 ? v : n - k0;
        if ((rc = launch_trsm_left_f64(false, false, true, B + k0, ldb, w, nrhs, L + k0 + k0 * ld, lda, st))) return rc;
        // B[0:k0] -= (L[k0:k0+w, 0:k0])^T B[k0:k0+w]
        if ((rc = launch_gemm_f64_sub_t(k0, nrhs, w, L + k0, lda, true, B + k0, ldb, false, B, ldb, false, nullptr,
                                        st)))
            return rc;
    }
    (void)lb;
    return CF_OK;
}

extern "C" int cf_residual(int m, int n, int nrhs, const double *A, int lda, const double *X, int ldx,
                           const double *B, int ldb, double *R, int ldr, cudaStream_t st) {
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (nrhs < 0) return -3;
    if (m > 0 && n > 0 && A == nullptr) return -4;
    if (lda < (m > 1 ? m : 1)) return -5;
    if (n > 0 && nrhs > 0 && X == nullptr) return -6;
    if (ldx < (n > 1 ? n : 1)) return -7;
    if (m > 0 && nrhs > 0 && B == nullptr) return -8;
    if (ldb < (m > 1 ? m : 1)) return -9;
    if (m > 0 && nrhs > 0 && R == nullptr) return -10;
    if (ldr < (m > 1 ? m : 1)) return -11;
    return launch_residual_f64(m, n, nrhs, A, lda, X, ldx, B, ldb, R, ldr, st);
}

extern "C" size_t cf_residual_pair_workspace_size(int m, int n, int nrhs) {
    (void)nrhs;
    return pair_residual_ws_bytes(m, n);
}

extern "C" int cf_residual_pair(int m, int n, int nrhs, const double *A, int lda, const double *X, int ldx,
                                const double *B, int ldb, double *R, int ldr, void *work, size_t lwork,
                                cudaStream_t st) {
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (nrhs < 0) return -3;
    if (m > 0 && n > 0 && A == nullptr) return -4;
    if (lda < (m > 1 ? m : 1)) return -5;
    if (n > 0 && nrhs > 0 && X == nullptr) return -6;
    if (ldx < (n > 1 ? n : 1)) return -7;
    if (m > 0 && nrhs > 0 && B == nullptr) return -8;
    if (ldb < (m > 1 ? m : 1)) return -9;
    if (m > 0 && nrhs > 0 && R == nullptr) return -10;
    if (ldr < (m > 1 ? m : 1)) return -11;
    if (m == 0 || nrhs == 0) return CF_OK;
    if (work == nullptr || lwork < pair_residual_ws_bytes(m, n)) return CF_ERR_WORKSPACE;
    return launch_residual_pair_auto(m, n, nrhs, A, lda, X, ldx, B, ldb, R, ldr, work, st);
}
