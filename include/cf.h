/*
 * cf.h -- C ABI of libcf: GB300 (sm_103a) dense LU with tournament pivoting
 * and Cholesky, after COnfLUX / COnfCHOX (Kwasniewski et al., "On the
 * Parallel I/O Optimality of Linear Algebra Kernels: Near-Optimal Matrix
 * Factorizations", SC'21, arXiv 2108.09337).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are column-major: element (i, j) of X with leading dimension
 *    ldx is X[i + j*ldx].  ld >= max(1, rows).  Sizes may be 0 (no-op).
 *  - Pointers are DEVICE pointers unless a parameter says "host".  The
 *    caller owns all memory.  Calls that need scratch take (work, lwork);
 *    the matching *_workspace_size() gives the bytes; lwork smaller than
 *    that returns CF_ERR_WORKSPACE before anything is enqueued.  The library
 *    never allocates device memory inside a call.
 *  - Every call enqueues its work on `stream` and returns without waiting,
 *    except where a parameter says it synchronises.
 *  - ipiv is int32, 1-based, LAPACK order: row i was interchanged with row
 *    ipiv[i]-1, for i = 0..n-1 in increasing order.
 *  - info is a device int32: 0 on success; k > 0 when U(k-1,k-1) is exactly
 *    zero (LU; the factorization still completes, as LAPACK dgetrf does), or
 *    when the leading minor of order k is not positive definite (Cholesky;
 *    the factorization stops there).
 *  - Return value (host): CF_OK, -i when argument i (1-based) is invalid, or
 *    one of the CF_ERR_* codes below.
 *  - Calls from several host threads, or overlapping on several streams,
 *    are safe when each has its own work buffer, with two device-wide
 *    exceptions: cf_getrf_noalloc's fixed scratch (such calls must not
 *    overlap on the GPU), and the status words of the bounded device waits
 *    (cf_device_status): a wait that runs out in one call may be reported,
 *    and cleared, by whichever call reads them next.
 */
#ifndef CF_H
#define CF_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    CF_OK = 0,
    CF_ERR_CUDA = -100,          /* a CUDA call failed; see cf_last_cuda_error */
    CF_ERR_WORKSPACE = -101,     /* lwork below the size *_workspace_size gave */
    CF_ERR_NOT_CONVERGED = -102, /* refinement stopped above the tolerance */
    CF_ERR_TIMEOUT = -103,       /* a bounded device-side wait ran out */
    CF_ERR_UNSUPPORTED = -104    /* valid but unsupported configuration */
};

typedef enum {
    CF_F64 = 0,
    CF_F32 = 1,
    CF_BF16 = 2,
    CF_F16 = 3,
    CF_FP8E4M3 = 4,
    CF_BF16X3 = 5      /* mixed solvers: each update operand as a BF16 pair
                          hi + lo, three products (hi.hi + hi.lo + lo.hi)
                          accumulated in FP32: 16 significant bits at three
                          times the tensor work */
} cf_prec;

/* Tunables.  Pass NULL for the defaults (in brackets); a field left 0 in v,
 * leaf_h, arity, tol, max_iter or gmres_restart also takes its default
 * (cf_default_options leaves v, leaf_h and arity 0, since their defaults
 * depend on the routine).  A value out of range makes the call return
 * CF_ERR_UNSUPPORTED (the size queries return 0) before anything is
 * enqueued.  The pivot sequence is a function of (v, leaf_h, arity) only;
 * the oracle takes the same three. */
typedef struct {
    int v;             /* block size of a step, 1..128 (Sec. 7.2, "Block size
                          v") [128; mixed LU: 64] */
    int leaf_h;        /* tournament leaf height: FP64 routines 1..128 [128];
                          mixed LU 1..512 with v <= 64 [512], 1..256 with
                          v > 64 [256] */
    int arity;         /* children per playoff node: FP64 routines 2..8 [8];
                          mixed LU with v <= 64: 2..8 and arity * v <= 512
                          [8], with v > 64: 2 [2] */
    int outer_V;       /* mixed LU/Cholesky: depth of the deferred update,
                          multiple of v [0 = auto: 2048 at n >= 16384,
                          1024 at n >= 8192, 512 below] */
    int lookahead;     /* LU-6 look-ahead [1]; 0 = one stream.  cf_getrf:
                          TournPivot of step t+1 on a high-priority stream
                          while the wide update of step t runs on a
                          low-priority one; mixed LU: the next panel's
                          columns are updated first and the rest of the
                          slab's update runs on a second stream beside
                          TournPivot of step t+1.  Results do not depend on
                          it; the other routines ignore it */
    double tol;        /* refinement stop: max backward error [1e-14] */
    int max_iter;      /* refinement iterations [30] */
    int gmres_restart; /* GMRES-IR Krylov dimension per correction, 1..256 [30] */
    int batch_cps;     /* batched calls: resident CTAs per SM, 1..3 (LU /
                          Cholesky) or 1..2 (mixed), 0 = as many as fit [0];
                          cf_batched_autotune picks it with v */
    int fp64_residual; /* mixed solvers: 1 = every residual and GMRES product
                          in FP64 arithmetic (overrides residual_kind); 0 =
                          as residual_kind says [0] */
    int residual_kind; /* mixed solvers' residuals and GMRES products: 0 = on
                          the tensor cores from digit slices of A
                          (cf_residual_tc; the workspace holds the slices,
                          16 n^2 bytes more) [0]; 2 = pair arithmetic
                          (cf_residual_pair) where the backward error allows
                          it, FP64 for the residual that decides convergence */
} cf_options;

void cf_default_options(cf_options *opt /* host */);

/* Statistics of a refined solve.  Written to host memory by the mixed
 * solvers (they synchronise `stream` once per refinement step). */
typedef struct {
    int iterations;    /* refinement steps taken (residual evaluations - 1) */
    int solver;        /* 0 = LU-IR / Cholesky-IR throughout, 1 = switched to
                          GMRES-IR (a classical step cut eta by less than
                          0.3x) */
    int converged;     /* 1 if eta <= tol */
    int info;          /* info of the low-precision factorization */
    double eta;        /* final max_j ||r_j||_inf / (||A||_inf ||x_j||_inf + ||b_j||_inf) */
    double eta0;       /* backward error of the unrefined solution */
    double shift;      /* diagonal shift added before factoring (0 if none) */
    double factor_ms;  /* device time of the factorization */
    double refine_ms;  /* device time of the refinement */
    double residual_ms;     /* device time inside the FP64 residual launches */
    double update_ms;       /* device time inside the K = V tensor-core updates */
    double update_flops;    /* algorithmic flops of those updates */
    int residual_launches;  /* FP64 products with A (residuals and GMRES steps) */
    int update_launches;
    int gmres_iterations;   /* inner GMRES steps over all GMRES-IR corrections */
    int escalated;          /* 1 if the solve refactored with CF_BF16X3 updates
                               after the requested precision stalled */
    double pair_ms;         /* device time inside the pair-arithmetic products */
    int pair_launches;      /* pair-arithmetic products with A */
    double tourn_ms;        /* device time inside the FP32 tournaments (LU) */
    int tourn_launches;
    double tourn_flops;     /* their elimination flops: per GEPP on r rows x w
                               columns, sum_j (r-j-1)(2(w-j-1) + 1) */
    double tc_ms;           /* device time inside the tensor-core residuals and
                               products with A */
    int tc_launches;        /* tensor-core products with A */
    double tc_prep_ms;      /* device time cutting A into its digit slices
                               (once per solve) */
} cf_refine_stats;

/* One workspace query for every call that takes (work, lwork): the bytes
 * that call needs, equal to its own *_workspace_size query.  n is the order
 * (rows of the panel for CF_OP_TOURN_SELECT, the batch size for the batched
 * calls); nrhs is the right-hand sides (the panel width for
 * CF_OP_TOURN_SELECT; ignored where the call has none); prec matters only for
 * the mixed solvers; opt may be NULL (defaults).  Host only; returns 0 for an
 * unknown op or an invalid configuration, and for calls that need no
 * workspace (CF_OP_POTRF, CF_OP_POTRS). */
typedef enum {
    CF_OP_GETRF = 0,
    CF_OP_POTRF = 1,
    CF_OP_GETRS = 2,
    CF_OP_POTRS = 3,
    CF_OP_GESV_MIXED = 4,
    CF_OP_POSV_MIXED = 5,
    CF_OP_GETRF_BATCHED = 6,
    CF_OP_POTRF_BATCHED = 7,
    CF_OP_FACTOR_BATCHED = 8,
    CF_OP_SOLVE_BATCHED_MIXED = 9,
    CF_OP_RESIDUAL_PAIR = 10,
    CF_OP_TOURN_SELECT = 11
} cf_op;
size_t cf_workspace_size(int op, int n, int nrhs, cf_prec prec, const cf_options *opt);

const char *cf_status_string(int status);
int cf_last_cuda_error(void);   /* last cudaError_t seen by the library */
/* Number of kernel launches the library has enqueued in this process so far
 * (a captured graph counts each of its kernels at every replay). */
long long cf_kernel_launches(void);

/* ------------------------------------------------------------------------
 * LU-1  TournPivot on one panel (Alg. 1; Sec. 7.3, "Tournament
 * Pivoting" / "Pivoting in COnfLUX").  Exposed for testing the selection
 * rule alone.
 *   panel   m x w FP64, ld ldp (read only)
 *   winners device int[min(m,w)]: 0-based panel rows of the pivots, in
 *           pivot order
 * Leaves are leaf_h consecutive rows; each playoff node stacks the winners
 * of `arity` adjacent children (original panel values) and keeps min(rows, w)
 * by partial-pivoting elimination; ties go to the smallest stacked position.
 * w <= 128, 1 <= leaf_h <= 128, 2 <= arity <= 8 (a playoff node is a
 * thread-block cluster of `arity` CTAs).
 * ------------------------------------------------------------------------ */
size_t cf_tourn_workspace_size(int m, int w, int leaf_h, int arity);
int cf_tourn_select(int m, int w, const double *panel, int ldp, int leaf_h,
                    int arity, int *winners, void *work, size_t lwork,
                    cudaStream_t stream);

/* The same selection on an FP32 panel, as the mixed-precision solvers run
 * it (elimination in FP32 with fused multiply-add; one register row per
 * thread).  Same arguments and workspace as cf_tourn_select, except the
 * shapes: w <= 64 with 1 <= leaf_h <= 512, 2 <= arity <= 8 and
 * arity * w <= 512; or w <= 128 with 1 <= leaf_h <= 256 and arity 2. */
int cf_tourn_select_f32(int m, int w, const float *panel, int ldp, int leaf_h,
                        int arity, int *winners, void *work, size_t lwork,
                        cudaStream_t stream);

/* ------------------------------------------------------------------------
 * cf_getrf -- FP64 LU with tournament pivoting, in place (Alg. 1; Sec. 7.2
 * routines TournPivot, Factorize A00/A10/A01/A11; Table 2).
 *   A     n x n FP64, lda: overwritten by L (unit, strictly below the
 *         diagonal) and U (upper) of P A = L U.
 *   ipiv  device int[n], 1-based interchanges (see above).
 *   info  device int[1].
 * ------------------------------------------------------------------------ */
size_t cf_getrf_workspace_size(int n, const cf_options *opt);
int cf_getrf(int n, double *A, int lda, int *ipiv, int *info, void *work,
             size_t lwork, const cf_options *opt, cudaStream_t stream);

/* cf_getrf_noalloc -- cf_getrf for callers that cannot allocate device
 * memory (code running under stream capture, plugins inside a framework
 * whose allocator owns the device memory, callers with memory partitioned up
 * front).  The paper has no counterpart; this is a deployment convenience.
 * Same arguments, results and kernels as cf_getrf, but the tournament
 * scratch lives in a 2 MiB array that the library places on every GPU that
 * loads it and holds until the process exits; nothing is allocated.
 *   - The scratch needed grows like n / leaf_h: n up to 393216 fits with
 *     leaf_h = 128 and the default arity 8 (196608 with leaf_h = 64; with
 *     arity 2, 131072 and 65536).  Larger requests return CF_ERR_WORKSPACE
 *     before anything is enqueued.
 *   - The first call on a device looks up the array's device address (once,
 *     with that device current); make that first call before any stream
 *     capture on that device.
 *   - All calls share the one array: calls whose work overlaps on the GPU
 *     (other streams, other host threads) race and corrupt each other.  The
 *     arrival counters are cleared at the start of every call.
 *   - It always runs the one-stream schedule on `stream` (opt->lookahead is
 *     ignored): the results equal cf_getrf's, the speed is that of cf_getrf
 *     with lookahead = 0.
 *   - The looked-up address is kept for the life of the process: after a
 *     cudaDeviceReset (or anything else that destroys the device's primary
 *     context) the next call on that device is invalid. */
int cf_getrf_noalloc(int n, double *A, int lda, int *ipiv, int *info,
                     const cf_options *opt, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * cf_potrf -- FP64 Cholesky, lower, in place (Listing "Cholesky
 * Factorization", Sec. 6.2; COnfCHOX, Sec. 7.5 and Table 2: potrf on A00,
 * trsm on the panel, triangular update of A11).  Only the lower triangle is
 * read or written.
 * ------------------------------------------------------------------------ */
size_t cf_potrf_workspace_size(int n, const cf_options *opt);
int cf_potrf(int n, double *A, int lda, int *info, void *work, size_t lwork,
             const cf_options *opt, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * S-1  Solves with the FP64 factors (paper silent; LAPACK getrs / potrs).
 *   B  n x nrhs FP64, ldb: overwritten by the solution.
 * cf_getrs needs work of cf_getrs_workspace_size(n, nrhs) bytes (the row
 * order and a permuted copy of B).
 * ------------------------------------------------------------------------ */
size_t cf_getrs_workspace_size(int n, int nrhs);
int cf_getrs(int n, int nrhs, const double *LU, int lda, const int *ipiv,
             double *B, int ldb, void *work, size_t lwork,
             cudaStream_t stream);
int cf_potrs(int n, int nrhs, const double *L, int lda, double *B, int ldb,
             cudaStream_t stream);

/* ------------------------------------------------------------------------
 * R-1  FP64 residual R = B - A X (A m x n; X n x nrhs; B, R m x nrhs).
 * R may alias B.
 * ------------------------------------------------------------------------ */
int cf_residual(int m, int n, int nrhs, const double *A, int lda,
                const double *X, int ldx, const double *B, int ldb, double *R,
                int ldr, cudaStream_t stream);

/* R-1 on the FP32 pipes: R = B - A X (A m x n FP64, lda; X n x nrhs FP64,
 * ldx; B, R m x nrhs FP64, column-major; R may alias B) in pair ("double-
 * float") arithmetic.  Each A element is split on the fly into two FP32
 * numbers after scaling by a power of two above max |a_ij| (computed here in
 * one extra pass over A), X once per call after scaling each column by a
 * power of two; every product is formed exactly as an FP32 pair and summed
 * with error-free transformations (Knuth's TwoSum), restarting into an FP64
 * accumulator every 16 terms.  Elements below 2^-74 max |a_ij| are dropped.
 * Accuracy: about 2^-48 sqrt(16) of the largest partial sums of 16 terms of
 * a row (1e-16 to a few 1e-14 of ||A||_inf ||x||_inf + ||b||_inf, the latter
 * on rows dominated by one term; ~1e-16 for cf_residual).  The mixed solvers
 * use this kernel for the residuals of refinement steps whose backward error
 * is above 1e-12 and for
 * the matrix-vector products of GMRES-IR, and cf_residual for the residual
 * that decides convergence.
 * work: cf_residual_pair_workspace_size(m, n, nrhs) bytes (device memory,
 * owned by the caller).  Errors: -k for the k-th argument out of range,
 * CF_ERR_WORKSPACE if work is null or too small.  Inf / NaN in A or X give
 * NaN in the affected rows. */
size_t cf_residual_pair_workspace_size(int m, int n, int nrhs);
int cf_residual_pair(int m, int n, int nrhs, const double *A, int lda,
                     const double *X, int ldx, const double *B, int ldb,
                     double *R, int ldr, void *work, size_t lwork,
                     cudaStream_t stream);

/* R-1 on the tensor cores at FP64 accuracy: R = B - A X (A m x n FP64, lda;
 * X n x nrhs FP64, ldx; B, R m x nrhs FP64; R may alias B; column-major).
 * Every a_ij is rounded to an integer q_ij = round(a_ij 2^(62 - E_i)) with
 * max_j |a_ij| < 2^E_i (X likewise per column) and cut into eight balanced
 * base-256 digits held exactly in BF16; the products of digit pairs whose
 * weights are at most 2^-56 below the leading pair are summed by tcgen05
 * MMAs with FP32 accumulation, exact because every 128-term chunk stays
 * below 2^24, then in int64; R is formed from those integer sums in
 * double-double.  Accuracy: a few 2^-63 of max_j |a_ij| ||x_k||_inf per term,
 * below the FP64 product's own rounding (the mixed solvers use it for every
 * residual and GMRES product by default).
 * work: cf_residual_tc_workspace_size(m, n, nrhs) bytes (16 m n bytes of
 * digit slices of A, cut on every call, plus 1 KB per row and 256 bytes per
 * column of scratch).  Inf / NaN in a row of A (column of X) give NaN in
 * that row (column) of R.  Errors: -k for the k-th argument, CF_ERR_WORKSPACE;
 * a bounded device wait that runs out is reported by cf_device_status. */
size_t cf_residual_tc_workspace_size(int m, int n, int nrhs);
int cf_residual_tc(int m, int n, int nrhs, const double *A, int lda,
                   const double *X, int ldx, const double *B, int ldb,
                   double *R, int ldr, void *work, size_t lwork,
                   cudaStream_t stream);

/* ------------------------------------------------------------------------
 * LU-5 / CH-3 building block, exposed for testing: C -= A_lp * B_lp^T on the
 * tensor cores (tcgen05, TMEM accumulators, TMA-fed), FP32 accumulate.
 *   A_lp  m x k low-precision, K-major: element (i, p) at A_lp[i*lda_k + p]
 *   B_lp  n x k low-precision, K-major: element (j, p) at B_lp[j*ldb_k + p]
 *   C     m x n FP32 column-major, ldc.
 *   prec  CF_BF16 or CF_F16.  lower != 0: only tiles on or below the
 *         diagonal of C are updated, and inside diagonal tiles only i >= j.
 * k must be a multiple of 64; lda_k, ldb_k multiples of 8 elements; both
 * operand pointers 16-byte aligned.
 * ------------------------------------------------------------------------ */
int cf_schur_update_lp(int m, int n, int k, const void *A_lp, int lda_k,
                       const void *B_lp, int ldb_k, float *C, int ldc,
                       cf_prec prec, int lower, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * CH-3 / LU-5 with FP8 operands (trailing SYRK/GEMM in FP8 e4m3 with
 * per-128 x 128-tile FP32 scales, FP32 accumulation; an addition of this
 * project, the paper has no low-precision update), exposed for testing.
 *
 * cf_quantize_e4m3: src is a rows x k FP32 block, column-major (lds).  For
 * every tile of 128 rows x 128 columns (K-block), scale = amax / 448 (1 for
 * an all-zero tile) and each element becomes the e4m3 code of x * (448 /
 * amax), rounded to nearest even and saturated to +-448.
 *   q       device bytes, K-major: code of (i, p) at q[i*ldq + p]; columns
 *           k .. kpad-1 (kpad = k rounded up to 128) are written as 0;
 *           ldq >= kpad, a multiple of 16
 *   scales  device float, scale of tile (rb, kb) at scales[rb*ld_scales + kb]
 *
 * cf_schur_update_fp8: C -= sum over K-blocks kb of
 *   sA[i/128, kb] * sB[j/128, kb] * (qA_kb qB_kb^T)
 * on the tensor cores (tcgen05 kind::f8f6f4, one TMEM accumulator per
 * K-block, promoted into FP32 with its tile-pair scale).  k a multiple of
 * 128; ldqa, ldqb multiples of 16 bytes; qA, qB 16-byte aligned; lower as
 * in cf_schur_update_lp.  A device wait that expires is reported by
 * cf_device_status.
 * ------------------------------------------------------------------------ */
/* Split-K form of cf_schur_update_lp (the paper's split of the reduction
 * dimension over processors, Sec. 7.1-7.2, at the scale of one GPU: when the
 * output has too few 128 x 256 tiles to occupy every SM, K is cut into
 * ksplit ranges that run as separate work units).  Each unit writes its FP32
 * partial product to work; then C -= the sum of the partials, added in range
 * order, so the result does not depend on the order the units ran in (it
 * differs from the one-range result by the rounding of the FP32 partial
 * sums).  ksplit in 1..64 (1: the plain update; more ranges than K blocks of
 * 64 are merged); work: cf_schur_update_lp_splitk_workspace_size(m, n, k,
 * ksplit) bytes (0 for ksplit = 1).  Other arguments and errors as
 * cf_schur_update_lp; -12 for ksplit out of range. */
size_t cf_schur_update_lp_splitk_workspace_size(int m, int n, int k, int ksplit);
int cf_schur_update_lp_splitk(int m, int n, int k, const void *A_lp, int lda_k,
                              const void *B_lp, int ldb_k, float *C, int ldc,
                              cf_prec prec, int lower, int ksplit, void *work,
                              size_t lwork, cudaStream_t stream);

int cf_quantize_e4m3(int rows, int k, const float *src, int lds, void *q,
                     int ldq, float *scales, int ld_scales,
                     cudaStream_t stream);
int cf_schur_update_fp8(int m, int n, int k, const void *qA, int ldqa,
                        const float *sA, int ldsa, const void *qB, int ldqb,
                        const float *sB, int ldsb, float *C, int ldc,
                        int lower, cudaStream_t stream);

/* Synchronises `stream` and returns, then clears, the status words of the
 * library's bounded device-side waits: CF_OK, or CF_ERR_TIMEOUT if a wait ran
 * out since the last call (the tensor-core kernels' waits on their TMA and
 * MMA barriers, the blocked triangular solves' waits on earlier blocks).  A
 * wait that runs out ends its kernel early or lets it finish with wrong
 * values; it never hangs, and the context stays usable.  The mixed solvers
 * read and clear these words themselves and return CF_ERR_TIMEOUT. */
int cf_device_status(cudaStream_t stream);

/* ------------------------------------------------------------------------
 * S-1 with FP32 factors: the blocked triangular solve that the mixed
 * solvers' refinement runs (paper silent; substitution by 128-row blocks).
 *   mode  0: X <- L^-1 X, L unit lower (the strictly lower part of T is
 *         read); 1: X <- U^-1 X, U upper; 2: X <- L^-1 X, L lower non-unit;
 *         3: X <- L^-T X, L lower non-unit.
 *   T     n x n FP32, ldt (read only); X n x nrhs FP32, ldx, nrhs <= 16,
 *         overwritten by the solution.
 *   work  cf_trsv_f32_workspace_size(n) bytes (inverses of the 128 x 128
 *         diagonal blocks, block flags).
 * The launch's CTAs take tickets in launch order and wait (bounded) only for
 * blocks with earlier tickets.
 * ------------------------------------------------------------------------ */
size_t cf_trsv_f32_workspace_size(int n);
int cf_trsv_f32(int mode, int n, int nrhs, const float *T, int ldt, float *X,
                int ldx, void *work, size_t lwork, cudaStream_t stream);

/* Failure-detection test of the bounded waits (no GPU fault, no hang): the
 * same solve with the first block withheld -- its ticket is taken before
 * the launch, so no CTA ever solves block 0 or raises its flag.  Every
 * CTA's wait for block 0 gives up after spin_limit polls (0 = the library's
 * limit, 2^22 polls of at least 20 ns), records CF_ERR_TIMEOUT for
 * cf_device_status, and the CTA goes on, so the kernel ends with X wrong.
 * Arguments as cf_trsv_f32; spin_limit < 0 returns -8. */
int cf_trsv_f32_withheld(int mode, int n, int nrhs, const float *T, int ldt,
                         float *X, int ldx, long long spin_limit, void *work,
                         size_t lwork, cudaStream_t stream);

/* ------------------------------------------------------------------------
 * BAT-1  Batched uneven factorizations in one persistent launch (an addition
 * of this project; the paper's small-N regime, Sec. 9).  All per-matrix arguments are DEVICE
 * arrays of length batch: n[i] (0 <= n[i] <= 512), lda[i], A[i] (device
 * pointer to an n x n column-major matrix), ipiv[i] (device int[n[i]]),
 * info[i].  kind[i] = 0 for LU (tournament rule with one leaf per panel, i.e.
 * partial pivoting, block size min(v, 32)), 1 for Cholesky (lower); kind ==
 * NULL means every matrix has default_kind.  ipiv may be NULL only when every
 * matrix is Cholesky by default (kind NULL, default_kind 1); otherwise it and
 * each LU matrix's ipiv[i] must be valid.  A NULL array argument returns its
 * own (negative) position.  One CTA factors one matrix at a
 * time (opt->batch_cps CTAs per SM; cf_batched_autotune picks it and v);
 * matrices are taken longest-first (decreasing n).  info[i] = -1 for
 * n[i] > 512.  Capturable in a CUDA graph (no host synchronisation, no
 * allocation); the workspace size depends on opt.
 * ------------------------------------------------------------------------ */
size_t cf_factor_batched_workspace_size(int batch, const cf_options *opt);
int cf_factor_batched(int batch, const int *kind, int default_kind,
                      const int *n, double *const *A, const int *lda,
                      int *const *ipiv, int *info, void *work, size_t lwork,
                      const cf_options *opt, cudaStream_t stream);
size_t cf_getrf_batched_workspace_size(int batch, const cf_options *opt);
int cf_getrf_batched(int batch, const int *n, double *const *A,
                     const int *lda, int *const *ipiv, int *info, void *work,
                     size_t lwork, const cf_options *opt, cudaStream_t stream);
size_t cf_potrf_batched_workspace_size(int batch, const cf_options *opt);
int cf_potrf_batched(int batch, const int *n, double *const *A,
                     const int *lda, int *info, void *work, size_t lwork,
                     const cf_options *opt, cudaStream_t stream);

/* Batched mixed-precision solve A_i x_i = b_i (one right-hand side each):
 * each matrix is factored in FP32 (same rule as above) in the CTA's own
 * scratch and its solution refined in FP64 (residual b - A x in FP64,
 * eta = ||r||_inf / (||A||_inf ||x||_inf + ||b||_inf)) until
 * eta <= opt->tol.  If the FP32 factorization breaks down, or eta does not
 * at least halve in one step, or opt->max_iter steps pass, that matrix is
 * refactored in FP64 and refined on (at most opt->max_iter more steps), the
 * per-matrix form of LAPACK dsgesv's fallback.  All in one launch.
 * A_i, b_i are not modified; X[i] (device double[n[i]]) receives x_i;
 * iters[i], eta[i] (device) the refinement steps and final backward error
 * (eta[i] > tol means not converged); info[i] = k > 0 if the FP64
 * factorization met a zero (LU) or non-positive (Cholesky) pivot at step k,
 * -1 if n[i] > 512.  solver (device, may be NULL): 32 or 64, the precision
 * of the factors that produced x_i. */
size_t cf_solve_batched_mixed_workspace_size(int batch, const cf_options *opt);
int cf_solve_batched_mixed(int batch, const int *kind, int default_kind,
                           const int *n, const double *const *A,
                           const int *lda, const double *const *B,
                           double *const *X, int *info, int *iters,
                           double *eta, int *solver, void *work, size_t lwork,
                           const cf_options *opt, cudaStream_t stream);

/* BAT-1 autotuner (block size and schedule chosen by measurement; no
 * counterpart in the paper).  Times every candidate block size
 * v in {8, 16, 32} with every resident-CTA count the hardware allows on up to
 * 512 synthetic matrices whose sizes are an evenly spaced sample of
 * n_host[0..batch) (host array; kind_host may be NULL: default_kind), for
 * the FP64 factorization (mixed = 0) or the mixed solve (mixed = 1), and
 * writes the fastest into opt->v and opt->batch_cps (opt is in/out, host;
 * its other fields are used as given).  best_ms (host, may be NULL) gets the
 * sample's time.  Synchronises `stream`.  The batch's own matrices are not
 * touched. */
size_t cf_batched_autotune_workspace_size(int batch, const int *n_host,
                                          const int *kind_host,
                                          int default_kind, int mixed);
int cf_batched_autotune(int batch, const int *n_host, const int *kind_host,
                        int default_kind, int mixed, void *work,
                        size_t lwork, cf_options *opt, float *best_ms,
                        cudaStream_t stream);

/* ------------------------------------------------------------------------
 * Mixed-precision refined solves (an addition of this project; the paper
 * cites GPU mixed LU + refinement as related work, Sec. 11).  A and B are never modified.
 * cf_posv_mixed factors the lower triangle but forms residuals with all of
 * A, which must hold both triangles.
 *   factor_prec  CF_BF16, CF_F16 or CF_BF16X3 (also CF_FP8E4M3 for
 *                cf_posv_mixed)
 *   X            n x nrhs FP64 solution, ldx
 *   info         device int[1], info of the low-precision factorization
 *   stats        host cf_refine_stats (may be NULL)
 * Refinement: classical (x += M^{-1} r with the FP32 factors M) while each
 * step cuts eta by at least 0.3x; after the first step that does not, GMRES-IR
 * (left-preconditioned GMRES with M, restart opt->gmres_restart) for every
 * remaining step.  Residuals and GMRES products with A: on the tensor cores
 * (cf_residual_tc, the digit slices of A cut once per solve) by default;
 * with opt->residual_kind = 2, in pair arithmetic (cf_residual_pair) while
 * the backward error predicted from the last two steps is at least 1e-12,
 * else in FP64 (a pair-arithmetic eta below 1e-12 is recomputed in FP64
 * before it is used, so convergence to tol < 1e-12 is decided on an FP64
 * residual), GMRES products in pair arithmetic; opt->fp64_residual = 1 takes
 * every product in FP64.
 * If refinement stalls (max_iter steps, a GMRES-IR step that fails to halve
 * eta or, with 16-bit factors, needs 12 or more inner steps to cut it by less
 * than 100x, or a breakdown of the low-precision factorization), the
 * matrix is refactored once with CF_BF16X3 updates and refinement continues
 * from the best iterate with a fresh step budget (stats->escalated = 1).
 * Returns CF_ERR_NOT_CONVERGED if that also stalls (max_iter more steps, or
 * two GMRES-IR steps in a row that fail to halve eta; X then holds the best
 * iterate and stats->eta its backward error).
 * ------------------------------------------------------------------------ */
size_t cf_gesv_mixed_workspace_size(int n, int nrhs, cf_prec factor_prec,
                                    const cf_options *opt);
int cf_gesv_mixed(int n, int nrhs, const double *A, int lda, const double *B,
                  int ldb, double *X, int ldx, cf_prec factor_prec, int *info,
                  cf_refine_stats *stats, void *work, size_t lwork,
                  const cf_options *opt, cudaStream_t stream);
size_t cf_posv_mixed_workspace_size(int n, int nrhs, cf_prec factor_prec,
                                    const cf_options *opt);
int cf_posv_mixed(int n, int nrhs, const double *A, int lda, const double *B,
                  int ldb, double *X, int ldx, cf_prec factor_prec, int *info,
                  cf_refine_stats *stats, void *work, size_t lwork,
                  const cf_options *opt, cudaStream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* CF_H */
