/*
 * cf_oracle.c -- plain, slow, FP64 CPU oracle for the COnfLUX / COnfCHOX hot
 * path (Kwasniewski et al., "On the Parallel I/O Optimality of Linear Algebra
 * Kernels: Near-Optimal Matrix Factorizations", SC'21, arXiv 2108.09337).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; it shares no code with the CUDA path.  It is compiled
 * with -O2 -ffp-contract=off so that every multiply and every subtract is a
 * separately rounded IEEE-754 binary64 operation (no FMA contraction), on x86
 * and on Arm alike.
 *
 * Storage: column-major, element (i,j) of a matrix with leading dimension ld
 * is X[i + j*ld].  Row and column indices are 0-based; ipiv is 1-based
 * (LAPACK convention).
 *
 * What each function follows:
 *   gepp_select        -- the local candidate choice of a tournament block:
 *                         each block runs a pivoted LU on its own rows and
 *                         keeps the rows it pivots on (Sec. 7.3, TournPivot,
 *                         and the pivot selection in the I/O-cost proof), realised as
 *                         unblocked Gaussian elimination with partial
 *                         pivoting.
 *   or_tourn_select    -- TournPivot (Alg. 1, Sec. 7.3): local
 *                         candidates on every leaf, then playoff rounds on
 *                         stacked candidate blocks until v winners remain.
 *   or_getrf           -- COnfLUX (Alg. 1): per step, TournPivot, then
 *                         Factorize A00 / A10 / A01 / A11 (Sec. 7.2, Table 2),
 *                         i.e. the column scaling A[i,k] /= A[k,k] and the
 *                         update A[i,j] -= A[i,k]*A[k,j] of the in-place LU
 *                         (Fig. "prog_rep", Sec. 6.1) applied to the
 *                         row-permuted matrix.
 *   or_potrf           -- Listing "Cholesky Factorization" (Sec. 6.2): the
 *                         pivot's square root, the column scaling and the
 *                         trailing update, on the lower triangle.
 *   or_getrs/or_potrs  -- forward and back substitution with the factors
 *                         (the paper is silent; plain textbook definition).
 *   or_residual        -- R = B - A*X with the compensated dot product Dot2 of
 *                         Ogita, Rump and Oishi (SIAM J. Sci. Comput. 26(6),
 *                         2005), so the residual is about twice as accurate
 *                         as a plain FP64 product.
 *
 * Readings of points the paper leaves open (each is also listed in the
 * design notes of the repository):
 *   - argmax ties: the candidate with the smallest position in the stacked
 *     block (its position before any elimination) wins; a NaN entry ranks
 *     below every number (NaN inputs are outside the contract; this only
 *     keeps the selection well defined);
 *   - tree: leaves are h consecutive rows of the current panel (the last leaf
 *     is shorter); each playoff node stacks the winners of `arity` adjacent
 *     children in child order; a group with a single child passes through;
 *   - a playoff node eliminates on the ORIGINAL (pre-elimination) panel
 *     values of its candidate rows;
 *   - a block with fewer rows than columns selects as many rows as it has;
 *   - the rows that remain after a step keep their physical order after the
 *     row swaps (the GPU swaps rows instead of masking them);
 *   - an exactly zero pivot in A00 sets info to its 1-based column (first
 *     occurrence) and the division by it is skipped, as LAPACK dgetf2 does.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define IX(i, j, ld) ((size_t)(i) + (size_t)(j) * (size_t)(ld))

/* ------------------------------------------------------------------------ */
/* Masked GEPP on a stacked candidate block.                                 */
/*                                                                           */
/* S is r x w (column-major, leading dimension lds) and is overwritten.      */
/* Rows are never physically swapped: a chosen row is marked as used and the */
/* rank-1 update touches the unused rows only, which selects exactly the     */
/* rows GEPP with row interchanges selects (up to the tie rule above).       */
/* order[j] = stacked index of the j-th pivot, j < min(r, w).                */
/* *min_gap = min over columns of 1 - |2nd largest| / |largest| among the    */
/* unused rows (1 when one row is left, 0 when the largest is 0).            */
/* Returns the number of pivots, min(r, w).                                  */
/* ------------------------------------------------------------------------ */
static int gepp_select(int r, int w, double *S, int lds, int *order,
                       double *min_gap)
{
    int npiv = r < w ? r : w;
    char *used = (char *)calloc((size_t)(r > 0 ? r : 1), 1);
    double gmin = 1.0;
    for (int j = 0; j < npiv; ++j) {
        int best = -1;
        double bestv = -1.0, second = -1.0;
        for (int i = 0; i < r; ++i) {
            if (used[i]) continue;
            double a = fabs(S[IX(i, j, lds)]);
            if (a != a) a = -0.5;       /* NaN ranks below every number */
            if (a > bestv) {            /* strict: ties keep the smaller i */
                second = bestv;
                bestv = a;
                best = i;
            } else if (a > second) {
                second = a;
            }
        }
        if (best < 0) best = 0;         /* unreachable for j < r */
        double gap;
        if (second < 0.0) gap = 1.0;    /* a single candidate left */
        else if (bestv > 0.0) gap = 1.0 - second / bestv;
        else gap = 0.0;
        if (gap < gmin) gmin = gap;
        order[j] = best;
        used[best] = 1;
        double piv = S[IX(best, j, lds)];
        if (piv != 0.0) {
            for (int i = 0; i < r; ++i) {
                if (used[i]) continue;
                double l = S[IX(i, j, lds)] / piv;
                for (int k = j + 1; k < w; ++k)
                    S[IX(i, k, lds)] = S[IX(i, k, lds)] - l * S[IX(best, k, lds)];
            }
        }
        /* piv == 0: every unused entry of column j is 0 as well; nothing to
           eliminate. */
    }
    free(used);
    if (min_gap) *min_gap = gmin;
    return npiv;
}

/* Copy the rows rows[0..cnt-1] of the panel P (m x w, ldp) into a stacked
 * block S (cnt x w, lds = cnt) and run gepp_select; write the selected panel
 * row indices to out[] in pivot order.  Returns the number selected. */
static int select_from_rows(const double *P, int ldp, int w, const int *rows,
                            int cnt, int *out, double *gap)
{
    double *S = (double *)malloc(sizeof(double) * (size_t)cnt * (size_t)w + 8);
    int *order = (int *)malloc(sizeof(int) * (size_t)(cnt + 1));
    for (int k = 0; k < w; ++k)
        for (int i = 0; i < cnt; ++i)
            S[IX(i, k, cnt)] = P[IX(rows[i], k, ldp)];
    int np = gepp_select(cnt, w, S, cnt, order, gap);
    for (int j = 0; j < np; ++j) out[j] = rows[order[j]];
    free(order);
    free(S);
    return np;
}

/* ------------------------------------------------------------------------ */
/* TournPivot on an m x w panel P (column-major, ldp).                       */
/* winners[0..min(m,w)-1] receives panel row indices in pivot order.         */
/* h >= 1 is the leaf height, arity >= 2 the number of children per playoff  */
/* node.  *min_gap is the smallest gap seen at any column of any node.       */
/* Returns min(m, w).                                                        */
/* ------------------------------------------------------------------------ */
int or_tourn_select(int m, int w, const double *P, int ldp, int h, int arity,
                    int *winners, double *min_gap)
{
    if (m <= 0 || w <= 0) {
        if (min_gap) *min_gap = 1.0;
        return 0;
    }
    if (h < 1) h = 1;
    if (arity < 2) arity = 2;
    int nnodes = (m + h - 1) / h;
    /* Each node keeps at most w candidates. */
    int *cand = (int *)malloc(sizeof(int) * (size_t)nnodes * (size_t)w);
    int *cnt = (int *)malloc(sizeof(int) * (size_t)nnodes);
    int *rows = (int *)malloc(sizeof(int) * (size_t)(h > arity * w ? h : arity * w));
    double gmin = 1.0, g;

    /* Leaves: local candidates of h consecutive rows. */
    for (int l = 0; l < nnodes; ++l) {
        int r0 = l * h, r1 = r0 + h < m ? r0 + h : m;
        for (int i = r0; i < r1; ++i) rows[i - r0] = i;
        cnt[l] = select_from_rows(P, ldp, w, rows, r1 - r0,
                                  cand + (size_t)l * w, &g);
        if (g < gmin) gmin = g;
    }
    /* Playoff rounds. */
    while (nnodes > 1) {
        int nnext = (nnodes + arity - 1) / arity;
        for (int gidx = 0; gidx < nnext; ++gidx) {
            int c0 = gidx * arity;
            int c1 = c0 + arity < nnodes ? c0 + arity : nnodes;
            if (c1 - c0 == 1) {         /* single child: passes through */
                if (gidx != c0) {
                    memmove(cand + (size_t)gidx * w, cand + (size_t)c0 * w,
                            sizeof(int) * (size_t)cnt[c0]);
                }
                cnt[gidx] = cnt[c0];
                continue;
            }
            int tot = 0;
            for (int c = c0; c < c1; ++c)
                for (int q = 0; q < cnt[c]; ++q)
                    rows[tot++] = cand[(size_t)c * w + q];
            cnt[gidx] = select_from_rows(P, ldp, w, rows, tot,
                                         cand + (size_t)gidx * w, &g);
            if (g < gmin) gmin = g;
        }
        nnodes = nnext;
    }
    int np = cnt[0];
    memcpy(winners, cand, sizeof(int) * (size_t)np);
    free(rows);
    free(cnt);
    free(cand);
    if (min_gap) *min_gap = gmin;
    return np;
}

static void swap_rows(int n, double *A, int lda, int r1, int r2)
{
    if (r1 == r2) return;
    for (int j = 0; j < n; ++j) {
        double t = A[IX(r1, j, lda)];
        A[IX(r1, j, lda)] = A[IX(r2, j, lda)];
        A[IX(r2, j, lda)] = t;
    }
}

/* ------------------------------------------------------------------------ */
/* COnfLUX LU with tournament pivoting (Alg. 1), in place.                   */
/*   A (n x n, lda) -> L (unit lower, below diagonal) and U (upper).         */
/*   ipiv[0..n-1]: row i was interchanged with row ipiv[i]-1, i = 0..n-1.    */
/*   *info: 0, or the 1-based column of the first exactly-zero pivot.        */
/*   step_gap[t] (optional, ceil(n/v) entries): smallest tournament gap of   */
/*   step t.  *n_upd (optional): number of updates A[i,j] -= A[i,k]A[k,j]. */
/* Returns 0, or -1 on a bad argument.                                       */
/* ------------------------------------------------------------------------ */
int or_getrf(int n, double *A, int lda, int v, int h, int arity, int *ipiv,
             int *info, double *step_gap, long long *n_upd)
{
    if (n < 0 || lda < (n > 1 ? n : 1) || v < 1) return -1;
    *info = 0;
    long long nupd = 0;
    int *win = (int *)malloc(sizeof(int) * (size_t)(v + 1));
    int *rowat = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    int *where = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    for (int k0 = 0, t = 0; k0 < n; k0 += v, ++t) {
        int w = v < n - k0 ? v : n - k0;
        int m = n - k0;
        double gap = 1.0;

        /* Step 2: TournPivot on the current panel A[k0:n, k0:k0+w]. */
        or_tourn_select(m, w, &A[IX(k0, k0, lda)], lda, h, arity, win, &gap);
        if (step_gap) step_gap[t] = gap;

        /* Bring the winners to the top in pivot order (row interchanges on
           all n columns; the paper masks instead, which a single copy of the
           matrix does not need). */
        for (int p = 0; p < m; ++p) { rowat[p] = p; where[p] = p; }
        for (int j = 0; j < w; ++j) {
            int lab = win[j];
            int p = where[lab];
            ipiv[k0 + j] = k0 + p + 1;
            if (p != j) {
                swap_rows(n, A, lda, k0 + j, k0 + p);
                int lj = rowat[j];
                rowat[j] = lab; where[lab] = j;
                rowat[p] = lj;  where[lj] = p;
            }
        }

        int ke = k0 + w;
        /* Factorize A00: scaling and update inside the w x w diagonal block. */
        for (int k = k0; k < ke; ++k) {
            double piv = A[IX(k, k, lda)];
            if (piv == 0.0) {
                if (*info == 0) *info = k + 1;
            } else {
                for (int i = k + 1; i < ke; ++i)
                    A[IX(i, k, lda)] = A[IX(i, k, lda)] / piv;
            }
            for (int j = k + 1; j < ke; ++j) {
                double akj = A[IX(k, j, lda)];
                for (int i = k + 1; i < ke; ++i)
                    A[IX(i, j, lda)] = A[IX(i, j, lda)] - A[IX(i, k, lda)] * akj;
            }
            nupd += (long long)(ke - k - 1) * (ke - k - 1);
        }
        /* Factorize A10: A10 <- A10 * U00^{-1} (scaling and update, rows below). */
        #pragma omp parallel for schedule(static)
        for (int i = ke; i < n; ++i) {
            for (int k = k0; k < ke; ++k) {
                double piv = A[IX(k, k, lda)];
                if (piv != 0.0) A[IX(i, k, lda)] = A[IX(i, k, lda)] / piv;
                double lik = A[IX(i, k, lda)];
                for (int j = k + 1; j < ke; ++j)
                    A[IX(i, j, lda)] = A[IX(i, j, lda)] - lik * A[IX(k, j, lda)];
            }
        }
        /* Factorize A01: A01 <- L00^{-1} * A01 (update on the pivot rows). */
        #pragma omp parallel for schedule(static)
        for (int j = ke; j < n; ++j) {
            for (int k = k0; k < ke; ++k) {
                double akj = A[IX(k, j, lda)];
                for (int i = k + 1; i < ke; ++i)
                    A[IX(i, j, lda)] = A[IX(i, j, lda)] - A[IX(i, k, lda)] * akj;
            }
        }
        /* Factorize A11: A11 <- A11 - A10 * A01 (update on the trailing block,
           one k at a time in increasing order, as in the unblocked loop). */
        #pragma omp parallel for schedule(static)
        for (int j = ke; j < n; ++j) {
            for (int k = k0; k < ke; ++k) {
                double akj = A[IX(k, j, lda)];
                for (int i = ke; i < n; ++i)
                    A[IX(i, j, lda)] = A[IX(i, j, lda)] - A[IX(i, k, lda)] * akj;
            }
        }
        for (int k = k0; k < ke; ++k)
            nupd += (long long)(n - ke) * (ke - k - 1) * 2   /* A10 and A01 */
                  + (long long)(n - ke) * (n - ke);          /* A11 */
    }
    free(where);
    free(rowat);
    free(win);
    if (n_upd) *n_upd = nupd;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Cholesky, Listing "Cholesky Factorization" (Sec. 6.2), lower, in place.   */
/* Only the lower triangle (i >= j) is read and written.                     */
/* *info: 0, or k+1 for the first k whose pivot is <= 0 or NaN (the         */
/* factorization stops there, as LAPACK dpotrf does).                        */
/* *n_upd (optional): number of trailing updates A[i,j] -= A[i,k]A[j,k].    */
/* ------------------------------------------------------------------------ */
int or_potrf(int n, double *A, int lda, int *info, long long *n_upd)
{
    if (n < 0 || lda < (n > 1 ? n : 1)) return -1;
    *info = 0;
    long long nupd = 0;
    for (int k = 0; k < n; ++k) {
        double d = A[IX(k, k, lda)];
        if (!(d > 0.0)) {               /* also catches NaN */
            *info = k + 1;
            break;
        }
        double lkk = sqrt(d);                               /* pivot */
        A[IX(k, k, lda)] = lkk;
        for (int i = k + 1; i < n; ++i)                     /* scaling */
            A[IX(i, k, lda)] = A[IX(i, k, lda)] / lkk;
        /* Update: the trailing lower triangle loses the outer product of the new
           column, a_ij - l_ik l_jk for k < j <= i; the loop order over (i, j)
           within one k does not change any element's arithmetic. */
        #pragma omp parallel for schedule(dynamic, 16)
        for (int j = k + 1; j < n; ++j) {
            double ljk = A[IX(j, k, lda)];
            for (int i = j; i < n; ++i)
                A[IX(i, j, lda)] = A[IX(i, j, lda)] - A[IX(i, k, lda)] * ljk;
        }
        nupd += (long long)(n - k - 1) * (n - k) / 2;
    }
    if (n_upd) *n_upd = nupd;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Solves with the factors.                                                  */
/* ------------------------------------------------------------------------ */
/* getrs: B <- A^{-1} B with A = P^T L U from or_getrf. */
int or_getrs(int n, int nrhs, const double *LU, int lda, const int *ipiv,
             double *B, int ldb)
{
    if (n < 0 || nrhs < 0) return -1;
    for (int c = 0; c < nrhs; ++c) {
        double *b = B + (size_t)c * ldb;
        for (int i = 0; i < n; ++i) {           /* apply the interchanges */
            int p = ipiv[i] - 1;
            if (p != i) { double t = b[i]; b[i] = b[p]; b[p] = t; }
        }
        for (int k = 0; k < n; ++k)             /* L y = P b, unit L */
            for (int i = k + 1; i < n; ++i)
                b[i] = b[i] - LU[IX(i, k, lda)] * b[k];
        for (int k = n - 1; k >= 0; --k) {      /* U x = y */
            b[k] = b[k] / LU[IX(k, k, lda)];
            for (int i = 0; i < k; ++i)
                b[i] = b[i] - LU[IX(i, k, lda)] * b[k];
        }
    }
    return 0;
}

/* potrs: B <- A^{-1} B with A = L L^T from or_potrf. */
int or_potrs(int n, int nrhs, const double *L, int lda, double *B, int ldb)
{
    if (n < 0 || nrhs < 0) return -1;
    for (int c = 0; c < nrhs; ++c) {
        double *b = B + (size_t)c * ldb;
        for (int k = 0; k < n; ++k) {           /* L y = b */
            b[k] = b[k] / L[IX(k, k, lda)];
            for (int i = k + 1; i < n; ++i)
                b[i] = b[i] - L[IX(i, k, lda)] * b[k];
        }
        for (int k = n - 1; k >= 0; --k) {      /* L^T x = y */
            double s = b[k];
            for (int i = k + 1; i < n; ++i)
                s = s - L[IX(i, k, lda)] * b[i];
            b[k] = s / L[IX(k, k, lda)];
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Residual R = B - A X, compensated (Dot2, Ogita-Rump-Oishi 2005).          */
/* Error-free transformations written from their definitions: TwoSum        */
/* (Knuth) and TwoProduct via Veltkamp splitting (Dekker), which need no FMA */
/* and are exact under round-to-nearest without contraction.                 */
/* ------------------------------------------------------------------------ */
static void two_sum(double a, double b, double *s, double *e)
{
    double x = a + b;
    double z = x - a;
    *e = (a - (x - z)) + (b - z);
    *s = x;
}

static void split(double a, double *hi, double *lo)
{
    const double factor = 134217729.0;          /* 2^27 + 1 */
    double c = factor * a;
    double x = c - (c - a);
    *hi = x;
    *lo = a - x;
}

static void two_prod(double a, double b, double *p, double *e)
{
    double x = a * b;
    double ah, al, bh, bl;
    split(a, &ah, &al);
    split(b, &bh, &bl);
    *e = al * bl - (((x - ah * bh) - al * bh) - ah * bl);
    *p = x;
}

int or_residual(int m, int n, int nrhs, const double *A, int lda,
                const double *X, int ldx, const double *B, int ldb,
                double *R, int ldr)
{
    if (m < 0 || n < 0 || nrhs < 0) return -1;
    #pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i) {
        for (int c = 0; c < nrhs; ++c) {
            double s = B[IX(i, c, ldb)], comp = 0.0;
            for (int j = 0; j < n; ++j) {
                double p, ep, es;
                two_prod(-A[IX(i, j, lda)], X[IX(j, c, ldx)], &p, &ep);
                two_sum(s, p, &s, &es);
                comp = comp + (ep + es);
            }
            R[IX(i, c, ldr)] = s + comp;
        }
    }
    return 0;
}
