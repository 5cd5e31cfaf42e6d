/* Drives every function of the C oracle over edge-case shapes (n = 0, 1,
 * ragged blocks, leaves of one row, arity 2..4, leading dimensions above the
 * row count, m < w, a zero column, a matrix that is not positive definite)
 * with buffers of exactly the documented sizes, so that a build with
 * -fsanitize=address,undefined stops at the first out-of-bounds access or
 * undefined operation.  Test infrastructure: it checks only that the oracle
 * runs cleanly; its numbers are checked elsewhere. */
#include <stdio.h>
#include <stdlib.h>

int or_tourn_select(int m, int w, const double *P, int ldp, int h, int arity, int *winners, double *min_gap);
int or_getrf(int n, double *A, int lda, int v, int h, int arity, int *ipiv, int *info, double *step_gap,
             long long *n_upd);
int or_potrf(int n, double *A, int lda, int *info, long long *n_upd);
int or_getrs(int n, int nrhs, const double *LU, int lda, const int *ipiv, double *B, int ldb);
int or_potrs(int n, int nrhs, const double *L, int lda, double *B, int ldb);
int or_residual(int m, int n, int nrhs, const double *A, int lda, const double *X, int ldx, const double *B, int ldb,
                double *R, int ldr);

static unsigned long long g_state = 88172645463325252ull;
static double uni(void) {            /* xorshift64, uniform in [-1, 1) */
    g_state ^= g_state << 13;
    g_state ^= g_state >> 7;
    g_state ^= g_state << 17;
    return (double)(g_state >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

static double *mat(int rows, int cols, int ld) {
    size_t sz = (size_t)ld * (size_t)(cols > 0 ? cols : 1);
    double *a = (double *)malloc(sizeof(double) * sz);
    for (size_t i = 0; i < sz; ++i) a[i] = uni();
    (void)rows;
    return a;
}

static int fails = 0;
#define CHECK(c) do { if (!(c)) { fprintf(stderr, "check failed: %s (line %d)\n", #c, __LINE__); ++fails; } } while (0)

int main(void) {
    /* tournament selection alone */
    const int shapes[][4] = {{1, 1, 1, 2}, {5, 8, 2, 2}, {17, 4, 1, 2}, {33, 7, 5, 3}, {100, 16, 7, 4},
                             {129, 128, 128, 2}, {300, 17, 40, 3}, {64, 64, 3, 4}};
    for (size_t s = 0; s < sizeof(shapes) / sizeof(shapes[0]); ++s) {
        const int m = shapes[s][0], w = shapes[s][1], h = shapes[s][2], ar = shapes[s][3];
        const int ldp = m + 3, np = m < w ? m : w;
        double *P = mat(m, w, ldp), gap = 0.0;
        int *win = (int *)malloc(sizeof(int) * (size_t)np);
        CHECK(or_tourn_select(m, w, P, ldp, h, ar, win, &gap) == np);
        for (int i = 0; i < np; ++i) CHECK(win[i] >= 0 && win[i] < m);
        free(win);
        free(P);
    }
    CHECK(or_tourn_select(0, 4, NULL, 1, 8, 2, NULL, NULL) == 0);

    /* LU, solves, residual */
    const int lu[][4] = {{1, 1, 1, 2}, {2, 1, 1, 2}, {3, 2, 128, 2}, {7, 3, 2, 3}, {33, 8, 5, 4},
                         {65, 32, 16, 2}, {130, 128, 128, 2}, {97, 16, 1, 2}};
    for (size_t s = 0; s < sizeof(lu) / sizeof(lu[0]); ++s) {
        const int n = lu[s][0], v = lu[s][1], h = lu[s][2], ar = lu[s][3];
        const int lda = n + 2, nrhs = 3, ldb = n + 1, steps = (n + v - 1) / v;
        double *A = mat(n, n, lda), *A0 = (double *)malloc(sizeof(double) * (size_t)lda * n);
        for (size_t i = 0; i < (size_t)lda * n; ++i) A0[i] = A[i];
        int *ipiv = (int *)malloc(sizeof(int) * (size_t)n), info = -1;
        double *gaps = (double *)malloc(sizeof(double) * (size_t)steps);
        long long nupd = 0;
        CHECK(or_getrf(n, A, lda, v, h, ar, ipiv, &info, gaps, &nupd) == 0);
        for (int i = 0; i < n; ++i) CHECK(ipiv[i] >= i + 1 && ipiv[i] <= n);
        double *B = mat(n, nrhs, ldb), *X = (double *)malloc(sizeof(double) * (size_t)ldb * nrhs);
        double *R = (double *)malloc(sizeof(double) * (size_t)(n + 4) * nrhs);
        for (size_t i = 0; i < (size_t)ldb * nrhs; ++i) X[i] = B[i];
        if (info == 0) CHECK(or_getrs(n, nrhs, A, lda, ipiv, X, ldb) == 0);
        CHECK(or_residual(n, n, nrhs, A0, lda, X, ldb, B, ldb, R, n + 4) == 0);
        free(A); free(A0); free(ipiv); free(gaps); free(B); free(X); free(R);
    }
    {   /* zero column: info set, factorization completes */
        const int n = 9, lda = 9;
        double *A = mat(n, n, lda);
        for (int i = 0; i < n; ++i) A[i + 4 * lda] = 0.0;
        int ipiv[9], info = 0;
        CHECK(or_getrf(n, A, lda, 4, 3, 2, ipiv, &info, NULL, NULL) == 0);
        CHECK(info == 5);
        free(A);
    }
    {   /* rectangular residual */
        const int m = 11, n = 6, nrhs = 2;
        double *A = mat(m, n, m + 1), *X = mat(n, nrhs, n), *B = mat(m, nrhs, m), *R = mat(m, nrhs, m);
        CHECK(or_residual(m, n, nrhs, A, m + 1, X, n, B, m, R, m) == 0);
        CHECK(or_residual(0, 0, 0, NULL, 1, NULL, 1, NULL, 1, NULL, 1) == 0);
        free(A); free(X); free(B); free(R);
    }

    /* Cholesky and its solve */
    const int ch[] = {1, 2, 5, 33, 130};
    for (size_t s = 0; s < sizeof(ch) / sizeof(ch[0]); ++s) {
        const int n = ch[s], lda = n + 1, nrhs = 2;
        double *A = mat(n, n, lda);
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                const double x = 0.5 * (A[i + j * lda] + A[j + i * lda]);
                A[i + j * lda] = x;
                A[j + i * lda] = x;
            }
        for (int i = 0; i < n; ++i) A[i + i * lda] += n;     /* diagonally dominant: SPD */
        int info = -1;
        long long nupd = 0;
        CHECK(or_potrf(n, A, lda, &info, &nupd) == 0);
        CHECK(info == 0);
        double *B = mat(n, nrhs, n);
        CHECK(or_potrs(n, nrhs, A, lda, B, n) == 0);
        free(A); free(B);
    }
    {   /* not positive definite: info = 2 */
        double A[4] = {1.0, 2.0, 2.0, 1.0};
        int info = 0;
        CHECK(or_potrf(2, A, 2, &info, NULL) == 0);
        CHECK(info == 2);
    }
    if (fails) return 1;
    printf("oracle ran cleanly under the sanitizers\n");
    return 0;
}
