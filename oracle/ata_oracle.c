/*
 * Oracle for C = A^t A and for the general product C = X^t Y (test
 * infrastructure only).
 *
 * This file is part of the test oracle.  Only the tests, the smoke check and
 * the CPU-baseline leg of the benchmark may load it; the product path never
 * does.  It shares no code, header or constant with the CUDA library.
 *
 * What it computes is the plain definition of the product the paper's ATA
 * algorithm produces (Section 3, Eq. "Cij" with the four blocks summed back
 * together; Algorithm 1 returns one triangle of it):
 *
 *     C[i][j] = sum_{k=0}^{m-1} A[k][i] * A[k][j],   0 <= i <= j < n,
 *
 * stored as the packed upper triangle in row-major order,
 *
 *     idx(i, j) = i*n - i*(i-1)/2 + (j - i)      (i <= j),
 *
 * which holds n(n+1)/2 entries (Section 3: only one triangle is kept, since
 * A^t A is symmetric).  The row-major packed upper order is the same memory
 * order as the paper's lower triangle read column by column.
 *
 * Arithmetic: IEEE binary64, one accumulator per entry, k ascending, a
 * separate multiply and add (built with -ffp-contract=off), so the result is
 * bit-reproducible for any thread count.  OpenMP only splits the rows i.
 * A is read through a column-major FP64 copy; the copy changes the memory
 * layout, not the arithmetic.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

static int64_t packed_row_start(int64_t i, int64_t n) { return i * n - i * (i - 1) / 2; }

/* Column-major FP64 copy: At[i*m + k] = A[k*lda + i]. Returns NULL on failure. */
static double* column_major_copy(const double* A, int64_t m, int64_t n, int64_t lda, int absval)
{
    size_t cnt = (size_t)m * (size_t)n;
    double* At = (double*)malloc(cnt ? cnt * sizeof(double) : 1);
    if (!At) return NULL;
    for (int64_t k = 0; k < m; ++k)
        for (int64_t i = 0; i < n; ++i) {
            double v = A[k * lda + i];
            At[i * m + k] = absval ? fabs(v) : v;
        }
    return At;
}

/* The definition over one column-major matrix, written into packed upper C. */
static void gram_packed(const double* At, int64_t m, int64_t n, double* C)
{
    int64_t i;
#pragma omp parallel for schedule(dynamic, 1)
    for (i = 0; i < n; ++i) {
        const double* ci = At + i * m;
        double* row = C + packed_row_start(i, n);
        for (int64_t j = i; j < n; ++j) {
            const double* cj = At + j * m;
            double acc = 0.0;
            for (int64_t k = 0; k < m; ++k) acc = acc + ci[k] * cj[k];
            row[j - i] = acc;
        }
    }
}

/* C_packed = A^t A (packed upper).  A is row-major m x n with leading
 * dimension lda >= n.  Returns 0 on success, -1 on bad arguments, -2 if out
 * of memory. */
int oracle_ata_packed(const double* A, int64_t m, int64_t n, int64_t lda, double* C)
{
    if (m < 0 || n < 0 || lda < n || (n > 0 && !C) || (m > 0 && n > 0 && !A)) return -1;
    if (n == 0) return 0;
    double* At = column_major_copy(A, m, n, lda, 0);
    if (!At) return -2;
    gram_packed(At, m, n, C);
    free(At);
    return 0;
}

/* G_packed = |A|^t |A| (packed upper): the denominator of the componentwise
 * error max |C - C_ref| / (|A|^t |A|)_ij. */
int oracle_abs_gram_packed(const double* A, int64_t m, int64_t n, int64_t lda, double* G)
{
    if (m < 0 || n < 0 || lda < n || (n > 0 && !G) || (m > 0 && n > 0 && !A)) return -1;
    if (n == 0) return 0;
    double* At = column_major_copy(A, m, n, lda, 1);
    if (!At) return -2;
    gram_packed(At, m, n, G);
    free(At);
    return 0;
}

/* Selected entries of A^t A: out[t] = sum_k A[k][I[t]] * A[k][J[t]], k
 * ascending, one accumulator, same arithmetic as oracle_ata_packed, so an
 * entry computed here is bitwise equal to the same entry of the full call.
 * Used where the full product is too large for the host (sampled parity).
 * If absval != 0, computes the same entries of |A|^t |A|. */
int oracle_ata_entries(const double* A, int64_t m, int64_t n, int64_t lda,
                       const int64_t* I, const int64_t* J, int64_t count,
                       int absval, double* out)
{
    if (m < 0 || n < 0 || lda < n || count < 0) return -1;
    if (count > 0 && (!I || !J || !out)) return -1;
    for (int64_t t = 0; t < count; ++t)
        if (I[t] < 0 || I[t] >= n || J[t] < 0 || J[t] >= n) return -1;
    int64_t t;
#pragma omp parallel for schedule(dynamic, 16)
    for (t = 0; t < count; ++t) {
        const int64_t ci = I[t], cj = J[t];
        double acc = 0.0;
        for (int64_t k = 0; k < m; ++k) {
            double a = A[k * lda + ci], b = A[k * lda + cj];
            if (absval) { a = fabs(a); b = fabs(b); }
            acc = acc + a * b;
        }
        out[t] = acc;
    }
    return 0;
}

/* Rows [i0, i1) of the packed upper triangle (entries j >= i), written to
 * out in packed order starting at idx(i0, i0).  Same arithmetic as above.
 * Used to time a bounded slice of the full product on the host. */
int oracle_ata_rows(const double* A, int64_t m, int64_t n, int64_t lda,
                    int64_t i0, int64_t i1, double* out)
{
    if (m < 0 || n < 0 || lda < n || i0 < 0 || i1 < i0 || i1 > n) return -1;
    if (i1 == i0) return 0;
    double* At = column_major_copy(A, m, n, lda, 0);
    if (!At) return -2;
    const int64_t base = packed_row_start(i0, n);
    int64_t i;
#pragma omp parallel for schedule(dynamic, 1)
    for (i = i0; i < i1; ++i) {
        const double* ci = At + i * m;
        double* row = out + (packed_row_start(i, n) - base);
        for (int64_t j = i; j < n; ++j) {
            const double* cj = At + j * m;
            double acc = 0.0;
            for (int64_t k = 0; k < m; ++k) acc = acc + ci[k] * cj[k];
            row[j - i] = acc;
        }
    }
    free(At);
    return 0;
}

/* General product C = X^t Y (the HASA step of Section 4.2.2 on two
 * operands; the off-diagonal block C_12 of the recursion is one such
 * product): X is m x p (ldx >= p), Y is m x r (ldy >= r), both row-major;
 * C is p x r row-major with ldc >= r,
 *
 *     C[i][j] = sum_{k=0}^{m-1} X[k][i] * Y[k][j],
 *
 * k ascending, one accumulator per entry, the same arithmetic as the
 * functions above (with X = Y = A the entries j >= i are bitwise those of
 * oracle_ata_packed).  If absval != 0, computes |X|^t |Y| (the denominator
 * of the componentwise error).  Returns 0, -1 on bad arguments, -2 if out of
 * memory. */
int oracle_gemm_tn(const double* X, int64_t m, int64_t p, int64_t ldx,
                   const double* Y, int64_t r, int64_t ldy,
                   double* C, int64_t ldc, int absval)
{
    if (m < 0 || p < 0 || r < 0 || ldx < p || ldy < r || ldc < r) return -1;
    if (p == 0 || r == 0) return 0;
    if (!C || (m > 0 && (!X || !Y))) return -1;
    double* Xt = column_major_copy(X, m, p, ldx, absval);
    double* Yt = column_major_copy(Y, m, r, ldy, absval);
    if (!Xt || !Yt) {
        free(Xt);
        free(Yt);
        return -2;
    }
    int64_t i;
#pragma omp parallel for schedule(dynamic, 1)
    for (i = 0; i < p; ++i) {
        const double* xi = Xt + i * m;
        for (int64_t j = 0; j < r; ++j) {
            const double* yj = Yt + j * m;
            double acc = 0.0;
            for (int64_t k = 0; k < m; ++k) acc = acc + xi[k] * yj[k];
            C[i * ldc + j] = acc;
        }
    }
    free(Xt);
    free(Yt);
    return 0;
}

/* Selected entries of X^t Y (or |X|^t |Y|): out[t] = C[I[t]][J[t]], the same
 * arithmetic as oracle_gemm_tn (sampled parity at sizes too large for the
 * full product on the host). */
int oracle_gemm_entries(const double* X, int64_t m, int64_t p, int64_t ldx,
                        const double* Y, int64_t r, int64_t ldy,
                        const int64_t* I, const int64_t* J, int64_t count,
                        int absval, double* out)
{
    if (m < 0 || p < 0 || r < 0 || ldx < p || ldy < r || count < 0) return -1;
    if (count > 0 && (!I || !J || !out)) return -1;
    for (int64_t t = 0; t < count; ++t)
        if (I[t] < 0 || I[t] >= p || J[t] < 0 || J[t] >= r) return -1;
    int64_t t;
#pragma omp parallel for schedule(dynamic, 16)
    for (t = 0; t < count; ++t) {
        double acc = 0.0;
        for (int64_t k = 0; k < m; ++k) {
            double a = X[k * ldx + I[t]], b = Y[k * ldy + J[t]];
            if (absval) { a = fabs(a); b = fabs(b); }
            acc = acc + a * b;
        }
        out[t] = acc;
    }
    return 0;
}

/* Number of OpenMP threads the oracle runs with. */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
