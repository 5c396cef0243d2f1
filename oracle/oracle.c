/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct FP64 CPU restatement of what the triangular
 * inversion path computes.  Only the test-suite, the smoke check and the bench's
 * CPU-baseline leg may load it; the product path never does.  It shares no code,
 * header, table or helper with the CUDA library.
 *
 * Storage convention: column-major, element (i, j) of a matrix M with leading
 * dimension ld is M[i + j*ld].  Every triangular routine works on the LOWER view of
 * its input: for an upper-triangular U the lower view is its transpose, because the
 * paper treats one orientation and obtains the other by transposition (Section 2,
 * after Eq. "defT").
 *
 * Compiled with -O2 -ffp-contract=off and without fast-math, so every product and
 * sum is an individually rounded IEEE binary64 operation in the order written here.
 * Threading (OpenMP) only splits independent columns or rows across threads; it never
 * changes the order of the operations that produce any single entry.
 *
 * Functions (with the passage each restates):
 *   oracle_tri_inv       column recurrence of CRIT (Section 4.2, Algorithm "CRIT"),
 *                        transposed to lower form: x_jj = 1/t_jj,
 *                        x_ij = -(1/t_ii) * sum_{k=j}^{i-1} t_ik x_kj.
 *   oracle_tri_inv_cols  the same recurrence for a chosen set of columns only
 *                        (oracle_view_*: the same against a lower view built once).
 *   oracle_crout         Crout LU with unit upper U, row by row as in SKUL
 *                        (Section 5.1, Algorithm "SKUL"): A = L U.
 *   oracle_gen_inv       A^-1 = U^-1 L^-1 from oracle_crout and oracle_tri_inv
 *                        (SKUL: "S K = A^-1"; BRSI with two blocks, Section 5.2).
 *   oracle_skul          Algorithm SKUL (Section 5.1) as printed: Crout L, U with the
 *                        inverse factors K = L^-1 (rows) and S = U^-1 (columns) built
 *                        alongside; A^-1 = S K.
 *   oracle_sqr           Algorithm SQR (Section 5.1): modified Gram-Schmidt A = Q R with
 *                        S = R^-1 built column by column; A^-1 = S Q^T.
 *   oracle_tri_grad      adjoint of X = T^-1 for a loss with cotangent G:
 *                        dT = -P(X^T G X^T), P the projection on T's free entries.
 *                        (Not in the paper; the plain definition from d(T^-1) =
 *                        -T^-1 dT T^-1.)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define AT(M, ld, i, j) ((M)[(int64_t)(i) + (int64_t)(j) * (int64_t)(ld)])

static int set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
    return nthreads;
#else
    (void)nthreads;
    return 1;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Lower view of a triangular matrix as a dense row-major copy: R[i*n + k] = t_ik
 * for k <= i, 0 above.  Only the referenced triangle of T is read.  A unit diagonal
 * is stored as 1 without reading T's diagonal. */
static double *lower_view_rowmajor(int upper, int unit, int64_t n, const double *T, int64_t ld) {
    double *R = (double *)calloc((size_t)(n * n > 0 ? n * n : 1), sizeof(double));
    if (!R) return NULL;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t k = 0; k < i; ++k)
            R[i * n + k] = upper ? AT(T, ld, k, i) : AT(T, ld, i, k);
        R[i * n + i] = unit ? 1.0 : AT(T, ld, i, i);
    }
    return R;
}

/* One column j of the lower inverse: forward substitution of T x = e_j, written as the
 * column recurrence.  R is the row-major lower view; x has length n. */
static void column_recurrence(int64_t n, const double *R, int64_t j, double *x) {
    for (int64_t i = 0; i < j; ++i) x[i] = 0.0;
    x[j] = 1.0 / R[j * n + j];
    for (int64_t i = j + 1; i < n; ++i) {
        const double *ti = R + i * n;
        double acc = 0.0;
        for (int64_t k = j; k < i; ++k) acc += ti[k] * x[k];
        x[i] = -acc / ti[i];
    }
}

/* Index of the first zero or non-finite diagonal entry of the lower view, or -1. */
static int64_t first_bad_pivot(int64_t n, const double *R) {
    for (int64_t i = 0; i < n; ++i) {
        double d = R[i * n + i];
        if (d == 0.0 || !isfinite(d)) return i;
    }
    return -1;
}

/* X = T^-1.  upper: T is upper triangular (X written upper), else lower.  unit: the
 * diagonal of T is taken as 1 and not read.  X receives the full n x n matrix with
 * zeros in the other triangle.  Returns -1, or the first singular pivot index (X is
 * then left unspecified). */
int64_t oracle_tri_inv(int upper, int unit, int64_t n, const double *T, int64_t ldt,
                       double *X, int64_t ldx, int nthreads) {
    if (n <= 0) return -1;
    double *R = lower_view_rowmajor(upper, unit, n, T, ldt);
    if (!R) return -2;
    int64_t bad = first_bad_pivot(n, R);
    if (bad >= 0) { free(R); return bad; }
    int nt = set_threads(nthreads);
    (void)nt;
#pragma omp parallel num_threads(nt)
    {
        double *x = (double *)malloc((size_t)n * sizeof(double));
#pragma omp for schedule(dynamic, 1)
        for (int64_t j = 0; j < n; ++j) {
            column_recurrence(n, R, j, x);
            for (int64_t i = 0; i < n; ++i) {
                if (upper) AT(X, ldx, j, i) = x[i];
                else AT(X, ldx, i, j) = x[i];
            }
        }
        free(x);
    }
    free(R);
    return -1;
}

/* Selected columns of the LOWER-VIEW inverse: out[:, c] = column cols[c] of
 * (lower view of T)^-1, n x ncols column-major with leading dimension n.  For an upper
 * T this is row cols[c] of T^-1. */
int64_t oracle_view_cols(int64_t n, const double *R, int64_t ncols, const int64_t *cols, double *out,
                         int nthreads);

int64_t oracle_tri_inv_cols(int upper, int unit, int64_t n, const double *T, int64_t ldt,
                            int64_t ncols, const int64_t *cols, double *out, int nthreads) {
    if (n <= 0) return -1;
    double *R = lower_view_rowmajor(upper, unit, n, T, ldt);
    if (!R) return -2;
    int64_t bad = oracle_view_cols(n, R, ncols, cols, out, nthreads);
    free(R);
    return bad;
}

/* The same column requests against a lower view prepared once (oracle_view_create), so
 * that repeated requests on one matrix do not rebuild it: the bench's CPU legs time only
 * the column recurrences. */
double *oracle_view_create(int upper, int unit, int64_t n, const double *T, int64_t ldt) {
    return n > 0 ? lower_view_rowmajor(upper, unit, n, T, ldt) : NULL;
}

void oracle_view_free(double *R) { free(R); }

int64_t oracle_view_cols(int64_t n, const double *R, int64_t ncols, const int64_t *cols, double *out,
                         int nthreads) {
    if (n <= 0) return -1;
    if (!R) return -2;
    int64_t bad = first_bad_pivot(n, R);
    if (bad >= 0) return bad;
    int nt = set_threads(nthreads);
    (void)nt;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 1)
    for (int64_t c = 0; c < ncols; ++c) column_recurrence(n, R, cols[c], out + c * n);
    return -1;
}

/* Crout LU in SKUL's row order: for each row i, first L_{i,j} (j <= i) then
 * U_{i,j} (j > i), with L non-unit lower and U unit upper:
 *   L_ij = A_ij - sum_{p<j} L_ip U_pj            (j <= i)
 *   U_ij = (A_ij - sum_{p<i} L_ip U_pj) / L_ii   (j > i)
 * L, U are full n x n column-major outputs (ld n), zero outside their triangles.
 * Returns -1, or the first row whose pivot L_ii is zero or non-finite (no pivoting). */
int64_t oracle_crout(int64_t n, const double *A, int64_t lda, double *L, double *U, int nthreads) {
    if (n <= 0) return -1;
    /* Row-major copy of L and column-major copy of U keep each dot product contiguous. */
    double *Lr = (double *)calloc((size_t)(n * n), sizeof(double));
    double *Uc = (double *)calloc((size_t)(n * n), sizeof(double));
    if (!Lr || !Uc) { free(Lr); free(Uc); return -2; }
    int64_t bad = -1;
    int nt = set_threads(nthreads);
    (void)nt;
    for (int64_t i = 0; i < n && bad < 0; ++i) {
        double *li = Lr + i * n;
        /* L_ij needs L_ip for p < j of the same row: sequential in j. */
        for (int64_t j = 0; j <= i; ++j) {
            const double *uj = Uc + j * n;
            double acc = 0.0;
            for (int64_t p = 0; p < j; ++p) acc += li[p] * uj[p];
            li[j] = AT(A, lda, i, j) - acc;
        }
        double piv = li[i];
        if (piv == 0.0 || !isfinite(piv)) { bad = i; break; }
        Uc[i * n + i] = 1.0;
        /* U_ij needs only row i of L and rows < i of U: independent in j. */
#pragma omp parallel for num_threads(nt) schedule(static) if (n - i > 256)
        for (int64_t j = i + 1; j < n; ++j) {
            double *uj = Uc + j * n;
            double acc = 0.0;
            for (int64_t p = 0; p < i; ++p) acc += li[p] * uj[p];
            uj[i] = (AT(A, lda, i, j) - acc) / piv;
        }
    }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) {
            AT(L, n, i, j) = Lr[i * n + j];
            AT(U, n, i, j) = Uc[j * n + i];
        }
    free(Lr);
    free(Uc);
    return bad;
}

/* A^-1 = U^-1 L^-1 (no pivoting).  X: n x n column-major, ld ldx.  Returns -1 or the
 * first bad pivot. */
int64_t oracle_gen_inv(int64_t n, const double *A, int64_t lda, double *X, int64_t ldx, int nthreads) {
    if (n <= 0) return -1;
    size_t sz = (size_t)(n * n);
    double *L = (double *)malloc(sz * sizeof(double));
    double *U = (double *)malloc(sz * sizeof(double));
    double *K = (double *)malloc(sz * sizeof(double)); /* L^-1, lower */
    double *S = (double *)malloc(sz * sizeof(double)); /* U^-1, unit upper */
    if (!L || !U || !K || !S) { free(L); free(U); free(K); free(S); return -2; }
    int64_t bad = oracle_crout(n, A, lda, L, U, nthreads);
    if (bad < 0) bad = oracle_tri_inv(0, 0, n, L, n, K, n, nthreads);
    if (bad < 0) bad = oracle_tri_inv(1, 1, n, U, n, S, n, nthreads);
    if (bad < 0) {
        /* (S K)_ij = sum_{k >= max(i,j)} S_ik K_kj: S upper, K lower. */
        double *Sr = L; /* reuse: row-major copy of S */
        for (int64_t i = 0; i < n; ++i)
            for (int64_t k = 0; k < n; ++k) Sr[i * n + k] = AT(S, n, i, k);
        int nt = set_threads(nthreads);
        (void)nt;
#pragma omp parallel for num_threads(nt) schedule(dynamic, 4)
        for (int64_t j = 0; j < n; ++j) {
            const double *kj = K + j * n;
            for (int64_t i = 0; i < n; ++i) {
                const double *si = Sr + i * n;
                int64_t k0 = i > j ? i : j;
                double acc = 0.0;
                for (int64_t k = k0; k < n; ++k) acc += si[k] * kj[k];
                AT(X, ldx, i, j) = acc;
            }
        }
    }
    free(L); free(U); free(K); free(S);
    return bad;
}

/* dT = -P(X^T G X^T) where X = T^-1 (triangular, same orientation as T), G the
 * cotangent of X and P keeps T's free entries: the lower triangle for lower T, the
 * upper triangle for upper T, with the diagonal cleared when the diagonal is unit.
 * Computed as the plain two products M = X^T G then (M X^T), restricted to P.
 * All matrices n x n column-major; dT receives zeros outside P. */
void oracle_tri_grad(int upper, int unit, int64_t n, const double *X, int64_t ldx,
                     const double *G, int64_t ldg, double *dT, int64_t ldd, int nthreads) {
    if (n <= 0) return;
    size_t sz = (size_t)(n * n);
    double *M = (double *)malloc(sz * sizeof(double)); /* row-major M[i*n+l] = (X^T G)_il */
    double *Xr = (double *)malloc(sz * sizeof(double)); /* row-major copy of X */
    if (!M || !Xr) { free(M); free(Xr); return; }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t k = 0; k < n; ++k) Xr[i * n + k] = AT(X, ldx, i, k);
    int nt = set_threads(nthreads);
    (void)nt;
    /* M_il = sum_k X_ki G_kl */
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t l = 0; l < n; ++l) {
            const double *gl = G + l * ldg;
            double acc = 0.0;
            for (int64_t k = 0; k < n; ++k) acc += AT(X, ldx, k, i) * gl[k];
            M[i * n + l] = acc;
        }
    }
    /* (M X^T)_ij = sum_l M_il X_jl */
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int64_t j = 0; j < n; ++j) {
        const double *xj = Xr + j * n;
        for (int64_t i = 0; i < n; ++i) {
            int keep = upper ? (i <= j) : (i >= j);
            if (unit && i == j) keep = 0;
            double v = 0.0;
            if (keep) {
                const double *mi = M + i * n;
                double acc = 0.0;
                for (int64_t l = 0; l < n; ++l) acc += mi[l] * xj[l];
                v = -acc;
            }
            AT(dT, ldd, i, j) = v;
        }
    }
    free(M);
    free(Xr);
}

/* Algorithm SKUL (Section 5.1), step by step in the paper's order, 0-based:
 *   L_{i,0} = A_{i,0};  U_ii = S_ii = K_ii = 1;  U_{0,j} = A_{0,j} / L_00;  D_00 = 1/L_00;
 *   for i = 1 .. n-1:
 *     L_ij = A_ij - sum_{p<j} L_ip U_pj                          (1 <= j <= i)
 *     D_ii = 1 / L_ii
 *     K_ij = -(sum_{p=j}^{i-1} L_ip K_pj) D_ii                   (j < i; unit-diagonal K)
 *     U_ij = (A_ij - sum_{p<i} L_ip U_pj) / L_ii                 (j > i)
 *     S_{l,i+1} = -sum_{p=l}^{i} S_lp U_{p,i+1}                  (l <= i, when i < n-1)
 *   (S_{0,1} = -U_{0,1} is the i = 0 case of the last line.)  Finally K <- K D.
 * The row of K is the CRIT recurrence on L run as each row of L appears, and the column
 * of S the CRIT* recurrence on U run as each column of U is complete.
 * Outputs: L, U, S, K full n x n column-major (ld n), zero outside their triangles.
 * Returns -1, the first row whose pivot L_ii is zero or non-finite, or -2 (no memory). */
int64_t oracle_skul(int64_t n, const double *A, int64_t lda, double *L, double *U, double *S, double *K) {
    if (n <= 0) return -1;
    memset(L, 0, sizeof(double) * (size_t)(n * n));
    memset(U, 0, sizeof(double) * (size_t)(n * n));
    memset(S, 0, sizeof(double) * (size_t)(n * n));
    memset(K, 0, sizeof(double) * (size_t)(n * n));
    double *D = (double *)calloc((size_t)n, sizeof(double));
    if (!D) return -2;
    int64_t bad = -1;
    for (int64_t i = 0; i < n; ++i) {
        AT(L, n, i, 0) = AT(A, lda, i, 0);
        AT(U, n, i, i) = 1.0;
        AT(S, n, i, i) = 1.0;
        AT(K, n, i, i) = 1.0;
    }
    double l00 = AT(L, n, 0, 0);
    if (l00 == 0.0 || !isfinite(l00)) { free(D); return 0; }
    for (int64_t j = 1; j < n; ++j) AT(U, n, 0, j) = AT(A, lda, 0, j) / l00;
    D[0] = 1.0 / l00;
    if (n > 1) AT(S, n, 0, 1) = -AT(U, n, 0, 1);
    for (int64_t i = 1; i < n && bad < 0; ++i) {
        for (int64_t j = 1; j <= i; ++j) {
            double acc = 0.0;
            for (int64_t p = 0; p < j; ++p) acc += AT(L, n, i, p) * AT(U, n, p, j);
            AT(L, n, i, j) = AT(A, lda, i, j) - acc;
        }
        const double lii = AT(L, n, i, i);
        if (lii == 0.0 || !isfinite(lii)) { bad = i; break; }
        D[i] = 1.0 / lii;
        for (int64_t j = 0; j < i; ++j) {
            double acc = 0.0;
            for (int64_t p = j; p < i; ++p) acc += AT(L, n, i, p) * AT(K, n, p, j);
            AT(K, n, i, j) = -acc * D[i];
        }
        for (int64_t j = i + 1; j < n; ++j) {
            double acc = 0.0;
            for (int64_t p = 0; p < i; ++p) acc += AT(L, n, i, p) * AT(U, n, p, j);
            AT(U, n, i, j) = (AT(A, lda, i, j) - acc) / lii;
        }
        if (i < n - 1)
            for (int64_t l = 0; l <= i; ++l) {
                double acc = 0.0;
                for (int64_t p = l; p <= i; ++p) acc += AT(S, n, l, p) * AT(U, n, p, i + 1);
                AT(S, n, l, i + 1) = -acc;
            }
    }
    if (bad < 0)
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = j; i < n; ++i) AT(K, n, i, j) *= D[j];
    free(D);
    return bad;
}

/* Algorithm SQR (Section 5.1): modified Gram-Schmidt QR of A with S = R^-1 built one
 * column at a time as the columns of R appear.  0-based, for j = 0 .. n-1:
 *     qh = a_j;  for i < j:  R_ij = qh . q_i;  qh <- qh - R_ij q_i     (MGS)
 *     R_jj = ||qh||_2  (stop if zero);  D_jj = 1/R_jj;  q_j = D_jj qh;  S_jj = 1
 *     S_ij = -(1/R_jj) sum_{p=i}^{j-1} S_ip R_pj                         (i < j)
 *   and finally S <- D S, so that A = Q R and A^-1 = S Q^T.
 * The printed algorithm lists the S update before R_jj although it divides by R_jj; the
 * update is taken after R_jj here.  Outputs full n x n column-major (ld n); Q
 * orthonormal, R and S upper.  Returns -1, the first column j with R_jj zero or
 * non-finite, or -2. */
int64_t oracle_sqr(int64_t n, const double *A, int64_t lda, double *Q, double *R, double *S) {
    if (n <= 0) return -1;
    memset(Q, 0, sizeof(double) * (size_t)(n * n));
    memset(R, 0, sizeof(double) * (size_t)(n * n));
    memset(S, 0, sizeof(double) * (size_t)(n * n));
    double *qh = (double *)malloc(sizeof(double) * (size_t)n);
    double *D = (double *)malloc(sizeof(double) * (size_t)n);
    if (!qh || !D) { free(qh); free(D); return -2; }
    int64_t bad = -1;
    for (int64_t j = 0; j < n && bad < 0; ++j) {
        for (int64_t r = 0; r < n; ++r) qh[r] = AT(A, lda, r, j);
        for (int64_t i = 0; i < j; ++i) {
            double dot = 0.0;
            for (int64_t r = 0; r < n; ++r) dot += qh[r] * AT(Q, n, r, i);
            AT(R, n, i, j) = dot;
            for (int64_t r = 0; r < n; ++r) qh[r] -= dot * AT(Q, n, r, i);
        }
        double ss = 0.0;
        for (int64_t r = 0; r < n; ++r) ss += qh[r] * qh[r];
        const double rjj = sqrt(ss);
        if (rjj == 0.0 || !isfinite(rjj)) { bad = j; break; }
        AT(R, n, j, j) = rjj;
        D[j] = 1.0 / rjj;
        for (int64_t r = 0; r < n; ++r) AT(Q, n, r, j) = D[j] * qh[r];
        AT(S, n, j, j) = 1.0;
        for (int64_t i = 0; i < j; ++i) {
            double acc = 0.0;
            for (int64_t p = i; p < j; ++p) acc += AT(S, n, i, p) * AT(R, n, p, j);
            AT(S, n, i, j) = -acc / rjj;
        }
    }
    if (bad < 0)
        for (int64_t j = 0; j < n; ++j)
            for (int64_t i = 0; i <= j; ++i) AT(S, n, i, j) *= D[i];
    free(qh);
    free(D);
    return bad;
}
