/*
 * Sequential CPU oracle for sparse triangular solves.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load this file.  The CUDA library never
 * includes, links or calls it, and this file includes nothing from the
 * library: the two share no code.
 *
 * Everything here is a plain restatement of Li, "On Parallel Solution of
 * Sparse Triangular Linear Systems in CUDA" (arXiv:1710.04985), in double
 * precision, one loop per formula, no blocking or reordering.
 *
 * Storage convention.  Sec. 3 keeps the strict triangle in CSR (ia, ja, a)
 * and the diagonal apart in a vector d.  Here the CSR arrays (rowptr, colidx,
 * vals) hold the diagonal inside its row; it is found by its column index.
 * Indices are 0-based int32.  With unit != 0 the diagonal is taken to be 1
 * and any stored diagonal entry is ignored.  Right-hand sides and solutions
 * are row-major [n][ld] with k columns in use.
 *
 * Levels are 0-based: the level of Sec. 4.1 minus one (roots get level 0).
 *
 * Parity status: every function below is pinned by tests against closed
 * forms, brute force or dense library solves (see the oracle pin tests).
 */
#include <stddef.h>

/* Level of each unknown by the row-wise loop of Sec. 4.1:
 * lev(i) = 1 + max{lev(j) : A_ij != 0, j != i}, with the maximum over an empty
 * set giving a root.  Lower triangles sweep i = 0..n-1 (forward
 * substitution); upper triangles sweep i = n-1..0 (backward substitution,
 * "the same way by reversing the order", Sec. 4.1).  Returns nlev. */
int oracle_levels_rowwise(int n, const int *rowptr, const int *colidx,
                          int upper, int *lev)
{
    int nlev = 0;
    for (int t = 0; t < n; ++t) {
        int i = upper ? n - 1 - t : t;
        int best = -1;
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int j = colidx[p];
            if (j == i) continue;
            if (lev[j] > best) best = lev[j];
        }
        lev[i] = best + 1;
        if (lev[i] + 1 > nlev) nlev = lev[i] + 1;
    }
    return nlev;
}

/* Levels of the TRANSPOSED system op(A) = A^T, computed with the
 * column-wise loop of Sec. 4.1: lev(i) = max(lev(j) + 1, lev(i)) for every i
 * with (A^T)_ij != 0, sweeping j in substitution order, lev initialised to
 * zero.  Column j of A^T is row j of A, so the CSR of A is read as the CSC of
 * A^T.  For lower A, A^T is upper and is swept j = n-1..0; for upper A,
 * A^T is lower and is swept j = 0..n-1.  Returns nlev. */
int oracle_levels_transpose(int n, const int *rowptr, const int *colidx,
                            int upper, int *lev)
{
    for (int i = 0; i < n; ++i) lev[i] = 0;
    int nlev = n > 0 ? 1 : 0;
    for (int t = 0; t < n; ++t) {
        int j = upper ? t : n - 1 - t;
        for (int p = rowptr[j]; p < rowptr[j + 1]; ++p) {
            int i = colidx[p];          /* (A^T)_{i j} = A_{j i} != 0 */
            if (i == j) continue;
            if (lev[j] + 1 > lev[i]) lev[i] = lev[j] + 1;
            if (lev[i] + 1 > nlev) nlev = lev[i] + 1;
        }
    }
    return nlev;
}

/* Level sets of Sec. 4.1: jlev lists the unknowns in nondecreasing level
 * order and ilev[m] points at the first unknown of level m in jlev
 * (ilev[nlev] = n).  Within a level, unknowns are listed in increasing
 * index order (a counting sort, which is stable). */
void oracle_level_sets(int n, const int *lev, int nlev, int *ilev, int *jlev)
{
    for (int m = 0; m <= nlev; ++m) ilev[m] = 0;
    for (int i = 0; i < n; ++i) ilev[lev[i] + 1] += 1;
    for (int m = 0; m < nlev; ++m) ilev[m + 1] += ilev[m];
    /* fill, using ilev as running cursors, then shift back */
    for (int i = 0; i < n; ++i) {
        int m = lev[i];
        jlev[ilev[m]] = i;
        ilev[m] += 1;
    }
    for (int m = nlev; m > 0; --m) ilev[m] = ilev[m - 1];
    ilev[0] = 0;
}

/* Row-wise substitution of Sec. 3.1 (forward for lower, reversed outer loop
 * for upper): x := f, then for each i in substitution order
 *   x(i) := x(i) - sum_{j != i} A_ij x(j);  x(i) := x(i) / A_ii.
 * Solves each of the k right-hand-side columns in turn. */
void oracle_solve(int n, const int *rowptr, const int *colidx,
                  const double *vals, int upper, int unit, int k,
                  const double *b, int ldb, double *x, int ldx)
{
    for (int c = 0; c < k; ++c) {
        for (int t = 0; t < n; ++t) {
            int i = upper ? n - 1 - t : t;
            double s = b[(size_t)i * ldb + c];
            double d = 1.0;
            for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                int j = colidx[p];
                if (j == i) {
                    if (!unit) d = vals[p];
                } else {
                    s -= vals[p] * x[(size_t)j * ldx + c];
                }
            }
            x[(size_t)i * ldx + c] = unit ? s : s / d;
        }
    }
}

/* Solve A^T y = g with the column-wise sweep of Sec. 3.2: the CSR of A is the
 * CSC of A^T.  y := g; then for each column j of A^T in substitution order
 * (j = n-1..0 when A is lower, since A^T is upper; j = 0..n-1 when A is
 * upper):  y(j) := y(j) / A_jj;  y(i) := y(i) - A_ji y(j) for i != j. */
void oracle_solve_transpose(int n, const int *rowptr, const int *colidx,
                            const double *vals, int upper, int unit, int k,
                            const double *g, int ldg, double *y, int ldy)
{
    for (int c = 0; c < k; ++c) {
        for (int i = 0; i < n; ++i) y[(size_t)i * ldy + c] = g[(size_t)i * ldg + c];
        for (int t = 0; t < n; ++t) {
            int j = upper ? t : n - 1 - t;
            double d = 1.0;
            if (!unit) {
                for (int p = rowptr[j]; p < rowptr[j + 1]; ++p)
                    if (colidx[p] == j) d = vals[p];
            }
            double yj = y[(size_t)j * ldy + c] / d;
            y[(size_t)j * ldy + c] = yj;
            for (int p = rowptr[j]; p < rowptr[j + 1]; ++p) {
                int i = colidx[p];
                if (i == j) continue;
                y[(size_t)i * ldy + c] -= vals[p] * yj;
            }
        }
    }
}

/* Gradient of a scalar loss through x = A^{-1} b with respect to the stored
 * entries of A.  Differentiating (1), A x = b, gives dx = -A^{-1} (dA) x, so
 * with y = A^{-T} (dloss/dx):  dloss/dA_ij = -sum_c y(i,c) x(j,c), for every
 * stored (i, j) including the diagonal.  With a unit diagonal the diagonal is
 * not a parameter and its gradient is zero. */
void oracle_grad_vals(int n, const int *rowptr, const int *colidx, int unit,
                      int k, const double *y, int ldy, const double *x,
                      int ldx, double *gvals)
{
    for (int i = 0; i < n; ++i) {
        for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
            int j = colidx[p];
            double s = 0.0;
            if (!(unit && j == i)) {
                for (int c = 0; c < k; ++c)
                    s += y[(size_t)i * ldy + c] * x[(size_t)j * ldx + c];
            }
            gvals[p] = -s;
        }
    }
}

/* Residual r = b - A x of system (1), A including its diagonal (taken as 1
 * when unit != 0), for k right-hand-side columns. */
void oracle_residual(int n, const int *rowptr, const int *colidx,
                     const double *vals, int unit, int k, const double *b,
                     int ldb, const double *x, int ldx, double *r, int ldr)
{
    for (int i = 0; i < n; ++i) {
        for (int c = 0; c < k; ++c) {
            double s = b[(size_t)i * ldb + c];
            for (int p = rowptr[i]; p < rowptr[i + 1]; ++p) {
                int j = colidx[p];
                if (unit && j == i) continue;   /* a stored diagonal is ignored ... */
                s -= x[(size_t)j * ldx + c] * vals[p];
            }
            if (unit) s -= x[(size_t)i * ldx + c];   /* ... and 1 is used, stored or not */
            r[(size_t)i * ldr + c] = s;
        }
    }
}
