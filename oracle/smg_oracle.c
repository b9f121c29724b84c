/*
 * Oracle for the surface multigrid hot path: plain, serial, obviously correct
 * CPU loops.  TEST INFRASTRUCTURE ONLY: only the tests, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library; the product path
 * never does.  It shares no code with the CUDA library.
 *
 * Contents
 *   oracle_greedy_colouring  graph colouring of Alg. 3 (App. "Multi-Color Gauss Seidel")
 *   oracle_gs_sweep_f64/f32  one Gauss-Seidel pass over a given row order (Sec. 5, Alg. 2
 *                            "Relaxation"; colour-major order as in App. "Multi-Color GS")
 *   oracle_cholesky          dense LL^T of the coarsest operator (Alg. 2 "direct solve")
 *   oracle_chol_solve        forward then backward substitution with that factor
 *
 * All sparse matrices are CSR with int64 indices; multi-right-hand-side vectors
 * are row-major n x nrhs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/*
 * Alg. 3 (greedy colouring with a move-to-back palette).  The graph is the set of
 * structural off-diagonal entries of the symmetric pattern (rowptr, col).
 * Readings where the text leaves a choice:
 *   - degree = number of off-diagonal entries in the row;
 *   - nodes are visited by degree, descending (the appendix text), ties by
 *     ascending index (a stable sort);
 *   - the palette is a list; the first listed colour unused by painted
 *     neighbours is taken and moved to the back; if none fits, a new colour with
 *     id = number of colours so far is appended.
 * Writes colour[i] and returns the number of colours, or -1 on allocation failure.
 */
int64_t oracle_greedy_colouring(int64_t n, const int64_t *rowptr, const int64_t *col,
                                int32_t *colour)
{
    int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!deg || !order) { free(deg); free(order); return -1; }
    int64_t maxdeg = 0;
    for (int64_t i = 0; i < n; i++) {
        int64_t d = 0;
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++)
            if (col[p] != i) d++;
        deg[i] = d;
        if (d > maxdeg) maxdeg = d;
    }
    /* stable counting sort by degree, descending */
    int64_t *cnt = (int64_t *)calloc((size_t)(maxdeg + 2), sizeof(int64_t));
    int64_t *palette = (int64_t *)malloc(sizeof(int64_t) * (size_t)(maxdeg + 2));
    int64_t *seen = (int64_t *)malloc(sizeof(int64_t) * (size_t)(maxdeg + 2));
    if (!cnt || !palette || !seen) { free(deg); free(order); free(cnt); free(palette); free(seen); return -1; }
    for (int64_t i = 0; i < n; i++) cnt[maxdeg - deg[i] + 1]++;
    for (int64_t d = 1; d <= maxdeg + 1; d++) cnt[d] += cnt[d - 1];
    for (int64_t i = 0; i < n; i++) order[cnt[maxdeg - deg[i]]++] = i;

    for (int64_t i = 0; i < n; i++) colour[i] = -1;
    for (int64_t c = 0; c < maxdeg + 2; c++) seen[c] = -1;
    int64_t ncol = 0;
    for (int64_t t = 0; t < n; t++) {
        int64_t v = order[t];
        /* gather colours of already painted neighbours */
        for (int64_t p = rowptr[v]; p < rowptr[v + 1]; p++) {
            int64_t u = col[p];
            if (u != v && colour[u] >= 0) seen[colour[u]] = v;
        }
        int64_t pos = -1;
        for (int64_t q = 0; q < ncol; q++)
            if (seen[palette[q]] != v) { pos = q; break; }
        int64_t c;
        if (pos < 0) {
            c = ncol;
            palette[ncol++] = c;               /* new colour, appended at the back */
        } else {
            c = palette[pos];                  /* move the chosen colour to the back */
            for (int64_t q = pos; q + 1 < ncol; q++) palette[q] = palette[q + 1];
            palette[ncol - 1] = c;
        }
        colour[v] = (int32_t)c;
    }
    free(deg); free(order); free(cnt); free(palette); free(seen);
    return ncol;
}

/*
 * One Gauss-Seidel pass: for each row i in `order` (in that order),
 *   x_i <- (b_i - sum_{j != i} a_ij x_j) / a_ii
 * using the newest values of x.  Returns 0, or -(i+1) if row i has no
 * positive-or-negative diagonal entry (a_ii == 0).
 */
int64_t oracle_gs_sweep_f64(int64_t n, const int64_t *rowptr, const int64_t *col,
                            const double *val, const int64_t *order, int64_t norder,
                            const double *b, double *x, int64_t nrhs)
{
    (void)n;
    for (int64_t t = 0; t < norder; t++) {
        int64_t i = order[t];
        for (int64_t r = 0; r < nrhs; r++) {
            double s = b[i * nrhs + r];
            double aii = 0.0;
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) {
                int64_t j = col[p];
                if (j == i) aii = val[p];
                else s -= val[p] * x[j * nrhs + r];
            }
            if (aii == 0.0) return -(i + 1);
            x[i * nrhs + r] = s / aii;
        }
    }
    return 0;
}

/* The same pass carried out entirely in single precision (inner cycle of the
 * mixed-precision form). */
int64_t oracle_gs_sweep_f32(int64_t n, const int64_t *rowptr, const int64_t *col,
                            const float *val, const int64_t *order, int64_t norder,
                            const float *b, float *x, int64_t nrhs)
{
    (void)n;
    for (int64_t t = 0; t < norder; t++) {
        int64_t i = order[t];
        for (int64_t r = 0; r < nrhs; r++) {
            float s = b[i * nrhs + r];
            float aii = 0.0f;
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) {
                int64_t j = col[p];
                if (j == i) aii = val[p];
                else s -= val[p] * x[j * nrhs + r];
            }
            if (aii == 0.0f) return -(i + 1);
            x[i * nrhs + r] = s / aii;
        }
    }
    return 0;
}

/*
 * Dense Cholesky A = L L^T (row-major n x n; the lower triangle of `a` is read,
 * `l` receives L with zeros above the diagonal).  Column-by-column textbook form:
 *   L_jj = sqrt(A_jj - sum_{k<j} L_jk^2),  L_ij = (A_ij - sum_{k<j} L_ik L_jk) / L_jj.
 * Returns 0, or -(j+1) when the j-th pivot is not positive (A not SPD).
 */
int64_t oracle_cholesky(int64_t n, const double *a, double *l)
{
    memset(l, 0, sizeof(double) * (size_t)(n * n));
    for (int64_t j = 0; j < n; j++) {
        double d = a[j * n + j];
        for (int64_t k = 0; k < j; k++) d -= l[j * n + k] * l[j * n + k];
        if (!(d > 0.0)) return -(j + 1);
        double ljj = sqrt(d);
        l[j * n + j] = ljj;
        for (int64_t i = j + 1; i < n; i++) {
            double s = a[i * n + j];
            for (int64_t k = 0; k < j; k++) s -= l[i * n + k] * l[j * n + k];
            l[i * n + j] = s / ljj;
        }
    }
    return 0;
}

/* Solve L L^T x = b for nrhs right-hand sides (row-major n x nrhs). */
void oracle_chol_solve(int64_t n, const double *l, const double *b, double *x, int64_t nrhs)
{
    double *y = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t r = 0; r < nrhs; r++) {
        for (int64_t i = 0; i < n; i++) {              /* L y = b */
            double s = b[i * nrhs + r];
            for (int64_t k = 0; k < i; k++) s -= l[i * n + k] * y[k];
            y[i] = s / l[i * n + i];
        }
        for (int64_t i = n - 1; i >= 0; i--) {         /* L^T x = y */
            double s = y[i];
            for (int64_t k = i + 1; k < n; k++) s -= l[k * n + i] * x[k * nrhs + r];
            x[i * nrhs + r] = s / l[i * n + i];
        }
    }
    free(y);
}
