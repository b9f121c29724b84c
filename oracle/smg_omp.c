/*
 * Multicolour OpenMP form of the oracle's cycle, for the all-cores CPU
 * baseline of the benchmark.
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of oracle/: the product library
 * never calls it.  It is the paper's own CPU parallelisation (App.
 * "Multi-Color Gauss Seidel": the rows of one colour class are independent,
 * so each class is updated in parallel), written as plain loops over the same
 * CSR data the serial oracle uses.  Every row sums its terms in CSR order, as
 * the serial loops do, so a Gauss-Seidel sweep gives the serial sweep's bits;
 * the transfers sum in CSR order of P^T and P.
 */
#include <omp.h>
#include <stdint.h>

/* Threads the parallel loops use (omp_get_max_threads). */
int64_t omp_threads(void) { return (int64_t)omp_get_max_threads(); }

/*
 * One Gauss-Seidel sweep over colour classes: class c holds rows
 * rows[cptr[c] .. cptr[c+1]), visited in order c = 0..k-1 (reverse: k-1..0);
 * inside a class the rows are independent (no two are coupled), so they run in
 * parallel: x_i <- (b_i - sum_{j != i} a_ij x_j) / a_ii, nrhs columns
 * row-major.  Returns 0, or -(i+1) for a zero diagonal in row i.
 */
int64_t omp_gs_sweep(int64_t ncol, const int64_t *cptr, const int64_t *rows, const int64_t *rowptr,
                     const int64_t *col, const double *val, const double *b, double *x, int64_t nrhs,
                     int64_t reverse)
{
    int64_t bad = 0;
    for (int64_t cc = 0; cc < ncol; cc++) {
        int64_t c = reverse ? ncol - 1 - cc : cc;
#pragma omp parallel for schedule(static) reduction(min : bad)
        for (int64_t t = cptr[c]; t < cptr[c + 1]; t++) {
            int64_t i = rows[t];
            for (int64_t r = 0; r < nrhs; r++) {
                double s = b[i * nrhs + r];
                double aii = 0.0;
                for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) {
                    int64_t j = col[p];
                    if (j == i) aii = val[p];
                    else s -= val[p] * x[j * nrhs + r];
                }
                if (aii == 0.0) bad = bad < -(i + 1) ? bad : -(i + 1);
                else x[i * nrhs + r] = s / aii;
            }
        }
        if (bad) return bad;
    }
    return 0;
}

/* r = b - A x over all n rows (nrhs columns), in parallel. */
void omp_residual(int64_t n, const int64_t *rowptr, const int64_t *col, const double *val, const double *b,
                  const double *x, double *r, int64_t nrhs)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)
        for (int64_t q = 0; q < nrhs; q++) {
            double s = b[i * nrhs + q];
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) s -= val[p] * x[col[p] * nrhs + q];
            r[i * nrhs + q] = s;
        }
}

/* y = M v for a CSR matrix M (m rows): restriction with M = P^T, prolongation
 * with M = P; add = 1 accumulates into y (x <- x + P c). */
void omp_spmv(int64_t m, const int64_t *rowptr, const int64_t *col, const double *val, const double *v, double *y,
              int64_t nrhs, int64_t add)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; i++)
        for (int64_t q = 0; q < nrhs; q++) {
            double s = 0.0;
            for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) s += val[p] * v[col[p] * nrhs + q];
            y[i * nrhs + q] = add ? y[i * nrhs + q] + s : s;
        }
}
