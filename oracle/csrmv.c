/* csrmv.c -- y = s A x for a complex128 CSR matrix.  TEST INFRASTRUCTURE (oracle).
 *
 * The plain definition of the sparse product of eq. arnoldi (arXiv 2205.15346,
 * Sec. 2.1, first line of the recurrence): y_i = s * sum_k A[i, col_k] x[col_k]
 * over the stored entries of row i, in storage order, with the textbook complex
 * product (ar xr - ai xi) + i (ar xi + ai xr) and no fused multiply-add.  Rows are
 * split over OpenMP threads; every row is summed by one thread in the same
 * order whatever the thread count, so the result is bitwise the same for one
 * thread and for all cores.  Only the oracle (oracle/native.py) loads this.
 */
#include <stdint.h>

void oracle_csrmv(int64_t d, const int64_t* rowptr, const int32_t* col, const double* val,
                  const double* x, double s, double* y, int threads) {
#pragma omp parallel for schedule(static) num_threads(threads)
    for (int64_t i = 0; i < d; ++i) {
        double re = 0.0, im = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            const double ar = val[2 * k], ai = val[2 * k + 1];
            const int64_t c = col[k];
            const double xr = x[2 * c], xi = x[2 * c + 1];
            re += ar * xr - ai * xi;
            im += ar * xi + ai * xr;
        }
        y[2 * i] = s * re;
        y[2 * i + 1] = s * im;
    }
}
