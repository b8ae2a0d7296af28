/* CSR sparse matrix-vector product y = A x in FP64 for the oracle's assembled operators.
 *
 * TEST INFRASTRUCTURE ONLY: the oracle's apply step (the global matrix of Eq. 4.1 times a vector),
 * used to time the oracle on all host cores.  Rows are split over OpenMP threads in static
 * blocks; each row is summed in column order, so the result does not depend on the thread count.
 * Built by oracle/spmv.py with gcc -O2 -fopenmp; it shares nothing with the CUDA library.
 */
#include <stdint.h>
#include <omp.h>

void oracle_csr_spmv(int64_t nrows, const int64_t* indptr, const int64_t* indices, const double* data,
                     const double* x, double* y) {
#pragma omp parallel for schedule(static)
  for (int64_t r = 0; r < nrows; ++r) {
    double s = 0.0;
    for (int64_t p = indptr[r]; p < indptr[r + 1]; ++p) s += data[p] * x[indices[p]];
    y[r] = s;
  }
}

int oracle_max_threads(void) { return omp_get_max_threads(); }

void oracle_set_threads(int n) { omp_set_num_threads(n); }
