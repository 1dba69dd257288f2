/*
 * Sparse matrix-vector product y = A x for a CSR matrix, rows divided among
 * OpenMP threads (static schedule).  Part of the FP64 CPU oracle: test
 * infrastructure only, used to time the oracle on all host cores.  It shares
 * no code with the CUDA library.
 *
 * Definition: y_i = sum_{k = rowptr[i]}^{rowptr[i+1]-1} val[k] x[col[k]],
 * summed in the order of the stored entries (one thread per row, so the
 * result does not depend on the thread count).
 */
#include <stdint.h>
#include <omp.h>

int oracle_spmv_threads(void) { return omp_get_max_threads(); }

void oracle_csr_mv_f64(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                       const double *x, double *y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += val[k] * x[col[k]];
    y[i] = s;
  }
}

/* Complex form: val, x, y hold interleaved (re, im) pairs of FP64. */
void oracle_csr_mv_c128(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val,
                        const double *x, double *y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double sr = 0.0, si = 0.0;
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const double ar = val[2 * k], ai = val[2 * k + 1];
      const double xr = x[2 * (int64_t)col[k]], xi = x[2 * (int64_t)col[k] + 1];
      sr += ar * xr - ai * xi;
      si += ar * xi + ai * xr;
    }
    y[2 * i] = sr;
    y[2 * i + 1] = si;
  }
}
