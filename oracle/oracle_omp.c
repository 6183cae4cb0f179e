/*
 * ORACLE -- TEST INFRASTRUCTURE ONLY (CPU baseline).
 *
 * Multi-threaded (OpenMP) forms of three oracle products, used only to time
 * the CPU baseline on all host cores. Each states the same definition as its
 * serial counterpart in oracle.c, with the outer loop -- rows for the
 * row-major products, listed columns for the column-major one -- divided
 * among threads:
 *   oracle_csr_pull_par        = oracle_csr_pull (Sec. II; Sec. IV-A (3,6)),
 *                                 per-row sums in ascending k, so the result
 *                                 is bit-identical to the serial one;
 *   oracle_spmspv_rowmajor_par = oracle_spmspv_rowmajor (Sec. IV-A (3,5));
 *   oracle_csc_push_par        = oracle_csc_push (Sec. IV-A (2,8)), with
 *                                 atomic additions into y, so the order of
 *                                 the additions (and the last bits of y) may
 *                                 differ from the serial loop.
 * Tests check them against the serial oracle. The library never calls them.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>

int oracle_par_threads(void) { return omp_get_max_threads(); }

void oracle_csr_pull_par(int64_t m, const int32_t* rowptr, const int32_t* col,
                         const double* val, const double* x, double* y, double* s) {
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < m; ++i) {
        double acc = 0.0, mag = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            double a = val ? val[k] : 1.0;
            double p = a * x[col[k]];
            acc += p;
            mag += fabs(p);
        }
        y[i] = acc;
        if (s) s[i] = mag;
    }
}

void oracle_spmspv_rowmajor_par(int64_t m, int64_t n, const int32_t* rowptr, const int32_t* col,
                                const double* val, int64_t nnz_x, const int32_t* xidx,
                                const double* xval, double* y, double* s, uint8_t* hit) {
    double* xd = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    uint8_t* in = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < nnz_x; ++t) {  /* listed columns are distinct */
        xd[xidx[t]] = xval ? xval[t] : 1.0;
        in[xidx[t]] = 1;
    }
#pragma omp parallel for schedule(dynamic, 4096)
    for (int64_t i = 0; i < m; ++i) {
        double acc = 0.0, mag = 0.0;
        uint8_t h = 0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            if (!in[col[k]]) continue;
            double a = val ? val[k] : 1.0;
            double p = a * xd[col[k]];
            acc += p;
            mag += fabs(p);
            h = 1;
        }
        y[i] = acc;
        if (s) s[i] = mag;
        if (hit) hit[i] = h;
    }
    free(xd);
    free(in);
}

void oracle_csc_push_par(int64_t m, const int32_t* colptr, const int32_t* rowidx,
                         const double* val, int64_t nnz_x, const int32_t* xidx,
                         const double* xval, double* y, uint8_t* touched) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        y[i] = 0.0;
        if (touched) touched[i] = 0;
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t t = 0; t < nnz_x; ++t) {
        int32_t j = xidx[t];
        double xj = xval ? xval[t] : 1.0;
        for (int64_t k = colptr[j]; k < colptr[j + 1]; ++k) {
            double a = val ? val[k] : 1.0;
            double p = a * xj;
#pragma omp atomic update
            y[rowidx[k]] += p;
            if (touched) {
#pragma omp atomic write
                touched[rowidx[k]] = 1;
            }
        }
    }
}
