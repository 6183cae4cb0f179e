/*
 * ORACLE -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, serial, obviously-correct CPU statement of what the adaptive
 * SpMV/SpMSpV path computes (Li, Ao, Yang, "Adaptive SpMV/SpMSpV on GPUs for
 * Input Vectors of Varied Sparsity"). Only the test suite, the smoke check and
 * the benchmark's CPU-baseline leg may call it; the library's product path
 * never does. It shares no code with the CUDA path and includes no CUDA header.
 *
 * Arithmetic is FP64 throughout (FP32 inputs are widened exactly by the caller
 * before they reach these functions). Loops run in the order the definition
 * states: no blocking, no fusion, no reordering.
 *
 * Pins (tests/test_oracle_pins.py) tie each function to something other than
 * itself: dense brute force with exactly representable values, A*e_j = column
 * j, linearity, the adjoint identity, closed forms of the 2-D Laplacian and
 * 27-point stencil, scipy's transpose and BFS distances, Graph500-style BFS
 * validation, Gini/std-dev special cases, and the PageRank mass invariant.
 * The kernel selector has no oracle counterpart (parity unpinned: the paper
 * prints no decision rules); see the design notes.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* -------------------------------------------------------------------------
 * Row-major (CSR) product, the "traditional SpMV" solution (3,6) of Sec. IV-A
 * and the problem statement of Sec. II: y_i = sum_{k in row i} a_k * x[col_k],
 * accumulated in ascending k. s_i = sum |a_k * x[col_k]| is the per-row scale
 * used by the parity tolerance. val == NULL means a pattern matrix (a_k = 1). */
void oracle_csr_pull(int64_t m, const int32_t* rowptr, const int32_t* col,
                     const double* val, const double* x, double* y, double* s) {
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

/* -------------------------------------------------------------------------
 * Row-major SpMSpV with value validation, solution (3,5) of Sec. IV-A: an
 * entry of row i is effective iff its column is in the structural nonzero set
 * of x (the index list as given, explicit zeros included; Sec. II "effective
 * nonzeros"). y_i sums the effective entries; hit_i = 1 iff row i has at least
 * one effective entry (the structural output set); s_i as in oracle_csr_pull.
 * x arrives as a list (xidx[nnz_x], xval[nnz_x]); xval == NULL means all-ones. */
void oracle_spmspv_rowmajor(int64_t m, int64_t n, const int32_t* rowptr, const int32_t* col,
                            const double* val, int64_t nnz_x, const int32_t* xidx,
                            const double* xval, double* y, double* s, uint8_t* hit) {
    double* xd = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    uint8_t* in = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    for (int64_t t = 0; t < nnz_x; ++t) {
        xd[xidx[t]] = xval ? xval[t] : 1.0;
        in[xidx[t]] = 1;
    }
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

/* -------------------------------------------------------------------------
 * Column-major SpMSpV, solution (2,8) of Sec. IV-A (vector-driven, no
 * validation): y <- 0; for each listed x nonzero j, for each entry k of column
 * j, y[rowidx_k] += a_k * x_j. An independent loop over the CSC arrays used to
 * cross-check oracle_csr_pull. touched_i = 1 iff row i received a contribution. */
void oracle_csc_push(int64_t m, const int32_t* colptr, const int32_t* rowidx,
                     const double* val, int64_t nnz_x, const int32_t* xidx,
                     const double* xval, double* y, uint8_t* touched) {
    for (int64_t i = 0; i < m; ++i) { y[i] = 0.0; if (touched) touched[i] = 0; }
    for (int64_t t = 0; t < nnz_x; ++t) {
        int32_t j = xidx[t];
        double xj = xval ? xval[t] : 1.0;
        for (int64_t k = colptr[j]; k < colptr[j + 1]; ++k) {
            double a = val ? val[k] : 1.0;
            y[rowidx[k]] += a * xj;
            if (touched) touched[rowidx[k]] = 1;
        }
    }
}

/* -------------------------------------------------------------------------
 * Column-major dot product (the adjoint): out_j = sum_{k in column j} a_k *
 * v[rowidx_k], i.e. A^T v read through the CSC arrays. Used for the backward
 * form dx = A^T dy. */
void oracle_csc_pull(int64_t n, const int32_t* colptr, const int32_t* rowidx,
                     const double* val, const double* v, double* out, double* s) {
    for (int64_t j = 0; j < n; ++j) {
        double acc = 0.0, mag = 0.0;
        for (int64_t k = colptr[j]; k < colptr[j + 1]; ++k) {
            double p = (val ? val[k] : 1.0) * v[rowidx[k]];
            acc += p;
            mag += fabs(p);
        }
        out[j] = acc;
        if (s) s[j] = mag;
    }
}

/* -------------------------------------------------------------------------
 * CSR -> CSC (Sec. VI-A keeps both formats resident). Counting sort of the
 * entries by column, stable in row order, so rows ascend within each column.
 * perm[p] = CSR position of the entry stored at CSC position p. */
void oracle_csr_to_csc(int64_t m, int64_t n, const int32_t* rowptr, const int32_t* col,
                       int32_t* colptr, int32_t* rowidx, int32_t* perm) {
    int64_t nnz = rowptr[m];
    for (int64_t j = 0; j <= n; ++j) colptr[j] = 0;
    for (int64_t k = 0; k < nnz; ++k) colptr[col[k] + 1]++;
    for (int64_t j = 0; j < n; ++j) colptr[j + 1] += colptr[j];
    int32_t* next = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t j = 0; j < n; ++j) next[j] = colptr[j];
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            int32_t p = next[col[k]]++;
            rowidx[p] = (int32_t)i;
            perm[p] = (int32_t)k;
        }
    }
    free(next);
}

/* -------------------------------------------------------------------------
 * Dense -> sparse vector conversion (Sec. II vector formats; Sec. VI-A online
 * conversion): the ascending indices j with x_j != 0 by IEEE comparison (so
 * -0.0 is a zero and NaN is a nonzero), and their values. Returns nnz_x. */
int64_t oracle_compact(int64_t n, const double* x, int32_t* idx, double* xval) {
    int64_t c = 0;
    for (int64_t j = 0; j < n; ++j) {
        if (x[j] != 0.0) {
            idx[c] = (int32_t)j;
            if (xval) xval[c] = x[j];
            ++c;
        }
    }
    return c;
}

/* -------------------------------------------------------------------------
 * Matrix features of Table 1 (models 1-3), computed once per matrix (Sec.
 * VI-C). Readings taken where the paper is silent:
 *  - avg_row = nnz / m;
 *  - relative_range = (max_row - min_row) / n, the denominator as printed;
 *  - var_nnz_row ("standard variation") = population standard deviation of
 *    the row lengths, two passes around the mean;
 *  - Gini coefficient over ascending row lengths d_(1..m):
 *        G = sum_i (2i - m - 1) d_(i) / (m * sum_i d_i),  0 when nnz = 0.
 * out[] = {m, n, nnz, max_row, min_row, avg_row, relative_range, var_nnz_row, gini}. */
static int cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

void oracle_matrix_features(int64_t m, int64_t n, const int32_t* rowptr, double* out) {
    int64_t nnz = m > 0 ? rowptr[m] : 0;
    int64_t mx = 0, mn = 0;
    for (int64_t i = 0; i < m; ++i) {
        int64_t d = rowptr[i + 1] - rowptr[i];
        if (i == 0 || d > mx) mx = d;
        if (i == 0 || d < mn) mn = d;
    }
    double avg = m > 0 ? (double)nnz / (double)m : 0.0;
    double ss = 0.0;
    for (int64_t i = 0; i < m; ++i) {
        double dev = (double)(rowptr[i + 1] - rowptr[i]) - avg;
        ss += dev * dev;
    }
    double var = m > 0 ? sqrt(ss / (double)m) : 0.0;
    double gini = 0.0;
    if (m > 0 && nnz > 0) {
        int64_t* d = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
        for (int64_t i = 0; i < m; ++i) d[i] = rowptr[i + 1] - rowptr[i];
        qsort(d, (size_t)m, sizeof(int64_t), cmp_i64);
        __int128 num = 0;
        for (int64_t i = 1; i <= m; ++i) num += (__int128)(2 * i - m - 1) * d[i - 1];
        gini = (double)num / ((double)m * (double)nnz);
        free(d);
    }
    out[0] = (double)m;
    out[1] = (double)n;
    out[2] = (double)nnz;
    out[3] = (double)mx;
    out[4] = (double)mn;
    out[5] = avg;
    out[6] = n > 0 ? (double)(mx - mn) / (double)n : 0.0;
    out[7] = var;
    out[8] = gini;
}

/* -------------------------------------------------------------------------
 * Vector features of Table 1 (models 1 and 3), per input vector:
 * nnz_x, x_sparsity = nnz_x / n, nnz_s = number of effective matrix nonzeros
 * = sum over listed j of the length of column j, m_sparsity = nnz_s / nnz.
 * out[] = {nnz_x, x_sparsity, nnz_s, m_sparsity}. */
void oracle_vector_features(int64_t n, int64_t nnz, const int32_t* colptr, int64_t nnz_x,
                            const int32_t* xidx, double* out) {
    int64_t s = 0;
    for (int64_t t = 0; t < nnz_x; ++t) s += colptr[xidx[t] + 1] - colptr[xidx[t]];
    out[0] = (double)nnz_x;
    out[1] = n > 0 ? (double)nnz_x / (double)n : 0.0;
    out[2] = (double)s;
    out[3] = nnz > 0 ? (double)s / (double)nnz : 0.0;
}

/* -------------------------------------------------------------------------
 * Boolean (OR, AND) semiring over a pattern matrix, the BFS use of Sec. I/VII:
 * y_i = 1 iff some entry of row i has x[col_k] != 0. */
void oracle_bool_pull(int64_t m, const int32_t* rowptr, const int32_t* col,
                      const uint8_t* x, uint8_t* y) {
    for (int64_t i = 0; i < m; ++i) {
        uint8_t h = 0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            if (x[col[k]]) { h = 1; break; }
        y[i] = h;
    }
}

/* -------------------------------------------------------------------------
 * Integer (+, x) semiring in 32-bit two's-complement wrap-around arithmetic:
 * y_i = sum_k a_k * x[col_k] mod 2^32. val == NULL means all-ones. */
void oracle_i32_pull(int64_t m, const int32_t* rowptr, const int32_t* col,
                     const int32_t* val, const int32_t* x, int32_t* y) {
    for (int64_t i = 0; i < m; ++i) {
        uint32_t acc = 0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k)
            acc += (uint32_t)(val ? val[k] : 1) * (uint32_t)x[col[k]];
        y[i] = (int32_t)acc;
    }
}

/* -------------------------------------------------------------------------
 * Queue BFS over the adjacency lists of a pattern matrix (row i lists the
 * neighbours of vertex i). level[v] = hop distance from root, -1 if not
 * reached. Returns the number of levels (max level + 1). This is the
 * application of Sec. VII whose frontiers are the SpMSpV inputs. */
int32_t oracle_bfs(int64_t n, const int32_t* rowptr, const int32_t* col, int32_t root,
                   int32_t* level) {
    for (int64_t v = 0; v < n; ++v) level[v] = -1;
    if (root < 0 || root >= n) return 0;
    int32_t* q = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t head = 0, tail = 0;
    q[tail++] = root;
    level[root] = 0;
    int32_t maxl = 0;
    while (head < tail) {
        int32_t u = q[head++];
        for (int64_t k = rowptr[u]; k < rowptr[u + 1]; ++k) {
            int32_t v = col[k];
            if (level[v] < 0) {
                level[v] = level[u] + 1;
                if (level[v] > maxl) maxl = level[v];
                q[tail++] = v;
            }
        }
    }
    free(q);
    return maxl + 1;
}

/* -------------------------------------------------------------------------
 * One PageRank power step on a pattern matrix (the incremental-PageRank
 * application of Sec. VII gives no formula; reading): with out-degree
 * deg_j = length of column j, x_j = r_j / deg_j (0 when deg_j = 0),
 * y = A x, r'_i = (1 - d)/N + d * y_i. Writes x, y and r'. */
void oracle_pagerank_step(int64_t N, const int32_t* rowptr, const int32_t* col,
                          const int32_t* colptr, const double* r, double d,
                          double* x, double* y, double* rnext) {
    for (int64_t j = 0; j < N; ++j) {
        int64_t deg = colptr[j + 1] - colptr[j];
        x[j] = deg > 0 ? r[j] / (double)deg : 0.0;
    }
    oracle_csr_pull(N, rowptr, col, NULL, x, y, NULL);
    for (int64_t i = 0; i < N; ++i) rnext[i] = (1.0 - d) / (double)N + d * y[i];
}

/* -------------------------------------------------------------------------
 * Gradient of y = A x with respect to the stored values of A, restricted to
 * A's pattern: dA_k = dy[row(k)] * x[col_k], in CSR order. */
void oracle_grad_values(int64_t m, const int32_t* rowptr, const int32_t* col,
                        const double* dy, const double* x, double* dA) {
    for (int64_t i = 0; i < m; ++i)
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) dA[k] = dy[i] * x[col[k]];
}
