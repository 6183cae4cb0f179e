/*
 * Seeded synthetic inputs for the adaptive SpMV/SpMSpV library and its oracle.
 *
 * This file only builds matrices and vectors; it holds none of the method's
 * arithmetic (no products, no sums of products). Both the CUDA path's tests and
 * benchmark and the CPU oracle take their inputs from here, so neither side
 * generates anything of its own.
 *
 * Every random draw is a pure function of (seed, stream, counter) through the
 * splitmix64 finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014), so results do not depend on thread count or order.
 *
 * Matrix shapes follow the paper's workload classes (Sec. VII, Table 3):
 * meshes/stencils stand in for the high-diameter graphs, R-MAT for the
 * low-diameter social/Kronecker graphs, lognormal/Zipf rows for the ML-style
 * data matrix of Sec. I, and a uniform Bernoulli pattern for a pruned layer.
 *
 * All CSR outputs are canonical: column indices strictly ascending in a row.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Counter-based draw: the i-th 64-bit word of stream `stream` under `seed`. */
static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t i) {
    uint64_t key = mix64(seed ^ mix64(stream * GOLDEN + 0x632BE59BD9B4E019ULL));
    return mix64(key + (i + 1) * GOLDEN);
}

/* Uniform in [0, 1) with 53 random bits. */
static inline double u01(uint64_t h) { return (double)(h >> 11) * 0x1.0p-53; }

/* Standard normal via Box-Muller from two counter draws. */
static inline double normal01(uint64_t seed, uint64_t stream, uint64_t i) {
    double u1 = u01(draw(seed, stream, 2 * i));
    double u2 = u01(draw(seed, stream, 2 * i + 1));
    if (u1 < 0x1.0p-60) u1 = 0x1.0p-60;
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

void gen_free(void* p) { free(p); }

/* ---------------------------------------------------------------- 2-D Laplacian
 * 5-point stencil on a g x g grid, natural ordering idx = p*g + q, Dirichlet
 * truncation at the boundary (missing neighbours are dropped): 4 on the
 * diagonal, -1 to each present N/W/E/S neighbour. nnz = 5 g^2 - 4 g.
 * Arrays: rowptr[g*g+1], col[nnz], val[nnz] (double). Returns nnz.           */
int64_t gen_laplace2d(int32_t g, int32_t* rowptr, int32_t* col, double* val) {
    int64_t k = 0;
    rowptr[0] = 0;
    for (int32_t p = 0; p < g; ++p) {
        for (int32_t q = 0; q < g; ++q) {
            int32_t i = p * g + q;
            if (p > 0)     { col[k] = i - g; val[k] = -1.0; ++k; }
            if (q > 0)     { col[k] = i - 1; val[k] = -1.0; ++k; }
            col[k] = i; val[k] = 4.0; ++k;
            if (q + 1 < g) { col[k] = i + 1; val[k] = -1.0; ++k; }
            if (p + 1 < g) { col[k] = i + g; val[k] = -1.0; ++k; }
            rowptr[i + 1] = (int32_t)k;
        }
    }
    return k;
}

/* ---------------------------------------------------------------- 3-D 27-point stencil
 * g^3 grid, idx = (z*g + y)*g + x, neighbours (dz,dy,dx) in {-1,0,1}^3 that lie
 * inside the grid (so column ids ascend in lexicographic offset order).
 * Off-diagonal values U(0.5, 1.5) drawn from (row, offset); the centre is
 * 1 + sum of the row's off-diagonal magnitudes (diagonally dominant), rounded
 * to float. rowsum[i] is the FP64 sum of the stored float values of row i,
 * accumulated while generating (an independent closed form for A*1).
 * nnz = (3g-2)^3. Arrays: rowptr[g^3+1], col[nnz], val[nnz] (float),
 * rowsum[g^3] (double, may be NULL). Returns nnz.                               */
int64_t gen_stencil27_nnz(int32_t g) {
    int64_t e = 3 * (int64_t)g - 2;
    return e * e * e;
}

int64_t gen_stencil27(int32_t g, uint64_t seed, int32_t* rowptr, int32_t* col,
                      float* val, double* rowsum) {
    int64_t m = (int64_t)g * g * g;
    rowptr[0] = 0;
    {   /* row lengths in closed form, then a serial prefix */
        int64_t acc = 0;
        for (int64_t i = 0; i < m; ++i) {
            int32_t x = (int32_t)(i % g), y = (int32_t)((i / g) % g), z = (int32_t)(i / ((int64_t)g * g));
            int cx = 3 - (x == 0) - (x == g - 1);
            int cy = 3 - (y == 0) - (y == g - 1);
            int cz = 3 - (z == 0) - (z == g - 1);
            if (g == 1) { cx = cy = cz = 1; }
            acc += (int64_t)cx * cy * cz;
            rowptr[i + 1] = (int32_t)acc;
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        int32_t x = (int32_t)(i % g), y = (int32_t)((i / g) % g), z = (int32_t)(i / ((int64_t)g * g));
        int64_t k = rowptr[i];
        int64_t kc = -1;
        double off = 0.0;
        for (int dz = -1; dz <= 1; ++dz) {
            int32_t zz = z + dz;
            if (zz < 0 || zz >= g) continue;
            for (int dy = -1; dy <= 1; ++dy) {
                int32_t yy = y + dy;
                if (yy < 0 || yy >= g) continue;
                for (int dx = -1; dx <= 1; ++dx) {
                    int32_t xx = x + dx;
                    if (xx < 0 || xx >= g) continue;
                    col[k] = (int32_t)(((int64_t)zz * g + yy) * g + xx);
                    if (dz == 0 && dy == 0 && dx == 0) {
                        kc = k;
                    } else {
                        int nb = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1);
                        float v = (float)(0.5 + u01(draw(seed, 1, (uint64_t)i * 27 + nb)));
                        val[k] = v;
                        off += (double)v;
                    }
                    ++k;
                }
            }
        }
        float c = (float)(1.0 + off);
        val[kc] = c;
        if (rowsum) rowsum[i] = (double)c + off;
    }
    return rowptr[m];
}

/* ---------------------------------------------------------------- helpers */
static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* Sort + deduplicate each row's column list in place, then compact the arrays.
 * rowptr is rewritten; returns the new nnz. Values (if any) follow their
 * columns; a duplicate keeps the value of its first occurrence in sorted order. */
static int64_t canonicalise_rows(int64_t m, int64_t* rowptr64, int32_t* col, int32_t* keep_len) {
#pragma omp parallel for schedule(dynamic, 1024)
    for (int64_t i = 0; i < m; ++i) {
        int64_t b = rowptr64[i], e = rowptr64[i + 1];
        if (e - b > 1) qsort(col + b, (size_t)(e - b), sizeof(int32_t), cmp_i32);
        int64_t w = b;
        for (int64_t k = b; k < e; ++k)
            if (k == b || col[k] != col[w - 1]) col[w++] = col[k];
        keep_len[i] = (int32_t)(w - b);
    }
    int64_t out = 0;
    for (int64_t i = 0; i < m; ++i) {
        int64_t b = rowptr64[i];
        int32_t L = keep_len[i];
        if (out != b) memmove(col + out, col + b, (size_t)L * sizeof(int32_t));
        rowptr64[i] = out;
        out += L;
    }
    rowptr64[m] = out;
    return out;
}

/* Seeded Fisher-Yates permutation of 0..n-1. */
static void permutation(int64_t n, uint64_t seed, uint64_t stream, int32_t* p) {
    for (int64_t i = 0; i < n; ++i) p[i] = (int32_t)i;
    for (int64_t i = n - 1; i > 0; --i) {
        int64_t j = (int64_t)(u01(draw(seed, stream, (uint64_t)i)) * (double)(i + 1));
        if (j > i) j = i;
        int32_t t = p[i]; p[i] = p[j]; p[j] = t;
    }
}

/* ---------------------------------------------------------------- R-MAT graph
 * Chakrabarti-Zhan-Faloutsos recursive matrix: 2^scale vertices,
 * edge_factor * 2^scale generated edges, quadrant probabilities (a, b, c,
 * 1-a-b-c) chosen independently at each of the `scale` levels. Vertex labels
 * are permuted with a seeded permutation; self-loops dropped; the edge set is
 * symmetrised and deduplicated. Output CSR (pattern only) is malloc'ed:
 * *rowptr_out[N+1], *col_out[nnz]; free with gen_free. Returns nnz.          */
int64_t gen_rmat(int32_t scale, int32_t edge_factor, double a, double b, double c,
                 uint64_t seed, int32_t** rowptr_out, int32_t** col_out) {
    int64_t N = (int64_t)1 << scale;
    int64_t E = (int64_t)edge_factor * N;
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    permutation(N, seed, 3, perm);
    int32_t* src = (int32_t*)malloc(sizeof(int32_t) * (size_t)E);
    int32_t* dst = (int32_t*)malloc(sizeof(int32_t) * (size_t)E);
    const double ab = a + b, abc = a + b + c;
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; ++e) {
        int64_t u = 0, v = 0;
        uint64_t h = 0;
        for (int32_t lev = 0; lev < scale; ++lev) {
            if ((lev & 3) == 0) h = draw(seed, 2, (uint64_t)e * 8 + (uint64_t)(lev >> 2));
            double r = (double)((h >> (16 * (lev & 3))) & 0xFFFF) * (1.0 / 65536.0);
            int bu, bv;
            if (r < a) { bu = 0; bv = 0; }
            else if (r < ab) { bu = 0; bv = 1; }
            else if (r < abc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        src[e] = perm[u];
        dst[e] = perm[v];
    }
    free(perm);
    int64_t* rp = (int64_t*)calloc((size_t)N + 1, sizeof(int64_t));
    for (int64_t e = 0; e < E; ++e) {
        if (src[e] == dst[e]) continue;
        rp[src[e] + 1]++;
        rp[dst[e] + 1]++;
    }
    for (int64_t i = 0; i < N; ++i) rp[i + 1] += rp[i];
    int64_t tot = rp[N];
    int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(tot > 0 ? tot : 1));
    int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * (size_t)N);
    memcpy(cur, rp, sizeof(int64_t) * (size_t)N);
    for (int64_t e = 0; e < E; ++e) {
        int32_t u = src[e], v = dst[e];
        if (u == v) continue;
        col[cur[u]++] = v;
        col[cur[v]++] = u;
    }
    free(cur); free(src); free(dst);
    int32_t* len = (int32_t*)malloc(sizeof(int32_t) * (size_t)N);
    int64_t nnz = canonicalise_rows(N, rp, col, len);
    free(len);
    int32_t* rowptr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(N + 1));
    for (int64_t i = 0; i <= N; ++i) rowptr[i] = (int32_t)rp[i];
    free(rp);
    *rowptr_out = rowptr;
    *col_out = (int32_t*)realloc(col, sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    return nnz;
}

/* ---------------------------------------------------------------- lognormal rows / Zipf columns
 * m rows over n columns. Row length L_i = round(exp(mu + sigma*N(0,1)))
 * clamped to [1, n]; each of the L_i draws picks a column rank r in 1..n with
 * P(r) ~ r^(-s) (inverse CDF on the exact finite Zipf distribution), mapped to
 * a column id by a permutation seeded with perm_seed (matrices sharing a
 * feature space share it, so their popular columns coincide). Duplicates
 * within a row are dropped. Values are U(0, 1] floats. Output malloc'ed;
 * free with gen_free. Returns nnz. */
int64_t gen_lognormal_zipf(int64_t m, int64_t n, double mu, double sigma, double s,
                           uint64_t seed, uint64_t perm_seed, int32_t** rowptr_out, int32_t** col_out,
                           float** val_out) {
    double* cdf = (double*)malloc(sizeof(double) * (size_t)n);
    double acc = 0.0;
    for (int64_t r = 0; r < n; ++r) { acc += pow((double)(r + 1), -s); cdf[r] = acc; }
    for (int64_t r = 0; r < n; ++r) cdf[r] /= acc;
    cdf[n - 1] = 1.0;
    int32_t* idmap = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    permutation(n, perm_seed, 5, idmap);
    int64_t* rp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m + 1));
    rp[0] = 0;
    for (int64_t i = 0; i < m; ++i) {
        double L = floor(exp(mu + sigma * normal01(seed, 4, (uint64_t)i)) + 0.5);
        if (L < 1.0) L = 1.0;
        if (L > (double)n) L = (double)n;
        rp[i + 1] = rp[i] + (int64_t)L;
    }
    int64_t draws = rp[m];
    int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(draws > 0 ? draws : 1));
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < draws; ++k) {
        double u = u01(draw(seed, 6, (uint64_t)k));
        int64_t lo = 0, hi = n - 1;
        while (lo < hi) { int64_t mid = (lo + hi) >> 1; if (cdf[mid] > u) hi = mid; else lo = mid + 1; }
        col[k] = idmap[lo];
    }
    free(cdf); free(idmap);
    int32_t* len = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
    int64_t nnz = canonicalise_rows(m, rp, col, len);
    free(len);
    float* val = (float*)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < nnz; ++k) val[k] = (float)(1.0 - u01(draw(seed, 7, (uint64_t)k)));
    int32_t* rowptr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    for (int64_t i = 0; i <= m; ++i) rowptr[i] = (int32_t)rp[i];
    free(rp);
    *rowptr_out = rowptr;
    *col_out = (int32_t*)realloc(col, sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    *val_out = val;
    return nnz;
}

/* ---------------------------------------------------------------- uniform Bernoulli pattern
 * Each cell (i, j) of an m x n matrix is kept with probability p (decided by a
 * draw keyed on the cell), values N(0, std) as floats. Output malloc'ed.      */
int64_t gen_bernoulli(int64_t m, int64_t n, double p, double std, uint64_t seed,
                      int32_t** rowptr_out, int32_t** col_out, float** val_out) {
    uint64_t thr = (p >= 1.0) ? UINT64_MAX : (uint64_t)(p * 18446744073709551616.0);
    int32_t* cnt = (int32_t*)malloc(sizeof(int32_t) * (size_t)m);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        int32_t c = 0;
        for (int64_t j = 0; j < n; ++j) c += draw(seed, 8, (uint64_t)(i * n + j)) < thr;
        cnt[i] = c;
    }
    int32_t* rowptr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m + 1));
    rowptr[0] = 0;
    for (int64_t i = 0; i < m; ++i) rowptr[i + 1] = rowptr[i] + cnt[i];
    free(cnt);
    int64_t nnz = rowptr[m];
    int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    float* val = (float*)malloc(sizeof(float) * (size_t)(nnz > 0 ? nnz : 1));
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < m; ++i) {
        int64_t k = rowptr[i];
        for (int64_t j = 0; j < n; ++j) {
            uint64_t cell = (uint64_t)(i * n + j);
            if (draw(seed, 8, cell) < thr) {
                col[k] = (int32_t)j;
                val[k] = (float)(std * normal01(seed, 9, cell));
                ++k;
            }
        }
    }
    *rowptr_out = rowptr; *col_out = col; *val_out = val;
    return nnz;
}

/* ---------------------------------------------------------------- random values
 * U(lo, hi) doubles / floats and half-normal |N(0, 1)| * scale floats,
 * indexed by position so any prefix is reproducible.                          */
void gen_uniform_f64(int64_t count, double lo, double hi, uint64_t seed, uint64_t stream, double* out) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < count; ++k) out[k] = lo + (hi - lo) * u01(draw(seed, 100 + stream, (uint64_t)k));
}

void gen_uniform_f32(int64_t count, double lo, double hi, uint64_t seed, uint64_t stream, float* out) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < count; ++k) out[k] = (float)(lo + (hi - lo) * u01(draw(seed, 100 + stream, (uint64_t)k)));
}

void gen_halfnormal_f32(int64_t count, double scale, uint64_t seed, uint64_t stream, float* out) {
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < count; ++k) out[k] = (float)(scale * fabs(normal01(seed, 200 + stream, (uint64_t)k)));
}

/* Small integers in [lo, hi] (inclusive) divided by `den`: exactly representable
 * test values for tolerance-free brute-force checks.                          */
void gen_small_ints_f64(int64_t count, int32_t lo, int32_t hi, double den, uint64_t seed,
                        uint64_t stream, double* out) {
    int64_t span = (int64_t)hi - lo + 1;
    for (int64_t k = 0; k < count; ++k)
        out[k] = (double)(lo + (int64_t)(u01(draw(seed, 300 + stream, (uint64_t)k)) * (double)span)) / den;
}

/* ---------------------------------------------------------------- sample without replacement
 * `count` distinct positions in [0, n), uniformly at random, returned ascending.
 * Partial Fisher-Yates over a scratch permutation (O(n) memory).             */
void gen_sample_positions(int64_t n, int64_t count, uint64_t seed, uint64_t stream, int32_t* out) {
    if (count <= 0) return;
    if (count > n) count = n;
    int32_t* p = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) p[i] = (int32_t)i;
    for (int64_t i = 0; i < count; ++i) {
        int64_t j = i + (int64_t)(u01(draw(seed, 400 + stream, (uint64_t)i)) * (double)(n - i));
        if (j >= n) j = n - 1;
        int32_t t = p[i]; p[i] = p[j]; p[j] = t;
    }
    memcpy(out, p, sizeof(int32_t) * (size_t)count);
    free(p);
    qsort(out, (size_t)count, sizeof(int32_t), cmp_i32);
}

/* Uniform random integers in [0, n) (with replacement), e.g. for picking rows. */
void gen_randint(int64_t count, int64_t n, uint64_t seed, uint64_t stream, int64_t* out) {
    for (int64_t k = 0; k < count; ++k) {
        int64_t v = (int64_t)(u01(draw(seed, 500 + stream, (uint64_t)k)) * (double)n);
        out[k] = v >= n ? n - 1 : v;
    }
}
