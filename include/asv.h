/*
 * asv.h -- C ABI of the adaptive SpMV/SpMSpV library for GB300 (sm_103a).
 *
 * Computes y = A x for a sparse m x n matrix A and an input vector x of any
 * density (Li, Ao, Yang, "Adaptive SpMV/SpMSpV on GPUs for Input Vectors of
 * Varied Sparsity"; problem statement Sec. II), choosing per call among a
 * family of candidate kernels built along the paper's three axes (Sec. IV):
 * computing pattern (row-major CSR pull, with or without value validation,
 * versus column-major CSC push over x's nonzeros), workload distribution
 * (one row/column per thread, a (sub-)warp per row/column, or an even split
 * of the nonzeros) and, for the push pattern, write-back (atomics, sort +
 * reduce-by-key, or privatised row-tile accumulation). The runtime procedure
 * of Sec. VI (matrix features once, vector features per call, cascaded
 * decision trees, conversion only when needed) runs on the device with no
 * host round-trip.
 *
 * Conventions for every entry point:
 *  - Pointers named d_* are device pointers (cudaMalloc'd or torch-owned);
 *    pointers named h_* are host pointers. Indices are int32, counts int64.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued on it; nothing synchronises unless the comment says so.
 *  - Every function returns an asv_status; nothing throws across the ABI.
 *    Argument errors are detected on the host before anything is enqueued.
 *    Errors that only the device can see (capacity overflow, bounded-wait
 *    timeouts, an over-long input list) are latched in a per-handle device status
 *    word and returned by the next call that synchronises (asv_get_status,
 *    asv_select, asv_matrix_features).
 *  - Value dtype is fixed per matrix handle; x and y use the same dtype:
 *    ASV_F32 float, ASV_F64 double, ASV_I32 int32 (wrap-around (+,x)),
 *    ASV_BOOL uint8 0/1 with the (OR, AND) semiring over a pattern matrix.
 *  - A handle serves one stream at a time: its workspaces are reused by every
 *    call, so calls on the same handle from different streams must be ordered
 *    by the caller.
 */
#ifndef ASV_H
#define ASV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t asv_status;
enum {
    ASV_OK = 0,
    ASV_ERR_ARG = 1,           /* null/negative argument, dtype mismatch, bad kernel id      */
    ASV_ERR_NONCANONICAL = 2,  /* ASV_VALIDATE: rowptr not monotone, column out of range,
                                  or columns not strictly ascending within a row           */
    ASV_ERR_OVERFLOW = 3,      /* nnz or a dimension does not fit the int32 index layout     */
    ASV_ERR_CAPACITY = 4,      /* sparse output larger than y_cap (the count is still written) */
    ASV_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up                          */
    ASV_ERR_CUDA = 6,          /* a CUDA runtime call failed (see asv_last_cuda_error)        */
                               /* 7 is reserved (no checked build exists)                    */
    ASV_ERR_NOMEM = 8,         /* device allocation failed                                    */
    ASV_ERR_UNSUPPORTED = 9    /* kernel/dtype/output combination not available               */
};

typedef enum { ASV_F32 = 0, ASV_F64 = 1, ASV_BOOL = 2, ASV_I32 = 3 } asv_dtype;
typedef enum { ASV_OUT_DENSE = 0, ASV_OUT_SPARSE = 1 } asv_out_mode;

/* Candidate kernels (Sec. IV and Sec. VI-A). The paper's eight are
 * K1 PULL_THREAD ("SpMV direct"), K2 PULL_BAL ("SpMV load-balanced"),
 * K3 MPULL_THREAD, K4 MPULL_BAL (row-major SpMSpV with bitvector validation),
 * K5 PUSH_THREAD_ATOM, K6 PUSH_THREAD_SORT, K7 PUSH_BAL_ATOM, K8 PUSH_BAL_SORT
 * (column-major SpMSpV). The (sub-)warp split and the privatised write-back
 * are additions on the same axes. */
typedef enum {
    ASV_K_AUTO = -1,
    ASV_K_PULL_THREAD = 0, ASV_K_PULL_WARP = 1, ASV_K_PULL_BAL = 2,
    ASV_K_MPULL_THREAD = 3, ASV_K_MPULL_WARP = 4, ASV_K_MPULL_BAL = 5,
    ASV_K_PUSH_THREAD_ATOM = 6, ASV_K_PUSH_WARP_ATOM = 7, ASV_K_PUSH_BAL_ATOM = 8,
    ASV_K_PUSH_THREAD_SORT = 9, ASV_K_PUSH_WARP_SORT = 10, ASV_K_PUSH_BAL_SORT = 11,
    ASV_K_PUSH_THREAD_PRIV = 12, ASV_K_PUSH_WARP_PRIV = 13, ASV_K_PUSH_BAL_PRIV = 14,
    ASV_K_COUNT = 15
} asv_kernel;

/* Handle creation flags. */
enum {
    ASV_BORROW = 0,         /* default: the caller keeps the CSR arrays alive and unchanged
                               for the handle's lifetime                                   */
    ASV_COPY = 1u << 0,     /* the handle copies the CSR arrays into memory it owns        */
    ASV_VALIDATE = 1u << 1  /* check canonical CSR on the device during create (syncs)     */
};

typedef struct asv_matrix_s* asv_matrix;

/* Matrix features of Table 1 (models 1 and 2), computed once per matrix on
 * the device (Sec. VI-C). relative_range = (max_row - min_row) / n as
 * printed; var_nnz_row is the population standard deviation of the row
 * lengths; gini is the Gini coefficient of the row lengths. */
typedef struct {
    int64_t m, n, nnz, max_row, min_row;
    double avg_row, relative_range, var_nnz_row, gini;
} asv_mfeat;

/* Vector features of Table 1 (models 1 and 3), per input vector:
 * nnz_s = number of effective matrix nonzeros = sum of the lengths of the
 * columns j listed in x; m_sparsity = nnz_s / nnz; x_sparsity = nnz_x / n. */
typedef struct {
    int64_t nnz_x, nnz_s;
    double x_sparsity, m_sparsity;
} asv_vfeat;

/* ---------------------------------------------------------------- handle */

/* Create a handle for the m x n CSR matrix (d_rowptr[m+1], d_colidx[nnz],
 * d_val[nnz] of `dtype`; d_val must be NULL for ASV_BOOL and may be NULL for
 * ASV_I32/ASV_F32/ASV_F64 to mean all-ones). Builds, on the device, the CSC
 * view (colptr[n+1], rowidx[nnz], values) with rows ascending in each column
 * and the CSC->CSR position map (Sec. VI-A: both formats stay resident so no
 * matrix conversion happens per call), the matrix features of Table 1, the
 * nnz-balanced tile partition, and all per-call workspaces. CSR must be
 * canonical (rowptr[0] = 0, non-decreasing, columns strictly ascending per
 * row); ASV_VALIDATE checks this and fails with ASV_ERR_NONCANONICAL.
 * Synchronises `stream` once at the end. The handle owns everything it
 * allocates; with ASV_BORROW it keeps pointers to the caller's CSR arrays. */
asv_status asv_matrix_create_csr(asv_matrix* out, int64_t m, int64_t n, int64_t nnz,
                                 const int32_t* d_rowptr, const int32_t* d_colidx,
                                 const void* d_val, int32_t dtype, uint32_t flags,
                                 void* stream);

/* Transposed view (Sec. II: row-major access reads A in CSR, column-major
 * access in CSC, and A's CSC arrays are exactly the CSR arrays of A^T):
 * *At becomes an n x m handle for A^T whose
 * CSR is A's CSC and whose CSC is A's CSR, borrowed from A with no copy of
 * any pointer, index or value array. The view computes its own Table 1
 * features (A^T's row lengths are A's column lengths), nnz-balanced
 * partition, long-row segments and per-call workspaces, and its CSC -> CSR
 * map (the inverse of A's), so every entry point taking a handle computes
 * with A^T: y = A^T x through asv_spmv / asv_spmspv with the selector or a
 * forced candidate. Lifetime: A must outlive At -- asv_matrix_destroy(A)
 * returns ASV_ERR_ARG while A has live views. Values: the view reads A's
 * arrays in place, so asv_matrix_update_values(A, ...) updates both, and
 * asv_matrix_update_values on the view returns ASV_ERR_UNSUPPORTED. The
 * current device must be A's (else ASV_ERR_ARG), and A's CSR arrays must
 * start on 16-byte boundaries (every cudaMalloc or torch allocation does,
 * as do ASV_COPY handles; else ASV_ERR_UNSUPPORTED), because the view's
 * column-major kernels read them with 16-byte loads. Synchronises `stream`. */
asv_status asv_matrix_transpose_view(asv_matrix A, asv_matrix* At, void* stream);

/* Release the handle and everything it owns (synchronises its device).
 * Returns ASV_ERR_ARG, and releases nothing, while transposed views of A
 * are alive. */
asv_status asv_matrix_destroy(asv_matrix A);

/* Copy the Table 1 matrix features to *h_out (synchronises). */
asv_status asv_matrix_features(asv_matrix A, asv_mfeat* h_out);

/* Expose the handle's device arrays (read-only, owned by the handle):
 * CSR (rowptr, colidx, val) and CSC (colptr, rowidx, val_csc, perm) where
 * perm[p] = CSR position of the entry at CSC position p. Any out-pointer may
 * be NULL. For ASV_BOOL the value pointers are NULL. */
asv_status asv_matrix_arrays(asv_matrix A, const int32_t** d_rowptr, const int32_t** d_colidx,
                             const void** d_val, const int32_t** d_colptr,
                             const int32_t** d_rowidx, const void** d_val_csc,
                             const int32_t** d_perm);

/* Copy the CSC view (Sec. VI-A) into caller-owned device buffers, any of
 * which may be NULL: d_colptr[n+1], d_rowidx[nnz], d_val_csc[nnz] (value
 * dtype; ignored for ASV_BOOL), d_perm[nnz] (CSC position -> CSR position).
 * Enqueued on `stream`. */
asv_status asv_matrix_copy_csc(asv_matrix A, int32_t* d_colptr, int32_t* d_rowidx, void* d_val_csc,
                               int32_t* d_perm, void* stream);

/* The stored values changed (same pattern): refresh the handle's CSC copy
 * of them. With d_val NULL, or equal to the array a borrowed handle reads,
 * the current CSR values are re-gathered; a handle created with ASV_COPY
 * first copies d_val[nnz] into its own array. Not for ASV_BOOL handles or
 * handles created without values (ASV_ERR_UNSUPPORTED). Enqueued on `stream`. */
asv_status asv_matrix_update_values(asv_matrix A, const void* d_val, void* stream);

/* ---------------------------------------------------------------- products */

/* y = A x with x dense (d_x[n]) and y dense (d_y[m]), overwritten
 * (the traditional SpMV of Sec. IV-A when a pull kernel runs); d_y must not
 * overlap d_x. `kernel` is a
 * candidate id or ASV_K_AUTO; with AUTO the device computes the vector
 * features of x, evaluates the selector and runs the chosen candidate
 * (which may be a push kernel when x is sparse in value). */
asv_status asv_spmv(asv_matrix A, const void* d_x, void* d_y, int32_t kernel, void* stream);

/* y = A x for x given either dense (d_x_dense[n], then d_nnz_x/d_xidx/d_xval
 * are ignored and x's nonzeros are those with x_j != 0 by IEEE comparison)
 * or sparse (d_x_dense NULL; *d_nnz_x is a device int64 count, d_xidx[nnz_x]
 * distinct column ids in [0, n) in any order -- NULL allowed only when the
 * count is 0 -- and d_xval[nnz_x] values, ignored for ASV_BOOL and NULL to
 * mean all-ones). A list longer than n latches ASV_ERR_ARG and is clamped. Listed entries are structural even when their value
 * is zero. Output (Sec. IV-B write-back):
 *  - ASV_OUT_DENSE: d_y[m] is overwritten with A x;
 *  - ASV_OUT_SPARSE: the structural output set -- rows with at least one
 *    effective entry (an entry whose column is a nonzero of x), ascending --
 *    is written to d_yidx[], its values to d_yval[] (NULL allowed for
 *    ASV_BOOL), and its size to the device int64 *d_nnz_y. At most y_cap
 *    entries are written; a larger set latches ASV_ERR_CAPACITY.
 * Dense/sparse conversion of x happens on the device only when the chosen
 * kernel needs the other format (Sec. VI-A/VI-C); a list of every column in
 * order (d_xidx[t] = t) is read in place, and a list output that holds every
 * row is written in place, so the output arrays (d_y, d_yidx, d_yval,
 * d_nnz_y) must not overlap any input array (x's count, list or dense
 * vector): the kernels may still read x while they write y. No
 * synchronisation. */
asv_status asv_spmspv(asv_matrix A, const int64_t* d_nnz_x, const int32_t* d_xidx,
                      const void* d_xval, const void* d_x_dense, int32_t out_mode,
                      void* d_y, int32_t* d_yidx, void* d_yval, int64_t* d_nnz_y,
                      int64_t y_cap, int32_t kernel, void* stream);

/* y = A x restricted by an output mask (an extension for the BFS application
 * of Sec. VII; the paper's kernels have no mask): d_ymask[(m + 31) / 32] is a
 * device bitmap, bit i (word i / 32, bit i % 32) set = row i is excluded.
 * Excluded rows are not computed by the pull kernels (their y_i is 0 in the
 * dense output) and never enter the sparse output set; the push kernels drop
 * their entries. Other arguments, errors and formats as asv_spmspv; d_ymask
 * must not be NULL (ASV_ERR_ARG) and must stay unchanged until the call has
 * run. The selector does not look at the mask. No synchronisation. */
asv_status asv_spmspv_masked(asv_matrix A, const uint32_t* d_ymask, const int64_t* d_nnz_x,
                             const int32_t* d_xidx, const void* d_xval, const void* d_x_dense,
                             int32_t out_mode, void* d_y, int32_t* d_yidx, void* d_yval,
                             int64_t* d_nnz_y, int64_t y_cap, int32_t kernel, void* stream);

/* Incremental (delta-form) PageRank over a square FP32 or FP64 handle (the
 * incremental PageRank application of Sec. VII; the paper gives no formula,
 * this is the delta iteration of the power method): rank = sum of delta_k,
 * delta_0 = (1 - damping)/n on every vertex, delta_{k+1} = damping *
 * A D^{-1} delta_k with D the column counts of A (a column without entries
 * contributes 0) and A's stored values as edge weights (all ones for the
 * plain PageRank). After each product the entries with |delta| < eps are
 * dropped, so the input vector of the product turns sparse as the iteration
 * converges and the selector (kernel = ASV_K_AUTO) moves from pull to push
 * kernels on its own; eps = 0 keeps every entry (the exact power series).
 * d_rank[n] (device, the handle's value type, caller-owned) receives the
 * rank; *h_iters (may be NULL) the number of products run (at most
 * max_iter; fewer when the delta list empties). The iterations run on the
 * device as one CUDA graph (a WHILE node over product + update, no host
 * round trip per iteration); the call synchronises `stream` once, at the
 * end, only when h_iters is given. The first call allocates the handle's
 * driver workspaces, the first call with each `kernel` builds its graph.
 * Errors: ASV_ERR_ARG (non-square, n = 0, damping outside [0, 1),
 * eps < 0, max_iter < 0, NULL d_rank), ASV_ERR_UNSUPPORTED (Boolean or int32
 * handle). */
asv_status asv_pagerank(asv_matrix A, double damping, double eps, int32_t max_iter, void* d_rank,
                        int32_t kernel, int32_t* h_iters, void* stream);

/* Breadth-first search from vertex `source` over the pattern of a square
 * handle (any value type; a Boolean handle is the cheap one): d_level[n]
 * (device int32, caller-owned) receives each vertex's level, 0 for the
 * source and -1 for vertices not reached. A vertex i is reached from j when
 * A stores entry (i, j) -- the direction of y = A x; for a symmetric pattern
 * this is the ordinary undirected search. Each level is one masked product
 * (frontier in, unvisited rows out, as a sparse list) run by `kernel`
 * (ASV_K_AUTO: the selector chooses per level). *h_depth (may be NULL)
 * receives the number of levels including the source's. The levels run on
 * the device as one CUDA graph (a WHILE node over product + level step, no
 * host round trip per level); the call synchronises `stream` once, at the
 * end, only when h_depth is given. The first call allocates the handle's
 * search workspaces (bitmap, two frontier lists), the first call with each
 * `kernel` builds its graph. The workspaces and graphs belong to the handle:
 * searches on one handle must not overlap in time. Errors: ASV_ERR_ARG for a
 * non-square handle, n = 0, a source outside [0, n) or a NULL d_level. */
asv_status asv_bfs(asv_matrix A, int32_t source, int32_t* d_level, int32_t kernel, int32_t* h_depth,
                   void* stream);

/* Run the feature pass and the selector for this x (same x arguments as
 * asv_spmspv) and an output in `out_mode` (the trees are per call format:
 * x dense or a list, y dense or the structural list), and return the kernel
 * an ASV_K_AUTO call with these arguments would run and the vector features
 * (Sec. V-A Table 1, Sec. VI-B cascaded trees). Nothing is written to any
 * output. Synchronises `stream`. */
asv_status asv_select(asv_matrix A, const int64_t* d_nnz_x, const int32_t* d_xidx,
                      const void* d_xval, const void* d_x_dense, int32_t out_mode,
                      int32_t* h_kernel, asv_vfeat* h_feat, void* stream);

/* The kernel id chosen by the most recent ASV_K_AUTO call on this handle
 * (synchronises `stream`). */
asv_status asv_last_kernel(asv_matrix A, int32_t* h_kernel, void* stream);

/* Dense -> sparse conversion of x (Sec. VI-A online conversion; Sec. VI-C
 * stream compaction): writes the ascending indices j with x_j != 0 (IEEE;
 * -0.0 is zero, NaN is nonzero) to d_idx[], their values to d_val[] (may be
 * NULL), and the count to the device int64 *d_count. d_idx must hold n
 * entries. Uses the handle's workspaces (x has length A's n). */
asv_status asv_compact(asv_matrix A, const void* d_x_dense, int32_t* d_idx, void* d_val,
                       int64_t* d_count, void* stream);

/* ---------------------------------------------------------------- batched */

/* Tiling of the batched product.
 * hot_columns = 0: the column-list kernel -- rows of A per work item (4, 8 or
 *   16) and vectors per group (rows * (vectors + 1) * 8 bytes of shared
 *   memory, one compensated FP32 pair per output, <= 200 KB).
 * hot_columns = 64 or 128: the hot-column kernel -- at most that many columns
 *   shared by many vectors are multiplied as a dense block (rows per item 8 or
 *   16, vectors per group 128 or 256 = threads per block), the other entries
 *   are added through shared-memory atomics (results within tolerance, not
 *   bitwise reproducible from call to call). Its workspaces (first use) take
 *   about 16 bytes per nonzero of A plus 4 * n * (B / vectors + 1) bytes.
 * Other values give ASV_ERR_ARG. */
typedef struct {
    int32_t rows_per_tile;
    int32_t vectors_per_group;
    int32_t hot_columns;
} asv_tune;

/* Y[b,:] = A x_b for B vectors at once (FP32 handles; a batched form of the
 * SpMSpV of Sec. II). The batch is a CSR of vectors -- d_xptr[B+1] device
 * int64 offsets (relative to d_xptr[0]), d_xidx column ids in [0, n),
 * distinct within a vector, d_xval values (NULL = ones) -- or, when
 * d_X_dense is not NULL, a dense row-major [B][n] array whose nonzeros are
 * taken. d_Y is a dense row-major [B][m] output, fully overwritten. max_entries
 * bounds the total number of listed entries (ignored for dense input); a
 * batch with more entries latches ASV_ERR_CAPACITY. `tune` may be NULL (use
 * the handle's setting, see asv_autotune_batched). One call is one CUDA-graph
 * launch of the captured pipeline (regroup by column with a radix sort, then
 * a persistent kernel over row-tile x vector-group work items); the first call
 * with a new B or tiling, or one that needs larger workspaces, allocates and
 * captures, so it should not itself be inside a stream capture. */
asv_status asv_spmspv_batched(asv_matrix A, int32_t B, int64_t max_entries, const int64_t* d_xptr,
                              const int32_t* d_xidx, const void* d_xval, const void* d_X_dense,
                              void* d_Y, const asv_tune* tune, void* stream);

/* Times the candidate tilings on this batch (same arguments as
 * asv_spmspv_batched), keeps the fastest in the handle and returns it in
 * *h_best (may be NULL). With cache_path, a line "<gpu>|<matrix>|B=..\tR\tGB"
 * is read if present (no timing) or appended. Synchronises `stream`. */
asv_status asv_autotune_batched(asv_matrix A, int32_t B, int64_t max_entries, const int64_t* d_xptr,
                                const int32_t* d_xidx, const void* d_xval, const void* d_X_dense,
                                void* d_Y, const char* cache_path, asv_tune* h_best, void* stream);

/* Backward pass of Y[b,:] = A x_b (FP32 handles, 1 <= B <= 128): given dense
 * row-major d_dY[B][m] (and d_X[B][n], needed for dA), writes
 * d_dX[B][n] = dY A (dx_b = A^T dy_b, read through the CSC view) and
 * d_dA[nnz] (CSR order) with dA_k = sum_b dy_b[row(k)] * x_b[col(k)], the
 * gradient of the stored values on A's pattern. Either output may be NULL. */
asv_status asv_spmspv_backward(asv_matrix A, int32_t B, const void* d_X, const void* d_dY, void* d_dX,
                               void* d_dA, void* stream);

/* ---------------------------------------------------------------- single-call tuning */

/* Launch shape of the pull candidates; it changes their speed, never their
 * result. lanes: lanes per row of the sub-warp pull (2, 4, 8, 16 or 32);
 * unroll: rows per lane group loaded together (2 or 4); tma: 1 = the
 * one-row-per-thread pull stages each warp's span with TMA bulk copies. */
typedef struct {
    int32_t lanes;
    int32_t unroll;
    int32_t tma;
} asv_pull_tune;

/* Per-matrix tuner of the single-call kernels (the counterpart of
 * asv_autotune_batched for the plain product): times the pull candidates'
 * launch shapes on a dense x of ones -- lanes x unroll of the sub-warp pull,
 * starting from the creation-time choice and moving outwards, then TMA
 * staging on or off for the one-row-per-thread pull -- until budget_ms of
 * wall time has passed, and keeps the fastest in the handle (later calls,
 * forced or selector-driven, use it). With cache_path, a line
 * "<gpu>|m=..|n=..|nnz=..|max_row=..|dtype=..|pull\tlanes\tunroll\ttma" is
 * read if present (no timing) or appended. *h_out (may be NULL) receives the
 * settings kept. Allocates and frees a scratch x and y; synchronises `stream`.
 * The handle's other calls must not run concurrently. */
asv_status asv_autotune(asv_matrix A, const char* cache_path, uint32_t budget_ms, asv_pull_tune* h_out,
                        void* stream);

/* The handle's current pull launch shape (creation-time choice or the
 * tuner's). */
asv_status asv_pull_tuning(asv_matrix A, asv_pull_tune* h_out);

/* Backward pass of the same product with the batch listed instead of dense:
 * X as a CSR of vectors -- d_xptr[B+1] device int64 offsets (relative to
 * d_xptr[0]), d_xidx column ids in [0, n), distinct within a vector, d_xval
 * values (NULL = ones) -- as asv_spmspv_batched takes it. Writes d_dX[B][n]
 * = dY A and d_dA[nnz] (CSR order), dA_k = sum_b dy_b[row(k)] * x_b[col(k)]
 * (only the listed entries of x contribute). The list is converted on the
 * device into the vector-minor dense layout the dA kernel reads; a column id
 * outside [0, n) is skipped and latches ASV_ERR_ARG. FP32 handles,
 * 1 <= B <= 128; either output may be NULL (d_xptr is needed for dA). */
asv_status asv_spmspv_backward_list(asv_matrix A, int32_t B, const int64_t* d_xptr,
                                    const int32_t* d_xidx, const void* d_xval, const void* d_dY,
                                    void* d_dX, void* d_dA, void* stream);

/* ---------------------------------------------------------------- selector */

/* Replace the handle's decision trees (cascaded CART trees: computing
 * pattern, then workload distribution given the pattern, then write-back for
 * the push pattern; Sec. V-B / VI-B). `nodes` holds n_nodes (<= 2048) records
 * of 5 doubles {feature, threshold, left, right, leaf_class}; feature < 0
 * marks a leaf. h_roots[20] holds five roots for each of the four call
 * formats (x dense, y dense), (x dense, y list), (x list, y dense),
 * (x list, y list): the pattern tree, the distribution trees applied after
 * pattern 0 (push), 1 (masked pull) and 2 (pull), and the write-back tree.
 * Feature indices: 0 m, 1 n, 2 nnz, 3 max_row, 4 min_row, 5 avg_row,
 * 6 relative_range, 7 var_nnz_row, 8 gini, 9 nnz_x, 10 x_sparsity, 11 nnz_s,
 * 12 m_sparsity. A node sends x left when feature <= threshold.
 * Pattern classes: 0 push, 1 masked pull, 2 pull. Distribution classes:
 * 0 thread, 1 warp, 2 balanced. Write-back classes: 0 atomic, 1 sort,
 * 2 privatised. Synchronises `stream`. */
asv_status asv_set_trees(asv_matrix A, const double* h_nodes, int32_t n_nodes,
                         const int32_t* h_roots, void* stream);

/* ---------------------------------------------------------------- allocation-free */

/* y = A x (FP32, x and y dense) for caller-owned CSR arrays d_rowptr[m+1],
 * d_colidx[nnz], d_val[nnz] (NULL = all ones), without allocating device
 * memory and without a handle. The paper has no counterpart: this is for
 * callers that must not allocate on their call path -- real-time loops in
 * which cudaMalloc or cudaFree would synchronise the device, runtimes that
 * give all device memory to their own pool at start-up, and one-off products
 * on borrowed arrays that cannot afford a handle (which allocates the CSC view
 * and workspaces). It runs the balanced (merge-path) candidate, whose scratch
 * -- the tile table and the carries of rows that span tiles -- lives in one
 * fixed 4 MB device array inside the library, held by every GPU that loads
 * the library until the process exits. Limit: m + nnz <= 2^29 (2^18 tiles of
 * 2048 items); larger sizes return ASV_ERR_CAPACITY before anything runs.
 * The arrays must be a valid CSR -- rowptr[0] = 0, rowptr non-decreasing,
 * rowptr[m] = nnz, 0 <= colidx[k] < n -- and are NOT checked (no handle, no
 * validation pass): the kernel only keeps every memory access inside the
 * stated array sizes, so malformed arrays give an unspecified y, never an
 * access outside them. The first call on a device looks up the array's device
 * address (once per device; the address is kept, so do not use this entry
 * point on a device after cudaDeviceReset), so make that first call before
 * any stream capture. All calls
 * share the array: calls whose work overlaps on the GPU (different streams,
 * or different host threads, without ordering) race on it. Each call
 * rewrites every scratch entry it reads, so nothing needs clearing between
 * calls. Enqueued on `stream`; no synchronisation. */
asv_status asv_spmv_noalloc_f32(int64_t m, int64_t n, int64_t nnz, const int32_t* d_rowptr,
                                const int32_t* d_colidx, const float* d_val, const float* d_x,
                                float* d_y, void* stream);

/* ---------------------------------------------------------------- testing hooks */

/* Default number of polls of a bounded device-side wait. */
#define ASV_WAIT_LIMIT_DEFAULT (1u << 24)

/* Failure injection for tests, on the host side of the device's bounded
 * waits (no GPU fault, trap or hang is ever provoked). Sets how many times
 * the first bounded wait of the handle's TMA-staged kernels (the one-row-per-
 * thread pull waiting for its bulk copies of a warp's span) polls its
 * mbarrier before it gives up and latches ASV_ERR_TIMEOUT; the warp then
 * waits for its copies again under the default bound, so none is left in
 * flight, and leaves its rows unwritten. polls = 0 makes every such wait
 * give up at once; ASV_WAIT_LIMIT_DEFAULT restores the default. The status
 * is read (and cleared) by asv_get_status. */
asv_status asv_debug_set_wait_limit(asv_matrix A, uint32_t polls);

/* Failure injection for tests: with countdown k > 0, the k-th device
 * allocation of a handle's arrays and workspaces (asv_matrix_create_csr,
 * asv_matrix_transpose_view) from now on fails as if the device were out of
 * memory; the creating call then releases whatever it had allocated and
 * returns ASV_ERR_NOMEM. 0 disarms it. Process-wide. */
void asv_debug_fail_alloc(int32_t countdown);

/* ---------------------------------------------------------------- status */

/* Latched device status of the handle (synchronises `stream`); clears it. */
asv_status asv_get_status(asv_matrix A, void* stream);

/* Last CUDA error code seen by the library on this thread (0 if none). */
int32_t asv_last_cuda_error(void);

/* Human-readable name of a status code (static string). */
const char* asv_status_string(asv_status s);

/* Library version as major*10000 + minor*100 + patch. */
int32_t asv_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ASV_H */
