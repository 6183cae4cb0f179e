// Host-side internals shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <vector>

#include "common.cuh"
#include "selector.cuh"

namespace asv {
// Per-call arguments of the vector-feature pass (written into the call descriptor).
struct DescInit {
    const void* x_dense;
    const uint32_t* xbits;
    const int32_t* xidx;
    const void* xval;
    void* y;
    int32_t* yidx;
    void* yval;
    int64_t* nnz_y;
    int64_t y_cap;
    const void* user_x_dense;
    const int32_t* user_xidx;
    const void* user_xval;
    const int64_t* user_nnz_x;
    const uint32_t* ymask;  // output mask (NULL = none)
    int32_t out_mode;
    int32_t x_sparse;
    // a list output whose set is every row when x reaches every column: the
    // matrix has no empty row, the output has values and room for m entries
    // (the output mask, set after this, is checked on the device)
    int32_t y_ident_ok;
};

// Device-resident state of a driver loop (BFS, PageRank). The loop graph is
// built once per handle with fixed pointers, so what changes from call to
// call -- the caller's output array and the scalar arguments -- is written
// here by the driver's init kernel and read by its step kernel.
struct LoopState {
    void* out;            // BFS: the level array; PageRank: the rank
    int64_t iter;         // BFS: level the next frontier gets; PageRank: products run
    int64_t max_iter;     // bound on iter (BFS: n, which no search reaches)
    double p0, p1;        // PageRank: damping, eps
    unsigned int ticket;  // last-block ticket of the step kernel, re-zeroed by that block
};
}  // namespace asv

// Workspaces of the batched forward/backward forms, grown on demand.
struct BatchWs {
    uint32_t* keys[2] = {nullptr, nullptr};
    uint64_t* pay[2] = {nullptr, nullptr};
    int64_t* xptr = nullptr;  // [cap_B+1] offsets, then the entry count
    int32_t* cptr = nullptr;  // [n+1] column pointers of the regrouped batch
    void* desc = nullptr;     // device BatchDesc
    unsigned long long* queue = nullptr;  // work queue + ticket (zero-invariant)
    int64_t cap_entries = 0;
    int32_t cap_B = 0;
    std::map<long long, cudaGraphExec_t> graphs;  // captured pipelines by (B, R, GB)
    void* dYt = nullptr;
    void* Xt = nullptr;
    void* dXt = nullptr;
    int32_t bwd_B = 0;
    // hot-column path: column -> hot slot, control words (histogram, threshold,
    // count), dense [hot][B] block of the batch's hot entries
    int32_t* hot_id = nullptr;
    int32_t* hot_ctl = nullptr;
    void* xh = nullptr;
    int64_t xh_cap = 0;
    // A's entries split per row into hot (slot, a) and cold (column, a) lists,
    // and the cold columns' vector-tile bounds
    int32_t* hrow = nullptr;
    int32_t* crow = nullptr;
    void* hent = nullptr;
    void* cent = nullptr;
    void* tb = nullptr;
    int64_t tb_cap = 0;
};

struct asv_matrix_s {
    int dev = 0;
    int32_t dtype = ASV_F32;
    int64_t m = 0, n = 0, nnz = 0;
    uint32_t flags = 0;
    int num_sms = 0;
    // CSR (borrowed or owned) and CSC (owned)
    const int32_t* rowptr = nullptr;
    const int32_t* col = nullptr;
    const void* val = nullptr;
    bool owns_val = false;
    int32_t* colptr = nullptr;
    int32_t* rowidx = nullptr;
    void* val_csc = nullptr;
    int32_t* perm = nullptr;
    // features (Table 1)
    asv::MatFeat* d_mfeat = nullptr;
    asv_mfeat h_mfeat{};
    // nnz-balanced (merge-path) partition of the pull pattern
    int32_t* tile_row = nullptr;
    int64_t ntiles = 0;
    int32_t* carry_row = nullptr;
    void* carry_val = nullptr;
    // rows over kLongRow entries, cut into segments of at most kLongSeg:
    // segment s = {row, begin, end, 1 if it is the whole row}: entries
    // [begin, end) of the row, at most kLongSeg of them; a row's segments are
    // consecutive and ascending. Rows with several segments are listed in
    // multi_row with their first segment in multi_base; their partial sums
    // go to long_part / long_hit.
    int4* seg = nullptr;
    uint64_t* long_part = nullptr;
    uint8_t* long_hit = nullptr;
    int32_t* multi_row = nullptr;
    int32_t* multi_base = nullptr;
    int64_t nseg = 0, nmulti = 0;
    // Boolean handles: pieces of long-row segments handed to the second pass
    // of a list-output product, and their count (reset by the feature pass)
    int4* long_rest = nullptr;
    unsigned int* long_rest_n = nullptr;
    int pull_lanes = 8;   // lanes per row of the (sub-)warp pull kernels
    int pull_unroll = 4;  // rows per lane group loaded together (2: more resident warps)
    bool pull_tma = true; // one-row-per-thread pull stages its spans with TMA bulk copies
    // polls of the first bounded wait on a TMA copy (asv_debug_set_wait_limit)
    uint32_t wait_limit = 1u << 24;
    // selector tables
    asv::TreeNode* d_trees = nullptr;
    // the table's roots and, per call format, the window of nodes a feature
    // pass stages (kernel arguments of every selector-enabled pass)
    int32_t h_roots[asv::kRootsLen] = {};
    int32_t win_lo[4] = {0, 0, 0, 0}, win_hi[4] = {0, 0, 0, 0};
    // per call format: its pattern tree starts with a feature that a listed
    // x gives for free (the lazy evaluation of the list feature pass)
    int32_t lazy_ok[4] = {0, 0, 0, 0};
    // per-call state
    asv::CallDesc* d_desc = nullptr;
    asv::Ws ws{};
    int32_t* d_last_kid = nullptr;
    // graphs of the selector-driven path, one per (x format, output mode)
    cudaGraph_t graph[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    cudaGraphExec_t gexec[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    cudaGraphNode_t feat_node[2][2] = {{nullptr, nullptr}, {nullptr, nullptr}};
    unsigned long long cond[2][2] = {{0, 0}, {0, 0}};
    asv::DescInit last_di[2][2];  // arguments the feature node of each graph was last given
    cudaStream_t cap_stream = nullptr;
    // while a direct candidate chain of a selector graph is captured: the
    // candidate whose chain it is (the Gate of its kernels), else -1
    int32_t gate_kid = -1;
    // an FP32 matrix whose rows have at most kNarrowRow entries: the push with
    // atomic write-back and a dense output adds in FP32, and the one-row-per-
    // thread pull sums a row with a plain FMA chain (their error bounds stay
    // within the FP32 tolerance, see push.cu and pull.cu)
    bool narrow_acc = false;
    // columns of more than kLongSeg entries: the hub count of a listed x that
    // holds every column, which the feature pass then need not gather
    int64_t hub_cols = 0;
    // the long-row pass of the thread and sub-warp pulls runs beside the
    // short-row kernel: a side stream joined by two events (in a graph
    // capture they become a fork and a join of the captured graph)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int G = 0;  // fixed grid of the scan / sort / compaction primitives
    BatchWs bws;
    int32_t tune_R = 8, tune_GB = 1024, tune_hot = 0;  // batched tiling chosen by the autotuner
    // breadth-first search (first asv_bfs call): visited bitmap, the current
    // and the next frontier list, their device counts, the loop state, a
    // pinned host scalar, and one loop graph per kernel id (AUTO first)
    uint32_t* bfs_visited = nullptr;
    int32_t* bfs_front[2] = {nullptr, nullptr};
    int64_t* bfs_count = nullptr;
    asv::LoopState* bfs_state = nullptr;
    int64_t* bfs_hcount = nullptr;
    cudaGraph_t bfs_graph[ASV_K_COUNT + 1] = {};
    cudaGraphExec_t bfs_exec[ASV_K_COUNT + 1] = {};
    // incremental PageRank (first asv_pagerank call): the product's input
    // list (index, scaled delta), its sparse output, the counts ([0] input,
    // [1] next input being appended, [2] output), the loop state and graphs
    int32_t* pr_xidx = nullptr;
    void* pr_xval = nullptr;
    int32_t* pr_yidx = nullptr;
    void* pr_yval = nullptr;
    int64_t* pr_count = nullptr;
    asv::LoopState* pr_state = nullptr;
    cudaGraph_t pr_graph[ASV_K_COUNT + 1] = {};
    cudaGraphExec_t pr_exec[ASV_K_COUNT + 1] = {};
    std::vector<void*> allocs;
    // transposed views: a view borrows its parent's CSR and CSC arrays, so
    // the parent counts its live views and is not destroyed before them
    asv_matrix_s* parent = nullptr;
    int views = 0;
};

namespace asv {

size_t vsize(int32_t dtype);

const char* kernel_name(int k);

// matrix.cu -- run once at handle creation
cudaError_t build_csc(asv_matrix_s* H, cudaStream_t s);
cudaError_t build_features(asv_matrix_s* H, cudaStream_t s);
cudaError_t build_partition(asv_matrix_s* H, cudaStream_t s);
// counts the long rows (synchronises), allocates and fills their segment list
cudaError_t build_long_rows(asv_matrix_s* H, cudaStream_t s);
// hub_cols: the columns longer than kLongSeg (synchronises)
cudaError_t count_hub_columns(asv_matrix_s* H, cudaStream_t s);
int64_t pull_tile_items(int32_t dtype);
cudaError_t validate_csr(asv_matrix_s* H, cudaStream_t s, int32_t* d_flag);
cudaError_t regather_values(asv_matrix_s* H, cudaStream_t s);
// inv[perm[p]] = p for p < nnz
cudaError_t invert_perm(const int32_t* perm, int64_t nnz, int32_t* inv, cudaStream_t s);

// bfs.cu -- the two driver loops, each run as a CUDA graph WHILE node whose
// body is one selector-driven product followed by the step kernel below;
// the step kernel's last block sets the loop condition
void launch_bfs_init(int32_t source, int64_t n, int32_t* level, uint32_t* visited, int32_t* front, int64_t* count,
                     LoopState* st, cudaStream_t s);
void launch_bfs_step(const int32_t* next, int64_t* count, int32_t* front, uint32_t* visited, LoopState* st,
                     unsigned long long loop, int grid, cudaStream_t s);
void launch_pr_init(int32_t dtype, int64_t n, double damping, double eps, int32_t max_iter, void* rank,
                    const int32_t* colptr, int32_t* xidx, void* xval, int64_t* count, LoopState* st, int grid,
                    cudaStream_t s);
void launch_pr_step(int32_t dtype, const int32_t* yidx, const void* yval, int64_t* count, const int32_t* colptr,
                    int32_t* xidx, void* xval, LoopState* st, unsigned long long loop, int grid, cudaStream_t s);

// shared scan launcher (device-side count allowed)
void scan_excl(const int32_t* in, int32_t* out, int64_t n_h, const int64_t* n_d, int32_t* blk, int G,
               bool write_total, cudaStream_t s);

// vector.cu -- per call
// A feature-pass launch whose argument storage lives in the struct.
struct FeatLaunch {
    void* func;
    dim3 grid, block;
    void* args[12];
    const void* xptr;
    int64_t hub_cols;
    const int64_t* nnz_x_dev;
    const int32_t* xidx;
    int64_t n, nnz;
    const int32_t* colptr;
    uint32_t* xbits;
    unsigned long long* counters;
    unsigned int* ticket;
    CallDesc* desc;
    DescInit di;
    int32_t* status;
    SelectArg sa;
};
void feature_launch(asv_matrix_s* H, const DescInit& di, const SelectArg& sa, FeatLaunch& fl);
void launch_features(asv_matrix_s* H, const DescInit& di, const SelectArg& sa, cudaStream_t s);
void launch_x_scatter(asv_matrix_s* H, bool set, bool bits, cudaStream_t s);
// the Gate of the kernels launched now (see gate_kid)
inline Gate gate_of(const asv_matrix_s* H) { return Gate{H->d_desc, H->gate_kid}; }
// bits_below > 0: skipped when x has fewer nonzeros than that (the warp push
// with atomics then reads the feature pass's bitmap instead of a list)
void launch_x_compact_list(asv_matrix_s* H, cudaStream_t s, int64_t bits_below = 0);
// narrow: the push accumulated into FP32 accumulators (narrow_acc)
void launch_finalize(asv_matrix_s* H, bool from_acc, int out_mode, cudaStream_t s, bool narrow = false);
void launch_compact_public(asv_matrix_s* H, const void* x, int32_t* idx, void* val, int64_t* count,
                           cudaStream_t s);

// pull.cu
struct PullIO {
    const void* x;
    const uint32_t* xbits;
    void* y;
    const uint32_t* ymask = nullptr;  // output mask: rows whose bit is set are not computed (y = 0)
};
void launch_pull(asv_matrix_s* H, int dist, bool masked, bool sparse_out, const PullIO* direct,
                 cudaStream_t s);

void launch_pull_bal_f32_raw(int64_t m, int64_t n, int64_t nnz, const int32_t* rowptr, const int32_t* col,
                             const float* val, const float* x, float* y, const int32_t* tile_row, int32_t* carry_row,
                             double* carry_val, int64_t ntiles, cudaStream_t s);
void launch_partition_raw(const int32_t* rowptr, int64_t m, int64_t nnz, int64_t ntiles, int32_t* tile_row,
                          cudaStream_t s);

// push.cu
// bits_below > 0 (the warp push on a dense x): an x of fewer nonzeros than
// that is read from the feature pass's bitmap, its list never built
void launch_push(asv_matrix_s* H, int dist, int wb, int out_mode, cudaStream_t s, int64_t bits_below = 0);

// batched.cu
cudaError_t batched_forward(asv_matrix_s* H, int32_t B, int64_t max_entries, const int64_t* xptr, const int32_t* xidx,
                            const float* xval, const float* Xdense, float* Y, int R, int GB, int hot,
                            cudaStream_t s);
// X dense [B][n], or (xptr != NULL) listed as a CSR of vectors
cudaError_t batched_backward(asv_matrix_s* H, int32_t B, const float* X, const float* dY, float* dX, float* dA,
                             cudaStream_t s, const int64_t* xptr = nullptr, const int32_t* xidx = nullptr,
                             const float* xval = nullptr);
void batch_release(asv_matrix_s* H);

// select.cu
// fmt: the call format 2 * (x listed) + (sparse output) the feature node
// serves; its trees, roots and lazy hint go into the arguments
SelectArg select_arg(asv_matrix_s* H, unsigned long long cond, int fmt);
// records a node table's roots and recomputes the per-format windows and
// lazy hints from it
void update_lazy(asv_matrix_s* H, const std::vector<TreeNode>& nodes, const int32_t* roots);
void default_trees(int32_t dtype, std::vector<TreeNode>& nodes, int32_t roots[kRootsLen]);

}  // namespace asv
