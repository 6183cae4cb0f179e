// C ABI of the adaptive SpMV/SpMSpV library: handle lifetime, per-call
// dispatch of the candidate kernels, and the selector-driven path (runtime
// procedure of Sec. VI): vector-feature pass -> decision trees on the device
// -> SWITCH conditional node of a CUDA graph whose branches are the
// candidates (with their own format conversion), so the chosen kernel runs
// with no host round-trip.
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <new>
#include <string>

#include "internal.h"

using namespace asv;

static thread_local int32_t g_last_cuda = 0;

#define CK(expr)                                      \
    do {                                              \
        cudaError_t e_ = (expr);                      \
        if (e_ != cudaSuccess) {                      \
            g_last_cuda = (int32_t)e_;                \
            return e_ == cudaErrorMemoryAllocation ? ASV_ERR_NOMEM : ASV_ERR_CUDA; \
        }                                             \
    } while (0)

namespace asv {
int64_t priv_bins(int64_t m);

const char* kernel_name(int k) {
    static const char* names[ASV_K_COUNT] = {
        "pull_thread", "pull_warp", "pull_bal", "mpull_thread", "mpull_warp", "mpull_bal",
        "push_thread_atom", "push_warp_atom", "push_bal_atom", "push_thread_sort", "push_warp_sort",
        "push_bal_sort", "push_thread_priv", "push_warp_priv", "push_bal_priv"};
    return (k >= 0 && k < ASV_K_COUNT) ? names[k] : "auto";
}
}  // namespace asv

// Testing hook (asv_debug_fail_alloc): when positive, the allocation that
// brings the countdown to zero fails as if the device were out of memory.
static std::atomic<int32_t> g_fail_alloc{0};

static asv_status dalloc(asv_matrix_s* H, void** p, size_t bytes, bool zero) {
    if (bytes < 16) bytes = 16;
    if (g_fail_alloc.load() > 0 && g_fail_alloc.fetch_sub(1) == 1) {
        *p = nullptr;
        return ASV_ERR_NOMEM;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        g_last_cuda = (int32_t)e;
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? ASV_ERR_NOMEM : ASV_ERR_CUDA;
    }
    H->allocs.push_back(*p);
    if (zero) {
        e = cudaMemset(*p, 0, bytes);
        if (e != cudaSuccess) {
            g_last_cuda = (int32_t)e;
            return ASV_ERR_CUDA;
        }
    }
    return ASV_OK;
}

#define AL(ptr, bytes, zero)                                               \
    do {                                                                   \
        void* p_ = nullptr;                                                \
        asv_status st_ = dalloc(H, &p_, (size_t)(bytes), zero);           \
        if (st_ != ASV_OK) { destroy_handle(H); return st_; }              \
        (ptr) = (decltype(ptr))p_;                                         \
    } while (0)

#define CKH(expr)                                                          \
    do {                                                                   \
        cudaError_t e_ = (expr);                                           \
        if (e_ != cudaSuccess) {                                           \
            g_last_cuda = (int32_t)e_;                                     \
            destroy_handle(H);                                             \
            return e_ == cudaErrorMemoryAllocation ? ASV_ERR_NOMEM : ASV_ERR_CUDA; \
        }                                                                  \
    } while (0)

static void destroy_handle(asv_matrix_s* H) {
    if (!H) return;
    cudaDeviceSynchronize();
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
            if (H->gexec[a][b]) cudaGraphExecDestroy(H->gexec[a][b]);
            if (H->graph[a][b]) cudaGraphDestroy(H->graph[a][b]);
        }
    batch_release(H);
    for (int k = 0; k <= ASV_K_COUNT; ++k) {
        if (H->bfs_exec[k]) cudaGraphExecDestroy(H->bfs_exec[k]);
        if (H->bfs_graph[k]) cudaGraphDestroy(H->bfs_graph[k]);
        if (H->pr_exec[k]) cudaGraphExecDestroy(H->pr_exec[k]);
        if (H->pr_graph[k]) cudaGraphDestroy(H->pr_graph[k]);
    }
    if (H->bfs_hcount) cudaFreeHost(H->bfs_hcount);
    if (H->cap_stream) cudaStreamDestroy(H->cap_stream);
    if (H->side_stream) cudaStreamDestroy(H->side_stream);
    if (H->ev_fork) cudaEventDestroy(H->ev_fork);
    if (H->ev_join) cudaEventDestroy(H->ev_join);
    for (void* p : H->allocs) cudaFree(p);
    delete H;
}

// Device, stream and events every handle needs; on failure H is released.
static asv_status init_handle(asv_matrix_s* H) {
    CKH(cudaGetDevice(&H->dev));
    CKH(cudaDeviceGetAttribute(&H->num_sms, cudaDevAttrMultiProcessorCount, H->dev));
    CKH(cudaStreamCreateWithFlags(&H->side_stream, cudaStreamNonBlocking));
    CKH(cudaEventCreateWithFlags(&H->ev_fork, cudaEventDisableTiming));
    CKH(cudaEventCreateWithFlags(&H->ev_join, cudaEventDisableTiming));
    H->G = H->num_sms * 4;
    return ASV_OK;
}

static asv_status finish_handle(asv_matrix* out, asv_matrix_s* H, cudaStream_t s, const asv_matrix_s* P);

static int pow2_floor(double v) {
    int p = 1;
    while (p * 2 <= v) p *= 2;
    return p;
}

extern "C" asv_status asv_matrix_create_csr(asv_matrix* out, int64_t m, int64_t n, int64_t nnz,
                                            const int32_t* d_rowptr, const int32_t* d_colidx, const void* d_val,
                                            int32_t dtype, uint32_t flags, void* stream) {
    if (!out) return ASV_ERR_ARG;
    *out = nullptr;
    if (m < 0 || n < 0 || nnz < 0) return ASV_ERR_ARG;
    if (dtype < ASV_F32 || dtype > ASV_I32) return ASV_ERR_ARG;
    if (m >= INT32_MAX || n >= INT32_MAX || nnz >= INT32_MAX) return ASV_ERR_OVERFLOW;
    if (!d_rowptr || (nnz > 0 && !d_colidx)) return ASV_ERR_ARG;
    if (dtype == ASV_BOOL && d_val) return ASV_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    asv_matrix_s* H = new (std::nothrow) asv_matrix_s();
    if (!H) return ASV_ERR_NOMEM;
    H->dtype = dtype;
    H->m = m;
    H->n = n;
    H->nnz = nnz;
    H->flags = flags;
    if (asv_status st = init_handle(H)) return st;
    const size_t vs = vsize(dtype);
    const bool has_val = (dtype != ASV_BOOL) && d_val != nullptr;

    // CSR: borrowed or copied
    if (flags & ASV_COPY) {
        int32_t *rp, *ci;
        void* v = nullptr;
        AL(rp, 4 * (m + 1), false);
        AL(ci, 4 * nnz, false);
        CKH(cudaMemcpyAsync(rp, d_rowptr, 4 * (m + 1), cudaMemcpyDeviceToDevice, s));
        if (nnz) CKH(cudaMemcpyAsync(ci, d_colidx, 4 * nnz, cudaMemcpyDeviceToDevice, s));
        if (has_val) {
            AL(v, vs * nnz, false);
            if (nnz) CKH(cudaMemcpyAsync(v, d_val, vs * nnz, cudaMemcpyDeviceToDevice, s));
        }
        H->rowptr = rp;
        H->col = ci;
        H->val = v;
        H->owns_val = true;
    } else {
        H->rowptr = d_rowptr;
        H->col = d_colidx;
        H->val = has_val ? d_val : nullptr;
    }

    if (flags & ASV_VALIDATE) {
        int32_t* flag;
        AL(flag, 4, true);
        CKH(validate_csr(H, s, flag));
        int32_t hf = 0;
        CKH(cudaMemcpyAsync(&hf, flag, 4, cudaMemcpyDeviceToHost, s));
        CKH(cudaStreamSynchronize(s));
        if (hf) {
            destroy_handle(H);
            return ASV_ERR_NONCANONICAL;
        }
    }
    return finish_handle(out, H, s, nullptr);
}

// Everything of a handle after its CSR arrays are set: the CSC view, the
// Table 1 features, the pull partition and long-row segments, the selector
// tables and the per-call workspaces. With a parent P the handle is P's
// transposed view: its CSC is P's CSR (borrowed, never written) and its
// CSC -> CSR position map is the inverse of P's.
static asv_status finish_handle(asv_matrix* out, asv_matrix_s* H, cudaStream_t s, const asv_matrix_s* P) {
    const int64_t m = H->m, n = H->n, nnz = H->nnz;
    const int32_t dtype = H->dtype;
    const size_t vs = vsize(dtype);
    const bool has_val = H->val != nullptr;
    const int64_t nw_n = (n + 31) / 32;
    const int G = H->G;
    // CSC view
    if (P) {
        H->colptr = const_cast<int32_t*>(P->rowptr);
        H->rowidx = const_cast<int32_t*>(P->col);
        H->val_csc = const_cast<void*>(P->val);
    } else {
        AL(H->colptr, 4 * (n + 1), false);
        AL(H->rowidx, 4 * nnz, false);
        if (has_val) AL(H->val_csc, vs * nnz, false);
    }
    AL(H->perm, 4 * nnz, false);
    // features / partition / selector
    AL(H->d_mfeat, sizeof(MatFeat), true);
    H->ntiles = (m + nnz + pull_tile_items(dtype) - 1) / pull_tile_items(dtype);
    AL(H->tile_row, 4 * (H->ntiles + 1), false);
    AL(H->carry_row, 4 * (H->ntiles + 1), false);
    AL(H->carry_val, 8 * (H->ntiles + 1), false);
    AL(H->d_trees, sizeof(TreeNode) * kMaxTreeNodes, false);
    AL(H->d_desc, sizeof(CallDesc), true);
    AL(H->d_last_kid, 4, true);
    // workspaces
    Ws& w = H->ws;
    AL(w.xbits_dense, 4 * nw_n, true);
    AL(w.xbits_scat, 4 * nw_n, true);
    AL(w.xdense, vs * n, true);
    AL(w.xlist_idx, 4 * n, false);
    AL(w.xlist_val, vs * n, false);
    AL(w.xscan, 4 * (n + 1), false);
    AL(w.acc, 8 * m, true);
    // padded to whole 512-row groups: the dense write-out loads the flags of
    // a group with 16-byte loads whatever m is
    AL(w.yflag, ((m + 511) & ~(int64_t)511) + 16, true);
    AL(w.ywork, vs * m, false);
    const size_t pv = vs == 8 ? 8 : 4;
    AL(w.pkeys[0], 4 * nnz, false);
    AL(w.pkeys[1], 4 * nnz, false);
    if (dtype != ASV_BOOL) {
        AL(w.pvals[0], pv * nnz, false);
        AL(w.pvals[1], pv * nnz, false);
    }
    w.pair_cap = nnz;
    const int64_t hist_n = std::max<int64_t>((int64_t)256 * G + 1, 2 * priv_bins(m) + 2);
    AL(w.hist, 4 * hist_n, false);
    AL(w.blk, 4 * (G + 1), false);
    AL(w.status, 4, true);
    AL(w.counters, 32, true);
    AL(w.ticket, 4, true);
    w.lcol_cap = (int32_t)std::min<int64_t>(nnz / kLongSeg + 1, (int64_t)1 << 30);
    AL(w.lcol, sizeof(int2) * (size_t)w.lcol_cap, false);
    AL(w.lcol_n, 4, true);
    AL(w.chunk_t0, 4 * (nnz / 256 + 2), false);
    {
        std::vector<int2> empty((size_t)w.lcol_cap, make_int2(-1, 0));
        CKH(cudaMemcpy(w.lcol, empty.data(), sizeof(int2) * empty.size(), cudaMemcpyHostToDevice));
    }
    CKH(cudaDeviceSynchronize());  // the zero-fills above ran on the legacy stream

    CKH(P ? invert_perm(P->perm, nnz, H->perm, s) : build_csc(H, s));
    CKH(build_features(H, s));  // synchronises
    H->narrow_acc = dtype == ASV_F32 && H->h_mfeat.max_row <= kNarrowRow;
    CKH(build_partition(H, s));
    CKH(build_long_rows(H, s));  // synchronises
    CKH(count_hub_columns(H, s));  // synchronises
    {
        std::vector<TreeNode> nodes;
        int32_t roots[kRootsLen];
        default_trees(dtype, nodes, roots);
        update_lazy(H, nodes, roots);
        CKH(cudaMemcpyAsync(H->d_trees, nodes.data(), sizeof(TreeNode) * nodes.size(), cudaMemcpyHostToDevice, s));
    }
    // lanes per row for the sub-warp pull: about six entries per lane; fewer
    // lanes also want two rows per group rather than four (measured on GB300)
    H->pull_lanes = std::min(32, std::max(2, pow2_floor(H->h_mfeat.avg_row / 6.0)));
    H->pull_unroll = H->pull_lanes <= 4 ? 2 : 4;
    if (const char* e = getenv("ASV_PULL_UNROLL")) H->pull_unroll = atoi(e) >= 4 ? 4 : 2;
    if (const char* e = getenv("ASV_PULL_TMA")) H->pull_tma = atoi(e) != 0;
    if (const char* e = getenv("ASV_PULL_LANES")) {
        const int l = atoi(e);
        if (l == 2 || l == 4 || l == 8 || l == 16 || l == 32) H->pull_lanes = l;
    }
    CKH(cudaStreamSynchronize(s));
    CKH(cudaGetLastError());
    *out = H;
    return ASV_OK;
}

extern "C" asv_status asv_matrix_transpose_view(asv_matrix A, asv_matrix* out, void* stream) {
    if (!out) return ASV_ERR_ARG;
    *out = nullptr;
    if (!A) return ASV_ERR_ARG;
    int dev = -1;
    CK(cudaGetDevice(&dev));
    if (dev != A->dev) return ASV_ERR_ARG;
    // the view reads A's CSR as its CSC, whose kernels take 16-byte loads
    // of the column pointers
    auto misaligned = [](const void* p) { return ((uintptr_t)p & 15) != 0; };
    if (misaligned(A->rowptr) || misaligned(A->col) || misaligned(A->val)) return ASV_ERR_UNSUPPORTED;
    asv_matrix_s* H = new (std::nothrow) asv_matrix_s();
    if (!H) return ASV_ERR_NOMEM;
    H->dtype = A->dtype;
    H->m = A->n;
    H->n = A->m;
    H->nnz = A->nnz;
    H->flags = ASV_BORROW;
    if (asv_status st = init_handle(H)) return st;
    // the CSR of A^T is A's CSC (rows of A^T = columns of A, ascending)
    H->rowptr = A->colptr;
    H->col = A->rowidx;
    H->val = A->val_csc;
    const asv_status st = finish_handle(out, H, (cudaStream_t)stream, A);
    if (st == ASV_OK) {
        H->parent = A;
        ++A->views;
    }
    return st;
}

extern "C" asv_status asv_matrix_destroy(asv_matrix A) {
    if (!A) return ASV_ERR_ARG;
    if (A->views > 0) return ASV_ERR_ARG;  // its transposed views read its arrays
    if (A->parent) --A->parent->views;
    destroy_handle(A);
    return ASV_OK;
}

extern "C" asv_status asv_matrix_features(asv_matrix A, asv_mfeat* h_out) {
    if (!A || !h_out) return ASV_ERR_ARG;
    *h_out = A->h_mfeat;
    return ASV_OK;
}

extern "C" asv_status asv_matrix_arrays(asv_matrix A, const int32_t** rp, const int32_t** ci, const void** v,
                                        const int32_t** cp, const int32_t** ri, const void** vc, const int32_t** perm) {
    if (!A) return ASV_ERR_ARG;
    if (rp) *rp = A->rowptr;
    if (ci) *ci = A->col;
    if (v) *v = A->val;
    if (cp) *cp = A->colptr;
    if (ri) *ri = A->rowidx;
    if (vc) *vc = A->val_csc;
    if (perm) *perm = A->perm;
    return ASV_OK;
}

extern "C" asv_status asv_matrix_copy_csc(asv_matrix A, int32_t* d_colptr, int32_t* d_rowidx, void* d_val_csc,
                                          int32_t* d_perm, void* stream) {
    if (!A) return ASV_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (d_colptr) CK(cudaMemcpyAsync(d_colptr, A->colptr, 4 * (A->n + 1), cudaMemcpyDeviceToDevice, s));
    if (A->nnz > 0) {
        if (d_rowidx) CK(cudaMemcpyAsync(d_rowidx, A->rowidx, 4 * A->nnz, cudaMemcpyDeviceToDevice, s));
        if (d_perm) CK(cudaMemcpyAsync(d_perm, A->perm, 4 * A->nnz, cudaMemcpyDeviceToDevice, s));
        if (d_val_csc && A->val_csc)
            CK(cudaMemcpyAsync(d_val_csc, A->val_csc, vsize(A->dtype) * A->nnz, cudaMemcpyDeviceToDevice, s));
    }
    return ASV_OK;
}

extern "C" asv_status asv_matrix_update_values(asv_matrix A, const void* d_val, void* stream) {
    if (!A) return ASV_ERR_ARG;
    if (A->dtype == ASV_BOOL || !A->val || A->parent) return ASV_ERR_UNSUPPORTED;
    cudaStream_t s = (cudaStream_t)stream;
    if (d_val && d_val != A->val) {
        if (!A->owns_val) return ASV_ERR_ARG;  // a borrowed handle reads the caller's array in place
        if (A->nnz) CK(cudaMemcpyAsync((void*)A->val, d_val, vsize(A->dtype) * A->nnz, cudaMemcpyDeviceToDevice, s));
    }
    CK(regather_values(A, s));
    return ASV_OK;
}

// ---------------------------------------------------------------- dispatch
// One candidate, including the vector-format conversion it needs: pull
// kernels on a sparse x first scatter it into the zero-invariant dense (and,
// when the kernel reads it, bitmap) workspaces and clear them afterwards;
// push kernels on a dense x first compact its bitmap into an ascending list.
static void enqueue_candidate(asv_matrix_s* H, int k, int x_sparse, int om, cudaStream_t s) {
    if (k < ASV_K_PUSH_THREAD_ATOM) {
        const bool masked = k >= ASV_K_MPULL_THREAD;
        const int dist = k % 3;
        // the bitmap serves validation, output flags and Boolean terms
        const bool bits = masked || om == ASV_OUT_SPARSE || H->dtype == ASV_BOOL;
        if (x_sparse) launch_x_scatter(H, true, bits, s);
        launch_pull(H, dist, masked, om == ASV_OUT_SPARSE, nullptr, s);
        if (om == ASV_OUT_SPARSE) launch_finalize(H, false, om, s);
        if (x_sparse) launch_x_scatter(H, false, bits, s);
    } else {
        const int q = k - ASV_K_PUSH_THREAD_ATOM;
        const int dist = q % 3, wb = q / 3;
        // the warp push with atomics reads a dense x's bitmap directly when x
        // has fewer nonzeros than its group form takes (two groups of 32 per
        // warp of its grid: 8 blocks of 8 warps per SM), so that list is
        // never compacted -- on matrices wide enough to give every warp of
        // that grid a stretch of 32 bitmap words (1,024 columns) and with
        // columns of at most 32 entries on average (group-walk columns): a
        // warp walks every column of its stretch, so on narrower matrices or
        // longer columns a few warps would hold all the work (a 16384-column
        // layer of 819-entry columns: 4.9 -> 53.7 ms for 64 products)
        const int64_t push_warps = (int64_t)H->num_sms * 64;
        const bool bits_ok = !x_sparse && k == ASV_K_PUSH_WARP_ATOM && H->n >= 1024 * push_warps &&
                             H->nnz <= 32 * H->n;
        const int64_t bits_below = bits_ok ? 64 * push_warps : 0;
        if (!x_sparse) launch_x_compact_list(H, s, bits_below);
        launch_push(H, dist, wb, om, s, bits_below);
    }
}

// The candidate whose chain runs beside the SWITCH node of a selector graph
// rather than as one of its branches: the warp push with atomic write-back,
// which the trees pick at the sparse end of the density range on matrices
// without hub columns, where a whole call takes a few tens of microseconds
// and the conditional node's own dispatch (about 10 us on GB300, measured
// with an empty branch) would add a fifth to a third to it. The chain
// depends on the feature node only, its kernels return at once unless the
// pass chose its candidate (Gate), and that candidate's SWITCH branch is
// empty; when it is chosen, the SWITCH node's dispatch overlaps the chain
// instead of preceding it. (More chains measured worse, for a cause not
// found: with the three atomic pushes as direct chains the R-MAT pull calls
// ran at half speed, and with the warp and balanced pushes the R-MAT BFS
// step took 6.3 ms instead of 4.9 ms, so one chain is kept.)
static constexpr int kDirect[1] = {ASV_K_PUSH_WARP_ATOM};

static bool is_direct(int k) {
    for (int d : kDirect)
        if (d == k) return true;
    return false;
}

// Captures the direct chains into graph g, each after node `after`; the
// nodes that end them are appended to *tails when it is given.
static cudaError_t capture_direct_chains(asv_matrix_s* H, cudaGraph_t g, cudaGraphNode_t after, int xs, int om,
                                         std::vector<cudaGraphNode_t>* tails) {
    cudaStream_t cs = H->cap_stream;
    for (int k : kDirect) {
        cudaError_t r = cudaStreamBeginCaptureToGraph(cs, g, &after, nullptr, 1, cudaStreamCaptureModeRelaxed);
        if (r != cudaSuccess) return r;
        H->gate_kid = k;
        enqueue_candidate(H, k, xs, om, cs);
        H->gate_kid = -1;
        if (tails) {
            cudaStreamCaptureStatus cst;
            const cudaGraphNode_t* deps = nullptr;
            size_t nd = 0;
            r = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &nd);
            if (r == cudaSuccess) tails->insert(tails->end(), deps, deps + nd);
        }
        cudaGraph_t cap;
        const cudaError_t e = cudaStreamEndCapture(cs, &cap);
        if (r != cudaSuccess) return r;
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// The selector-driven graph of one (x format, output mode): a feature-pass
// node whose last block also walks the trees and sets the SWITCH value, then
// the SWITCH node with one branch per candidate, and beside it the direct
// chains of the atomic pushes. The feature node's arguments are replaced
// before every launch, so one graph serves all calls.
static asv_status build_auto_graph(asv_matrix_s* H, int xs, int om, const DescInit& di) {
    if (H->gexec[xs][om]) return ASV_OK;
    if (!H->cap_stream) CK(cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = H->cap_stream;
    cudaGraph_t g;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    CK(cudaGraphConditionalHandleCreate(&h, g, ASV_K_PULL_BAL, cudaGraphCondAssignDefault));
    CK(cudaStreamBeginCaptureToGraph(cs, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    launch_features(H, di, select_arg(H, (unsigned long long)h, 2 * xs + om), cs);
    cudaGraph_t g2;
    CK(cudaStreamEndCapture(cs, &g2));
    cudaGraphNode_t feat;
    size_t nn = 1;
    CK(cudaGraphGetNodes(g, &feat, &nn));
    if (nn != 1) return ASV_ERR_CUDA;
    alignas(cudaGraphNodeParams) unsigned char cp_raw[sizeof(cudaGraphNodeParams)];
    memset(cp_raw, 0, sizeof(cp_raw));
    cudaGraphNodeParams& cp = *reinterpret_cast<cudaGraphNodeParams*>(cp_raw);
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeSwitch;
    cp.conditional.size = ASV_K_COUNT;
    cudaGraphNode_t cn;
    CK(cudaGraphAddNode(&cn, g, &feat, nullptr, 1, &cp));
    for (int k = 0; k < ASV_K_COUNT; ++k) {
        if (is_direct(k)) continue;  // an empty branch
        CK(cudaStreamBeginCaptureToGraph(cs, cp.conditional.phGraph_out[k], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeRelaxed));
        enqueue_candidate(H, k, xs, om, cs);
        cudaGraph_t bk;
        CK(cudaStreamEndCapture(cs, &bk));
    }
    CK(capture_direct_chains(H, g, feat, xs, om, nullptr));
    cudaGraphExec_t ex;
    CK(cudaGraphInstantiate(&ex, g, 0));
    H->graph[xs][om] = g;
    H->gexec[xs][om] = ex;
    H->feat_node[xs][om] = feat;
    H->cond[xs][om] = (unsigned long long)h;
    return ASV_OK;
}

static asv_status launch_auto(asv_matrix_s* H, const DescInit& di, int om, cudaStream_t s) {
    const int xs = di.x_sparse;
    asv_status st = build_auto_graph(H, xs, om, di);
    if (st != ASV_OK) return st;
    // the feature node's arguments change only when the call's pointers do
    if (memcmp(&H->last_di[xs][om], &di, sizeof(di)) != 0) {
        FeatLaunch fl;
        feature_launch(H, di, select_arg(H, H->cond[xs][om], 2 * xs + om), fl);
        cudaKernelNodeParams kp;
        memset(&kp, 0, sizeof(kp));
        kp.func = fl.func;
        kp.gridDim = fl.grid;
        kp.blockDim = fl.block;
        kp.sharedMemBytes = 0;
        kp.kernelParams = fl.args;
        kp.extra = nullptr;
        CK(cudaGraphExecKernelNodeSetParams(H->gexec[xs][om], H->feat_node[xs][om], &kp));
        H->last_di[xs][om] = di;
    }
    CK(cudaGraphLaunch(H->gexec[xs][om], s));
    return ASV_OK;
}

static asv_status prepare_call(asv_matrix_s* H, const int64_t* d_nnz_x, const int32_t* d_xidx, const void* d_xval,
                               const void* d_x_dense, int32_t om, void* d_y, int32_t* d_yidx, void* d_yval,
                               int64_t* d_nnz_y, int64_t y_cap, DescInit& di) {
    if (om != ASV_OUT_DENSE && om != ASV_OUT_SPARSE) return ASV_ERR_ARG;
    if (om == ASV_OUT_DENSE && !d_y && H->m > 0) return ASV_ERR_ARG;
    if (om == ASV_OUT_SPARSE && (!d_yidx || !d_nnz_y || y_cap < 0)) return ASV_ERR_ARG;
    const bool xs = d_x_dense == nullptr;
    if (xs && !d_nnz_x) return ASV_ERR_ARG;  // d_xidx may be NULL when *d_nnz_x == 0
    if (!xs && H->n > 0 && !d_x_dense) return ASV_ERR_ARG;
    memset(&di, 0, sizeof(di));
    di.y = d_y;
    di.yidx = d_yidx;
    di.yval = d_yval;
    di.nnz_y = d_nnz_y;
    di.y_cap = y_cap;
    di.out_mode = om;
    di.x_sparse = xs ? 1 : 0;
    di.y_ident_ok = om == ASV_OUT_SPARSE && H->dtype != ASV_BOOL && d_yval != nullptr && H->m > 0 &&
                    H->h_mfeat.min_row >= 1 && y_cap >= H->m;
    if (xs) {
        di.x_dense = H->ws.xdense;
        di.xbits = H->ws.xbits_scat;
        di.xidx = d_xidx;
        di.xval = (H->dtype == ASV_BOOL) ? nullptr : d_xval;
        di.user_xidx = d_xidx;
        di.user_xval = di.xval;
        di.user_nnz_x = d_nnz_x;
    } else {
        di.x_dense = d_x_dense;
        di.xbits = H->ws.xbits_dense;
        di.xidx = H->ws.xlist_idx;
        di.xval = (H->dtype == ASV_BOOL) ? nullptr : H->ws.xlist_val;
        di.user_x_dense = d_x_dense;
    }
    return ASV_OK;
}

static asv_status spmspv_impl(asv_matrix A, const uint32_t* d_ymask, const int64_t* d_nnz_x, const int32_t* d_xidx,
                              const void* d_xval, const void* d_x_dense, int32_t out_mode, void* d_y, int32_t* d_yidx,
                              void* d_yval, int64_t* d_nnz_y, int64_t y_cap, int32_t kernel, cudaStream_t s) {
    if (!A) return ASV_ERR_ARG;
    if (kernel < ASV_K_AUTO || kernel >= ASV_K_COUNT) return ASV_ERR_ARG;
    DescInit di;
    asv_status st = prepare_call(A, d_nnz_x, d_xidx, d_xval, d_x_dense, out_mode, d_y, d_yidx, d_yval, d_nnz_y, y_cap, di);
    if (st != ASV_OK) return st;
    di.ymask = d_ymask;
    if (kernel == ASV_K_AUTO) {
        st = launch_auto(A, di, out_mode, s);
        if (st != ASV_OK) return st;
    } else {
        SelectArg none = select_arg(A, 0ull, 2 * di.x_sparse + out_mode);
        none.enabled = 0;
        launch_features(A, di, none, s);
        enqueue_candidate(A, kernel, di.x_sparse, out_mode, s);
    }
    CK(cudaGetLastError());
    return ASV_OK;
}

extern "C" asv_status asv_spmspv(asv_matrix A, const int64_t* d_nnz_x, const int32_t* d_xidx, const void* d_xval,
                                 const void* d_x_dense, int32_t out_mode, void* d_y, int32_t* d_yidx, void* d_yval,
                                 int64_t* d_nnz_y, int64_t y_cap, int32_t kernel, void* stream) {
    return spmspv_impl(A, nullptr, d_nnz_x, d_xidx, d_xval, d_x_dense, out_mode, d_y, d_yidx, d_yval, d_nnz_y, y_cap,
                       kernel, (cudaStream_t)stream);
}

extern "C" asv_status asv_spmspv_masked(asv_matrix A, const uint32_t* d_ymask, const int64_t* d_nnz_x,
                                        const int32_t* d_xidx, const void* d_xval, const void* d_x_dense,
                                        int32_t out_mode, void* d_y, int32_t* d_yidx, void* d_yval, int64_t* d_nnz_y,
                                        int64_t y_cap, int32_t kernel, void* stream) {
    if (!d_ymask && A && A->m > 0) return ASV_ERR_ARG;
    return spmspv_impl(A, d_ymask, d_nnz_x, d_xidx, d_xval, d_x_dense, out_mode, d_y, d_yidx, d_yval, d_nnz_y, y_cap,
                       kernel, (cudaStream_t)stream);
}

// ---------------------------------------------------------------- driver loops
// BFS and PageRank run their iterations as one CUDA graph each: a WHILE node
// (condition 1 at every launch) whose body is the product of one iteration
// -- list x in, sparse y out; the feature pass, then either the SWITCH over
// all candidates that the feature pass's selector sets (AUTO) or the forced
// candidate -- followed by the driver's step kernel, whose last block sets
// the WHILE condition. The graph holds fixed workspace pointers; the
// per-call arguments live in the driver's device LoopState. `step` enqueues
// the step kernel given the WHILE handle.
template <class Step>
static asv_status build_loop_graph(asv_matrix_s* H, const DescInit& di, int32_t kernel, Step step, cudaGraph_t* g_out,
                                   cudaGraphExec_t* ex_out) {
    if (!H->cap_stream) CK(cudaStreamCreateWithFlags(&H->cap_stream, cudaStreamNonBlocking));
    cudaStream_t cs = H->cap_stream;
    cudaGraph_t g;
    CK(cudaGraphCreate(&g, 0));
    cudaGraphExec_t ex = nullptr;
    cudaError_t e = [&]() -> cudaError_t {
        cudaError_t r;
#define CKL(expr) if ((r = (expr)) != cudaSuccess) return r
        cudaGraphConditionalHandle hw;
        CKL(cudaGraphConditionalHandleCreate(&hw, g, 1, cudaGraphCondAssignDefault));
        alignas(cudaGraphNodeParams) unsigned char wp_raw[sizeof(cudaGraphNodeParams)];
        memset(wp_raw, 0, sizeof(wp_raw));
        cudaGraphNodeParams& wp = *reinterpret_cast<cudaGraphNodeParams*>(wp_raw);
        wp.type = cudaGraphNodeTypeConditional;
        wp.conditional.handle = hw;
        wp.conditional.type = cudaGraphCondTypeWhile;
        wp.conditional.size = 1;
        cudaGraphNode_t wn;
        CKL(cudaGraphAddNode(&wn, g, nullptr, nullptr, 0, &wp));
        cudaGraph_t body = wp.conditional.phGraph_out[0];
        if (kernel != ASV_K_AUTO) {
            SelectArg none = select_arg(H, 0ull, 2 + ASV_OUT_SPARSE);
            none.enabled = 0;
            CKL(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
            launch_features(H, di, none, cs);
            enqueue_candidate(H, kernel, 1, ASV_OUT_SPARSE, cs);
            step(cs, (unsigned long long)hw);
            cudaGraph_t cap;
            CKL(cudaStreamEndCapture(cs, &cap));
        } else {
            cudaGraphConditionalHandle hs;
            CKL(cudaGraphConditionalHandleCreate(&hs, body, ASV_K_PULL_BAL, cudaGraphCondAssignDefault));
            CKL(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
            launch_features(H, di, select_arg(H, (unsigned long long)hs, 2 + ASV_OUT_SPARSE), cs);
            cudaGraph_t cap;
            CKL(cudaStreamEndCapture(cs, &cap));
            cudaGraphNode_t feat;
            size_t nn = 1;
            CKL(cudaGraphGetNodes(body, &feat, &nn));
            if (nn != 1) return cudaErrorInvalidValue;
            alignas(cudaGraphNodeParams) unsigned char sp_raw[sizeof(cudaGraphNodeParams)];
            memset(sp_raw, 0, sizeof(sp_raw));
            cudaGraphNodeParams& sp = *reinterpret_cast<cudaGraphNodeParams*>(sp_raw);
            sp.type = cudaGraphNodeTypeConditional;
            sp.conditional.handle = hs;
            sp.conditional.type = cudaGraphCondTypeSwitch;
            sp.conditional.size = ASV_K_COUNT;
            cudaGraphNode_t sn;
            CKL(cudaGraphAddNode(&sn, body, &feat, nullptr, 1, &sp));
            for (int k = 0; k < ASV_K_COUNT; ++k) {
                if (is_direct(k)) continue;  // an empty branch
                CKL(cudaStreamBeginCaptureToGraph(cs, sp.conditional.phGraph_out[k], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeRelaxed));
                enqueue_candidate(H, k, 1, ASV_OUT_SPARSE, cs);
                CKL(cudaStreamEndCapture(cs, &cap));
            }
            // the step waits for the SWITCH node and every direct chain
            std::vector<cudaGraphNode_t> join{sn};
            CKL(capture_direct_chains(H, body, feat, 1, ASV_OUT_SPARSE, &join));
            CKL(cudaStreamBeginCaptureToGraph(cs, body, join.data(), nullptr, join.size(),
                                              cudaStreamCaptureModeRelaxed));
            step(cs, (unsigned long long)hw);
            CKL(cudaStreamEndCapture(cs, &cap));
        }
        CKL(cudaGraphInstantiate(&ex, g, 0));
#undef CKL
        return cudaSuccess;
    }();
    if (e != cudaSuccess) {
        g_last_cuda = (int32_t)e;
        cudaGraphDestroy(g);
        return e == cudaErrorMemoryAllocation ? ASV_ERR_NOMEM : ASV_ERR_CUDA;
    }
    *g_out = g;
    *ex_out = ex;
    return ASV_OK;
}

// Incremental PageRank, delta form: rank = sum of delta_k, delta_0 = (1 - d)/N
// on every vertex, delta_{k+1} = d A D^{-1} delta_k with entries below eps
// dropped. Each iteration is one selector-driven product (list in, sparse
// list out) and one step kernel that adds d y to the rank and keeps the
// entries at or above eps, scaled, as the next input list.
extern "C" asv_status asv_pagerank(asv_matrix A, double damping, double eps, int32_t max_iter, void* d_rank,
                                   int32_t kernel, int32_t* h_iters, void* stream) {
    if (!A || !d_rank) return ASV_ERR_ARG;
    if (A->dtype != ASV_F32 && A->dtype != ASV_F64) return ASV_ERR_UNSUPPORTED;
    if (A->m != A->n || A->n == 0 || max_iter < 0 || !(damping >= 0.0 && damping < 1.0) || !(eps >= 0.0))
        return ASV_ERR_ARG;
    if (kernel < ASV_K_AUTO || kernel >= ASV_K_COUNT) return ASV_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    asv_matrix_s* H = A;
    const size_t vs = vsize(H->dtype);
    if (!H->pr_count) {  // workspaces of the driver, allocated on the first call
        CK(cudaStreamSynchronize(s));
        void* p[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
        const size_t bytes[6] = {4 * (size_t)H->n, vs * H->n, 4 * (size_t)H->n, vs * H->n, 32, sizeof(LoopState)};
        for (int i = 0; i < 6; ++i) {
            asv_status st = dalloc(H, &p[i], bytes[i], i >= 4);
            if (st != ASV_OK) return st;
        }
        H->pr_xidx = (int32_t*)p[0];
        H->pr_xval = p[1];
        H->pr_yidx = (int32_t*)p[2];
        H->pr_yval = p[3];
        H->pr_count = (int64_t*)p[4];
        H->pr_state = (LoopState*)p[5];
        if (!H->bfs_hcount) CK(cudaMallocHost((void**)&H->bfs_hcount, sizeof(int64_t)));
    }
    const int grid = H->num_sms * 4;
    const int slot = kernel + 1;
    if (!H->pr_exec[slot]) {
        DescInit di;
        asv_status st = prepare_call(H, H->pr_count, H->pr_xidx, H->pr_xval, nullptr, ASV_OUT_SPARSE, nullptr,
                                     H->pr_yidx, H->pr_yval, H->pr_count + 2, H->n, di);
        if (st != ASV_OK) return st;
        auto step = [H, grid](cudaStream_t cs, unsigned long long loop) {
            launch_pr_step(H->dtype, H->pr_yidx, H->pr_yval, H->pr_count, H->colptr, H->pr_xidx, H->pr_xval,
                           H->pr_state, loop, grid, cs);
        };
        st = build_loop_graph(H, di, kernel, step, &H->pr_graph[slot], &H->pr_exec[slot]);
        if (st != ASV_OK) return st;
    }
    launch_pr_init(H->dtype, H->n, damping, eps, max_iter, d_rank, H->colptr, H->pr_xidx, H->pr_xval, H->pr_count,
                   H->pr_state, grid, s);
    if (max_iter > 0) CK(cudaGraphLaunch(H->pr_exec[slot], s));
    if (h_iters) {
        CK(cudaMemcpyAsync(H->bfs_hcount, &H->pr_state->iter, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        *h_iters = (int32_t)*H->bfs_hcount;
    }
    CK(cudaGetLastError());
    return ASV_OK;
}

// Level-synchronous BFS through the masked product: frontier_{d+1} =
// (A frontier_d) restricted to the unvisited rows, as the ascending list the
// sparse output mode produces; each level is one selector-driven product (or
// the forced candidate), so the pattern, distribution and write-back adapt
// from level to level, and one step kernel that records the levels.
extern "C" asv_status asv_bfs(asv_matrix A, int32_t source, int32_t* d_level, int32_t kernel, int32_t* h_depth,
                              void* stream) {
    if (!A || !d_level) return ASV_ERR_ARG;
    if (A->m != A->n || A->n == 0 || source < 0 || source >= A->n) return ASV_ERR_ARG;
    if (kernel < ASV_K_AUTO || kernel >= ASV_K_COUNT) return ASV_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    asv_matrix_s* H = A;
    if (!H->bfs_count) {  // workspaces of the search, allocated on the first call
        CK(cudaStreamSynchronize(s));
        void* p[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
        const size_t bytes[5] = {(size_t)4 * ((H->n + 31) / 32), (size_t)4 * H->n, (size_t)4 * H->n, 16,
                                 sizeof(LoopState)};
        for (int i = 0; i < 5; ++i) {
            asv_status st = dalloc(H, &p[i], bytes[i], i == 0 || i >= 3);
            if (st != ASV_OK) return st;
        }
        H->bfs_visited = (uint32_t*)p[0];
        H->bfs_front[0] = (int32_t*)p[1];
        H->bfs_front[1] = (int32_t*)p[2];
        H->bfs_count = (int64_t*)p[3];
        H->bfs_state = (LoopState*)p[4];
        if (!H->bfs_hcount) CK(cudaMallocHost((void**)&H->bfs_hcount, sizeof(int64_t)));
    }
    const int slot = kernel + 1;
    if (!H->bfs_exec[slot]) {
        DescInit di;
        asv_status st = prepare_call(H, H->bfs_count, H->bfs_front[0], nullptr, nullptr, ASV_OUT_SPARSE, nullptr,
                                     H->bfs_front[1], nullptr, H->bfs_count + 1, H->n, di);
        if (st != ASV_OK) return st;
        di.ymask = H->bfs_visited;
        const int grid = H->num_sms * 4;
        auto step = [H, grid](cudaStream_t cs, unsigned long long loop) {
            launch_bfs_step(H->bfs_front[1], H->bfs_count, H->bfs_front[0], H->bfs_visited, H->bfs_state, loop, grid,
                            cs);
        };
        st = build_loop_graph(H, di, kernel, step, &H->bfs_graph[slot], &H->bfs_exec[slot]);
        if (st != ASV_OK) return st;
    }
    CK(cudaMemsetAsync(d_level, 0xff, 4 * (size_t)H->n, s));
    CK(cudaMemsetAsync(H->bfs_visited, 0, 4 * (size_t)((H->n + 31) / 32), s));
    launch_bfs_init(source, H->n, d_level, H->bfs_visited, H->bfs_front[0], H->bfs_count, H->bfs_state, s);
    CK(cudaGraphLaunch(H->bfs_exec[slot], s));
    if (h_depth) {
        CK(cudaMemcpyAsync(H->bfs_hcount, &H->bfs_state->iter, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        *h_depth = (int32_t)*H->bfs_hcount;
    }
    CK(cudaGetLastError());
    return ASV_OK;
}

extern "C" asv_status asv_spmv(asv_matrix A, const void* d_x, void* d_y, int32_t kernel, void* stream) {
    if (!A) return ASV_ERR_ARG;
    if (kernel < ASV_K_AUTO || kernel >= ASV_K_COUNT) return ASV_ERR_ARG;
    if ((!d_x && A->n > 0) || (!d_y && A->m > 0)) return ASV_ERR_ARG;
    if (kernel >= ASV_K_PULL_THREAD && kernel <= ASV_K_PULL_BAL) {
        // the plain SpMV needs neither the feature pass nor the descriptor
        PullIO io{d_x, nullptr, d_y};
        launch_pull(A, kernel, false, false, &io, (cudaStream_t)stream);
        CK(cudaGetLastError());
        return ASV_OK;
    }
    return asv_spmspv(A, nullptr, nullptr, nullptr, d_x, ASV_OUT_DENSE, d_y, nullptr, nullptr, nullptr, 0, kernel, stream);
}

extern "C" asv_status asv_select(asv_matrix A, const int64_t* d_nnz_x, const int32_t* d_xidx, const void* d_xval,
                                 const void* d_x_dense, int32_t out_mode, int32_t* h_kernel, asv_vfeat* h_feat,
                                 void* stream) {
    if (!A) return ASV_ERR_ARG;
    if (out_mode != ASV_OUT_DENSE && out_mode != ASV_OUT_SPARSE) return ASV_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    DescInit di;
    // no candidate runs: the output pointers only have to be valid, never written
    asv_status st = prepare_call(A, d_nnz_x, d_xidx, d_xval, d_x_dense, out_mode, A->ws.ywork, A->ws.xlist_idx,
                                 A->ws.ywork, (int64_t*)A->ws.hist, 0, di);
    if (st != ASV_OK) return st;
    // the full pass: every feature is reported, so no lazy evaluation
    SelectArg sa = select_arg(A, 0ull, 2 * di.x_sparse + out_mode);
    sa.lazy = 0;
    launch_features(A, di, sa, s);
    CallDesc hd;
    CK(cudaMemcpyAsync(&hd, A->d_desc, sizeof(hd), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h_kernel) *h_kernel = hd.kid;
    if (h_feat) {
        h_feat->nnz_x = hd.nnz_x;
        h_feat->nnz_s = hd.nnz_s;
        h_feat->x_sparsity = hd.vfeat[1];
        h_feat->m_sparsity = hd.vfeat[3];
    }
    return ASV_OK;
}

extern "C" asv_status asv_last_kernel(asv_matrix A, int32_t* h_kernel, void* stream) {
    if (!A || !h_kernel) return ASV_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(h_kernel, A->d_last_kid, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return ASV_OK;
}

extern "C" asv_status asv_compact(asv_matrix A, const void* d_x_dense, int32_t* d_idx, void* d_val, int64_t* d_count,
                                  void* stream) {
    if (!A || (!d_x_dense && A->n > 0) || !d_idx || !d_count) return ASV_ERR_ARG;
    launch_compact_public(A, d_x_dense, d_idx, d_val, d_count, (cudaStream_t)stream);
    CK(cudaGetLastError());
    return ASV_OK;
}

extern "C" asv_status asv_set_trees(asv_matrix A, const double* h_nodes, int32_t n_nodes, const int32_t* h_roots,
                                    void* stream) {
    if (!A || !h_nodes || !h_roots || n_nodes <= 0 || n_nodes > kMaxTreeNodes) return ASV_ERR_ARG;
    std::vector<TreeNode> nodes(n_nodes);
    for (int i = 0; i < n_nodes; ++i) {
        const double* r = h_nodes + 5 * i;
        TreeNode& t = nodes[i];
        t.feature = (int32_t)r[0];
        t.thr = r[1];
        t.left = (int32_t)r[2];
        t.right = (int32_t)r[3];
        t.leaf = (int32_t)r[4];
        if (t.feature >= 13) return ASV_ERR_ARG;
        if (t.feature >= 0 && (t.left < 0 || t.left >= n_nodes || t.right < 0 || t.right >= n_nodes)) return ASV_ERR_ARG;
        if (t.feature < 0 && (t.leaf < 0 || t.leaf > 2)) return ASV_ERR_ARG;
    }
    int32_t r[kRootsLen];
    for (int i = 0; i < kRootsLen - 1; ++i) {
        if (h_roots[i] < 0 || h_roots[i] >= n_nodes) return ASV_ERR_ARG;
        r[i] = h_roots[i];
    }
    r[kRootsLen - 1] = n_nodes;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaMemcpyAsync(A->d_trees, nodes.data(), sizeof(TreeNode) * n_nodes, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    update_lazy(A, nodes, r);
    // the selector graphs' feature nodes take the new roots, windows and lazy
    // hints at their next call; the BFS and PageRank graphs hold them in
    // their captured feature nodes, so they are rebuilt at their next call
    // (a graph still executing is freed when it completes)
    memset(A->last_di, 0xff, sizeof(A->last_di));
    for (int k = 0; k <= ASV_K_COUNT; ++k) {
        if (A->bfs_exec[k]) cudaGraphExecDestroy(A->bfs_exec[k]);
        if (A->bfs_graph[k]) cudaGraphDestroy(A->bfs_graph[k]);
        if (A->pr_exec[k]) cudaGraphExecDestroy(A->pr_exec[k]);
        if (A->pr_graph[k]) cudaGraphDestroy(A->pr_graph[k]);
        A->bfs_exec[k] = A->pr_exec[k] = nullptr;
        A->bfs_graph[k] = A->pr_graph[k] = nullptr;
    }
    return ASV_OK;
}

// ---------------------------------------------------------------- batched forms
static asv_status batched_args(asv_matrix A, int32_t B, int64_t max_entries, const int64_t* d_xptr,
                               const void* d_X_dense, void* d_Y) {
    if (!A || B < 0 || !d_Y) return ASV_ERR_ARG;
    if (A->dtype != ASV_F32) return ASV_ERR_UNSUPPORTED;
    if (!d_X_dense && (!d_xptr || max_entries < 0)) return ASV_ERR_ARG;
    if ((int64_t)B * A->m >= ((int64_t)1 << 40)) return ASV_ERR_OVERFLOW;
    if (d_X_dense && (int64_t)B * A->n >= INT32_MAX) return ASV_ERR_OVERFLOW;
    if (max_entries >= INT32_MAX) return ASV_ERR_OVERFLOW;
    return ASV_OK;
}

static bool tune_ok(const asv_tune& t, int32_t B) {
    if (B < 0) return false;
    if (t.hot_columns != 0) {
        return (t.hot_columns == 64 || t.hot_columns == 128) && (t.rows_per_tile == 8 || t.rows_per_tile == 16) &&
               (t.vectors_per_group == 128 || t.vectors_per_group == 256);
    }
    const bool r_ok = t.rows_per_tile == 4 || t.rows_per_tile == 8 || t.rows_per_tile == 16;
    return r_ok && t.vectors_per_group >= 1 && (int64_t)t.rows_per_tile * (t.vectors_per_group + 1) * 8 <= 200 * 1024;
}

extern "C" asv_status asv_spmspv_batched(asv_matrix A, int32_t B, int64_t max_entries, const int64_t* d_xptr,
                                         const int32_t* d_xidx, const void* d_xval, const void* d_X_dense, void* d_Y,
                                         const asv_tune* tune, void* stream) {
    asv_status st = batched_args(A, B, max_entries, d_xptr, d_X_dense, d_Y);
    if (st != ASV_OK) return st;
    if (B == 0 || A->m == 0) return ASV_OK;
    asv_tune t{A->tune_R, A->tune_GB, A->tune_hot};
    if (tune) t = *tune;
    if (!tune_ok(t, B)) return ASV_ERR_ARG;
    if (t.hot_columns != 0 && (int64_t)t.hot_columns * B >= INT32_MAX) return ASV_ERR_OVERFLOW;
    if (t.hot_columns == 0) t.vectors_per_group = std::min(t.vectors_per_group, B);
    CK(batched_forward(A, B, max_entries, d_xptr, d_xidx, (const float*)d_xval, (const float*)d_X_dense,
                       (float*)d_Y, t.rows_per_tile, t.vectors_per_group, t.hot_columns, (cudaStream_t)stream));
    return ASV_OK;
}

static std::string tune_key(asv_matrix A, int32_t B) {
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, A->dev);
    char buf[512];
    snprintf(buf, sizeof(buf), "%s|m=%lld|n=%lld|nnz=%lld|max_row=%lld|B=%d", p.name, (long long)A->m,
             (long long)A->n, (long long)A->nnz, (long long)A->h_mfeat.max_row, B);
    return buf;
}

extern "C" asv_status asv_autotune_batched(asv_matrix A, int32_t B, int64_t max_entries, const int64_t* d_xptr,
                                           const int32_t* d_xidx, const void* d_xval, const void* d_X_dense,
                                           void* d_Y, const char* cache_path, asv_tune* h_best, void* stream) {
    asv_status st = batched_args(A, B, max_entries, d_xptr, d_X_dense, d_Y);
    if (st != ASV_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const std::string key = tune_key(A, B);
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "r")) {
            char line[1024];
            while (fgets(line, sizeof(line), f)) {
                int r = 0, g = 0, hc = 0;
                char k[600];
                const int got = sscanf(line, "%599[^\t]\t%d\t%d\t%d", k, &r, &g, &hc);
                if (got >= 3 && key == k) {
                    asv_tune t{r, g, got == 4 ? hc : 0};
                    if (tune_ok(t, B)) {
                        A->tune_R = r;
                        A->tune_GB = g;
                        A->tune_hot = t.hot_columns;
                        if (h_best) *h_best = t;
                        fclose(f);
                        return ASV_OK;
                    }
                }
            }
            fclose(f);
        }
    }
    const asv_tune cands[] = {{4, 4096, 0},   {4, 2048, 0},   {8, 512, 0},    {8, 1024, 0},  {8, 2048, 0},
                              {4, 1024, 0},   {16, 256, 0},   {16, 512, 0},   {16, 1024, 0}, {16, 1536, 0},
                              {8, 256, 128},  {16, 256, 128}, {16, 128, 128}, {16, 256, 64}};
    float best = 1e30f;
    asv_tune bt{A->tune_R, A->tune_GB, A->tune_hot};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (const asv_tune& c : cands) {
        if (!tune_ok(c, B) ||
            (c.hot_columns == 0 && c.vectors_per_group > 2 * std::max(B, 1) && c.vectors_per_group > 256))
            continue;
        st = asv_spmspv_batched(A, B, max_entries, d_xptr, d_xidx, d_xval, d_X_dense, d_Y, &c, stream);
        if (st != ASV_OK) break;
        float tsum = 0.f;
        for (int r = 0; r < 3; ++r) {
            CK(cudaEventRecord(e0, s));
            st = asv_spmspv_batched(A, B, max_entries, d_xptr, d_xidx, d_xval, d_X_dense, d_Y, &c, stream);
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e0, e1));
            tsum += ms;
        }
        if (tsum < best) {
            best = tsum;
            bt = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != ASV_OK) return st;
    A->tune_R = bt.rows_per_tile;
    A->tune_GB = bt.vectors_per_group;
    A->tune_hot = bt.hot_columns;
    if (h_best) *h_best = bt;
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "a")) {
            fprintf(f, "%s\t%d\t%d\t%d\n", key.c_str(), bt.rows_per_tile, bt.vectors_per_group, bt.hot_columns);
            fclose(f);
        }
    }
    return ASV_OK;
}

// ---------------------------------------------------------------- single-call tuner
// The pull kernels' launch shape -- lanes per row and rows per lane group of
// the sub-warp pull, TMA staging of the one-row-per-thread pull -- changes
// their speed, never their result. The tuner times the candidates on a dense
// x of ones through the direct (descriptor-free) launch path, within the time
// budget, and keeps the fastest of each in the handle.
static std::string pull_tune_key(asv_matrix A) {
    cudaDeviceProp p;
    cudaGetDeviceProperties(&p, A->dev);
    char buf[512];
    snprintf(buf, sizeof(buf), "%s|m=%lld|n=%lld|nnz=%lld|max_row=%lld|dtype=%d|pull", p.name, (long long)A->m,
             (long long)A->n, (long long)A->nnz, (long long)A->h_mfeat.max_row, (int)A->dtype);
    return buf;
}

static bool pull_tune_ok(const asv_pull_tune& t) {
    const int l = t.lanes;
    return (l == 2 || l == 4 || l == 8 || l == 16 || l == 32) && (t.unroll == 2 || t.unroll == 4) &&
           (t.tma == 0 || t.tma == 1);
}

extern "C" asv_status asv_autotune(asv_matrix A, const char* cache_path, uint32_t budget_ms, asv_pull_tune* h_out,
                                   void* stream) {
    if (!A) return ASV_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    auto current = [&]() { return asv_pull_tune{A->pull_lanes, A->pull_unroll, A->pull_tma ? 1 : 0}; };
    const std::string key = pull_tune_key(A);
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "r")) {
            char line[1024];
            while (fgets(line, sizeof(line), f)) {
                asv_pull_tune t{0, 0, 0};
                char k[600];
                if (sscanf(line, "%599[^\t]\t%d\t%d\t%d", k, &t.lanes, &t.unroll, &t.tma) == 4 && key == k &&
                    pull_tune_ok(t)) {
                    fclose(f);
                    A->pull_lanes = t.lanes;
                    A->pull_unroll = t.unroll;
                    A->pull_tma = t.tma != 0;
                    if (h_out) *h_out = t;
                    return ASV_OK;
                }
            }
            fclose(f);
        }
    }
    if (A->m == 0 || A->nnz == 0) {
        if (h_out) *h_out = current();
        return ASV_OK;
    }
    // a dense x of ones and a y, owned by the tuner for its duration
    const size_t vs = vsize(A->dtype);
    void *x = nullptr, *y = nullptr;
    CK(cudaMalloc(&x, vs * std::max<int64_t>(A->n, 1)));
    {
        cudaError_t e = cudaMalloc(&y, vs * A->m);
        if (e != cudaSuccess) {
            cudaFree(x);
            g_last_cuda = (int32_t)e;
            return e == cudaErrorMemoryAllocation ? ASV_ERR_NOMEM : ASV_ERR_CUDA;
        }
    }
    {
        std::vector<unsigned char> ones(vs * std::max<int64_t>(A->n, 1));
        for (int64_t j = 0; j < std::max<int64_t>(A->n, 1); ++j) {
            unsigned char* q = ones.data() + vs * j;
            switch (A->dtype) {
                case ASV_F32: { const float o = 1.f; memcpy(q, &o, 4); break; }
                case ASV_F64: { const double o = 1.0; memcpy(q, &o, 8); break; }
                case ASV_I32: { const int32_t o = 1; memcpy(q, &o, 4); break; }
                default: q[0] = 1; break;
            }
        }
        cudaError_t e = cudaMemcpyAsync(x, ones.data(), ones.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaFree(x);
            cudaFree(y);
            g_last_cuda = (int32_t)e;
            return ASV_ERR_CUDA;
        }
    }
    const PullIO io{x, nullptr, y};
    const auto t_start = std::chrono::steady_clock::now();
    auto elapsed_ms = [&]() {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // one warm-up and three timed launches of `dist` with the handle's
    // current settings; the median of the three
    auto time_pull = [&](int dist) -> float {
        launch_pull(A, dist, false, false, &io, s);
        float t[3];
        for (int r = 0; r < 3; ++r) {
            cudaEventRecord(e0, s);
            launch_pull(A, dist, false, false, &io, s);
            cudaEventRecord(e1, s);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&t[r], e0, e1);
        }
        std::sort(t, t + 3);
        return t[1];
    };
    const asv_pull_tune start = current();
    asv_pull_tune best = start;
    // the sub-warp pull: lanes per row x rows per lane group, starting from
    // the creation-time choice, then its neighbours outwards
    float bw = time_pull(1);
    const int lanes[] = {2, 4, 8, 16, 32};
    std::vector<asv_pull_tune> cands;
    for (int l : lanes)
        for (int u : {2, 4})
            if (l != start.lanes || u != start.unroll) cands.push_back({l, u, start.tma});
    std::stable_sort(cands.begin(), cands.end(), [&](const asv_pull_tune& p, const asv_pull_tune& q) {
        auto d = [&](const asv_pull_tune& t) { return std::abs(__builtin_ctz(t.lanes) - __builtin_ctz(start.lanes)); };
        return d(p) < d(q);
    });
    for (const asv_pull_tune& c : cands) {
        if (elapsed_ms() > budget_ms) break;
        A->pull_lanes = c.lanes;
        A->pull_unroll = c.unroll;
        const float t = time_pull(1);
        if (t < bw) {
            bw = t;
            best.lanes = c.lanes;
            best.unroll = c.unroll;
        }
    }
    A->pull_lanes = best.lanes;
    A->pull_unroll = best.unroll;
    // TMA staging of the one-row-per-thread pull (arithmetic types only)
    if (A->dtype != ASV_BOOL && elapsed_ms() <= budget_ms) {
        const float t_cur = time_pull(0);
        A->pull_tma = !A->pull_tma;
        const float t_alt = time_pull(0);
        if (t_alt < t_cur) best.tma = A->pull_tma ? 1 : 0;
        A->pull_tma = best.tma != 0;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const cudaError_t e = cudaGetLastError();
    cudaFree(x);
    cudaFree(y);
    if (e != cudaSuccess) {
        g_last_cuda = (int32_t)e;
        return ASV_ERR_CUDA;
    }
    if (h_out) *h_out = best;
    if (cache_path) {
        if (FILE* f = fopen(cache_path, "a")) {
            fprintf(f, "%s\t%d\t%d\t%d\n", key.c_str(), best.lanes, best.unroll, best.tma);
            fclose(f);
        }
    }
    return ASV_OK;
}

extern "C" asv_status asv_pull_tuning(asv_matrix A, asv_pull_tune* h_out) {
    if (!A || !h_out) return ASV_ERR_ARG;
    *h_out = asv_pull_tune{A->pull_lanes, A->pull_unroll, A->pull_tma ? 1 : 0};
    return ASV_OK;
}

extern "C" asv_status asv_spmspv_backward(asv_matrix A, int32_t B, const void* d_X, const void* d_dY, void* d_dX,
                                          void* d_dA, void* stream) {
    if (!A || B < 0 || !d_dY || (d_dA && !d_X)) return ASV_ERR_ARG;
    if (A->dtype != ASV_F32) return ASV_ERR_UNSUPPORTED;
    if (B > 128) return ASV_ERR_UNSUPPORTED;
    if (B == 0) return ASV_OK;
    CK(batched_backward(A, B, (const float*)d_X, (const float*)d_dY, (float*)d_dX, (float*)d_dA,
                        (cudaStream_t)stream));
    return ASV_OK;
}

extern "C" asv_status asv_spmspv_backward_list(asv_matrix A, int32_t B, const int64_t* d_xptr, const int32_t* d_xidx,
                                               const void* d_xval, const void* d_dY, void* d_dX, void* d_dA,
                                               void* stream) {
    if (!A || B < 0 || !d_dY || (d_dA && !d_xptr)) return ASV_ERR_ARG;
    if (A->dtype != ASV_F32) return ASV_ERR_UNSUPPORTED;
    if (B > 128) return ASV_ERR_UNSUPPORTED;
    if (B == 0) return ASV_OK;
    CK(batched_backward(A, B, nullptr, (const float*)d_dY, (float*)d_dX, (float*)d_dA, (cudaStream_t)stream,
                        d_dA ? d_xptr : nullptr, d_xidx, (const float*)d_xval));
    return ASV_OK;
}

extern "C" asv_status asv_get_status(asv_matrix A, void* stream) {
    if (!A) return ASV_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t v = 0;
    CK(cudaMemcpyAsync(&v, A->ws.status, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemsetAsync(A->ws.status, 0, 4, s));
    CK(cudaStreamSynchronize(s));
    return v;
}

extern "C" int32_t asv_last_cuda_error(void) { return g_last_cuda; }

extern "C" asv_status asv_debug_set_wait_limit(asv_matrix A, uint32_t polls) {
    if (!A) return ASV_ERR_ARG;
    A->wait_limit = polls;
    return ASV_OK;
}

extern "C" void asv_debug_fail_alloc(int32_t countdown) { g_fail_alloc.store(countdown > 0 ? countdown : 0); }

extern "C" const char* asv_status_string(asv_status s) {
    switch (s) {
        case ASV_OK: return "ok";
        case ASV_ERR_ARG: return "invalid argument";
        case ASV_ERR_NONCANONICAL: return "non-canonical CSR";
        case ASV_ERR_OVERFLOW: return "size overflows the int32 index layout";
        case ASV_ERR_CAPACITY: return "sparse output exceeds y_cap";
        case ASV_ERR_TIMEOUT: return "bounded device wait timed out";
        case ASV_ERR_CUDA: return "CUDA runtime error";
        case ASV_ERR_NOMEM: return "out of device memory";
        case ASV_ERR_UNSUPPORTED: return "unsupported combination";
    }
    return "unknown status";
}

extern "C" int32_t asv_version(void) { return 100; }
