// Device-side evaluation of the cascaded decision trees (Sec. V-B, VI-B),
// shared by the standalone selector kernel and the last block of the
// vector-feature pass.
#pragma once
#include "common.cuh"

namespace asv {

// roots[5*f + t] for format f = 2*(x arrives as a list) + (sparse output):
// t = 0 the pattern tree, t = 1 + p the distribution tree used once pattern p
// (0 push, 1 masked pull, 2 pull) is chosen, t = 4 the write-back tree;
// roots[20] holds the number of nodes in the shared node table.
constexpr int kRootsPerFormat = 5;
constexpr int kRootsLen = 4 * kRootsPerFormat + 1;

// What the selector needs besides the call descriptor. cond is the SWITCH
// node's conditional handle (0 = none).
struct SelectArg {
    double mf[9];  // Table 1 matrix features 0..8, by value (no load on the critical path)
    const TreeNode* trees;
    const int32_t* roots;
    int32_t* last_kid;
    unsigned long long cond;
    int32_t enabled;
    // lazy evaluation hint: the call format's pattern tree starts with a
    // feature a listed x gives without a pass over it (see k_feat_sparse)
    int32_t lazy;
    // the push kernels' hub-column queue, reset by every feature pass, and
    // the count of long-row pieces of the Boolean pull's second pass
    int2* lcol;
    unsigned int* lcol_n;
    int32_t lcol_cap;
    unsigned int* long_rest_n;
};

// Nodes [lo, hi) of the table are staged in shared memory (sn); a node
// outside that window is read from global memory. Features with an index of
// nknown or more are not available: a node testing one makes the walk give
// up (*unknown set).
__device__ __forceinline__ int eval_tree(const TreeNode* sn, int lo, int hi, const TreeNode* nodes, int root,
                                         const double* f, int nknown = 13, bool* unknown = nullptr) {
    int node = root;
    for (int depth = 0; depth < 64; ++depth) {
        const TreeNode nd = (node >= lo && node < hi) ? sn[node - lo] : nodes[node];
        if (nd.feature < 0) return nd.leaf;
        if (nd.feature >= nknown) {
            *unknown = true;
            return 0;
        }
        node = (f[nd.feature] <= nd.thr) ? nd.left : nd.right;
    }
    return 0;
}

// Called by every thread of a block: stages the trees of call format `fmt`
// in shared memory. The trained tables store the five trees of a format
// contiguously, so the window from the format's lowest root to the next
// root above its highest root holds all of them (about a quarter of the
// table: one load per thread).
__device__ __forceinline__ const int* stage_trees(const SelectArg& sa, int fmt, TreeNode* sn, int& lo, int& hi) {
    const int cnt = min(sa.roots[kRootsLen - 1], kMaxTreeNodes);
    const int* r = sa.roots + kRootsPerFormat * fmt;
    lo = cnt;
    int mx = -1;
    for (int t = 0; t < kRootsPerFormat; ++t) {
        lo = min(lo, r[t]);
        mx = max(mx, r[t]);
    }
    hi = cnt;
    for (int q = 0; q < kRootsLen - 1; ++q)
        if (sa.roots[q] > mx && sa.roots[q] < hi) hi = sa.roots[q];
    lo = max(lo, 0);
    hi = min(hi, lo + kTreeWindow);
    for (int i = lo + (int)threadIdx.x; i < hi; i += blockDim.x) sn[i - lo] = sa.trees[i];
    __syncthreads();
    return r;
}

// The cascade of Sec. VI-B (pattern, then distribution, then write-back for
// the push pattern) over features f[0 .. nknown); -1 when a tree on the path
// needs a feature beyond them.
__device__ __forceinline__ int pick_kernel(const TreeNode* sn, int lo, int hi, const TreeNode* nodes, const int* r,
                                           const double* f, int nknown) {
    bool unknown = false;
    const int pattern = min(max(eval_tree(sn, lo, hi, nodes, r[0], f, nknown, &unknown), 0), 2);
    const int dist = eval_tree(sn, lo, hi, nodes, r[1 + pattern], f, nknown, &unknown);
    int kid;
    if (pattern == 2) {
        kid = ASV_K_PULL_THREAD + dist;  // 0 thread, 1 warp, 2 balanced
    } else if (pattern == 1) {
        kid = ASV_K_MPULL_THREAD + dist;
    } else {
        const int wb = eval_tree(sn, lo, hi, nodes, r[4], f, nknown, &unknown);  // 0 atomic, 1 sort, 2 privatised
        kid = ASV_K_PUSH_THREAD_ATOM + 3 * wb + dist;
    }
    if (unknown) return -1;
    return (kid < 0 || kid >= ASV_K_COUNT) ? ASV_K_PULL_BAL : kid;
}

// Records the choice and sets the graph's SWITCH value when a handle is given.
__device__ __forceinline__ void commit_kernel(const SelectArg& sa, CallDesc* desc, int kid) {
    desc->kid = kid;
    *sa.last_kid = kid;
    if (sa.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)sa.cond, (unsigned)kid);
}

// Called by every thread of one block once the descriptor holds all the
// features: stages the call format's trees, then thread 0 walks them.
__device__ __forceinline__ void run_selector(const SelectArg& sa, CallDesc* desc, TreeNode* sn) {
    int lo, hi;
    const int* r = stage_trees(sa, desc->x_sparse * 2 + desc->out_mode, sn, lo, hi);
    if (threadIdx.x != 0) return;
    double f[13];
#pragma unroll
    for (int q = 0; q < 9; ++q) f[q] = sa.mf[q];
    f[9] = desc->vfeat[0];
    f[10] = desc->vfeat[1];
    f[11] = desc->vfeat[2];
    f[12] = desc->vfeat[3];
    commit_kernel(sa, desc, pick_kernel(sn, lo, hi, sa.trees, r, f, 13));
}

}  // namespace asv
