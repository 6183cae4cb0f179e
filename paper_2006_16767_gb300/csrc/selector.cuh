// Device-side evaluation of the cascaded decision trees (Sec. V-B, VI-B) by
// the vector-feature pass: its last block once the features are complete,
// or, for a listed x, every block that takes part when the features the
// list gives for free decide.
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
// node's conditional handle (0 = none). The call format's five roots and the
// bounds of the node window that holds its trees are computed on the host
// from the table (they change only with it), so a feature pass stages the
// window with one round of loads at its start and walks the trees without
// reading the roots first.
struct SelectArg {
    double mf[9];  // Table 1 matrix features 0..8, by value (no load on the critical path)
    const TreeNode* trees;
    int32_t root[kRootsPerFormat];  // the call format's roots (see above)
    int32_t win_lo, win_hi;         // its node window [win_lo, win_hi), at most kTreeWindow nodes
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
                                         const double* f, int nknown, bool* unknown) {
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

// Called by every thread of a block (B threads) of a selector-enabled pass:
// copies the call format's node window into shared memory, as 8-byte words,
// four loads in flight per thread. The copy is visible to the block after
// its next __syncthreads.
template <int B>
__device__ __forceinline__ void stage_window(const SelectArg& sa, TreeNode* sn) {
    static_assert(sizeof(TreeNode) == 24, "a node is three 8-byte words");
    const int nw = 3 * (sa.win_hi - sa.win_lo);
    const long long* __restrict__ src = reinterpret_cast<const long long*>(sa.trees + sa.win_lo);
    long long* dst = reinterpret_cast<long long*>(sn);
#pragma unroll 4
    for (int q = (int)threadIdx.x; q < nw; q += B) dst[q] = __ldg(src + q);
}

// The cascade of Sec. VI-B (pattern, then distribution, then write-back for
// the push pattern) over features f[0 .. nknown) (f in shared memory), taken
// by one whole warp: lanes 0..4 walk the format's five trees at once (the
// pattern tree, the three distribution trees, the write-back tree) and the
// cascade then takes the leaves on its path, so the walk costs the deepest
// tree rather than the sum of three. The result is the sequential cascade's:
// the kernel id, or -1 when a tree on the path needs a feature beyond
// nknown. Every lane returns it.
__device__ __forceinline__ int pick_kernel(const SelectArg& sa, const TreeNode* sn, const double* f, int nknown) {
    const int lane = threadIdx.x & 31;
    int leaf = 0;
    bool unk = false;
    if (lane < kRootsPerFormat) leaf = eval_tree(sn, sa.win_lo, sa.win_hi, sa.trees, sa.root[lane], f, nknown, &unk);
    const unsigned um = __ballot_sync(0xffffffffu, unk);
    const int p0 = __shfl_sync(0xffffffffu, leaf, 0);
    const int pattern = min(max(p0, 0), 2);
    const int dist = __shfl_sync(0xffffffffu, leaf, 1 + pattern);
    const int wb = __shfl_sync(0xffffffffu, leaf, 4);  // 0 atomic, 1 sort, 2 privatised
    // the trees on the path: pattern, its distribution tree, and the
    // write-back tree for the push pattern
    const unsigned path = 1u | (1u << (1 + pattern)) | (pattern == 0 ? (1u << 4) : 0u);
    if (um & path) return -1;
    int kid;
    if (pattern == 2) kid = ASV_K_PULL_THREAD + dist;  // 0 thread, 1 warp, 2 balanced
    else if (pattern == 1) kid = ASV_K_MPULL_THREAD + dist;
    else kid = ASV_K_PUSH_THREAD_ATOM + 3 * wb + dist;
    return (kid < 0 || kid >= ASV_K_COUNT) ? ASV_K_PULL_BAL : kid;
}

// Records the choice and sets the graph's SWITCH value when a handle is given.
__device__ __forceinline__ void commit_kernel(const SelectArg& sa, CallDesc* desc, int kid) {
    desc->kid = kid;
    *sa.last_kid = kid;
    if (sa.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)sa.cond, (unsigned)kid);
}

// Called by every thread of the block that published the descriptor, once
// it holds all the features (vf: the four vector features as published, in
// shared memory); the call format's window was staged at the start of the
// pass. Warp 0 walks the trees and lane 0 commits the choice.
__device__ __forceinline__ void run_selector(const SelectArg& sa, CallDesc* desc, const TreeNode* sn,
                                             const double* vf) {
    __shared__ double s_f[13];
    if (threadIdx.x < 32) {
        if (threadIdx.x == 0) {
#pragma unroll
            for (int q = 0; q < 9; ++q) s_f[q] = sa.mf[q];
#pragma unroll
            for (int q = 0; q < 4; ++q) s_f[9 + q] = vf[q];
        }
        __syncwarp();
        const int kid = pick_kernel(sa, sn, s_f, 13);
        if (threadIdx.x == 0) commit_kernel(sa, desc, kid);
    }
}

}  // namespace asv
