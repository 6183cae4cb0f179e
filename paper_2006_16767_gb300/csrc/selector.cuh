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
    const MatFeat* mf;
    const TreeNode* trees;
    const int32_t* roots;
    int32_t* last_kid;
    unsigned long long cond;
    int32_t enabled;
};

__device__ __forceinline__ int eval_tree(const TreeNode* nodes, int root, const double* f) {
    int node = root;
    for (int depth = 0; depth < 64 && nodes[node].feature >= 0; ++depth)
        node = (f[nodes[node].feature] <= nodes[node].thr) ? nodes[node].left : nodes[node].right;
    return nodes[node].feature >= 0 ? 0 : nodes[node].leaf;
}

// Called by every thread of one block: stages the node table in shared
// memory, then thread 0 walks the trees, records the choice and sets the
// graph's SWITCH value when a handle is given.
__device__ __forceinline__ void run_selector(const SelectArg& sa, CallDesc* desc, TreeNode* sn) {
    const int cnt = min(sa.roots[kRootsLen - 1], kMaxTreeNodes);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) sn[i] = sa.trees[i];
    __syncthreads();
    if (threadIdx.x != 0) return;
    const MatFeat* mf = sa.mf;
    double f[13];
    f[0] = (double)mf->m;
    f[1] = (double)mf->n;
    f[2] = (double)mf->nnz;
    f[3] = (double)mf->max_row;
    f[4] = (double)mf->min_row;
    f[5] = mf->avg_row;
    f[6] = mf->relative_range;
    f[7] = mf->var_nnz_row;
    f[8] = mf->gini;
    f[9] = desc->vfeat[0];
    f[10] = desc->vfeat[1];
    f[11] = desc->vfeat[2];
    f[12] = desc->vfeat[3];
    const int* r = sa.roots + kRootsPerFormat * (desc->x_sparse * 2 + desc->out_mode);
    const int pattern = min(max(eval_tree(sn, r[0], f), 0), 2);  // 0 push, 1 masked pull, 2 pull
    const int dist = eval_tree(sn, r[1 + pattern], f);            // 0 thread, 1 warp, 2 balanced
    int kid;
    if (pattern == 2) {
        kid = ASV_K_PULL_THREAD + dist;
    } else if (pattern == 1) {
        kid = ASV_K_MPULL_THREAD + dist;
    } else {
        const int wb = eval_tree(sn, r[4], f);  // 0 atomic, 1 sort, 2 privatised
        kid = ASV_K_PUSH_THREAD_ATOM + 3 * wb + dist;
    }
    if (kid < 0 || kid >= ASV_K_COUNT) kid = ASV_K_PULL_BAL;
    desc->kid = kid;
    *sa.last_kid = kid;
    if (sa.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)sa.cond, (unsigned)kid);
}

}  // namespace asv
