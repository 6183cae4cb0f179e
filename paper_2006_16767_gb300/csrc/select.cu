// Kernel selector (Sec. V and Sec. VI-B): three cascaded decision trees over
// the Table 1 features -- computing pattern first, then workload
// distribution, then (for the push pattern) write-back -- evaluated by one
// device thread right after the vector-feature pass, with no host round-trip.
// Inside the selector-driven CUDA graph the chosen id becomes the value of a
// SWITCH conditional node whose branches are the candidate kernels.
#include "internal.h"
#include "trees_default.h"

namespace asv {

__device__ __forceinline__ int eval_tree(const TreeNode* nodes, int root, const double* f) {
    int node = root;
    for (int depth = 0; depth < 64 && nodes[node].feature >= 0; ++depth)
        node = (f[nodes[node].feature] <= nodes[node].thr) ? nodes[node].left : nodes[node].right;
    return nodes[node].feature >= 0 ? 0 : nodes[node].leaf;
}

// The block first copies the node table into shared memory (one burst), so
// the walk down the trees is a chain of shared-memory reads, not of global
// loads. roots[3] holds the number of nodes.
__global__ void __launch_bounds__(128) k_select(const MatFeat* __restrict__ mf, CallDesc* desc,
                                                const TreeNode* __restrict__ trees, const int32_t* __restrict__ roots,
                                                int32_t* last_kid, unsigned long long cond, int set_cond) {
    __shared__ TreeNode sn[kMaxTreeNodes];
    const int cnt = min(__ldg(roots + 3), kMaxTreeNodes);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) sn[i] = trees[i];
    __syncthreads();
    trees = sn;
    if (threadIdx.x != 0) return;
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
    const int pattern = eval_tree(trees, roots[0], f);  // 0 push, 1 masked pull, 2 pull
    const int dist = eval_tree(trees, roots[1], f);     // 0 thread, 1 warp, 2 balanced
    int kid;
    if (pattern == 2) {
        kid = ASV_K_PULL_THREAD + dist;
    } else if (pattern == 1) {
        kid = ASV_K_MPULL_THREAD + dist;
    } else {
        const int wb = eval_tree(trees, roots[2], f);  // 0 atomic, 1 sort, 2 privatised
        kid = ASV_K_PUSH_THREAD_ATOM + 3 * wb + dist;
    }
    if (kid < 0 || kid >= ASV_K_COUNT) kid = ASV_K_PULL_BAL;
    desc->kid = kid;
    *last_kid = kid;
    if (set_cond) cudaGraphSetConditional((cudaGraphConditionalHandle)cond, (unsigned)kid);
}

void launch_select(asv_matrix_s* H, unsigned long long cond_handle, bool set_cond, cudaStream_t s) {
    k_select<<<1, 128, 0, s>>>(H->d_mfeat, H->d_desc, H->d_trees, H->d_roots, H->d_last_kid, cond_handle,
                              set_cond ? 1 : 0);
}

void default_trees(std::vector<TreeNode>& nodes, int32_t roots[4]) {
    nodes.clear();
    for (int i = 0; i < kDefaultTreeNodes; ++i) {
        TreeNode t;
        t.feature = (int32_t)kDefaultTrees[i][0];
        t.thr = kDefaultTrees[i][1];
        t.left = (int32_t)kDefaultTrees[i][2];
        t.right = (int32_t)kDefaultTrees[i][3];
        t.leaf = (int32_t)kDefaultTrees[i][4];
        nodes.push_back(t);
    }
    for (int i = 0; i < 3; ++i) roots[i] = kDefaultTreeRoots[i];
    roots[3] = (int32_t)nodes.size();
}

}  // namespace asv
