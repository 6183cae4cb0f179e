// Kernel selector (Sec. V and Sec. VI-B): three cascaded decision trees over
// the Table 1 features -- computing pattern first, then workload
// distribution, then (for the push pattern) write-back. In the
// selector-driven path the trees are walked by the last block of the
// vector-feature pass, inside the CUDA graph whose SWITCH node runs the
// chosen candidate (selector.cuh); this file holds the host-side tables.
#include "internal.h"
#include "selector.cuh"
#include "trees_default.h"

namespace asv {

static_assert(kTreeNodesF32 <= kMaxTreeNodes && kTreeNodesBool <= kMaxTreeNodes,
              "compiled-in trees exceed the selector's node table");

void update_lazy(asv_matrix_s* H, const std::vector<TreeNode>& nodes, const int32_t* roots) {
    const int cnt = std::min((int)nodes.size(), kMaxTreeNodes);
    for (int q = 0; q < kRootsLen; ++q) H->h_roots[q] = roots[q];
    for (int f = 0; f < 4; ++f) {
        const int32_t* r = roots + kRootsPerFormat * f;
        // a leaf, or a split on a matrix feature, nnz_x or x_sparsity (ids 0..10)
        H->lazy_ok[f] = (f >= 2 && r[0] >= 0 && r[0] < cnt && nodes[r[0]].feature < 11) ? 1 : 0;
        // the format's window: from its lowest root to the next root of any
        // format above its highest one (the trained tables store a format's
        // five trees contiguously), at most kTreeWindow nodes; a node outside
        // it is read from global memory by the walk
        int lo = cnt, mx = -1;
        for (int t = 0; t < kRootsPerFormat; ++t) {
            lo = std::min(lo, r[t]);
            mx = std::max(mx, r[t]);
        }
        int hi = cnt;
        for (int q = 0; q < kRootsLen - 1; ++q)
            if (roots[q] > mx && roots[q] < hi) hi = roots[q];
        lo = std::max(lo, 0);
        hi = std::max(lo, std::min(hi, lo + kTreeWindow));
        H->win_lo[f] = lo;
        H->win_hi[f] = hi;
    }
}

// fmt = 2 * (x arrives as a list) + (sparse output), the call format whose
// trees the pass walks.
SelectArg select_arg(asv_matrix_s* H, unsigned long long cond, int fmt) {
    SelectArg sa;
    const asv_mfeat& m = H->h_mfeat;
    const double mf[9] = {(double)m.m, (double)m.n, (double)m.nnz, (double)m.max_row, (double)m.min_row,
                          m.avg_row, m.relative_range, m.var_nnz_row, m.gini};
    for (int q = 0; q < 9; ++q) sa.mf[q] = mf[q];
    const int f = (fmt >= 0 && fmt < 4) ? fmt : 0;
    sa.trees = H->d_trees;
    for (int t = 0; t < kRootsPerFormat; ++t) sa.root[t] = H->h_roots[kRootsPerFormat * f + t];
    sa.win_lo = H->win_lo[f];
    sa.win_hi = H->win_hi[f];
    sa.last_kid = H->d_last_kid;
    sa.cond = cond;
    sa.enabled = 1;
    sa.lazy = f >= 2 ? H->lazy_ok[f] : 0;
    sa.lcol = H->ws.lcol;
    sa.lcol_n = H->ws.lcol_n;
    sa.lcol_cap = H->ws.lcol_cap;
    sa.long_rest_n = H->long_rest_n;
    return sa;
}

// The compiled-in trees of a value type: the Boolean table for ASV_BOOL, the
// FP32 table for every arithmetic type.
void default_trees(int32_t dtype, std::vector<TreeNode>& nodes, int32_t roots[kRootsLen]) {
    const bool b = dtype == ASV_BOOL;
    const int cnt = b ? kTreeNodesBool : kTreeNodesF32;
    const double (*tab)[5] = b ? kTreesBool : kTreesF32;
    const int* rt = b ? kTreeRootsBool : kTreeRootsF32;
    nodes.clear();
    for (int i = 0; i < cnt; ++i) {
        TreeNode t;
        t.feature = (int32_t)tab[i][0];
        t.thr = tab[i][1];
        t.left = (int32_t)tab[i][2];
        t.right = (int32_t)tab[i][3];
        t.leaf = (int32_t)tab[i][4];
        nodes.push_back(t);
    }
    for (int i = 0; i < kRootsLen - 1; ++i) roots[i] = rt[i];
    roots[kRootsLen - 1] = cnt;
}

}  // namespace asv
