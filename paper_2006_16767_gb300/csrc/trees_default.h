// Decision trees compiled into the library as its default selector.
// Records: {feature, threshold, left, right, leaf_class}; feature < 0 = leaf.
// Feature ids: 0 m, 1 n, 2 nnz, 3 max_row, 4 min_row, 5 avg_row,
// 6 relative_range, 7 var_nnz_row, 8 gini, 9 nnz_x, 10 x_sparsity,
// 11 nnz_s, 12 m_sparsity.
//
// These are hand-set starting rules (push when x is very sparse, the plain
// SpMV when it is dense, the validated row-major kernel in between; balanced
// splits for skewed row lengths), used until trees trained on GB300 timings
// replace them.
#pragma once

namespace asv {

static const int kDefaultTreeNodes = 11;
static const double kDefaultTrees[kDefaultTreeNodes][5] = {
    // pattern tree (root 0)
    {10, 0.01, 1, 2, 0},   // 0: x_sparsity <= 0.01 ?
    {-1, 0, 0, 0, 0},      // 1: push
    {10, 0.25, 3, 4, 0},   // 2: x_sparsity <= 0.25 ?
    {-1, 0, 0, 0, 1},      // 3: masked pull
    {-1, 0, 0, 0, 2},      // 4: pull
    // distribution tree (root 5)
    {8, 0.5, 6, 7, 0},     // 5: gini <= 0.5 ?
    {-1, 0, 0, 0, 1},      // 6: warp
    {-1, 0, 0, 0, 2},      // 7: balanced
    // write-back tree (root 8)
    {11, 1e9, 9, 10, 0},   // 8: nnz_s <= 1e9 ?
    {-1, 0, 0, 0, 0},      // 9: atomic
    {-1, 0, 0, 0, 0},      // 10: atomic
};
static const int kDefaultTreeRoots[3] = {0, 5, 8};

}  // namespace asv
