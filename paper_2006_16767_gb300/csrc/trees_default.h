// Decision trees compiled into the library as its default selector.
// Records: {feature, threshold, left, right, leaf_class}; feature < 0 = leaf.
// Feature ids: 0 m, 1 n, 2 nnz, 3 max_row, 4 min_row, 5 avg_row,
// 6 relative_range, 7 var_nnz_row, 8 gini, 9 nnz_x, 10 x_sparsity,
// 11 nnz_s, 12 m_sparsity. Roots, five per call format -- pattern, distribution
// after push / masked pull / pull, write-back -- for (x dense, y dense),
// (x dense, y list), (x list, y dense), (x list, y list).
//
// Hand-set starting rules (push when x is very sparse, the plain SpMV when it
// is dense, the validated row-major kernel in between; balanced splits for
// skewed row lengths), used until trees trained on this GPU replace them.
#pragma once

namespace asv {

static const int kTreeNodesF32 = 11;
static const double kTreesF32[][5] = {
    {10, 0.005, 1, 2, 0}, {-1, 0, 0, 0, 0}, {10, 0.25, 3, 4, 0}, {-1, 0, 0, 0, 1}, {-1, 0, 0, 0, 2},
    {8, 0.5, 6, 7, 0},    {-1, 0, 0, 0, 1}, {-1, 0, 0, 0, 2},
    {11, 1e9, 9, 10, 0},  {-1, 0, 0, 0, 0}, {-1, 0, 0, 0, 0},
};
static const int kTreeRootsF32[20] = {0, 5, 5, 5, 8, 0, 5, 5, 5, 8, 0, 5, 5, 5, 8, 0, 5, 5, 5, 8};

static const int kTreeNodesBool = 11;
static const double kTreesBool[][5] = {
    {10, 0.005, 1, 2, 0}, {-1, 0, 0, 0, 0}, {10, 0.25, 3, 4, 0}, {-1, 0, 0, 0, 1}, {-1, 0, 0, 0, 2},
    {8, 0.5, 6, 7, 0},    {-1, 0, 0, 0, 1}, {-1, 0, 0, 0, 2},
    {11, 1e9, 9, 10, 0},  {-1, 0, 0, 0, 0}, {-1, 0, 0, 0, 0},
};
static const int kTreeRootsBool[20] = {0, 5, 5, 5, 8, 0, 5, 5, 5, 8, 0, 5, 5, 5, 8, 0, 5, 5, 5, 8};

}  // namespace asv
