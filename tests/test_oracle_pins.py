"""Pins for the oracle: each test ties an oracle function to something other than
itself (a brute-force dense product, a library routine, a closed form or an
invariant), chosen so that a dropped term, a wrong index or sign, or a
transposed operand fails at least one of them. CPU only."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csgraph

import gen
import oracle


def dense_of(m, n, rowptr, col, val=None):
    """Dense matrix from CSR by direct placement (rows expanded with np.repeat)."""
    D = np.zeros((m, n), np.float64)
    rows = np.repeat(np.arange(m), np.diff(rowptr))
    D[rows, col] = 1.0 if val is None else val
    return D


def pattern_of(m, n, rowptr, col):
    P = np.zeros((m, n), np.int64)
    rows = np.repeat(np.arange(m), np.diff(rowptr))
    P[rows, col] = 1
    return P


SHAPES = [(1, 1, 1.0), (7, 5, 0.5), (33, 64, 0.2), (64, 17, 0.3), (64, 64, 0.05), (5, 9, 0.0)]


@pytest.mark.parametrize("m,n,dens", SHAPES)
def test_csr_pull_dense_bruteforce_exact(m, n, dens):
    # values in {-2..2}/4: every product and partial sum is exact in FP64,
    # so the oracle must equal the dense product bit for bit.
    rowptr, col, val = gen.random_csr(m, n, dens, seed=11 + m)
    x = gen.small_ints(n, -2, 2, 4.0, seed=5, stream=m)
    D = dense_of(m, n, rowptr, col, val)
    y, s = oracle.csr_pull(rowptr, col, val, x)
    assert np.array_equal(y, D @ x)
    assert np.array_equal(s, np.abs(D) @ np.abs(x))


@pytest.mark.parametrize("m,n,dens", SHAPES)
def test_csc_push_matches_dense_and_structural_set(m, n, dens):
    rowptr, col, val = gen.random_csr(m, n, dens, seed=21 + n)
    x = gen.small_ints(n, -2, 2, 4.0, seed=6, stream=n)
    x[::3] = 0.0
    colptr, rowidx, perm = oracle.csr_to_csc(m, n, rowptr, col)
    xidx, xval = oracle.compact(x)
    y, touched = oracle.csc_push(m, colptr, rowidx, val[perm], xidx, xval)
    D = dense_of(m, n, rowptr, col, val)
    assert np.array_equal(y, D @ x)
    P = pattern_of(m, n, rowptr, col)
    assert np.array_equal(touched.astype(bool), (P @ (x != 0).astype(np.int64)) > 0)


@pytest.mark.parametrize("m,n,dens", SHAPES)
def test_spmspv_rowmajor_dense_and_explicit_zeros(m, n, dens):
    rowptr, col, val = gen.random_csr(m, n, dens, seed=31 + m)
    idx = gen.sample_positions(n, max(1, n // 3), seed=7, stream=m)
    xv = gen.small_ints(len(idx), -2, 2, 4.0, seed=8, stream=m)
    xv[::2] = 0.0  # explicit zeros stay structural
    y, s, hit = oracle.spmspv_rowmajor(n, rowptr, col, val, idx, xv)
    D = dense_of(m, n, rowptr, col, val)
    xd = gen.densify(n, idx, xv)
    assert np.array_equal(y, D @ xd)
    mask = np.zeros(n, np.int64)
    mask[idx] = 1
    P = pattern_of(m, n, rowptr, col)
    assert np.array_equal(hit.astype(bool), (P @ mask) > 0)


def test_transpose_matches_scipy_and_round_trips():
    for (m, n, dens, seed) in [(50, 80, 0.1, 1), (80, 50, 0.2, 2), (1, 300, 0.5, 3), (300, 1, 0.5, 4)]:
        rowptr, col, _ = gen.random_csr(m, n, dens, seed=seed)
        nnz = len(col)
        tag = np.arange(nnz, dtype=np.float64) + 1.0
        colptr, rowidx, perm = oracle.csr_to_csc(m, n, rowptr, col)
        ref = sp.csr_matrix((tag, col, rowptr), shape=(m, n)).tocsc()
        ref.sort_indices()
        assert np.array_equal(colptr, ref.indptr)
        assert np.array_equal(rowidx, ref.indices)
        assert np.array_equal(tag[perm], ref.data)
        assert np.array_equal(np.sort(perm), np.arange(nnz))
        # transposing the transpose (CSC of A is CSR of A^T) gives A back
        rp2, c2, perm2 = oracle.csr_to_csc(n, m, colptr, rowidx)
        assert np.array_equal(rp2, rowptr) and np.array_equal(c2, col)
        assert np.array_equal(perm[perm2], np.arange(nnz))


def test_unit_vectors_give_columns_exactly():
    m, n = 40, 30
    rowptr, col, val = gen.random_csr(m, n, 0.2, seed=9, values="uniform")
    D = dense_of(m, n, rowptr, col, val)
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        y, _ = oracle.csr_pull(rowptr, col, val, e)
        assert np.array_equal(y, D[:, j])
        colptr, rowidx, perm = oracle.csr_to_csc(m, n, rowptr, col)
        yp, _ = oracle.csc_push(m, colptr, rowidx, val[perm], np.array([j]), np.array([1.0]))
        assert np.array_equal(yp, D[:, j])


def test_linearity_and_adjoint():
    m, n = 300, 200
    rowptr, col, val = gen.random_csr(m, n, 0.05, seed=12, values="uniform")
    x = gen.uniform(n, -1, 1, seed=1, stream=1)
    z = gen.uniform(n, -1, 1, seed=1, stream=2)
    a, b = 0.75, -1.3
    yx, sx = oracle.csr_pull(rowptr, col, val, x)
    yz, sz = oracle.csr_pull(rowptr, col, val, z)
    yc, _ = oracle.csr_pull(rowptr, col, val, a * x + b * z)
    assert np.all(np.abs(yc - (a * yx + b * yz)) <= 1e-12 * (abs(a) * sx + abs(b) * sz) + 1e-300)
    # <dy, A x> = <A^T dy, x>, A^T read through the CSC arrays
    colptr, rowidx, perm = oracle.csr_to_csc(m, n, rowptr, col)
    dy = gen.uniform(m, -1, 1, seed=1, stream=3)
    atdy, _ = oracle.csc_pull(colptr, rowidx, val[perm], dy)
    lhs, rhs = float(dy @ yx), float(atdy @ x)
    scale = float(np.abs(dy) @ sx)
    assert abs(lhs - rhs) <= 1e-12 * scale
    # and A^T dy equals the transpose's dense product
    D = dense_of(m, n, rowptr, col, val)
    assert np.allclose(atdy, D.T @ dy, rtol=0, atol=1e-12)


@pytest.mark.parametrize("g", [1, 2, 3, 8, 64])
def test_laplace2d_closed_forms(g):
    rowptr, col, val = gen.laplace2d(g)
    m = g * g
    assert rowptr[-1] == 5 * g * g - 4 * g
    p, q = np.divmod(np.arange(m), g)
    top, bot, left, right = (p == 0), (p == g - 1), (q == 0), (q == g - 1)
    # A*1 = number of missing neighbours
    y1, _ = oracle.csr_pull(rowptr, col, val, np.ones(m))
    assert np.array_equal(y1, (top.astype(int) + bot + left + right).astype(np.float64))
    # a linear field is annihilated in the interior; at the boundary the result is
    # the sum of the missing neighbours' values of the linearly extended field
    yp, _ = oracle.csr_pull(rowptr, col, val, p.astype(np.float64))
    expect = -1.0 * top + g * bot + p * left + p * right
    assert np.array_equal(yp, expect.astype(np.float64))
    yq, _ = oracle.csr_pull(rowptr, col, val, q.astype(np.float64))
    expect_q = q * top + q * bot - 1.0 * left + g * right
    assert np.array_equal(yq, expect_q.astype(np.float64))


def test_stencil27_row_sums_and_dominance():
    g = 12
    rowptr, col, val, rowsum = gen.stencil27(g, seed=gen.config_seed(5))
    m = g ** 3
    assert rowptr[-1] == (3 * g - 2) ** 3
    y, s = oracle.csr_pull(rowptr, col, val.astype(np.float64), np.ones(m))
    assert np.all(np.abs(y - rowsum) <= 1e-13 * s)
    # diagonally dominant: centre >= sum of off-diagonal magnitudes
    rows = np.repeat(np.arange(m), np.diff(rowptr))
    diag = val[col == rows].astype(np.float64)
    assert len(diag) == m
    assert np.all(2 * diag >= y)


def test_compact_ieee_semantics():
    x = np.array([0.0, -0.0, 1.0, np.nan, -np.inf, 5e-324, 0.0, -2.5, np.inf, -0.0])
    idx, val = oracle.compact(x)
    ref = np.flatnonzero(x)
    assert np.array_equal(idx, ref)
    assert np.array_equal(val, x[ref], equal_nan=True)
    rng_x = gen.uniform(10000, -1, 1, seed=3)
    rng_x[gen.sample_positions(10000, 7000, seed=4)] = 0.0
    idx, val = oracle.compact(rng_x)
    assert np.array_equal(idx, np.flatnonzero(rng_x))
    assert oracle.compact(np.zeros(0))[0].size == 0


def gini_pairwise(d):
    d = np.asarray(d, np.float64)
    m = len(d)
    return np.abs(d[:, None] - d[None, :]).sum() / (2.0 * m * m * d.mean())


def test_matrix_features_special_cases_and_definitions():
    # equal row lengths: Gini 0, std 0
    rowptr, col, val = gen.laplace2d(1)
    f = oracle.matrix_features(1, 1, rowptr)
    assert f["gini"] == 0.0 and f["var_nnz_row"] == 0.0
    rp = np.arange(0, 4 * 10 + 1, 4, dtype=np.int32)
    f = oracle.matrix_features(10, 50, rp)
    assert f["gini"] == 0.0 and f["var_nnz_row"] == 0.0 and f["avg_row"] == 4.0
    assert f["relative_range"] == 0.0
    # one nonempty row out of m: Gini = (m - 1) / m
    for m in (1, 2, 7, 100):
        rp = np.zeros(m + 1, np.int32)
        rp[-1] = 5
        f = oracle.matrix_features(m, 10, rp)
        assert abs(f["gini"] - (m - 1) / m) <= 1e-15
    # random degree sequences against the pairwise-difference definition and numpy
    for seed in range(5):
        m = 200 + seed
        d = (gen.uniform(m, 0, 1, seed=seed) ** 3 * 50).astype(np.int32)
        rp = np.concatenate([[0], np.cumsum(d)]).astype(np.int32)
        f = oracle.matrix_features(m, 77, rp)
        assert f["m"] == m and f["n"] == 77 and f["nnz"] == d.sum()
        assert f["max_row"] == d.max() and f["min_row"] == d.min()
        assert f["avg_row"] == d.sum() / m
        assert f["relative_range"] == (d.max() - d.min()) / 77
        assert abs(f["var_nnz_row"] - np.std(d.astype(np.float64))) <= 1e-12 * max(1.0, np.std(d))
        assert abs(f["gini"] - gini_pairwise(d)) <= 1e-12
    # empty matrix
    f = oracle.matrix_features(3, 4, np.zeros(4, np.int32))
    assert f["gini"] == 0.0 and f["nnz"] == 0


def test_vector_features_counts():
    m, n = 120, 90
    rowptr, col, _ = gen.random_csr(m, n, 0.1, seed=17)
    colptr, _, _ = oracle.csr_to_csc(m, n, rowptr, col)
    nnz = len(col)
    f = oracle.vector_features(n, nnz, colptr, np.arange(n, dtype=np.int32))
    assert f["nnz_s"] == nnz and f["m_sparsity"] == 1.0 and f["x_sparsity"] == 1.0
    idx = gen.sample_positions(n, 13, seed=2)
    f = oracle.vector_features(n, nnz, colptr, idx)
    assert f["nnz_s"] == np.isin(col, idx).sum()
    assert f["nnz_x"] == 13 and f["x_sparsity"] == 13 / n
    assert f["m_sparsity"] == f["nnz_s"] / nnz


def test_bool_pull_bruteforce():
    for seed in range(4):
        m, n = 50 + seed, 60
        rowptr, col, _ = gen.random_csr(m, n, 0.05, seed=seed)
        x = (gen.uniform(n, 0, 1, seed=seed, stream=9) < 0.2).astype(np.uint8)
        y = oracle.bool_pull(rowptr, col, x)
        P = pattern_of(m, n, rowptr, col)
        assert np.array_equal(y.astype(bool), (P @ x.astype(np.int64)) > 0)


def test_i32_wraparound():
    m, n = 40, 40
    rowptr, col, _ = gen.random_csr(m, n, 0.3, seed=3)
    val = (gen.uniform(len(col), -2**31, 2**31 - 1, seed=1).astype(np.int64)).astype(np.int32)
    x = (gen.uniform(n, -2**31, 2**31 - 1, seed=2).astype(np.int64)).astype(np.int32)
    y = oracle.i32_pull(rowptr, col, val, x)
    P = dense_of(m, n, rowptr, col, None).astype(np.int64)
    rows = np.repeat(np.arange(m), np.diff(rowptr))
    ref = np.zeros(m, np.uint64)
    prod = (val.astype(np.int64).astype(np.uint64) * x[col].astype(np.int64).astype(np.uint64))
    np.add.at(ref, rows, prod)  # uint64 wrap, then reduce mod 2^32
    assert np.array_equal(y, (ref & np.uint64(0xFFFFFFFF)).astype(np.uint32).view(np.int32))
    assert P.sum() == len(col)


def graph500_validate(n, rowptr, col, root, level):
    assert level[root] == 0
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    lu, lv = level[rows], level[col]
    both = (lu >= 0) & (lv >= 0)
    assert np.all(np.abs(lu[both] - lv[both]) <= 1)
    assert np.all((lu >= 0) == (lv >= 0))  # an edge never leaves the reached set
    # every reached non-root vertex has a neighbour one level up
    has_parent = np.zeros(n, bool)
    ok = both & (lv == lu - 1)
    has_parent[rows[ok]] = True
    reached = level > 0
    assert np.all(has_parent[reached])


@pytest.mark.parametrize("scale,seed", [(8, 1), (10, 2), (12, 3)])
def test_bfs_vs_scipy_and_frontier_recurrence(scale, seed):
    rowptr, col = gen.rmat(scale, 8, seed=seed)
    n = 1 << scale
    deg = np.diff(rowptr)
    root = int(np.flatnonzero(deg > 0)[0])
    level, L = oracle.bfs(n, rowptr, col, root)
    A = sp.csr_matrix((np.ones(len(col)), col, rowptr), shape=(n, n))
    dist = csgraph.shortest_path(A, method="D", unweighted=True, indices=root)
    ref = np.where(np.isinf(dist), -1, dist).astype(np.int32)
    assert np.array_equal(level, ref)
    graph500_validate(n, rowptr, col, root, level)
    # frontier_{l+1} = (A * frontier_l) AND NOT visited_l
    fr = oracle.frontiers(n, rowptr, col, root)
    assert len(fr) == L
    visited = np.zeros(n, np.uint8)
    for l in range(L):
        f = np.zeros(n, np.uint8)
        f[fr[l]] = 1
        visited |= f
        nxt = oracle.bool_pull(rowptr, col, f) & (1 - visited)
        want = np.flatnonzero(nxt)
        if l + 1 < L:
            assert np.array_equal(want, fr[l + 1])
        else:
            assert want.size == 0


def test_pagerank_mass_invariant():
    rowptr, col = gen.rmat(11, 8, seed=4)
    N = 1 << 11
    colptr, _, _ = oracle.csr_to_csc(N, N, rowptr, col)
    r = gen.uniform(N, 0, 1, seed=5)
    r /= r.sum()
    x, y, rn = oracle.pagerank_step(N, rowptr, col, colptr, r, 0.85)
    deg = np.diff(colptr)
    # each column j hands out r_j/deg_j to deg_j rows: total mass is preserved
    assert abs(y.sum() - r[deg > 0].sum()) <= 1e-12
    assert np.all(x[deg == 0] == 0.0)
    assert abs(rn.sum() - (0.15 + 0.85 * y.sum())) <= 1e-12


def test_grad_values_finite_difference():
    m, n = 30, 20
    rowptr, col, val = gen.random_csr(m, n, 0.2, seed=23, values="uniform")
    x = gen.uniform(n, -1, 1, seed=2)
    w = gen.uniform(m, -1, 1, seed=3)
    dA = oracle.grad_values(rowptr, col, w, x)
    # L(A) = w^T A x is linear in the values, so central differences are exact up to roundoff
    h = 1e-3
    for k in range(len(col)):
        vp, vm = val.copy(), val.copy()
        vp[k] += h
        vm[k] -= h
        Lp = float(w @ oracle.csr_pull(rowptr, col, vp, x)[0])
        Lm = float(w @ oracle.csr_pull(rowptr, col, vm, x)[0])
        assert abs((Lp - Lm) / (2 * h) - dA[k]) <= 1e-9 * max(1.0, abs(dA[k]))
    # and equals the outer product dy x^T restricted to the pattern
    rows = np.repeat(np.arange(m), np.diff(rowptr))
    assert np.array_equal(dA, np.outer(w, x)[rows, col])


def test_empty_shapes():
    y, s = oracle.csr_pull(np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0), np.zeros(5))
    assert y.size == 0
    rp = np.zeros(4, np.int32)
    y, s = oracle.csr_pull(rp, np.zeros(0, np.int32), np.zeros(0), np.zeros(2))
    assert np.array_equal(y, np.zeros(3)) and np.array_equal(s, np.zeros(3))
    colptr, rowidx, perm = oracle.csr_to_csc(3, 2, rp, np.zeros(0, np.int32))
    assert np.array_equal(colptr, np.zeros(3)) and rowidx.size == 0
    y, t = oracle.csc_push(3, colptr, rowidx, np.zeros(0), np.zeros(0, np.int32), np.zeros(0))
    assert np.array_equal(y, np.zeros(3)) and not t.any()


def test_pagerank_delta_equals_the_linear_solve_without_threshold():
    """With eps = 0 the delta iteration sums the Neumann series of
    (I - d A D^-1)^-1 (1-d)/N; pinned against numpy's dense solve of that
    system on a small symmetric graph with a dangling (isolated) vertex."""
    rp, c = gen.rmat(7, 4, seed=12)
    n = 1 << 7
    Ad = np.zeros((n, n))
    for i in range(n):
        Ad[i, c[rp[i]:rp[i + 1]]] = 1.0
    deg = Ad.sum(axis=0)
    assert (deg == 0).any()
    M = 0.85 * Ad / np.where(deg > 0, deg, 1.0)[None, :]
    want = np.linalg.solve(np.eye(n) - M, np.full(n, 0.15 / n))
    r, it, _ = oracle.pagerank_delta(n, rp, c, None, 0.85, 0.0, 400)
    np.testing.assert_allclose(r, want, rtol=1e-12, atol=1e-15)


def test_pagerank_delta_threshold_drops_and_stops():
    # a large eps stops after the first product, which must equal one plain pull step
    rp, c = gen.rmat(8, 4, seed=13)
    n = 1 << 8
    r1, it1, _ = oracle.pagerank_delta(n, rp, c, None, 0.85, 1.0, 50)
    assert it1 == 1
    deg = np.bincount(c, minlength=n)
    x = np.where(deg > 0, (0.15 / n) / np.maximum(deg, 1), 0.0)
    y, _ = oracle.csr_pull(rp, c, np.ones(len(c)), x)
    np.testing.assert_allclose(r1, 0.15 / n + 0.85 * y, rtol=1e-14)
