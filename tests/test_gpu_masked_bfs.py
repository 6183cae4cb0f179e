"""The output-masked product and the breadth-first search built on it,
against the oracle (through the C ABI).

Masked product: y = A x with the rows whose mask bit is set excluded -- the
oracle's product with those rows zeroed and removed from the structural set
-- for every candidate, x dense or listed, y dense or sparse; FP32/FP64
within the per-row tolerances, Boolean and int32 bit for bit. BFS: the level
of every vertex equals the oracle's queue BFS, bit for bit, for the selector
and for forced candidates of each pattern, on a power-law graph, a mesh and
a graph with several components; long paths run thousands of iterations of
the device-side loop. PageRank: the delta iteration against the oracle's.
"""
import numpy as np
import pytest
import torch

import gen
import oracle
from tests._util import assert_rows_close

pytestmark = pytest.mark.gpu
asv = pytest.importorskip("paper_2006_16767_gb300")
DEV = "cuda"
ALL_K = list(asv.KERNELS)


def to_dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def mask_bits(m, rows):
    w = np.zeros((m + 31) // 32, np.uint32)
    for r in rows:
        w[r >> 5] |= np.uint32(1) << np.uint32(r & 31)
    return w.view(np.int32)


def long_and_skewed(dtype):
    # R-MAT rows plus rows across the long-row split (256) and several segments (4096)
    rp, c = gen.rmat(13, 8, seed=21)
    n = 1 << 13
    rows = [c[rp[i]:rp[i + 1]] for i in range(n)]
    for t, L in enumerate((257, 300, 4097, 8192)):
        rows[11 + t] = gen.sample_positions(n, L, seed=22, stream=t)
    rp2 = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    c2 = np.concatenate(rows).astype(np.int32)
    v2 = gen.uniform(len(c2), -1, 1, seed=23, dtype=np.float64).astype(dtype)
    return n, n, rp2, c2, v2


@pytest.mark.parametrize("k", ["auto"] + ALL_K)
@pytest.mark.parametrize("dtype,tag", [(np.float32, "f32"), (np.float64, "f64")])
def test_masked_product_all_kernels(k, dtype, tag):
    m, n, rp, c, v = long_and_skewed(dtype)
    A = asv.Matrix(m, n, to_dev(rp), to_dev(c), to_dev(v))
    masked = gen.sample_positions(m, m // 3, seed=24)
    mk = to_dev(mask_bits(m, masked))
    keep = np.ones(m, bool)
    keep[masked] = False
    for rho in (1.0, 0.05, 0.002):
        idx, val = gen.sparse_x(n, max(1, int(rho * n)), seed=25, stream=int(rho * 1000), dtype=np.float64)
        y_ref, s, hit = oracle.spmspv_rowmajor(n, rp, c, v.astype(np.float64), idx, val)
        y_ref = np.where(keep, y_ref, 0.0)
        s = np.where(keep, s, 0.0)
        want = np.flatnonzero(hit.astype(bool) & keep)
        xv = val.astype(dtype)
        for dense_in in (True, False):
            kw = dict(x_dense=to_dev(gen.densify(n, idx, xv, dtype))) if dense_in else \
                dict(xidx=to_dev(idx), xval=to_dev(xv))
            what = f"masked {tag} k={k} rho={rho} dense_in={dense_in}"
            y = A.spmspv(kernel=k, ymask=mk, **kw).cpu().numpy()
            assert_rows_close(y, y_ref, s, tag, what)
            assert np.all(y[masked] == 0), what + " (masked rows not zero)"
            yidx, yval, nnz_y = A.spmspv(kernel=k, ymask=mk, sparse_out=True, **kw)
            cnt = int(nnz_y.item())
            got = yidx[:cnt].cpu().numpy()
            assert np.array_equal(got, want), what + " (structural set)"
            assert_rows_close(yval[:cnt].cpu().numpy(), y_ref[got], s[got], tag, what)


@pytest.mark.parametrize("k", ["auto"] + ALL_K)
def test_masked_boolean_and_int32_bit_exact(k):
    m, n, rp, c, _ = long_and_skewed(np.float32)
    masked = gen.sample_positions(m, m // 2, seed=26)
    mk = to_dev(mask_bits(m, masked))
    keep = np.ones(m, bool)
    keep[masked] = False
    Ab = asv.Matrix(m, n, to_dev(rp), to_dev(c), None)
    for rho in (0.3, 0.01):
        idx = gen.sample_positions(n, max(1, int(rho * n)), seed=27, stream=int(rho * 100))
        xb = np.zeros(n, np.uint8)
        xb[idx] = 1
        want = (oracle.bool_pull(rp, c, xb) != 0) & keep
        y = Ab.spmspv(x_dense=to_dev(xb), kernel=k, ymask=mk).cpu().numpy()
        assert np.array_equal(y != 0, want), f"bool masked k={k}"
        yidx, _, nnz_y = Ab.spmspv(xidx=to_dev(idx), kernel=k, ymask=mk, sparse_out=True)
        assert np.array_equal(yidx[:int(nnz_y.item())].cpu().numpy(), np.flatnonzero(want)), f"bool masked list k={k}"
    val = gen.uniform(len(c), -2**31, 2**31 - 1, seed=28).astype(np.int64).astype(np.int32)
    x = gen.uniform(n, -2**31, 2**31 - 1, seed=29).astype(np.int64).astype(np.int32)
    x[gen.sample_positions(n, n // 2, seed=30)] = 0
    Ai = asv.Matrix(m, n, to_dev(rp), to_dev(c), to_dev(val))
    want = np.where(keep, oracle.i32_pull(rp, c, val, x), 0)
    assert np.array_equal(Ai.spmspv(x_dense=to_dev(x), kernel=k, ymask=mk).cpu().numpy(), want), f"int32 masked k={k}"


def symmetric(n, rows):
    """Pattern of rows plus its transpose, canonical (sorted, no duplicates)."""
    import scipy.sparse as sp
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])])
    c = np.concatenate(rows) if rows else np.zeros(0, np.int32)
    M = sp.csr_matrix((np.ones(len(c)), c, rp), shape=(n, n))
    M = ((M + M.T) > 0).tocsr()
    M.sort_indices()
    return M.indptr.astype(np.int32), M.indices.astype(np.int32)


def bfs_graphs():
    rp, c = gen.rmat(13, 8, seed=31)  # power law, isolated vertices, hubs
    yield "rmat13", 1 << 13, rp, c
    rp, c, _ = gen.laplace2d(48)  # high diameter (94 levels from a corner)
    yield "grid48", 48 * 48, rp, c
    # several components, one with long rows
    n = 6000
    rows = [np.zeros(0, np.int32) for _ in range(n)]
    rows[0] = gen.sample_positions(3000, 2900, seed=32)
    for i in range(3000, n - 1):
        if i % 7:
            rows[i] = np.array([i + 1], np.int32)
    rp, c = symmetric(n, rows)
    yield "components", n, rp, c


@pytest.mark.parametrize("k", ["auto", "pull_thread", "mpull_bal", "push_thread_atom", "push_warp_sort",
                               "push_bal_priv", "pull_warp"])
def test_bfs_levels_match_oracle(k):
    for name, n, rp, c in bfs_graphs():
        A = asv.Matrix(n, n, to_dev(rp), to_dev(c), None)
        deg = np.diff(rp)
        roots = [int(np.argmax(deg)), int(np.flatnonzero(deg > 0)[-1]), 0]
        for root in roots:
            want, L = oracle.bfs(n, rp, c, root)
            level, depth = A.bfs(root, kernel=k)
            got = level.cpu().numpy()
            assert np.array_equal(got, want), f"bfs {name} root={root} k={k}"
            assert depth == L, f"bfs depth {name} root={root} k={k}: {depth} vs {L}"


def test_bfs_on_a_float_handle_and_argument_errors():
    rp, c = gen.rmat(11, 8, seed=33)
    n = 1 << 11
    A = asv.Matrix(n, n, to_dev(rp), to_dev(c), to_dev(np.ones(len(c), np.float32)))
    root = int(np.argmax(np.diff(rp)))
    want, L = oracle.bfs(n, rp, c, root)
    level, depth = A.bfs(root)
    assert np.array_equal(level.cpu().numpy(), want) and depth == L
    for bad in (-1, n):
        with pytest.raises(asv.AsvError):
            A.bfs(bad)
    rp2, c2, _ = gen.random_csr(n, n // 2, 0.01, seed=1)
    R = asv.Matrix(n, n // 2, to_dev(rp2), to_dev(c2), None)
    with pytest.raises(asv.AsvError):
        R.bfs(0)


def path_graph(n, start=0):
    """Undirected path start - start+1 - ... - n-1; vertices below start isolated."""
    rows = [np.array([i + 1], np.int32) if start <= i < n - 1 else np.zeros(0, np.int32) for i in range(n)]
    return symmetric(n, rows)


@pytest.mark.parametrize("k", ["auto", "push_warp_atom", "mpull_thread", "pull_bal"])
def test_bfs_device_loop_long_paths_and_isolated_source(k):
    # a 5000-vertex path: 5000 iterations of the device-side loop, one vertex per level
    n = 5000
    rp, c = path_graph(n)
    A = asv.Matrix(n, n, to_dev(rp), to_dev(c), None)
    for root in (0, n // 2, n - 1):
        want, L = oracle.bfs(n, rp, c, root)
        level, depth = A.bfs(root, kernel=k)
        assert np.array_equal(level.cpu().numpy(), want), f"path root={root} k={k}"
        assert depth == L, f"path depth root={root} k={k}: {depth} vs {L}"
    # a source without edges: one (empty) product, every other vertex unreached
    rp, c = path_graph(64, start=1)
    A = asv.Matrix(64, 64, to_dev(rp), to_dev(c), None)
    level, depth = A.bfs(0, kernel=k)
    want = np.full(64, -1, np.int32)
    want[0] = 0
    assert np.array_equal(level.cpu().numpy(), want) and depth == 1, f"isolated source k={k}"
    level, depth = A.bfs(5, kernel=k)
    assert np.array_equal(level.cpu().numpy(), oracle.bfs(64, rp, c, 5)[0]) and depth == 59


def test_drivers_share_a_handle_and_run_without_host_scalars():
    rp, c = gen.rmat(12, 8, seed=43)
    n = 1 << 12
    A = asv.Matrix(n, n, to_dev(rp), to_dev(c), to_dev(np.ones(len(c), np.float64)))
    deg = np.diff(rp)
    r0, r1 = int(np.argmax(deg)), int(np.flatnonzero(deg > 0)[0])
    # PageRank first, then BFS on the same handle: each driver keeps its own workspaces
    want_pr, it, _ = oracle.pagerank_delta(n, rp, c, None, 0.85, 1e-9, 50)
    rank, iters = A.pagerank(0.85, 1e-9, 50)
    assert iters == it and np.max(np.abs(rank.cpu().numpy() - want_pr) / want_pr) <= 1e-11
    level, depth = A.bfs(r0)
    want0, L0 = oracle.bfs(n, rp, c, r0)
    assert np.array_equal(level.cpu().numpy(), want0) and depth == L0
    # without host scalars the calls only enqueue; results are read after a synchronisation
    lv = [torch.empty(n, dtype=torch.int32, device=DEV) for _ in range(2)]
    rk = torch.empty(n, dtype=torch.float64, device=DEV)
    assert A.bfs(r1, level=lv[0], wait=False)[1] is None
    assert A.pagerank(0.85, 1e-9, 50, rank=rk, wait=False)[1] is None
    assert A.bfs(r0, level=lv[1], kernel="push_bal_atom", wait=False)[1] is None
    torch.cuda.synchronize()
    assert np.array_equal(lv[0].cpu().numpy(), oracle.bfs(n, rp, c, r1)[0])
    assert np.array_equal(lv[1].cpu().numpy(), want0)
    assert np.max(np.abs(rk.cpu().numpy() - want_pr) / want_pr) <= 1e-11
    # one product only, and the exact series cut at 3 products
    for mi in (1, 3):
        want, it, _ = oracle.pagerank_delta(n, rp, c, None, 0.85, 0.0, mi)
        rank, iters = A.pagerank(0.85, 0.0, mi)
        assert iters == it == mi and np.max(np.abs(rank.cpu().numpy() - want) / want) <= 1e-12


@pytest.mark.parametrize("k", ["auto", "pull_warp", "push_bal_atom", "push_thread_sort", "mpull_thread"])
def test_incremental_pagerank_fp64_matches_oracle(k):
    rp, c = gen.rmat(12, 8, seed=41)
    n = 1 << 12
    A = asv.Matrix(n, n, to_dev(rp), to_dev(c), to_dev(np.ones(len(c), np.float64)))
    for eps in (0.0, 1e-9):
        want, it, margin = oracle.pagerank_delta(n, rp, c, None, 0.85, eps, 60)
        assert margin > 1e-6, "a keep/drop decision of the oracle run sits on the threshold"
        rank, iters = A.pagerank(0.85, eps, 60, kernel=k)
        got = rank.cpu().numpy()
        assert iters == it, f"pagerank k={k} eps={eps}: {iters} products vs {it}"
        assert np.max(np.abs(got - want) / want) <= 1e-11, f"pagerank k={k} eps={eps}"


@pytest.mark.parametrize("k", ["auto", "pull_warp", "push_bal_atom"])
def test_incremental_pagerank_fp32_matches_oracle(k):
    # Every value of the iteration is nonnegative (A's entries, the deltas,
    # the column scaling), so sum |a x| of a product row equals the row's
    # value and the FP32 product bound 2e-6 * sum |a x| is a relative bound.
    # A delta after k products then carries a relative error of at most
    # k (2e-6 + 3u) (the product, the division by the column count, the
    # scaling by the damping; u = 2^-24), and so does each vertex's rank,
    # which adds them up in FP32 (one more u per product). The threshold is
    # one where every keep/drop decision of the oracle's run lies at least
    # 1.9e-3 (relative) away from eps -- far beyond that error -- so both
    # runs keep the same entries and run the same number of products.
    rp, c = gen.rmat(10, 8, seed=42)
    n = 1 << 10
    eps = 1.8112434987143081e-06
    A = asv.Matrix(n, n, to_dev(rp), to_dev(c), to_dev(np.ones(len(c), np.float32)))
    want, it, margin = oracle.pagerank_delta(n, rp, c, None, 0.85, eps, 100)
    tol = it * (2e-6 + 4 * 2.0 ** -24)
    assert it < 100 and margin > 10 * tol
    rank, iters = A.pagerank(0.85, eps, 100, kernel=k)
    got = rank.cpu().numpy().astype(np.float64)
    assert iters == it, f"pagerank k={k}: {iters} products vs {it}"
    rel = np.abs(got - want) / want
    assert np.all(rel <= tol), f"pagerank k={k}: max relative error {rel.max():.3g} > {tol:.3g}"


def test_incremental_pagerank_fp32_arguments():
    rp, c = gen.rmat(12, 8, seed=42)
    n = 1 << 12
    A = asv.Matrix(n, n, to_dev(rp), to_dev(c), to_dev(np.ones(len(c), np.float32)))
    r0, i0 = A.pagerank(0.85, 1e-8, 0)
    assert i0 == 0 and np.allclose(r0.cpu().numpy(), 0.15 / n)
    for bad in (dict(damping=1.0), dict(damping=-0.1), dict(eps=-1.0), dict(max_iter=-1)):
        kw = dict(damping=0.85, eps=1e-8, max_iter=5)
        kw.update(bad)
        with pytest.raises(asv.AsvError):
            A.pagerank(**kw)
    Ab = asv.Matrix(n, n, to_dev(rp), to_dev(c), None)
    with pytest.raises(asv.AsvError):
        Ab.pagerank()
