"""Parity of the CUDA path against the oracle (through the C ABI).

Every candidate kernel, with x given dense or as a list and with dense or
sparse output, on small seeded inputs that span several tiles and a ragged
tail: FP64 within 1e-12 * sum|a x| per row, FP32 within 2e-6 * sum|a x|,
Boolean and int32 and every index set bit for bit."""
import numpy as np
import pytest
import torch

import gen
import oracle
from tests._util import TOL, assert_rows_close, sparse_result

pytestmark = pytest.mark.gpu

asv = pytest.importorskip("paper_2006_16767_gb300")
DEV = "cuda"
ALL_K = list(asv.KERNELS)


def to_dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def make(m, n, rowptr, col, val, **kw):
    return asv.Matrix(m, n, to_dev(rowptr), to_dev(col), to_dev(val), **kw)


# ------------------------------------------------------------------ matrices under test
def mat_laplace():
    rp, c, v = gen.laplace2d(64)
    return "laplace64", 4096, 4096, rp, c, v


def mat_random(dtype):
    rp, c, v = gen.random_csr(3001, 2503, 0.004, seed=77, values="uniform", dtype=dtype)
    return "random", 3001, 2503, rp, c, v


def mat_skewed(dtype):
    # R-MAT rows (hubs, empty rows) plus two rows longer than a balanced tile
    rp, c = gen.rmat(12, 8, seed=5)
    n = 1 << 12
    deg = np.diff(rp).astype(np.int64)
    rows = [c[rp[i]:rp[i + 1]] for i in range(n)]
    rows[7] = np.arange(0, n, 1, dtype=np.int32)
    rows[8] = np.arange(0, n, 2, dtype=np.int32)
    rp2 = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    c2 = np.concatenate(rows).astype(np.int32)
    v2 = gen.uniform(len(c2), -1, 1, seed=9, dtype=np.float64).astype(dtype)
    return "skewed", n, n, rp2, c2, v2


LONG_LENS = (0, 1, 255, 256, 257, 300, 1023, 1024, 1025, 2049, 4096, 4097, 8192, 8193, 12289, 20000)


def long_rows_pattern(n=20000, short=700, seed=31):
    """Rows of every length class of the long-row split (at and around 256,
    one segment, exactly 4096, several segments, a full row) between short
    random rows."""
    rows = []
    for t, L in enumerate(LONG_LENS):
        rows.append(gen.sample_positions(n, L, seed=seed, stream=100 + t))
        for q in range(short // len(LONG_LENS)):
            rows.append(gen.sample_positions(n, q % 9, seed=seed, stream=1000 + 97 * t + q))
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    return len(rows), n, rp, np.concatenate(rows).astype(np.int32)


def mat_long(dtype):
    m, n, rp, c = long_rows_pattern()
    v = gen.uniform(len(c), -1, 1, seed=13, dtype=np.float64).astype(dtype)
    return "long_rows", m, n, rp, c, v


def x_cases(n, seed, dtype=np.float64):
    out = []
    for rho in (1.0, 0.1, 0.01, 0.001):
        k = max(1, int(round(rho * n)))
        idx, val = gen.sparse_x(n, k, seed=seed, stream=int(rho * 1000), dtype=np.float64)
        out.append((rho, idx, val.astype(dtype)))
    return out


def run(A, k, idx, val, n, dtype, dense_in, sparse_out):
    it, vt = to_dev(idx), to_dev(val)
    if dense_in:
        xd = to_dev(gen.densify(n, idx, val, dtype))
        return A.spmspv(x_dense=xd, kernel=k, sparse_out=sparse_out)
    return A.spmspv(xidx=it, xval=vt, kernel=k, sparse_out=sparse_out)


def check(A, k, name, n, rp, c, v, idx, val, dtype, tag, dense_in, sparse_out):
    vv = None if v is None else v.astype(np.float64)
    xv = val.astype(np.float64)
    if dense_in:
        # a dense x's nonzeros are its IEEE nonzeros
        nzm = xv != 0
        idx, xv = idx[nzm], xv[nzm]
    y_ref, s, hit = oracle.spmspv_rowmajor(n, rp, c, vv, idx, xv)
    out = run(A, k, idx, xv.astype(dtype), n, dtype, dense_in, sparse_out)
    what = f"{name} {tag} k={k} dense_in={dense_in} sparse_out={sparse_out}"
    if sparse_out:
        yidx, yval, nnz_y = out
        cnt = int(nnz_y.item())
        got_idx = yidx[:cnt].cpu().numpy()
        assert np.array_equal(got_idx, np.flatnonzero(hit)), what + " (structural set)"
        assert_rows_close(yval[:cnt].cpu().numpy(), y_ref[got_idx], s[got_idx], tag, what)
    else:
        assert_rows_close(out.cpu().numpy(), y_ref, s, tag, what)


@pytest.mark.parametrize("k", ["auto"] + ALL_K)
def test_laplace_f64_all_kernels(k):
    name, m, n, rp, c, v = mat_laplace()
    A = make(m, n, rp, c, v)
    for rho, idx, val in x_cases(n, gen.config_seed(1)):
        for dense_in in (True, False):
            for sparse_out in (False, True):
                check(A, k, name, n, rp, c, v, idx, val, np.float64, "f64", dense_in, sparse_out)


@pytest.mark.parametrize("k", ["auto"] + ALL_K)
@pytest.mark.parametrize("dtype,tag", [(np.float32, "f32"), (np.float64, "f64")])
def test_random_and_skewed_all_kernels(k, dtype, tag):
    for maker in (mat_random, mat_skewed, mat_long):
        name, m, n, rp, c, v = maker(dtype)
        A = make(m, n, rp, c, v)
        for rho, idx, val in x_cases(n, 123, dtype):
            for dense_in in (True, False):
                for sparse_out in (False, True):
                    check(A, k, name, n, rp, c, v, idx, val, dtype, tag, dense_in, sparse_out)


@pytest.mark.parametrize("k", ["auto"] + ALL_K)
def test_boolean_bit_exact(k):
    rp, c = gen.rmat(12, 8, seed=3)
    n = 1 << 12
    A = make(n, n, rp, c, None)
    for rho in (0.5, 0.05, 0.002):
        idx = gen.sample_positions(n, max(1, int(rho * n)), seed=11, stream=int(rho * 1000))
        xb = np.zeros(n, np.uint8)
        xb[idx] = 1
        want = oracle.bool_pull(rp, c, xb)
        y1 = A.spmspv(x_dense=to_dev(xb), kernel=k).cpu().numpy()
        assert np.array_equal(y1 != 0, want != 0), f"bool dense-in k={k} rho={rho}"
        y2 = A.spmspv(xidx=to_dev(idx), kernel=k).cpu().numpy()
        assert np.array_equal(y2 != 0, want != 0), f"bool list-in k={k} rho={rho}"
        yidx, yval, nnz_y = A.spmspv(xidx=to_dev(idx), kernel=k, sparse_out=True)
        cnt = int(nnz_y.item())
        assert np.array_equal(yidx[:cnt].cpu().numpy(), np.flatnonzero(want)), f"bool sparse-out k={k}"


@pytest.mark.parametrize("k", ["auto"] + ALL_K)
def test_long_rows_boolean_and_int32_bit_exact(k):
    m, n, rp, c = long_rows_pattern()
    A = make(m, n, rp, c, None)
    # x with no column of the long rows (every long row is walked to its end,
    # as for a BFS frontier past the hubs), then a dense-ish one (early exits)
    longc = np.unique(np.concatenate([c[rp[i]:rp[i + 1]] for i in range(m) if rp[i + 1] - rp[i] > 256]))
    free = np.setdiff1d(np.arange(n, dtype=np.int32), longc)
    for idx in (free[gen.sample_positions(len(free), min(len(free), 40), seed=5)],
                gen.sample_positions(n, n // 3, seed=6)):
        idx = idx.astype(np.int32)
        xb = np.zeros(n, np.uint8)
        xb[idx] = 1
        want = oracle.bool_pull(rp, c, xb)
        y1 = A.spmspv(x_dense=to_dev(xb), kernel=k).cpu().numpy()
        assert np.array_equal(y1 != 0, want != 0), f"bool long rows dense-in k={k}"
        yidx, yval, nnz_y = A.spmspv(xidx=to_dev(idx), kernel=k, sparse_out=True)
        cnt = int(nnz_y.item())
        assert np.array_equal(yidx[:cnt].cpu().numpy(), np.flatnonzero(want)), f"bool long rows sparse-out k={k}"
    val = gen.uniform(len(c), -2**31, 2**31 - 1, seed=14).astype(np.int64).astype(np.int32)
    x = gen.uniform(n, -2**31, 2**31 - 1, seed=15).astype(np.int64).astype(np.int32)
    x[gen.sample_positions(n, n // 2, seed=16)] = 0
    Ai = make(m, n, rp, c, val)
    want = oracle.i32_pull(rp, c, val, x)
    assert np.array_equal(Ai.spmspv(x_dense=to_dev(x), kernel=k).cpu().numpy(), want), f"int32 long rows k={k}"


def long_columns_pattern():
    """The transpose of long_rows_pattern: columns of every length class of the
    hub-column queue of the thread and warp push (over 64, over 4096, several
    segments)."""
    m0, n0, rp, c = long_rows_pattern()
    colptr, rowidx, _ = oracle.csr_to_csc(m0, n0, rp, c)
    return n0, m0, colptr.astype(np.int32), rowidx.astype(np.int32)


@pytest.mark.parametrize("k", ["auto"] + ALL_K)
def test_long_columns_all_kernels(k):
    m, n, rp, c = long_columns_pattern()
    deg = np.bincount(c, minlength=n)
    hubs = np.flatnonzero(deg > 64).astype(np.int32)
    v = gen.uniform(len(c), -1, 1, seed=17, dtype=np.float64).astype(np.float32)
    A = make(m, n, rp, c, v)
    Ab = make(m, n, rp, c, None)
    # the hub columns, every column in order and in a seeded shuffled order
    # (a list of every column takes the feature pass's shortcut: no gathers),
    # and a fifth of the columns
    every_shuffled = np.argsort(gen.uniform(n, 0, 1, seed=20)).astype(np.int32)
    # Each as a list and as a dense x (the warp push reads a dense x of this
    # size from its bitmap, hub columns queued by column id).
    for idx in (hubs, np.arange(n, dtype=np.int32), every_shuffled, gen.sample_positions(n, n // 5, seed=18)):
        xv = gen.uniform(len(idx), -1, 1, seed=19, dtype=np.float64)
        for dense_in in (False, True):
            for sparse_out in (False, True):
                check(A, k, "long_columns", n, rp, c, v, idx, xv, np.float32, "f32", dense_in, sparse_out)
        xb = np.zeros(n, np.uint8)
        xb[idx] = 1
        want = oracle.bool_pull(rp, c, xb)
        y = Ab.spmspv(xidx=to_dev(idx), kernel=k).cpu().numpy()
        assert np.array_equal(y != 0, want != 0), f"bool long columns k={k}"
        y = Ab.spmspv(x_dense=to_dev(xb), kernel=k).cpu().numpy()
        assert np.array_equal(y != 0, want != 0), f"bool long columns dense x k={k}"


@pytest.mark.parametrize("k", ["auto"] + ALL_K)
def test_int32_wraparound_bit_exact(k):
    rp, c, _ = gen.random_csr(1500, 1200, 0.01, seed=8)
    val = gen.uniform(len(c), -2**31, 2**31 - 1, seed=1).astype(np.int64).astype(np.int32)
    x = gen.uniform(1200, -2**31, 2**31 - 1, seed=2).astype(np.int64).astype(np.int32)
    x[gen.sample_positions(1200, 900, seed=3)] = 0
    want = oracle.i32_pull(rp, c, val, x)
    A = make(1500, 1200, rp, c, val)
    got = A.spmspv(x_dense=to_dev(x), kernel=k).cpu().numpy()
    assert np.array_equal(got, want), f"int32 k={k}"
    idx = np.flatnonzero(x).astype(np.int32)
    got2 = A.spmspv(xidx=to_dev(idx), xval=to_dev(x[idx]), kernel=k).cpu().numpy()
    assert np.array_equal(got2, want), f"int32 list k={k}"


def test_transpose_bit_exact():
    for (m, n, seed) in [(5000, 3000, 1), (3000, 5000, 2), (1, 700, 3), (700, 1, 4)]:
        rp, c, v = gen.random_csr(m, n, 0.01, seed=seed, values="uniform", dtype=np.float32)
        A = make(m, n, rp, c, v)
        colptr, rowidx, valc, perm = A.csc()
        cp_ref, ri_ref, pm_ref = oracle.csr_to_csc(m, n, rp, c)
        assert np.array_equal(colptr.cpu().numpy(), cp_ref)
        assert np.array_equal(rowidx.cpu().numpy(), ri_ref)
        assert np.array_equal(perm.cpu().numpy(), pm_ref)
        assert np.array_equal(valc.cpu().numpy(), v[pm_ref])


def test_matrix_features_match_oracle():
    for name, m, n, rp, c, v in (mat_laplace(), mat_random(np.float32), mat_skewed(np.float32)):
        A = make(m, n, rp, c, v)
        got = A.features()
        want = oracle.matrix_features(m, n, rp)
        for key in ("m", "n", "nnz", "max_row", "min_row"):
            assert got[key] == want[key], (name, key)
        for key in ("avg_row", "relative_range", "var_nnz_row", "gini"):
            assert abs(got[key] - want[key]) <= 1e-12 * max(1.0, abs(want[key])), (name, key, got[key], want[key])


def test_vector_features_and_selection():
    name, m, n, rp, c, v = mat_skewed(np.float32)
    A = make(m, n, rp, c, v)
    colptr, _, _ = oracle.csr_to_csc(m, n, rp, c)
    for rho, idx, val in x_cases(n, 5, np.float32):
        kid, f = A.select(xidx=to_dev(idx), xval=to_dev(val))
        want = oracle.vector_features(n, len(c), colptr, idx)
        assert f["nnz_x"] == want["nnz_x"] and f["nnz_s"] == want["nnz_s"]
        assert f["x_sparsity"] == want["x_sparsity"] and abs(f["m_sparsity"] - want["m_sparsity"]) <= 1e-15
        assert 0 <= kid < asv.ASV_K_COUNT
        xd = to_dev(gen.densify(n, idx, val))
        kid2, f2 = A.select(x_dense=xd)
        nzi = idx[val != 0]
        want2 = oracle.vector_features(n, len(c), colptr, nzi)
        assert f2["nnz_x"] == want2["nnz_x"] and f2["nnz_s"] == want2["nnz_s"]
        # the auto call runs the kernel the selector names for its call
        # format (the trees differ between a dense and a list output)
        A.spmspv(xidx=to_dev(idx), xval=to_dev(val))
        assert A.last_kernel() == kid
        kid3, f3 = A.select(xidx=to_dev(idx), xval=to_dev(val), sparse_out=True)
        assert f3 == f
        A.spmspv(xidx=to_dev(idx), xval=to_dev(val), sparse_out=True)
        assert A.last_kernel() == kid3


def test_compaction_ieee_bit_exact():
    n = 70001
    x = gen.uniform(n, -1, 1, seed=4)
    x[gen.sample_positions(n, 60000, seed=5)] = 0.0
    x[10] = -0.0
    x[11] = np.nan
    x[12] = np.inf
    x[13] = 5e-324
    rp, c, v = gen.random_csr(10, n, 0.001, seed=1, values="uniform")
    A = make(10, n, rp, c, v)
    idx = torch.empty(n, dtype=torch.int32, device=DEV)
    val = torch.empty(n, dtype=torch.float64, device=DEV)
    cnt = torch.zeros(1, dtype=torch.int64, device=DEV)
    asv.asv_compact(A.handle, to_dev(x), idx, val, cnt)
    k = int(cnt.item())
    ref_idx, ref_val = oracle.compact(x)
    assert np.array_equal(idx[:k].cpu().numpy(), ref_idx)
    assert np.array_equal(val[:k].cpu().numpy(), ref_val, equal_nan=True)


def test_edge_cases():
    # empty x (list of length 0), all-zero dense x, empty matrix, single row/column
    name, m, n, rp, c, v = mat_random(np.float64)
    A = make(m, n, rp, c, v)
    for k in ["auto"] + ALL_K:
        y = A.spmspv(xidx=torch.zeros(0, dtype=torch.int32, device=DEV),
                     xval=torch.zeros(0, dtype=torch.float64, device=DEV), kernel=k)
        assert torch.count_nonzero(y).item() == 0, k
        y = A.spmspv(x_dense=torch.zeros(n, dtype=torch.float64, device=DEV), kernel=k)
        assert torch.count_nonzero(y).item() == 0, k
        yidx, yval, nnz_y = A.spmspv(xidx=torch.zeros(0, dtype=torch.int32, device=DEV),
                                     xval=torch.zeros(0, dtype=torch.float64, device=DEV), kernel=k,
                                     sparse_out=True)
        assert int(nnz_y.item()) == 0, k
    E = make(50, 40, np.zeros(51, np.int32), np.zeros(0, np.int32), np.zeros(0, np.float64))
    for k in ["auto"] + ALL_K:
        y = E.spmspv(x_dense=torch.ones(40, dtype=torch.float64, device=DEV), kernel=k)
        assert torch.count_nonzero(y).item() == 0, k
    for (mm, nn) in [(1, 900), (900, 1)]:
        rp, c, v = gen.random_csr(mm, nn, 0.5, seed=2, values="uniform")
        B = make(mm, nn, rp, c, v)
        x = gen.uniform(nn, -1, 1, seed=3)
        y_ref, s = oracle.csr_pull(rp, c, v, x)
        for k in ["auto"] + ALL_K:
            assert_rows_close(B.spmspv(x_dense=to_dev(x), kernel=k).cpu().numpy(), y_ref, s, "f64", f"{mm}x{nn} {k}")


def test_sparse_output_capacity_is_reported():
    name, m, n, rp, c, v = mat_random(np.float64)
    A = make(m, n, rp, c, v)
    x = torch.ones(n, dtype=torch.float64, device=DEV)
    _, s, hit = oracle.spmspv_rowmajor(n, rp, c, v, np.arange(n, dtype=np.int32), np.ones(n))
    assert A.status() == 0
    for k in ("pull_bal", "push_bal_atom", "push_thread_sort"):
        yidx, yval, nnz_y = A.spmspv(x_dense=x, kernel=k, sparse_out=True, y_cap=10)
        assert int(nnz_y.item()) == int(hit.sum())
        assert A.status() == asv.ASV_ERR_CAPACITY
        assert A.status() == 0


def test_validation_rejects_noncanonical():
    rp = np.array([0, 2, 3], np.int32)
    c = np.array([1, 0, 2], np.int32)  # row 0 not ascending
    with pytest.raises(asv.AsvError) as e:
        make(2, 3, rp, c, np.ones(3), validate=True)
    assert e.value.status == asv.ASV_ERR_NONCANONICAL
    c_ok = np.array([0, 1, 2], np.int32)
    make(2, 3, rp, c_ok, np.ones(3), validate=True).close()
    c_bad = np.array([0, 1, 3], np.int32)  # out of range
    with pytest.raises(asv.AsvError):
        make(2, 3, rp, c_bad, np.ones(3), validate=True)


def test_spmv_entry_point_and_copy_flag():
    name, m, n, rp, c, v = mat_skewed(np.float32)
    vt = to_dev(v)
    A = asv.Matrix(m, n, to_dev(rp), to_dev(c), vt, copy=True)
    vt.zero_()  # the handle owns its copy
    x = gen.uniform(n, -1, 1, seed=6).astype(np.float32)
    y_ref, s = oracle.csr_pull(rp, c, v.astype(np.float64), x.astype(np.float64))
    for k in ["auto"] + ALL_K:
        y = A.spmv(to_dev(x), kernel=k)
        assert_rows_close(y.cpu().numpy(), y_ref, s, "f32", f"spmv {k}")


def test_set_trees_drives_the_switch_branch():
    name, m, n, rp, c, v = mat_random(np.float32)
    A = make(m, n, rp, c, v)
    x = gen.uniform(n, -1, 1, seed=12).astype(np.float32)
    y_ref, s = oracle.csr_pull(rp, c, v.astype(np.float64), x.astype(np.float64))
    for pat, dist, wb in [(0, 2, 1), (1, 0, 0), (2, 1, 0), (0, 0, 2), (0, 1, 0)]:
        nodes = [(-1, 0, 0, 0, pat), (-1, 0, 0, 0, dist), (-1, 0, 0, 0, wb)]
        A.set_trees(nodes, [0, 1, 1, 1, 2] * 4)
        want = {2: dist, 1: 3 + dist, 0: 6 + 3 * wb + dist}[pat]
        for dense_in in (True, False):
            if dense_in:
                y = A.spmspv(x_dense=to_dev(x))
            else:
                idx = np.flatnonzero(x).astype(np.int32)
                y = A.spmspv(xidx=to_dev(idx), xval=to_dev(x[idx]))
            assert A.last_kernel() == want
            assert_rows_close(y.cpu().numpy(), y_ref, s, "f32", f"trees -> {asv.KERNELS[want]}")
        kid, _ = A.select(x_dense=to_dev(x))
        assert kid == want
    with pytest.raises(asv.AsvError):
        A.set_trees([(0, 1.0, 5, 6, 0)], [0] * 20)  # child index out of range


def test_lazy_feature_evaluation_for_listed_x():
    # trees whose list-format pattern root splits on x_sparsity (a free
    # feature of a listed x): below the threshold the decision needs
    # m_sparsity (full feature pass), above it the pull / masked pull / warp
    # push named by the leaves is decided without the pass. Every call must
    # give the oracle's result and run the kernel the full walk (asv_select)
    # names; the structural output set must match too.
    name, m, n, rp, c, v = mat_skewed(np.float32)
    A = make(m, n, rp, c, v)
    for hi_pat, hi_dist, lo_pat in [(2, 1, 0), (1, 0, 2), (0, 1, 1), (0, 2, 2)]:
        # 0: x_sparsity <= 0.05 ? node 1 : leaf hi_pat; 1: m_sparsity <= 0.5 ? leaf lo_pat : leaf 0
        nodes = [(10, 0.05, 1, 2, 0), (12, 0.5, 3, 4, 0), (-1, 0, 0, 0, hi_pat), (-1, 0, 0, 0, lo_pat),
                 (-1, 0, 0, 0, 0), (-1, 0, 0, 0, hi_dist), (-1, 0, 0, 0, 0)]
        A.set_trees(nodes, [0, 5, 5, 5, 6] * 4)
        for rho in (0.01, 0.2):
            k = int(rho * n)
            idx, val = gen.sparse_x(n, k, 33, 11, np.float32)
            y_ref, s, hit = oracle.spmspv_rowmajor(n, rp, c, v.astype(np.float64), idx, val.astype(np.float64))
            kid_d, _ = A.select(xidx=to_dev(idx), xval=to_dev(val))
            y = A.spmspv(xidx=to_dev(idx), xval=to_dev(val))
            assert A.last_kernel() == kid_d
            assert_rows_close(y.cpu().numpy(), y_ref, s, "f32", f"lazy {asv.KERNELS[kid_d]} rho={rho}")
            kid_s, _ = A.select(xidx=to_dev(idx), xval=to_dev(val), sparse_out=True)
            yi, yv, ny = A.spmspv(xidx=to_dev(idx), xval=to_dev(val), sparse_out=True)
            assert A.last_kernel() == kid_s
            got_idx, got_val = sparse_result(yi, yv, ny)
            assert np.array_equal(got_idx, np.flatnonzero(hit))
            assert_rows_close(got_val, y_ref[got_idx], s[got_idx], "f32", f"lazy list out rho={rho}")
            assert A.status() == asv.ASV_OK


def test_single_call_autotuner_keeps_results_and_caches(tmp_path):
    # the tuner changes only the pull kernels' launch shape: every setting it
    # keeps must give the oracle's result, and a cached setting is reused
    for dt in (np.float32, np.float64):
        name, m, n, rp, c, v = mat_skewed(dt)
        A = make(m, n, rp, c, v)
        cache = tmp_path / "pull.tsv"
        t1 = A.autotune(cache_path=cache, budget_ms=3000)
        assert t1[0] in (2, 4, 8, 16, 32) and t1[1] in (2, 4) and t1[2] in (0, 1)
        assert A.pull_tuning() == t1
        lines = cache.read_text().strip().splitlines()
        assert len(lines) >= 1 and lines[-1].endswith("\t".join(str(q) for q in t1))
        B = make(m, n, rp, c, v)
        assert B.autotune(cache_path=cache, budget_ms=0) == t1 and B.pull_tuning() == t1
        assert len(cache.read_text().strip().splitlines()) == len(lines)  # read, not appended
        x = gen.uniform(n, -1, 1, 91).astype(dt)
        y_ref, s = oracle.csr_pull(rp, c, v.astype(np.float64), x.astype(np.float64))
        for k in ("pull_thread", "pull_warp", "auto"):
            y = A.spmv(to_dev(x), kernel=k).cpu().numpy()
            assert_rows_close(y, y_ref, s, "f32" if dt == np.float32 else "f64", f"tuned {k}")
        # a zero budget still returns a valid setting (the creation-time one)
        assert make(m, n, rp, c, v).autotune(budget_ms=0)[0] in (2, 4, 8, 16, 32)


def short_rows_pattern(m, n, row_len, seed):
    """Every row holds exactly row_len entries at random columns."""
    rows = [gen.sample_positions(n, row_len, seed=seed, stream=i) for i in range(m)]
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    return rp, np.concatenate(rows).astype(np.int32)


@pytest.mark.parametrize("row_len", [32, 33])
@pytest.mark.parametrize("k", ["push_thread_atom", "push_warp_atom", "push_bal_atom", "pull_thread", "mpull_thread",
                               "auto"])
def test_fp32_push_accumulation_stays_in_tolerance(row_len, k):
    # rows of 32 entries: the FP32 atomic push adds in FP32 and the thread
    # pull sums each row with a plain FMA chain (32 products, each rounded
    # once, in any order stay within 32 * 2^-24 < 2e-6 of sum |a x|); 33
    # entries keep FP64 accumulators and the compensated sum. Values spread
    # over six decades with both signs, so the sums cancel and rounding is at
    # its worst relative to the scale.
    m, n = 3000, 2048
    rp, c = short_rows_pattern(m, n, row_len, seed=41)
    mag = 10.0 ** gen.uniform(len(c), -3, 3, seed=42, dtype=np.float64)
    sign = np.where(gen.uniform(len(c), 0, 1, seed=43, dtype=np.float64) < 0.5, -1.0, 1.0)
    v = (mag * sign).astype(np.float32)
    A = make(m, n, rp, c, v)
    for rho, idx, val in x_cases(n, seed=44, dtype=np.float32):
        for dense_in in (False, True):
            for sparse_out in (False, True):
                check(A, k, f"rows{row_len}", n, rp, c, v, idx, val, np.float32, "f32", dense_in, sparse_out)
