"""The transposed view A^T (asv_matrix_transpose_view) against the oracle.

The view borrows A's CSC as its CSR and A's CSR as its CSC, so every
candidate kernel run on it computes y = A^T x. The expected values come from
the oracle's own transpose (stable counting sort) and its row-major product
on the transposed CSR; the oracle's column-major push over A's CSR (read as
the CSC of A^T, no transpose built) cross-checks that route. FP64 within
1e-12 * sum|a x| per row, FP32 within 2e-6, Boolean and index sets bit for
bit, matrix features as the oracle's over A^T's row lengths."""
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


def transposed(m, n, rp, c, v):
    """A^T in CSR from the oracle: (colptr, rowidx, values in A^T's CSR order)."""
    colptr, rowidx, perm = oracle.csr_to_csc(m, n, rp, c)
    return colptr, rowidx, (None if v is None else v[perm]), perm


def skewed_rect():
    """A rectangular matrix with hub rows and hub columns: in the view the
    hub columns become rows longer than a long-row segment and the hub rows
    become long columns of the push kernels."""
    m, n = 5000, 9000
    rows = [gen.sample_positions(n, (i * 7) % 13, seed=41, stream=i) for i in range(m)]
    rows[5] = np.arange(0, n, 1, dtype=np.int32)            # a full row: a long column of A^T
    rows[6] = np.arange(0, n, 3, dtype=np.int32)
    for i in range(m):                                       # column 17 in every row: a row of
        rows[i] = np.union1d(rows[i], [17]).astype(np.int32)  # A^T over two long-row segments
    for i in range(0, m, 3):                                 # column 18 in every third row
        rows[i] = np.union1d(rows[i], [18]).astype(np.int32)  # (one segment)
    rp = np.concatenate([[0], np.cumsum([len(r) for r in rows])]).astype(np.int32)
    return m, n, rp, np.concatenate(rows).astype(np.int32)


@pytest.mark.parametrize("k", ["auto"] + ALL_K)
@pytest.mark.parametrize("dtype,tag", [(np.float64, "f64"), (np.float32, "f32")])
def test_view_products_all_kernels(k, dtype, tag):
    m, n, rp, c = skewed_rect()
    v = gen.uniform(len(c), -1, 1, seed=43, dtype=np.float64).astype(dtype)
    A = asv.Matrix(m, n, to_dev(rp), to_dev(c), to_dev(v))
    At = A.transpose_view()
    assert (At.m, At.n, At.nnz) == (n, m, A.nnz)
    tp, tc, tv, _ = transposed(m, n, rp, c, v.astype(np.float64))
    for rho in (1.0, 0.05, 0.002):
        kx = max(1, int(round(rho * m)))
        idx, xv = gen.sparse_x(m, kx, seed=44, stream=int(rho * 1000), dtype=np.float64)
        xv = xv.astype(dtype).astype(np.float64)  # the values the kernels see, widened exactly
        y_ref, s, hit = oracle.spmspv_rowmajor(m, tp, tc, tv, idx, xv)
        # A's CSR read as the CSC of A^T: the oracle's column-major push over
        # it gives A^T x without the oracle's transpose
        y_alt, touched = oracle.csc_push(n, rp, c, v.astype(np.float64), idx, xv)
        assert_rows_close(y_alt, y_ref, s, "f64", "oracle routes disagree")
        assert np.array_equal(touched != 0, hit != 0)
        xd = to_dev(gen.densify(m, idx, xv.astype(dtype), dtype))
        y = At.spmspv(x_dense=xd, kernel=k).cpu().numpy()
        assert_rows_close(y, y_ref, s, tag, f"A^T x dense k={k} rho={rho}")
        yidx, yval, nnz_y = At.spmspv(xidx=to_dev(idx), xval=to_dev(xv.astype(dtype)), kernel=k, sparse_out=True)
        cnt = int(nnz_y.item())
        got = yidx[:cnt].cpu().numpy()
        assert np.array_equal(got, np.flatnonzero(hit)), f"A^T x structural set k={k} rho={rho}"
        assert_rows_close(yval[:cnt].cpu().numpy(), y_ref[got], s[got], tag, f"A^T x sparse k={k}")
    del At
    A.close()


@pytest.mark.parametrize("k", ["auto"] + ALL_K)
def test_view_boolean_bit_exact(k):
    rp, c = gen.rmat(12, 8, seed=21)
    n = 1 << 12
    # drop the lower triangle so that A is not symmetric and A^T differs from A
    keep = np.concatenate([c[rp[i]:rp[i + 1]] >= i for i in range(n)])
    rows = np.repeat(np.arange(n), np.diff(rp))[keep]
    c2 = c[keep].astype(np.int32)
    rp2 = np.concatenate([[0], np.cumsum(np.bincount(rows, minlength=n))]).astype(np.int32)
    A = asv.Matrix(n, n, to_dev(rp2), to_dev(c2), None)
    At = A.transpose_view()
    tp, tc, _, _ = transposed(n, n, rp2, c2, None)
    for rho in (0.3, 0.01):
        idx = gen.sample_positions(n, max(1, int(rho * n)), seed=22, stream=int(rho * 1000))
        xb = np.zeros(n, np.uint8)
        xb[idx] = 1
        want = oracle.bool_pull(tp, tc, xb)
        y = At.spmspv(x_dense=to_dev(xb), kernel=k).cpu().numpy()
        assert np.array_equal(y != 0, want != 0), f"bool A^T x k={k} rho={rho}"
        yidx, _, nnz_y = At.spmspv(xidx=to_dev(idx), kernel=k, sparse_out=True)
        cnt = int(nnz_y.item())
        assert np.array_equal(yidx[:cnt].cpu().numpy(), np.flatnonzero(want)), f"bool A^T sparse k={k}"
    del At
    A.close()


def test_view_arrays_features_lifetime_and_values():
    m, n, rp, c = skewed_rect()
    v = gen.uniform(len(c), -1, 1, seed=45, dtype=np.float64)
    A = asv.Matrix(m, n, to_dev(rp), to_dev(c), to_dev(v))
    At = A.transpose_view()
    # the view's CSC is A's CSR; its CSC -> CSR map is the inverse of A's
    _, _, _, permA = A.csc()
    colptr, rowidx, valc, perm = At.csc()
    assert np.array_equal(colptr.cpu().numpy(), rp)
    assert np.array_equal(rowidx.cpu().numpy(), c)
    assert np.array_equal(valc.cpu().numpy(), v)
    assert np.array_equal(perm.cpu().numpy()[permA.cpu().numpy()], np.arange(A.nnz))
    # Table 1 features over A^T's rows (A's columns)
    tp, _, _, _ = transposed(m, n, rp, c, v)
    want = oracle.matrix_features(n, m, tp)
    got = At.features()
    for key, w in want.items():
        assert got[key] == pytest.approx(w, rel=1e-12, abs=0), key
    # A stays alive while its view exists; values are updated through A only
    with pytest.raises(asv.AsvError):
        A.close()
    with pytest.raises(asv.AsvError):
        At.update_values()
    v2 = gen.uniform(len(c), -1, 1, seed=46, dtype=np.float64)
    A.val.copy_(to_dev(v2))
    A.update_values()
    x = gen.uniform(m, -1, 1, seed=47, dtype=np.float64)
    y = At.spmv(to_dev(x)).cpu().numpy()
    tp2, tc2, tv2, _ = transposed(m, n, rp, c, v2)
    y_ref, s = oracle.csr_pull(tp2, tc2, tv2, x)
    assert_rows_close(y, y_ref, s, "f64", "A^T x after a value update of A")
    # the view of the view multiplies by A again
    Att = At.transpose_view()
    xn = gen.uniform(n, -1, 1, seed=48, dtype=np.float64)
    y2 = Att.spmv(to_dev(xn)).cpu().numpy()
    y2_ref, s2 = oracle.csr_pull(rp, c, v2, xn)
    assert_rows_close(y2, y2_ref, s2, "f64", "(A^T)^T x")
    with pytest.raises(asv.AsvError):
        At.close()
    Att.close()
    At.close()
    A.close()
