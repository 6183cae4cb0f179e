"""Lists that name every column, against the oracle through the C ABI.

A listed x of n entries is every column. When it is also in order
(xidx[t] = t, as an ascending list of every column is), the feature pass
marks it and the pull kernels read the list's values in place: the scatter
into the dense workspace is replaced by setting the bitmap, and the clear
afterwards by clearing it. These cases check that path and its neighbours:
the in-order list with structural zeros among its values, the same columns
in another order (the ordinary scatter), the in-order list without values
(all ones), and a partial list right after, which would read whatever the
in-order call left in the workspaces. On a matrix without empty rows, a
list of every column reaches every row, so an unmasked list output is every
row in order: the pull kernels then write its values in place and the
compaction only writes the indices. Every pull candidate and the selector,
dense and list output, with and without an output mask; FP32 and FP64 within
the per-row tolerances, int32 bit for bit. The matrices have empty rows (the
R-MAT graph), no empty row (the rectangular one), rows long enough for the
long-row pass, and a column count that leaves the bitmap's last word partly
used.
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
PULLS = ["pull_thread", "pull_warp", "pull_bal", "mpull_thread", "mpull_warp", "mpull_bal", "auto"]


def to_dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def mask_bits(m, rows):
    w = np.zeros((m + 31) // 32, np.uint32)
    np.bitwise_or.at(w, rows >> 5, (np.uint32(1) << (rows & 31).astype(np.uint32)))
    return w.view(np.int32)


def matrices(dtype):
    """R-MAT scale 12 (isolated vertices give empty rows, hubs give rows over
    the long-row threshold) and a rectangular Bernoulli matrix of 5,003
    columns (the bitmap's last word holds 11 columns)."""
    rp, c = gen.rmat(12, 16, seed=71)
    n = 1 << 12
    v = gen.uniform(len(c), -1, 1, 72, 0, np.float64).astype(dtype)
    yield "rmat12", rp, c, v, n
    rp2, c2, _ = gen.bernoulli(3001, 5003, 0.004, 1.0, 73)
    v2 = gen.uniform(len(c2), -1, 1, 74, 0, np.float64).astype(dtype)
    yield "bernoulli3001x5003", rp2, c2, v2, 5003


def full_lists(n, dtype, seed):
    """(label, idx, val) for the in-order list with exact zeros among its
    values, every column in another order, the in-order list without values,
    and a partial ascending list."""
    val = gen.uniform(n, -1, 1, seed, 0, np.float64).astype(dtype)
    val[gen.sample_positions(n, n // 10, seed, 1)] = 0  # listed zeros stay structural
    ident = np.arange(n, dtype=np.int32)
    perm = np.random.default_rng(seed).permutation(n).astype(np.int32)
    half, hv = gen.sparse_x(n, n // 2, seed, 2, np.float64)
    return [("in order", ident, val), ("permuted", perm, val[perm]), ("in order, no values", ident, None),
            ("partial", half.astype(np.int32), hv.astype(dtype))]


def check(A, rp, c, v, n, tag, dtype, name, seed):
    m = len(rp) - 1
    masked = gen.sample_positions(m, m // 4, seed, 3)
    keep = np.ones(m, bool)
    keep[masked] = False
    mk = to_dev(mask_bits(m, masked.astype(np.int64)))
    for label, idx, val in full_lists(n, dtype, seed):
        vx = np.ones(len(idx)) if val is None else val.astype(np.float64)
        y_ref, s, hit = oracle.spmspv_rowmajor(n, rp, c, v.astype(np.float64), idx, vx)
        for k in PULLS:
            for use_mask in (False, True):
                ym = np.where(keep, y_ref, 0.0) if use_mask else y_ref
                sm = np.where(keep, s, 0.0) if use_mask else s
                want = np.flatnonzero(hit.astype(bool) & keep) if use_mask else np.flatnonzero(hit)
                extra = dict(ymask=mk) if use_mask else {}
                what = f"{name} {tag} {label} k={k} masked={use_mask}"
                xv = to_dev(val)
                y = A.spmspv(xidx=to_dev(idx), xval=xv, kernel=k, **extra).cpu().numpy()
                if tag == "i32":
                    assert np.array_equal(y, ym.astype(np.int32)), what
                else:
                    assert_rows_close(y, ym, sm, tag, what)
                yidx, yval, nnz_y = A.spmspv(xidx=to_dev(idx), xval=xv, kernel=k, sparse_out=True, **extra)
                cnt = int(nnz_y.item())
                got = yidx[:cnt].cpu().numpy()
                assert np.array_equal(got, want), what + " (structural set)"
                gv = yval[:cnt].cpu().numpy()
                if tag == "i32":
                    assert np.array_equal(gv, ym[got].astype(np.int32)), what
                else:
                    assert_rows_close(gv, ym[got], sm[got], tag, what)


@pytest.mark.parametrize("dtype,tag", [(np.float32, "f32"), (np.float64, "f64")])
def test_full_lists_values(dtype, tag):
    for name, rp, c, v, n in matrices(dtype):
        A = asv.Matrix(len(rp) - 1, n, to_dev(rp), to_dev(c), to_dev(v))
        check(A, rp, c, v, n, tag, dtype, name, 75)


def test_full_lists_int32_bit_exact():
    rp, c = gen.rmat(12, 16, seed=76)
    n = 1 << 12
    v = gen.small_ints(len(c), -50, 50, 1.0, seed=77).astype(np.int32)
    A = asv.Matrix(n, n, to_dev(rp), to_dev(c), to_dev(v))
    ident = np.arange(n, dtype=np.int32)
    xi = gen.small_ints(n, -50, 50, 0.9, seed=78).astype(np.int32)
    for label, idx, val in (("in order", ident, xi), ("in order, no values", ident, None)):
        x = np.ones(n, np.int32) if val is None else val
        want = oracle.i32_pull(rp, c, v, x)
        for k in PULLS:
            y = A.spmspv(xidx=to_dev(idx), xval=to_dev(val), kernel=k).cpu().numpy()
            assert np.array_equal(y, want), f"int32 {label} k={k}"


def test_long_list_in_order_and_with_one_swap():
    # a list of 2^21 + 5 columns spans several rounds of every thread of the
    # feature pass's order check; the same list with two entries swapped
    # (one in the first and one in the last round) must take the scatter
    m = (1 << 21) + 5
    i = np.arange(m, dtype=np.int64)
    cols = np.stack([i - 1, i, i + 1], axis=1)
    ok = (cols >= 0) & (cols < m)
    rp = np.concatenate([[0], np.cumsum(ok.sum(axis=1))]).astype(np.int32)
    c = cols[ok].astype(np.int32)
    v = gen.uniform(len(c), -1, 1, 79, 0, np.float64).astype(np.float32)
    A = asv.Matrix(m, m, to_dev(rp), to_dev(c), to_dev(v))
    val = gen.uniform(m, -1, 1, 80, 0, np.float64).astype(np.float32)
    ident = np.arange(m, dtype=np.int32)
    swap = ident.copy()
    swap[[17, m - 9]] = swap[[m - 9, 17]]
    for label, idx in (("in order", ident), ("one swap", swap)):
        xv = val[idx]
        y_ref, s, hit = oracle.spmspv_rowmajor(m, rp, c, v.astype(np.float64), idx, xv.astype(np.float64))
        for k in ("pull_thread", "auto"):
            y = A.spmspv(xidx=to_dev(idx), xval=to_dev(xv), kernel=k).cpu().numpy()
            assert_rows_close(y, y_ref, s, "f32", f"tridiagonal {m} {label} k={k}")
            yidx, yval, nnz_y = A.spmspv(xidx=to_dev(idx), xval=to_dev(xv), kernel=k, sparse_out=True)
            cnt = int(nnz_y.item())
            got = yidx[:cnt].cpu().numpy()
            assert np.array_equal(got, np.flatnonzero(hit)), f"tridiagonal {m} {label} k={k} (structural set)"
            assert_rows_close(yval[:cnt].cpu().numpy(), y_ref[got], s[got], "f32", f"tridiagonal {m} {label} k={k}")
