"""The warp push on lists long enough for groups of 32 columns per warp
(lane l loading column l's pointers, four short columns walked per step),
against the oracle through the C ABI.

The group form runs once a list holds two groups of 32 per warp of the
launch's grid (4,096 entries per SM); the cases here are sized from the
device's SM count so that it does. A 27-point stencil (FP32 rows of at most
32 entries, so a dense output accumulates in FP32) and a tridiagonal matrix
with a ragged last group of list entries, unmasked and with an output mask;
FP32/FP64 within the per-row tolerances; Boolean and int32 bit for bit.
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
KS = ["push_warp_atom", "push_warp_sort"]


def to_dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def group_threshold():
    # 8 blocks per SM of 8 warps each, two groups of 32 columns per warp
    return 4096 * torch.cuda.get_device_properties(0).multi_processor_count


def mask_bits(m, rows):
    w = np.zeros((m + 31) // 32, np.uint32)
    np.bitwise_or.at(w, rows >> 5, (np.uint32(1) << (rows & 31).astype(np.uint32)))
    return w.view(np.int32)


def tridiagonal(m, seed):
    i = np.arange(m, dtype=np.int64)
    cols = np.stack([i - 1, i, i + 1], axis=1)
    ok = (cols >= 0) & (cols < m)
    rp = np.concatenate([[0], np.cumsum(ok.sum(axis=1))]).astype(np.int32)
    c = cols[ok].astype(np.int32)
    v = gen.uniform(len(c), -1, 1, seed=seed, dtype=np.float64).astype(np.float32)
    return rp, c, v


def lists(n, seed):
    thr = group_threshold()
    out = []
    for rho in (1.0, 0.75):
        k = int(rho * n)
        assert k >= thr, f"a list of {k} entries stays below the group form's {thr}"
        idx, val = gen.sparse_x(n, k, seed=seed, stream=int(rho * 100))
        out.append((rho, idx, val))
    return out


def check_values(A, k, n, rp, c, v, dtype, tag, seed, name):
    m = len(rp) - 1
    masked = gen.sample_positions(m, m // 3, seed=seed + 1)
    keep = np.ones(m, bool)
    keep[masked] = False
    mk = to_dev(mask_bits(m, masked.astype(np.int64)))
    for rho, idx, val in lists(n, seed):
        y_ref, s, hit = oracle.spmspv_rowmajor(n, rp, c, v.astype(np.float64), idx, val)
        xv = val.astype(dtype)
        for dense_in in (False, True):
            kw = dict(x_dense=to_dev(gen.densify(n, idx, xv, dtype))) if dense_in else \
                dict(xidx=to_dev(idx), xval=to_dev(xv))
            for use_mask in (False, True):
                ym = np.where(keep, y_ref, 0.0) if use_mask else y_ref
                sm = np.where(keep, s, 0.0) if use_mask else s
                want = np.flatnonzero(hit.astype(bool) & keep) if use_mask else np.flatnonzero(hit)
                extra = dict(ymask=mk) if use_mask else {}
                what = f"{name} {tag} k={k} rho={rho} dense_in={dense_in} masked={use_mask}"
                y = A.spmspv(kernel=k, **kw, **extra).cpu().numpy()
                assert_rows_close(y, ym, sm, tag, what)
                if use_mask:
                    assert np.all(y[masked] == 0), what + " (masked rows not zero)"
                yidx, yval, nnz_y = A.spmspv(kernel=k, sparse_out=True, **kw, **extra)
                cnt = int(nnz_y.item())
                got = yidx[:cnt].cpu().numpy()
                assert np.array_equal(got, want), what + " (structural set)"
                assert_rows_close(yval[:cnt].cpu().numpy(), ym[got], sm[got], tag, what)


@pytest.mark.parametrize("k", KS)
def test_stencil_long_lists_f32(k):
    g = 100
    rp, c, v, _ = gen.stencil27(g, gen.config_seed(5))
    n = g ** 3
    A = asv.Matrix(n, n, to_dev(rp), to_dev(c), to_dev(v))
    check_values(A, k, n, rp, c, v, np.float32, "f32", 61, "stencil27 100^3")


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("dtype,tag", [(np.float32, "f32"), (np.float64, "f64")])
def test_tridiagonal_ragged_tail(k, dtype, tag):
    m = 4096 * 256 + 3  # the list's last group of 32 is ragged
    rp, c, v = tridiagonal(m, seed=62)
    v = v.astype(dtype)
    A = asv.Matrix(m, m, to_dev(rp), to_dev(c), to_dev(v))
    check_values(A, k, m, rp, c, v, dtype, tag, 63, f"tridiagonal {m}")


@pytest.mark.parametrize("k", KS)
def test_stencil_long_lists_boolean_and_int32_bit_exact(k):
    g = 100
    rp, c, _, _ = gen.stencil27(g, gen.config_seed(5))
    n = g ** 3
    B = asv.Matrix(n, n, to_dev(rp), to_dev(c), None)
    vi = gen.small_ints(len(c), -50, 50, 1.0, seed=64).astype(np.int32)
    I = asv.Matrix(n, n, to_dev(rp), to_dev(c), to_dev(vi))
    for rho, idx, _ in lists(n, 65):
        xb = np.zeros(n, np.uint8)
        xb[idx] = 1
        want = oracle.bool_pull(rp, c, xb)
        yidx, _, nnz_y = B.spmspv(xidx=to_dev(idx), kernel=k, sparse_out=True)
        got = yidx[:int(nnz_y.item())].cpu().numpy()
        assert np.array_equal(got, np.flatnonzero(want)), f"bool list k={k} rho={rho}"
        y = B.spmspv(xidx=to_dev(idx), kernel=k).cpu().numpy()
        assert np.array_equal(y != 0, want != 0), f"bool dense-out k={k} rho={rho}"
        xi = gen.small_ints(len(idx), -50, 50, 1.0, seed=66, stream=int(rho * 100)).astype(np.int32)
        x = np.zeros(n, np.int32)
        x[idx] = xi
        wi = oracle.i32_pull(rp, c, vi, x)
        keep = xi != 0
        got = I.spmspv(xidx=to_dev(idx[keep]), xval=to_dev(xi[keep]), kernel=k).cpu().numpy()
        assert np.array_equal(got, wi), f"int32 list k={k} rho={rho}"


def test_dense_x_read_from_the_bitmap():
    # A dense x of fewer nonzeros than the group threshold, on a matrix wide
    # enough (1,024 columns per warp of the push's grid) with columns of at
    # most 32 entries on average: the warp push reads the feature pass's
    # bitmap instead of a compacted list. A tridiagonal matrix plus one column
    # of 10,000 entries (a hub, queued by its column id); x at three
    # densities, the last above the threshold (list and group form); FP32 and
    # FP64 within their per-row tolerances, int32 and Boolean bit for bit.
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    m = 1024 * 64 * sms + 5
    rp0, c0, _ = tridiagonal(m, seed=81)
    # column 5 joins rows 0, 7, ..., 69993 (the first 70,000 rows are rebuilt)
    cut = 70000
    head = np.repeat(np.arange(cut, dtype=np.int64), np.diff(rp0[:cut + 1]))
    hub_rows = np.arange(0, 10000, dtype=np.int64) * 7
    key = np.unique(np.concatenate([head * m + c0[:rp0[cut]], hub_rows * m + 5]))
    rp_head = np.cumsum(np.bincount(key // m, minlength=cut))
    rp = np.concatenate([[0], rp_head, rp_head[-1] + (rp0[cut + 1:] - rp0[cut])]).astype(np.int32)
    c = np.concatenate([(key % m), c0[rp0[cut]:]]).astype(np.int32)
    v64 = gen.uniform(len(c), -1, 1, seed=82, dtype=np.float64)
    v = v64.astype(np.float32)
    A = asv.Matrix(m, m, to_dev(rp), to_dev(c), to_dev(v))
    A64 = asv.Matrix(m, m, to_dev(rp), to_dev(c), to_dev(v64))
    vi = gen.small_ints(len(c), -50, 50, 1.0, seed=86).astype(np.int32)
    I = asv.Matrix(m, m, to_dev(rp), to_dev(c), to_dev(vi))
    B = asv.Matrix(m, m, to_dev(rp), to_dev(c), None)
    masked = gen.sample_positions(m, m // 5, seed=83)
    keep = np.ones(m, bool)
    keep[masked] = False
    mk = to_dev(mask_bits(m, masked.astype(np.int64)))
    for rho in (1e-4, 1e-2, 0.1):
        idx, val = gen.sparse_x(m, int(rho * m), seed=84, stream=int(rho * 1e4))
        idx = np.union1d(idx, [5]).astype(np.int32)  # the hub column is always in x
        val = gen.uniform(len(idx), -1, 1, seed=85, stream=int(rho * 1e4), dtype=np.float64)
        y_ref, s, hit = oracle.spmspv_rowmajor(m, rp, c, v.astype(np.float64), idx, val)
        xd = to_dev(gen.densify(m, idx, val.astype(np.float32), np.float32))
        for k in ("push_warp_atom", "auto"):
            for use_mask in (False, True):
                ym = np.where(keep, y_ref, 0.0) if use_mask else y_ref
                sm = np.where(keep, s, 0.0) if use_mask else s
                want = np.flatnonzero(hit.astype(bool) & keep) if use_mask else np.flatnonzero(hit)
                extra = dict(ymask=mk) if use_mask else {}
                what = f"bitmap push rho={rho} k={k} masked={use_mask}"
                y = A.spmspv(x_dense=xd, kernel=k, **extra).cpu().numpy()
                assert_rows_close(y, ym, sm, "f32", what)
                yidx, yval, nnz_y = A.spmspv(x_dense=xd, kernel=k, sparse_out=True, **extra)
                cnt = int(nnz_y.item())
                got = yidx[:cnt].cpu().numpy()
                assert np.array_equal(got, want), what + " (structural set)"
                assert_rows_close(yval[:cnt].cpu().numpy(), ym[got], sm[got], "f32", what)
        y64_ref, s64, _ = oracle.spmspv_rowmajor(m, rp, c, v64, idx, val)
        y64 = A64.spmspv(x_dense=to_dev(gen.densify(m, idx, val, np.float64)), kernel="push_warp_atom").cpu().numpy()
        assert_rows_close(y64, y64_ref, s64, "f64", f"bitmap push FP64 rho={rho}")
        xi = np.zeros(m, np.int32)
        xi[idx] = gen.small_ints(len(idx), -50, 50, 1.0, seed=87, stream=int(rho * 1e4)).astype(np.int32)
        wi = oracle.i32_pull(rp, c, vi, xi)
        yi = I.spmspv(x_dense=to_dev(xi), kernel="push_warp_atom").cpu().numpy()
        assert np.array_equal(yi, wi), f"bitmap push int32 rho={rho}"
        xb = np.zeros(m, np.uint8)
        xb[idx] = 1
        wb = oracle.bool_pull(rp, c, xb)
        yb = B.spmspv(x_dense=to_dev(xb), kernel="push_warp_atom").cpu().numpy()
        assert np.array_equal(yb != 0, wb != 0), f"bitmap push Boolean rho={rho}"
