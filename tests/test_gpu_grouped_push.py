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
