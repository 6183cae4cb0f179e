"""Parity at the benchmark's full sizes, through the same selector-driven
calls the benchmark times: outputs sampled row by row (or vector by vector)
against the oracle, and properties that hold at any size. Slower than the
small-case parity tests (the inputs take seconds to generate), so they run
last among the GPU tests but the test_zz file."""
import numpy as np
import pytest
import torch

import gen
import oracle
from tests._util import assert_rows_close

pytestmark = pytest.mark.gpu
asv = pytest.importorskip("paper_2006_16767_gb300")
DEV = "cuda"


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def sub_csr(rp, c, v, rows):
    """The sampled rows of a CSR matrix as a CSR matrix of their own."""
    lens = (rp[rows + 1] - rp[rows]).astype(np.int64)
    rp_s = np.concatenate([[0], np.cumsum(lens)]).astype(np.int32)
    sel = np.concatenate([np.arange(rp[r], rp[r + 1]) for r in rows])
    return rp_s, c[sel], (None if v is None else v[sel])


def test_stencil256_dense_and_listed_x():
    g = 256
    rp, c, v, rowsum = gen.stencil27(g, gen.config_seed(5))
    m = n = g ** 3
    A = asv.Matrix(m, n, to_dev(rp), to_dev(c), to_dev(v))
    # closed form on every row: A 1 = the row sums (all terms positive, so s_i = row sum)
    y = A.spmv(torch.ones(n, dtype=torch.float32, device=DEV), kernel="auto").cpu().numpy()
    assert_rows_close(y, rowsum, rowsum, "f32", "stencil256 A*1")
    rows = np.sort(gen.randint(4096, m, 51)).astype(np.int64)
    rp_s, c_s, v_s = sub_csr(rp, c, v, rows)
    x = gen.uniform(n, -1, 1, 52).astype(np.float32)
    y = A.spmv(to_dev(x), kernel="auto").cpu().numpy()
    ref, s = oracle.csr_pull(rp_s, c_s, v_s.astype(np.float64), x.astype(np.float64))
    assert_rows_close(y[rows], ref, s, "f32", "stencil256 dense x")
    for rho in (1e-5, 1e-3, 0.1):
        idx, val = gen.sparse_x(n, int(rho * n), gen.config_seed(5), 11, np.float32)
        yd = A.spmspv(xidx=to_dev(idx), xval=to_dev(val), kernel="auto").cpu().numpy()
        ref, s, _ = oracle.spmspv_rowmajor(n, rp_s, c_s, v_s.astype(np.float64), idx, val.astype(np.float64))
        assert_rows_close(yd[rows], ref, s, "f32", f"stencil256 listed x rho={rho}")


def test_stencil256_benchmark_step_calls():
    # the twelve selector-driven products of the benchmark step, in its launch
    # configuration: per density, x listed -> the structural output list (the
    # whole index set bit for bit, values on sampled rows), and x dense -> y
    # dense (sampled rows)
    g = 256
    rp, c, v, _ = gen.stencil27(g, gen.config_seed(5))
    m = n = g ** 3
    A = asv.Matrix(m, n, to_dev(rp), to_dev(c), to_dev(v))
    colptr, rowidx, _ = oracle.csr_to_csc(m, n, rp, c)
    rows = np.sort(gen.randint(4096, m, 54)).astype(np.int64)
    rp_s, c_s, v_s = sub_csr(rp, c, v, rows)
    v_s = v_s.astype(np.float64)
    yidx = torch.empty(m, dtype=torch.int32, device=DEV)
    yval = torch.empty(m, dtype=torch.float32, device=DEV)
    nnz_y = torch.zeros(1, dtype=torch.int64, device=DEV)
    yd = torch.empty(m, dtype=torch.float32, device=DEV)
    for rho in (1e-5, 1e-4, 1e-3, 1e-2, 1e-1, 1.0):
        k = max(1, int(round(rho * n)))
        idx, val = gen.sparse_x(n, k, gen.config_seed(5), 11, np.float32)
        it, vt = to_dev(idx), to_dev(val)
        cnt = torch.tensor([k], dtype=torch.int64, device=DEV)
        asv.asv_spmspv(A.handle, cnt, it, vt, None, asv.ASV_OUT_SPARSE, None, yidx, yval, nnz_y, m, "auto")
        xd = torch.zeros(n, dtype=torch.float32, device=DEV)
        xd[it.long()] = vt
        asv.asv_spmspv(A.handle, None, None, None, xd, asv.ASV_OUT_DENSE, yd, kernel="auto")
        assert A.status() == asv.ASV_OK
        touched = np.flatnonzero(oracle.csc_push(m, colptr, rowidx, None, idx, None)[1])
        ny = int(nnz_y.item())
        got_idx = yidx[:ny].cpu().numpy()
        assert np.array_equal(got_idx, touched), f"rho={rho}: output index set"
        ref, s, hit = oracle.spmspv_rowmajor(n, rp_s, c_s, v_s, idx, val.astype(np.float64))
        pos = np.searchsorted(got_idx, rows)
        inset = hit.astype(bool)
        assert np.array_equal(inset, (pos < ny) & (got_idx[np.minimum(pos, ny - 1)] == rows))
        gv = yval[:ny].cpu().numpy()[pos[inset]]
        assert_rows_close(gv, ref[inset], s[inset], "f32", f"stencil256 list->list rho={rho}")
        assert_rows_close(yd.cpu().numpy()[rows], ref, s, "f32", f"stencil256 dense->dense rho={rho}")


def test_rmat22_bfs_levels_products_and_pagerank():
    rp, c = gen.rmat(22, 16, gen.config_seed(2))
    n = 1 << 22
    Ab = asv.Matrix(n, n, to_dev(rp), to_dev(c), None)
    deg = np.diff(rp)
    cand = np.flatnonzero(deg > 0)
    roots = [int(cand[i]) for i in gen.randint(8, len(cand), gen.config_seed(2), stream=7)]
    # a whole search through the masked product, every level bit for bit
    want, L = oracle.bfs(n, rp, c, roots[0])
    level, depth = Ab.bfs(roots[0])
    assert np.array_equal(level.cpu().numpy(), want) and depth == L
    # the unmasked level products of the benchmark (list in, list out), bit for bit on every row
    fronts = oracle.frontiers(n, rp, c, roots[1])
    for f in (fronts[1], max(fronts, key=len), fronts[-1]):
        xb = np.zeros(n, np.uint8)
        xb[f] = 1
        hit = np.flatnonzero(oracle.bool_pull(rp, c, xb))
        yidx, _, nnz_y = Ab.spmspv(xidx=to_dev(f), sparse_out=True, kernel="auto")
        got = yidx[:int(nnz_y.item())].cpu().numpy()
        assert np.array_equal(got, hit), f"rmat22 level product, frontier of {len(f)}"
    # the FP32 PageRank step (dense x), sampled rows
    Af = asv.Matrix(n, n, to_dev(rp), to_dev(c), to_dev(np.ones(len(c), np.float32)))
    r = gen.uniform(n, 0.0, 1.0, gen.config_seed(2), stream=8)
    r /= r.sum()
    x = np.where(deg > 0, r / np.maximum(deg, 1), 0.0).astype(np.float32)
    y = Af.spmv(to_dev(x), kernel="auto").cpu().numpy()
    rows = np.sort(gen.randint(4096, n, 53)).astype(np.int64)
    rp_s, c_s, _ = sub_csr(rp, c, None, rows)
    ref, s = oracle.csr_pull(rp_s, c_s, np.ones(len(c_s)), x.astype(np.float64))
    assert_rows_close(y[rows], ref, s, "f32", "rmat22 PageRank step")


def test_zipf_batch_of_4096_sampled_vectors():
    m, n, B = 1_000_000, 131_072, 4096
    rp, c, v = gen.lognormal_zipf(m, n, np.log(40), 1.0, 1.2, gen.config_seed(3))
    xrp_all, xc_all, xv_all = gen.lognormal_zipf(65_536, n, np.log(40), 1.0, 1.2, gen.config_seed(3) + 100,
                                                 perm_seed=gen.config_seed(3))
    pick = gen.randint(B, 65_536, gen.config_seed(3), 1)
    lens = (xrp_all[pick + 1] - xrp_all[pick]).astype(np.int64)
    xptr = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    xc = np.concatenate([xc_all[xrp_all[p]:xrp_all[p + 1]] for p in pick]).astype(np.int32)
    xv = np.concatenate([xv_all[xrp_all[p]:xrp_all[p + 1]] for p in pick]).astype(np.float32)
    A = asv.Matrix(m, n, to_dev(rp), to_dev(c), to_dev(v))
    Y = torch.empty((B, m), dtype=torch.float32, device=DEV)
    vs = gen.randint(6, B, 54)
    for tune in ((8, 256, 128), (4, 1024, 0)):
        A.spmspv_batched(to_dev(xptr), to_dev(xc), to_dev(xv), Y=Y, tune=tune)
        for b in vs:
            lo, hi = xptr[b], xptr[b + 1]
            ref, s, _ = oracle.spmspv_rowmajor(n, rp, c, v.astype(np.float64), xc[lo:hi], xv[lo:hi].astype(np.float64))
            assert_rows_close(Y[b].cpu().numpy(), ref, s, "f32", f"zipf batch tune={tune} vector {b}")
    del Y


def test_layer_16384_forward_and_backward_sampled():
    m = n = 16384
    B = 64
    rp, c, v = gen.bernoulli(m, n, 0.05, 0.02, gen.config_seed(4))
    dens = gen.uniform(B, 0.05, 0.5, gen.config_seed(4), 1)
    X = gen.halfnormal(B * n, 1.0, gen.config_seed(4), 2).reshape(B, n)
    X = np.where(gen.uniform(B * n, 0, 1, gen.config_seed(4), 3).reshape(B, n) < dens[:, None], X, 0).astype(np.float32)
    dY = gen.uniform(B * m, -1, 1, gen.config_seed(4), 4, np.float32).reshape(B, m)
    A = asv.Matrix(m, n, to_dev(rp), to_dev(c), to_dev(v))
    Y = A.spmspv_batched(X_dense=to_dev(X)).cpu().numpy()
    dX, dA = A.backward(to_dev(X), to_dev(dY))
    dX, dA = dX.cpu().numpy(), dA.cpu().numpy()
    colptr, rowidx, perm = oracle.csr_to_csc(m, n, rp, c)
    vv = v.astype(np.float64)
    for b in gen.randint(4, B, 55):
        ref, s = oracle.csr_pull(rp, c, vv, X[b].astype(np.float64))
        assert_rows_close(Y[b], ref, s, "f32", f"layer forward vector {b}")
        ref, s = oracle.csc_pull(colptr, rowidx, vv[perm], dY[b].astype(np.float64))
        assert_rows_close(dX[b], ref, s, "f32", f"layer dx vector {b}")
    ks = np.sort(gen.randint(20000, len(c), 56)).astype(np.int64)
    rows = np.searchsorted(rp, ks, "right") - 1
    terms = dY[:, rows].astype(np.float64) * X[:, c[ks]].astype(np.float64)
    assert_rows_close(dA[ks], terms.sum(axis=0), np.abs(terms).sum(axis=0), "f32", "layer dA sampled entries")
