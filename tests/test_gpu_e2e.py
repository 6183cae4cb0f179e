"""The benchmark's end-to-end steps (inputs from pinned host memory, every
result copied back while later products run) return what the device-resident
step computes, for both workloads at small sizes: index sets and Boolean
results bit for bit, FP32 values within the tolerance of two results that
each meet the FP32 contract (the push's atomics land in any order)."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def asv():
    import __graft_entry__ as ge
    ge.build()
    import paper_2006_16767_gb300 as m
    return m


def test_stencil_e2e_step_returns_the_device_results(asv):
    import bench
    W = bench.Stencil256(side=40)
    W.setup_gpu(asv, torch, torch.device("cuda"))
    W.run_step()
    torch.cuda.synchronize()
    ny = W.nnz_y.cpu().numpy()
    want_list = {c["i"]: (W.yidx[c["i"]][:ny[c["i"]]].cpu().numpy(), W.yval[c["i"]][:ny[c["i"]]].cpu().numpy())
                 for c in W.calls if c["fmt"] == "list"}
    want_dense = {c["i"]: W.yd[c["i"]].cpu().numpy() for c in W.calls if c["fmt"] == "dense"}
    # per-row scale sum |a x| of every product (the oracle), for the FP32 bound
    scale = {}
    for rho, idx, val, _ in W.xs:
        i = [c["i"] for c in W.calls if W.RHOS[c["i"]] == rho][0]
        _, s, _ = oracle.spmspv_rowmajor(W.n, W.rowptr, W.col, W.val.astype(np.float64), idx,
                                         val.astype(np.float64))
        scale[i] = s
    tol = 2 * 2e-6
    W.e2e_setup(torch)
    for _ in range(2):  # the second step reuses every buffer of the first
        for t in W.h_yd:
            t.fill_(np.nan)
        W.e2e_step()
        torch.cuda.synchronize()
        for i, (idx, val) in want_list.items():
            k = int(W.h_nnzy[i])
            assert k == len(idx)
            np.testing.assert_array_equal(W.h_yidx[i][:k].numpy(), idx)
            got = W.h_yval[i][:k].numpy().astype(np.float64)
            assert np.all(np.abs(got - val) <= tol * scale[i][idx]), i
        for i, y in want_dense.items():
            got = W.h_yd[i].numpy().astype(np.float64)
            assert np.all(np.abs(got - y) <= tol * scale[i]), i


def test_rmat_e2e_step_returns_the_device_results(asv):
    import bench
    W = bench.Rmat22(scale=12, edge_factor=16, roots=3)
    W.setup_gpu(asv, torch, torch.device("cuda"))
    W.run_step()
    torch.cuda.synchronize()
    nf = len(W.frontiers)
    ny = W.nnz_y.cpu().numpy()
    want = [W.yidx[i][:ny[i]].cpu().numpy() for i in range(nf)]
    want_pr = W.y_pr.cpu().numpy()
    W.e2e_setup(torch)
    for _ in range(2):
        W.h_ypr.fill_(np.nan)
        W.e2e_step()
        torch.cuda.synchronize()
        for i in range(nf):
            k = int(W.h_nnzy[i])
            assert k == len(want[i])
            np.testing.assert_array_equal(W.h_yidx[i][:k].numpy(), want[i])
        np.testing.assert_array_equal(W.h_ypr.numpy(), want_pr)
