"""The allocation-free entry point (asv_spmv_noalloc_f32) against the handle path.

It serves callers that cannot allocate device memory on their call path, so
it takes caller-owned CSR arrays and keeps its scratch in a fixed array inside
the library. Two calls in a row (the second reuses the scratch the first left
behind) must each agree with the existing handle-based balanced kernel within
the FP32 tolerance of the parity tests. The file sorts last so that a run
stopping at the first failure has run every other test."""
import numpy as np
import pytest
import torch

import gen
import oracle

pytestmark = pytest.mark.gpu
asv = pytest.importorskip("paper_2006_16767_gb300")
DEV = "cuda"
TOL = 2e-6


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def test_no_alloc_matches_the_handle_path_on_two_calls():
    # skewed rows (hubs longer than a tile, empty rows) plus a stencil block
    rp, c = gen.rmat(13, 16, seed=61)
    n = m = 1 << 13
    v = gen.uniform(len(c), -1, 1, 62, 0, np.float32)
    rpd, cd, vd = to_dev(rp), to_dev(c), to_dev(v)
    A = asv.Matrix(m, n, rpd, cd, vd)
    for call, seed in enumerate((63, 64)):
        x = gen.uniform(n, -1, 1, seed, 0, np.float32)
        xd = to_dev(x)
        y_handle = A.spmv(xd, kernel="pull_bal")
        y = torch.full((m,), float("nan"), dtype=torch.float32, device=DEV)
        asv.asv_spmv_noalloc_f32(m, n, rpd, cd, vd, xd, y)
        torch.cuda.synchronize()
        _, s = oracle.csr_pull(rp, c, v.astype(np.float64), x.astype(np.float64))
        err = np.abs(y.cpu().numpy().astype(np.float64) - y_handle.cpu().numpy().astype(np.float64))
        assert np.all(err <= TOL * s), f"call {call}: {int((err > TOL * s).sum())} rows differ"
    g = 64
    rp2, c2, v2, _ = gen.stencil27(g, 65)
    x2 = gen.uniform(g ** 3, -1, 1, 66, 0, np.float32)
    B = asv.Matrix(g ** 3, g ** 3, to_dev(rp2), to_dev(c2), to_dev(v2))
    y_handle = B.spmv(to_dev(x2), kernel="pull_bal")
    y = torch.empty(g ** 3, dtype=torch.float32, device=DEV)
    asv.asv_spmv_noalloc_f32(g ** 3, g ** 3, to_dev(rp2), to_dev(c2), to_dev(v2), to_dev(x2), y)
    _, s = oracle.csr_pull(rp2, c2, v2.astype(np.float64), x2.astype(np.float64))
    err = np.abs(y.cpu().numpy().astype(np.float64) - y_handle.cpu().numpy().astype(np.float64))
    assert np.all(err <= TOL * s)


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    # m + nnz beyond 2^29 is refused on the host before any device work
    t = torch.zeros(16, dtype=torch.int32, device=DEV)
    f = torch.zeros(16, dtype=torch.float32, device=DEV)
    st = asv.lib().asv_spmv_noalloc_f32(2 ** 29, 2 ** 29, 16, t.data_ptr(), t.data_ptr(), f.data_ptr(),
                                        f.data_ptr(), f.data_ptr(), None)
    assert st == asv.ASV_ERR_CAPACITY
