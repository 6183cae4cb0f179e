"""The allocation-free entry point (asv_spmv_noalloc_f32) against the oracle.

It serves callers that cannot allocate device memory on their call path --
real-time loops where cudaMalloc/cudaFree would synchronise the device,
runtimes that own all device memory through their own pool -- so it takes
caller-owned CSR arrays and keeps its scratch in a fixed array inside the
library. Every call here is checked row by row against the FP64 CPU oracle
within the FP32 tolerance of the parity tests, and against the handle's
entry point on the same arrays within the same tolerance, in an order that makes a call
follow a larger one (the scratch then holds more tiles than the call uses),
and once with no value array (all ones). The file sorts last so that a run
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


def check_call(rp, c, v, x, m, n, label):
    """One allocation-free product, compared per row with the oracle:
    |y - y_ref| <= 2e-6 * sum |a x|, and exactly 0 where that sum is 0; and
    with the handle's own entry point (asv_spmv, which allocates its
    workspaces once at handle creation) on the same arrays, within the same
    per-row tolerance."""
    y = torch.full((m,), float("nan"), dtype=torch.float32, device=DEV)
    st = asv.asv_spmv_noalloc_f32(m, n, to_dev(rp), to_dev(c), None if v is None else to_dev(v), to_dev(x), y)
    assert st is None or st == asv.ASV_OK
    torch.cuda.synchronize()
    vv = np.ones(len(c)) if v is None else v.astype(np.float64)
    y_ref, s = oracle.csr_pull(rp, c, vv, x.astype(np.float64))
    got = y.cpu().numpy().astype(np.float64)
    err = np.abs(got - y_ref)
    bad = ~(err <= TOL * s)
    assert not bad.any(), f"{label}: {int(bad.sum())} rows outside 2e-6 * sum|a x|"
    vh = np.ones(len(c), np.float32) if v is None else v
    A = asv.Matrix(m, n, to_dev(rp), to_dev(c), to_dev(vh))
    yh = A.spmv(to_dev(x), kernel="pull_bal").cpu().numpy().astype(np.float64)
    bad = ~(np.abs(got - yh) <= TOL * s)
    assert not bad.any(), f"{label}: {int(bad.sum())} rows differ from asv_spmv by more than 2e-6 * sum|a x|"


def test_no_alloc_matches_the_oracle_on_consecutive_calls():
    # skewed rows (hubs longer than a 2048-item tile, empty rows)
    rp, c = gen.rmat(13, 16, seed=61)
    n = m = 1 << 13
    v = gen.uniform(len(c), -1, 1, 62, 0, np.float32)
    # a larger product in between: 64^3 27-point stencil (~3,500 tiles)
    g = 64
    rp2, c2, v2, _ = gen.stencil27(g, 65)
    x2 = gen.uniform(g ** 3, -1, 1, 66, 0, np.float32)
    check_call(rp, c, v, gen.uniform(n, -1, 1, 63, 0, np.float32), m, n, "R-MAT, first call")
    check_call(rp2, c2, v2, x2, g ** 3, g ** 3, "stencil, larger call")
    # a smaller call right after the larger one: the scratch still holds the
    # larger call's tiles and carries beyond this call's
    check_call(rp, c, v, gen.uniform(n, -1, 1, 64, 0, np.float32), m, n, "R-MAT after the larger call")
    # no value array: every stored entry is one
    check_call(rp, c, None, gen.uniform(n, -1, 1, 67, 0, np.float32), m, n, "R-MAT, all-ones values")


def test_no_alloc_rejects_sizes_beyond_its_scratch():
    # m + nnz beyond 2^29 is refused on the host before any device work
    t = torch.zeros(16, dtype=torch.int32, device=DEV)
    f = torch.zeros(16, dtype=torch.float32, device=DEV)
    st = asv.lib().asv_spmv_noalloc_f32(2 ** 29, 2 ** 29, 16, t.data_ptr(), t.data_ptr(), f.data_ptr(),
                                        f.data_ptr(), f.data_ptr(), None)
    assert st == asv.ASV_ERR_CAPACITY
