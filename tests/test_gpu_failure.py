"""Failure detection without a GPU fault.

A bounded device wait is made to give up at once (its poll limit set to 0
through a testing hook) while the bulk copies it waits for are still in
flight: the kernel latches ASV_ERR_TIMEOUT in the handle's status word, waits
for its copies again under the normal bound (so none is left in flight when
the warp leaves) and returns. The host reads the status; the context stays
usable and the next call, with the normal limit, is correct. An allocation
failure is injected on the host (the k-th allocation of handle creation
reports out-of-memory): creation returns ASV_ERR_NOMEM and releases every
allocation it had made. Nothing here faults, traps or hangs a GPU."""
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


def test_expired_wait_latches_timeout_and_the_handle_recovers():
    # 27-point stencil: a warp's 32 rows span ~864 entries, so the
    # one-row-per-thread pull stages them with TMA bulk copies
    g = 32
    rp, c, v, _ = gen.stencil27(g, 71)
    m = n = g ** 3
    A = asv.Matrix(m, n, to_dev(rp), to_dev(c), to_dev(v))
    x = gen.uniform(n, -1, 1, 72, 0, np.float32)
    xd = to_dev(x)
    assert A.status() == asv.ASV_OK
    asv.asv_debug_set_wait_limit(A.handle, 0)
    A.spmv(xd, kernel="pull_thread")
    assert A.status() == asv.ASV_ERR_TIMEOUT
    assert A.status() == asv.ASV_OK  # reading the status cleared it
    asv.asv_debug_set_wait_limit(A.handle, asv.ASV_WAIT_LIMIT_DEFAULT)
    y = A.spmv(xd, kernel="pull_thread")
    assert A.status() == asv.ASV_OK
    y_ref, s = oracle.csr_pull(rp, c, v.astype(np.float64), x.astype(np.float64))
    assert_rows_close(y.cpu().numpy(), y_ref, s, "f32", "pull_thread after the expired wait")


def test_injected_allocation_failure_returns_nomem_and_releases_everything():
    rp, c, v = gen.random_csr(3001, 2503, 0.004, seed=73, values="uniform", dtype=np.float32)
    rpd, cd, vd = to_dev(rp), to_dev(c), to_dev(v)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        for k in (1, 2, 7, 19, 30):
            asv.asv_debug_fail_alloc(k)
            with pytest.raises(asv.AsvError) as ei:
                asv.Matrix(3001, 2503, rpd, cd, vd)
            assert ei.value.status == asv.ASV_ERR_NOMEM, k
    finally:
        asv.asv_debug_fail_alloc(0)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    assert free0 - free1 < (8 << 20), f"{(free0 - free1) >> 20} MB not released"
    A = asv.Matrix(3001, 2503, rpd, cd, vd)
    x = gen.uniform(2503, -1, 1, 74, 0, np.float32)
    y = A.spmv(to_dev(x), kernel="pull_bal")
    y_ref, s = oracle.csr_pull(rp, c, v.astype(np.float64), x.astype(np.float64))
    assert_rows_close(y.cpu().numpy(), y_ref, s, "f32", "handle created after the injected failures")
