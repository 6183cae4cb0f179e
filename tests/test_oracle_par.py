"""The multi-threaded oracle forms (CPU-baseline only) against the serial
oracle: the row-parallel products are bit-identical (each row still sums in
ascending order), the column-parallel push agrees within the FP64 tolerance
(its atomic additions land in any order) and touches the same rows."""
import numpy as np
import pytest

import gen
import oracle


@pytest.fixture(scope="module")
def stencil():
    g = 24
    rp, c, v, _ = gen.stencil27(g, 81)
    return g ** 3, rp, c, v.astype(np.float64)


def test_row_parallel_pull_is_bit_identical(stencil):
    n, rp, c, v = stencil
    x = gen.uniform(n, -1, 1, 82)
    y1, s1 = oracle.csr_pull(rp, c, v, x)
    y2, s2 = oracle.csr_pull_par(rp, c, v, x)
    assert np.array_equal(y1, y2) and np.array_equal(s1, s2)


def test_row_parallel_spmspv_is_bit_identical(stencil):
    n, rp, c, v = stencil
    idx, xv = gen.sparse_x(n, n // 50, 83, 11, np.float64)
    a = oracle.spmspv_rowmajor(n, rp, c, v, idx, xv)
    b = oracle.spmspv_rowmajor_par(n, rp, c, v, idx, xv)
    for p, q in zip(a, b):
        assert np.array_equal(p, q)


def test_column_parallel_push_within_fp64_tolerance(stencil):
    n, rp, c, v = stencil
    idx, xv = gen.sparse_x(n, n // 20, 84, 11, np.float64)
    cp, ri, pm = oracle.csr_to_csc(n, n, rp, c)
    y1, t1 = oracle.csc_push(n, cp, ri, v[pm], idx, xv)
    y2, t2 = oracle.csc_push_par(n, cp, ri, v[pm], idx, xv)
    _, s, _ = oracle.spmspv_rowmajor(n, rp, c, v, idx, xv)
    assert np.array_equal(t1, t2)
    assert np.all(np.abs(y1 - y2) <= 1e-12 * s)
    assert oracle.par_threads() >= 1
