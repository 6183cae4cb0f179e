"""Shared helpers of the parity tests (test code; imports the oracle)."""
import numpy as np

import oracle

# Tolerances fixed by the method's numerics contract: per row,
# |y - y_ref| <= tol * sum_k |a_k x_k| (FP64: 1e-12, FP32: 2e-6); integer and
# Boolean semirings and all index sets are compared bit for bit.
TOL = {"f32": 2e-6, "f64": 1e-12}


def assert_rows_close(y, y_ref, s, dtype, what=""):
    y = np.asarray(y, np.float64)
    tol = TOL[dtype]
    err = np.abs(y - y_ref)
    bad = ~(err <= tol * s)
    if bad.any():
        i = int(np.flatnonzero(bad)[0])
        raise AssertionError(f"{what}: {int(bad.sum())} rows out of tolerance; first row {i}: "
                             f"got {y[i]!r} want {y_ref[i]!r} scale {s[i]!r}")


def ref_spmspv(n, rowptr, col, val, xidx, xval):
    """Oracle y, scale and structural set of a (possibly sparse) x."""
    return oracle.spmspv_rowmajor(n, rowptr, col, val, xidx, xval)


def sparse_result(yidx, yval, nnz_y):
    k = int(nnz_y.item())
    return yidx[:k].cpu().numpy(), (yval[:k].cpu().numpy() if yval is not None else None)
