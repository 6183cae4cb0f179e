"""Regression of the oracle against its stored C1 fixture (tests/golden/,
written by tests/golden/make_golden.py from the oracle), and the device
features of the same inputs against it."""
import json
import os

import numpy as np
import pytest

import gen
import oracle

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "c1_laplace64.json")))


def test_oracle_reproduces_the_c1_fixture():
    rp, c, v = gen.laplace2d(64)
    n = 4096
    assert oracle.matrix_features(n, n, rp) == GOLDEN["matrix_features"]
    colptr, _, _ = oracle.csr_to_csc(n, n, rp, c)
    for rec in GOLDEN["vectors"]:
        idx, val = gen.sparse_x(n, rec["nnz_x"], seed=gen.config_seed(1), stream=int(rec["rho"] * 1000))
        assert oracle.vector_features(n, len(c), colptr, idx) == rec["features"]
        y, s, hit = oracle.spmspv_rowmajor(n, rp, c, v, idx, val)
        assert float(y.sum()) == rec["sum_y"] and int(hit.sum()) == rec["nnz_y"]


@pytest.mark.gpu
def test_device_features_match_the_c1_fixture():
    import torch
    asv = pytest.importorskip("paper_2006_16767_gb300")
    rp, c, v = gen.laplace2d(64)
    n = 4096
    A = asv.Matrix(n, n, torch.from_numpy(rp).cuda(), torch.from_numpy(c).cuda(), torch.from_numpy(v).cuda())
    f = A.features()
    for k, want in GOLDEN["matrix_features"].items():
        assert abs(f[k] - want) <= 1e-12 * max(1.0, abs(want)), k
    for rec in GOLDEN["vectors"]:
        idx, val = gen.sparse_x(n, rec["nnz_x"], seed=gen.config_seed(1), stream=int(rec["rho"] * 1000))
        _, vf = A.select(xidx=torch.from_numpy(idx).cuda(), xval=torch.from_numpy(val).cuda())
        assert vf["nnz_x"] == rec["features"]["nnz_x"] and vf["nnz_s"] == rec["features"]["nnz_s"]
        yidx, yval, nnz_y = A.spmspv(xidx=torch.from_numpy(idx).cuda(), xval=torch.from_numpy(val).cuda(),
                                     sparse_out=True)
        assert int(nnz_y.item()) == rec["nnz_y"]
        k = int(nnz_y.item())
        assert abs(float(yval[:k].double().sum().item()) - rec["sum_y"]) <= 1e-12 * max(1.0, rec["sum_abs_y"])
