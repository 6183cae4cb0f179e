"""Writes tests/golden/c1_laplace64.json from the oracle (and the seeded
generators) only: the Table 1 matrix features of the 64 x 64 5-point
Laplacian (config C1) and, for x at densities 1, 0.1, 0.01, 0.001, the vector
features and a checksum of the oracle product. Run from the repository root:
    python tests/golden/make_golden.py
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import gen  # noqa: E402
import oracle  # noqa: E402


def main():
    rp, c, v = gen.laplace2d(64)
    n = 64 * 64
    colptr, _, _ = oracle.csr_to_csc(n, n, rp, c)
    out = {"what": "C1: 2-D 5-point Laplacian 64x64, FP64; written by oracle/ via tests/golden/make_golden.py",
           "matrix_features": oracle.matrix_features(n, n, rp), "vectors": []}
    for rho in (1.0, 0.1, 0.01, 0.001):
        k = max(1, int(round(rho * n)))
        idx, val = gen.sparse_x(n, k, seed=gen.config_seed(1), stream=int(rho * 1000))
        y, s, hit = oracle.spmspv_rowmajor(n, rp, c, v, idx, val)
        out["vectors"].append({"rho": rho, "nnz_x": int(k), "features": oracle.vector_features(n, len(c), colptr, idx),
                               "sum_y": float(y.sum()), "sum_abs_y": float(np.abs(y).sum()),
                               "nnz_y": int(hit.sum())})
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c1_laplace64.json")
    json.dump(out, open(path, "w"), indent=1)
    print(path)


if __name__ == "__main__":
    main()
