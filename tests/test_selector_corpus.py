"""Host-side checks of the selector's training inputs (no GPU): every corpus
vector is a valid duplicate-free ascending list, and the Zipf matrices get
vectors drawn as rows over the same feature space, whose effective nonzeros
are a far larger share of the matrix than their own density."""
import numpy as np

import gen
from paper_2006_16767_gb300 import selector_train as st


def test_feature_rows_are_valid_lists_reaching_popular_columns():
    name = "zipf_100k_32k"
    m, n, mu, sg, zs, sd = st.ZIPF[name]
    rp, c, _ = gen.lognormal_zipf(m, n, mu, sg, zs, st.CORPUS_SEED + sd)
    deg = np.bincount(c, minlength=n)
    rows = st.feature_rows(name)
    assert len(rows) >= 20
    for rho, idx in rows:
        assert len(idx) and np.all(np.diff(idx) > 0) and idx[0] >= 0 and idx[-1] < n
        assert rho == len(idx) / n
    # the typical row reaches hub columns: m_sparsity well above x_sparsity
    ratio = np.median([deg[idx].sum() / len(c) / (len(idx) / n) for _, idx in rows])
    assert ratio > 10


def test_vectors_of_a_zipf_matrix_include_feature_rows():
    name = "zipf_100k_32k"
    n = st.ZIPF[name][1]
    rp = np.zeros(2, np.int32)
    out = st.vectors(name, rp, np.zeros(0, np.int32), n, 1)
    assert len(out) == len(st.densities(n)) + len(st.feature_rows(name))
