"""Host checks of the selector's training labels (no GPU).

The paper prints no rule for turning measured times into the three models'
labels; the readings used are: the pattern label is the pattern of the
fastest candidate, each pattern's distribution label its fastest
distribution, the write-back label the fastest write-back at the best push
distribution, and candidates within 2 % of the fastest count as tied, the
lowest kernel id winning. These tests pin those readings on hand-made timing
rows, and the host-side tree walk on a hand-made tree table."""
import numpy as np

from paper_2006_16767_gb300 import selector_train as st

PULL, MPULL, PUSH = 2, 1, 0


def times(**over):
    t = [10.0] * st.NK
    for name, v in over.items():
        t[st.kernel_id(*{"pt": (2, 0, 0), "pw": (2, 1, 0), "pb": (2, 2, 0),
                          "mt": (1, 0, 0), "mw": (1, 1, 0), "mb": (1, 2, 0),
                          "hta": (0, 0, 0), "hwa": (0, 1, 0), "hba": (0, 2, 0),
                          "hts": (0, 0, 1), "hws": (0, 1, 1), "hbs": (0, 2, 1),
                          "htp": (0, 0, 2), "hwp": (0, 1, 2), "hbp": (0, 2, 2)}[name])] = v
    return t


def test_kernel_ids_and_parts_are_inverse():
    seen = set()
    for k in range(st.NK):
        p, d, w = st.kernel_parts(k)
        assert st.kernel_id(p, d, w) == k
        seen.add((p, d, w))
    assert len(seen) == st.NK
    # the paper's eight: pull K1/K2, validated pull K3/K4, push with atomics K5/K7, with sort K6/K8
    assert st.kernel_parts(0) == (PULL, 0, 0) and st.kernel_parts(2) == (PULL, 2, 0)
    assert st.kernel_parts(8) == (PUSH, 2, 0) and st.kernel_parts(11) == (PUSH, 2, 1)


def test_pattern_and_distribution_of_the_fastest():
    pat, dpush, dmpull, dpull, wb = st.labels(times(pw=3.0, pb=4.0, hba=5.0, mt=6.0))
    assert (pat, dpull, dpush, dmpull, wb) == (PULL, 1, 2, 0, 0)


def test_ties_within_two_percent_go_to_the_lower_id():
    # pull_thread within 2 % of pull_warp: the simpler kernel is the label
    assert st.labels(times(pt=3.05, pw=3.0))[3] == 0
    # 3 % slower is not a tie
    assert st.labels(times(pt=3.09, pw=3.0))[3] == 1
    # the pattern label follows the tie too: push_thread_atom (id 6) ties a
    # masked pull (id 3) only if within 2 % -- the lower id (masked pull) wins
    assert st.labels(times(mt=3.02, hta=3.0))[0] == MPULL
    assert st.labels(times(mt=3.2, hta=3.0))[0] == PUSH


def test_write_back_label_at_the_best_push_distribution():
    # the fastest push kernel is the balanced split with sort + reduce-by-key
    t = times(hwa=4.0, hws=3.5, hwp=3.9, hta=6.0, hba=6.0, hbs=2.0)
    pat, dpush, _, _, wb = st.labels(t)
    assert (pat, dpush, wb) == (PUSH, 2, 1)
    # a tie inside push: thread/atomic within 2 % of bal/sort takes both labels
    t = times(hta=2.03, hbs=2.0)
    pat, dpush, _, _, wb = st.labels(t)
    assert (pat, dpush, wb) == (PUSH, 0, 0)


def test_missing_times_never_win():
    t = times(pw=3.0)
    t[st.kernel_id(2, 0, 0)] = None
    assert st.labels(t)[3] == 1


def test_host_tree_walk_follows_thresholds():
    # pattern tree: m_sparsity (feature 12) <= 0.1 -> push else pull; the
    # push distribution tree: nnz_x (feature 9) <= 100 -> warp else bal;
    # write-back tree: a single atomic leaf
    nodes = [(12, 0.1, 1, 2, 0), (-1, 0.0, 0, 0, PUSH), (-1, 0.0, 0, 0, PULL),
             (9, 100.0, 4, 5, 0), (-1, 0.0, 0, 0, 1), (-1, 0.0, 0, 0, 2),
             (-1, 0.0, 0, 0, 0), (-1, 0.0, 0, 0, 1), (-1, 0.0, 0, 0, 0)]
    roots = [0, 3, 6, 7, 8] * 4
    trees = {"f32": {"nodes": nodes, "roots": roots}}
    f = np.zeros(13)
    f[12], f[9] = 0.05, 50
    assert st.predict(trees, "f32", 0, f) == st.kernel_id(PUSH, 1, 0)
    f[9] = 500
    assert st.predict(trees, "f32", 2, f) == st.kernel_id(PUSH, 2, 0)
    f[12] = 0.5
    assert st.predict(trees, "f32", 3, f) == st.kernel_id(PULL, 1, 0)


def _walk(nodes, root, feat):
    i = root
    path = []
    while nodes[i][0] >= 0:
        f, thr, l, r, _ = nodes[i]
        path.append(f)
        i = l if feat[f] <= thr else r
    return nodes[i][4], path


def test_cost_ordered_tree_tests_cheap_features_first():
    import pytest
    pytest.importorskip("sklearn")
    # labels: x_sparsity (feature 10, cheap) splits pull from the rest; among
    # the sparse samples, m_sparsity (feature 12, a pass over the list)
    # separates push from masked pull
    rng = np.random.default_rng(3)
    X = np.zeros((600, 13))
    X[:, 10] = rng.uniform(0, 1, 600)
    X[:, 12] = rng.uniform(0, 1, 600)
    X[:, 2] = 1e6
    y = np.where(X[:, 10] > 0.5, PULL, np.where(X[:, 12] > 0.3, MPULL, PUSH)).astype(np.int64)
    nodes, _ = st._fit_cost_ordered(X, y, tuple(range(13)), seed=0)
    n = len(nodes)
    for (f, thr, l, r, lf) in nodes:  # a valid table: children inside it
        assert f < 0 or (0 <= l < n and 0 <= r < n)
    assert nodes[0][0] in st.CHEAP  # the root splits on a cheap feature
    agree = 0
    for x, lab in zip(X, y):
        got, path = _walk(nodes, 0, x)
        agree += got == lab
        if lab == PULL:  # the dense side is decided from cheap features alone
            assert all(f in st.CHEAP for f in path)
    assert agree / len(y) > 0.97


def test_lazy_walk_decides_only_on_cheap_paths():
    # pattern tree: x_sparsity <= 0.5 -> test m_sparsity, else pull; pull and
    # masked-pull distribution trees: thread; push trees: warp, atomic
    nodes = [(10, 0.5, 1, 2, 0), (12, 0.1, 3, 4, 0), (-1, 0.0, 0, 0, PULL), (-1, 0.0, 0, 0, PUSH),
             (-1, 0.0, 0, 0, MPULL), (-1, 0.0, 0, 0, 0), (-1, 0.0, 0, 0, 1), (-1, 0.0, 0, 0, 0)]
    roots = [0, 6, 5, 5, 7] * 4
    trees = {"f32": {"nodes": nodes, "roots": roots}}
    feat = [0.0] * 13
    feat[10] = 0.9
    assert st.lazy_walk(trees, "f32", 3, feat) == st.kernel_id(PULL, 0, 0)
    assert st.lazy_walk(trees, "f32", 0, feat) is None  # dense x: no lazy path
    feat[10] = 0.1
    assert st.lazy_walk(trees, "f32", 2, feat) is None  # needs m_sparsity
