"""Training of the kernel selector for the GPU at hand (Sec. V-B).

The paper labels every (matrix, vector) sample with the fastest candidate,
trains three decision trees -- computing pattern, workload distribution,
write-back -- on the Table 1 features, and retrains per hardware because the
switch points move between GPUs. This module does the same on synthetic
matrices:

  collect(path)   on a GPU: for every corpus matrix, value type, call format
                  (x dense or a list; y dense or a list) and x density, time
                  every candidate through the C ABI and append one JSON row
                  {features, times} to `path`;
  fit(path)       on any host with scikit-learn: grid-searched CART per
                  (value type, format, model) as in Sec. V-B, labels as in
                  the design notes (pattern of the fastest kernel; fastest
                  distribution inside that pattern; fastest write-back inside
                  push at the best push distribution; ties within 2% go to the
                  lower kernel id);
  emit(trees)     the C table compiled into the library (csrc/trees_default.h);
  regret(path, trees)  selected-kernel time over best-candidate time.

Usage:  python -m paper_2006_16767_gb300.selector_train collect out.jsonl
        python -m paper_2006_16767_gb300.selector_train fit out.jsonl
"""
from __future__ import annotations

import json
import os
import sys
import time
import zlib

import numpy as np

FEATURES = ("m", "n", "nnz", "max_row", "min_row", "avg_row", "relative_range", "var_nnz_row", "gini",
            "nnz_x", "x_sparsity", "nnz_s", "m_sparsity")
# Table 1: model 1 sees every feature, model 2 the matrix ones, model 3 the sizes and vector ones
MODEL_FEATURES = (tuple(range(13)), tuple(range(9)), (0, 1, 2, 9, 10, 11, 12))
NK = 15
TIE = 1.02


def kernel_parts(k):
    """(pattern, distribution, write-back) of kernel id k; pattern 0 push, 1 masked pull, 2 pull."""
    if k < 3:
        return 2, k, 0
    if k < 6:
        return 1, k - 3, 0
    q = k - 6
    return 0, q % 3, q // 3


def kernel_id(pattern, dist, wb):
    if pattern == 2:
        return dist
    if pattern == 1:
        return 3 + dist
    return 6 + 3 * wb + dist


# ------------------------------------------------------------------ corpus
CORPUS_SEED = 7919
# lognormal-row / Zipf-column matrices of the corpus: (m, n, ln of the median
# row length, its sigma, Zipf exponent, seed offset)
ZIPF = {"zipf_200k": (200_000, 131_072, np.log(40), 1.0, 1.2, 1),
        "zipf_1m_64k": (1_000_000, 65_536, np.log(20), 1.0, 1.1, 2),
        "zipf_500k_256k": (500_000, 262_144, np.log(30), 0.8, 1.3, 7),
        "zipf_100k_32k": (100_000, 32_768, np.log(80), 1.2, 1.0, 8),
        # a million rows over 131,072 columns: the row count at which a hub-heavy
        # list's push (atomics on rows every hub reaches) loses to the pull
        "zipf_1m_131k": (1_000_000, 131_072, np.log(40), 1.0, 1.2, 11)}


def corpus():
    """Synthetic training matrices (none of them is a benchmark matrix)."""
    import gen
    s = CORPUS_SEED
    items = []
    for g in (48, 96, 128, 160, 192, 224):
        items.append((f"stencil27_{g}", lambda g=g: gen.stencil27(g, s + g)[:3] + (g ** 3,)))
    for g in (256, 512, 1024, 2048):
        items.append((f"laplace2d_{g}", lambda g=g: gen.laplace2d(g) + (g * g,)))
    for sc, ef in ((14, 16), (16, 8), (16, 16), (17, 32), (18, 8), (19, 16), (20, 8), (20, 16), (21, 16), (22, 16)):
        items.append((f"rmat_{sc}_{ef}", lambda sc=sc, ef=ef: rmat_vals(sc, ef, s + sc * 7 + ef)))
    items.append(("rmat_er_18", lambda: rmat_vals(18, 16, s + 5, a=0.25, b=0.25, c=0.25)))
    items.append(("rmat_mild_19", lambda: rmat_vals(19, 16, s + 6, a=0.45, b=0.22, c=0.22)))
    for name, (m, n, mu, sg, zs, sd) in ZIPF.items():
        items.append((name, lambda m=m, n=n, mu=mu, sg=sg, zs=zs, sd=sd:
                      gen.lognormal_zipf(m, n, mu, sg, zs, CORPUS_SEED + sd) + (n,)))
    for name, k, p, sd in (("bern_8192_1pct", 8192, 0.01, 3), ("bern_4096_5pct", 4096, 0.05, 4),
                           ("bern_16384_02pct", 16384, 0.002, 9)):
        items.append((name, lambda k=k, p=p, sd=sd: gen.bernoulli(k, k, p, 0.02, s + sd) + (k,)))
    return items


def rmat_vals(scale, ef, seed, a=0.57, b=0.19, c=0.19):
    import gen
    rp, c = gen.rmat(scale, ef, seed, a, b, c)
    return rp, c, gen.uniform(len(c), 0.5, 1.5, seed, 3, np.float32), 1 << scale


def densities(n):
    rhos = sorted(set([10.0 ** e for e in np.arange(-6, 0.01, 0.25)] + [0.15, 0.2, 0.3, 0.4, 0.5, 0.6, 0.8]))
    out = []
    for r in rhos:
        k = int(round(r * n))
        if k >= 1 and (not out or k > out[-1][1]):
            out.append((r, min(k, n)))
    return out


def bfs_levels(rp, c, n, root):
    """Host BFS levels over the pattern (scipy), -1 = unreached."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import breadth_first_order
    A = sp.csr_matrix((np.ones(len(c), np.int8), c, rp), shape=(n, n))
    order, pred = breadth_first_order(A, root, directed=True, return_predecessors=True)
    level = np.full(n, -1, np.int64)
    level[root] = 0
    for v in order[1:]:  # BFS order: a vertex's predecessor is settled before it
        level[v] = level[pred[v]] + 1
    return level


def feature_rows(name, count=24):
    """x drawn as rows of a second matrix over the same feature space as the
    Zipf corpus matrix `name` (same rank -> column map, so the same popular
    columns): a few dozen entries that reach the hub columns, so nnz_s / nnz
    is far above nnz_x / n -- the sparse-data inputs that uniform positions
    do not produce. Rows picked at spread-out length quantiles."""
    import gen
    m, n, mu, sg, zs, sd = ZIPF[name]
    xrp, xc, _ = gen.lognormal_zipf(4096, n, mu, sg, zs, CORPUS_SEED + sd + 100, perm_seed=CORPUS_SEED + sd)
    lens = np.diff(xrp)
    order = np.argsort(lens, kind="stable")
    picks = order[np.linspace(0, len(order) - 1, num=count).astype(np.int64)]
    return [(float(lens[r]) / n, np.unique(xc[xrp[r]:xrp[r + 1]]).astype(np.int32)) for r in picks if lens[r] > 0]


def vectors(name, rp, c, n, m, roots=2, max_levels=8):
    """The x of one training matrix: seeded uniform positions at every
    density; for the Zipf matrices, rows of a second matrix over the same
    feature space; and -- for square matrices -- BFS frontiers (the inputs of
    the graph applications, whose structure uniform positions do not have)
    from a few seeded roots, at most max_levels per root spread over the
    search."""
    import gen
    out = []
    for rho, k in densities(n):
        out.append((rho, gen.sample_positions(n, k, seed=zlib.crc32(f"{name}/{k}".encode()), stream=1)))
    if name in ZIPF:
        out.extend(feature_rows(name))
    if m == n and n > 1:
        deg = np.diff(rp)
        cand = np.flatnonzero(deg > 0)
        picks = gen.randint(roots, len(cand), zlib.crc32(f"{name}/roots".encode()), 3) if len(cand) else []
        for r in picks:
            level = bfs_levels(rp, c, n, int(cand[r]))
            L = int(level.max()) + 1
            for l in sorted(set(np.linspace(1, L - 1, num=min(max_levels, max(L - 1, 0))).astype(int).tolist())):
                f = np.flatnonzero(level == l).astype(np.int32)
                if len(f):
                    out.append((len(f) / n, f))
    return out


# ------------------------------------------------------------------ collection (GPU)
def collect(path, budget_s=900.0, reps=3, dtypes=("f32", "bool"), graphs=True, only=None):
    import torch

    import gen
    import paper_2006_16767_gb300 as asv
    dev = torch.device("cuda")
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    t_start = time.time()
    out = open(path, "a")
    for name, make in corpus():
        if time.time() - t_start > budget_s:
            break
        if only and name not in only:
            continue
        rp, c, v, n = make()
        m = len(rp) - 1
        rpt, ct = torch.from_numpy(rp).to(dev), torch.from_numpy(c).to(dev)
        for dt in dtypes:
            vt = torch.from_numpy(np.asarray(v, np.float32)).to(dev) if dt == "f32" else None
            A = asv.Matrix(m, n, rpt, ct, vt)
            tdt = A.tdtype
            y = torch.empty(m, dtype=tdt, device=dev)
            yidx = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
            yval = torch.empty(max(m, 1), dtype=tdt, device=dev)
            nnz_y = torch.zeros(1, dtype=torch.int64, device=dev)
            for rho, idx in vectors(name, rp, c, n, m):
                if time.time() - t_start > budget_s:
                    break
                it = torch.from_numpy(idx).to(dev)
                if dt == "f32":
                    xv = torch.from_numpy(gen.uniform(len(idx), -1, 1, 5, 2, np.float32)).to(dev)
                    xd = torch.zeros(n, dtype=tdt, device=dev)
                    xd[it.long()] = xv
                else:
                    xv = None
                    xd = torch.zeros(n, dtype=tdt, device=dev)
                    xd[it.long()] = 1
                cnt = torch.tensor([len(idx)], dtype=torch.int64, device=dev)
                for xs in (0, 1):
                    _, vf = asv.asv_select(A.handle, cnt, it, xv, None if xs else xd)
                    feats = [float(A.features()[f]) for f in FEATURES[:9]] + [
                        float(vf["nnz_x"]), float(vf["x_sparsity"]), float(vf["nnz_s"]), float(vf["m_sparsity"])]
                    for om in (0, 1):
                        kid, _ = asv.asv_select(A.handle, cnt, it, xv, None if xs else xd, out_mode=om)
                        times = [None] * NK
                        best = float("inf")
                        for kk in range(NK):
                            def call():
                                if om == 0:
                                    asv.asv_spmspv(A.handle, cnt, it, xv, None if xs else xd, 0, y, kernel=kk)
                                else:
                                    asv.asv_spmspv(A.handle, cnt, it, xv, None if xs else xd, 1, None, yidx,
                                                   yval, nnz_y, m, kernel=kk)
                            call()
                            # the candidate as one CUDA graph launch, as the
                            # selector-driven call runs it (a forced call from
                            # the host adds a host launch per kernel)
                            run = call
                            if graphs:
                                try:
                                    torch.cuda.synchronize()
                                    g = torch.cuda.CUDAGraph()
                                    with torch.cuda.graph(g):
                                        call()
                                    run = g.replay
                                except RuntimeError:
                                    torch.cuda.synchronize()
                                    run = call
                            ts = []
                            for r in range(reps):
                                flush.zero_()
                                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                                e0.record()
                                run()
                                e1.record()
                                torch.cuda.synchronize()
                                ts.append(e0.elapsed_time(e1))
                                if ts[-1] > 30 * best:
                                    break
                            times[kk] = float(np.median(ts))
                            best = min(best, times[kk])
                        out.write(json.dumps({"matrix": name, "dtype": dt, "fmt": 2 * xs + om, "rho": rho,
                                              "feat": feats, "t": times, "auto": kid}) + "\n")
                out.flush()
            A.close()
    out.close()


# ------------------------------------------------------------------ labels and fitting (host)
def labels(times):
    """Per-model labels of one sample (Sec. V-B readings): the pattern of the
    fastest kernel; for each pattern, its fastest distribution (for push at
    its best write-back); the fastest write-back at the best push distribution."""
    t = np.asarray([x if x is not None else np.inf for x in times])

    def pick(cands):
        best = min(t[k] for k in cands)
        for k in sorted(cands):
            if t[k] <= best * TIE:
                return k
        return min(cands, key=lambda k: t[k])

    pat = kernel_parts(pick(range(NK)))[0]
    dists = []
    for p in range(3):
        in_p = [k for k in range(NK) if kernel_parts(k)[0] == p]
        dists.append(kernel_parts(pick(in_p))[1])
    wb = kernel_parts(pick([kernel_id(0, dists[0], w) for w in range(3)]))[2]
    return pat, dists[0], dists[1], dists[2], wb


def load(path):
    rows = [json.loads(l) for l in open(path) if l.strip()]
    return [r for r in rows if all(x is not None for x in r["t"])]


# feature columns of the five trees of a format: pattern (Table 1 model 1),
# distribution after push / masked pull / pull (model 2, here with the vector
# features too: which split is best for push depends on x), write-back (model 3)
TREE_FEATURES = (MODEL_FEATURES[0], tuple(range(13)), tuple(range(13)), tuple(range(13)), MODEL_FEATURES[2])


def _fit_one(X, y, seed, leaf_nodes=(8, 16, 24)):
    from sklearn.model_selection import GridSearchCV, train_test_split
    from sklearn.tree import DecisionTreeClassifier
    if len(set(y.tolist())) < 2 or len(y) < 10:
        leaf = int(np.bincount(y).argmax()) if len(y) else 0
        return None, leaf, 1.0
    Xtr, Xte, ytr, yte = train_test_split(X, y, test_size=0.3, random_state=seed)
    folds = max(2, min(5, int(np.bincount(ytr).min()) if len(set(ytr.tolist())) > 1 else 2))
    # max_leaf_nodes keeps the 20 trees of a value type within the selector's
    # 2048-node table (at most 47 nodes each, 135 for a cost-ordered one)
    gs = GridSearchCV(DecisionTreeClassifier(random_state=seed),
                      {"max_depth": list(range(1, 11)), "class_weight": [None, "balanced"],
                       "max_leaf_nodes": list(leaf_nodes)}, cv=folds)
    gs.fit(Xtr, ytr)
    acc = float(gs.score(Xte, yte))
    clf = DecisionTreeClassifier(random_state=seed, **gs.best_params_).fit(X, y)
    return clf, None, acc


# Features a listed x gives without a pass over it: the matrix features,
# nnz_x and x_sparsity (nnz_s and m_sparsity need the list's column pointers).
CHEAP = tuple(range(11))
# the trees a lazy decision walks: pattern, then the masked-pull or pull
# distribution (the push kernels the lazy path may run need no other tree)
LAZY_TREES = (0, 2, 3)


def _fit_cost_ordered(X, y, cols, seed, impure=0.05, min_leaf=20):
    """A tree whose upper levels test only the cheap features (Sec. VI-C:
    rules on cheap features first): a CART tree fitted on the cheap columns,
    whose leaves that still mix labels (more than `impure` of their samples
    off the majority) are replaced by a small tree fitted on every column of
    the tree's samples there. Returns (nodes, accuracy of stage one)."""
    from sklearn.tree import DecisionTreeClassifier
    c1 = [c for c in cols if c in CHEAP]
    clf1, leaf1, acc1 = _fit_one(X[:, c1], y, seed, leaf_nodes=(4, 8))
    if clf1 is None:
        return [(-1, 0.0, 0, 0, leaf1)], acc1
    out = export_tree(clf1, c1)
    leaves = clf1.apply(X[:, c1])
    for li in sorted(set(leaves.tolist())):
        sel = leaves == li
        ys = y[sel]
        if len(ys) < min_leaf or len(set(ys.tolist())) < 2:
            continue
        if float(np.mean(ys != np.bincount(ys).argmax())) <= impure:
            continue
        clf2 = DecisionTreeClassifier(random_state=seed, max_leaf_nodes=8, min_samples_leaf=3).fit(X[sel][:, cols], ys)
        sub = export_tree(clf2, cols)
        base = len(out)
        # sub's root takes the leaf's place; its other nodes are appended
        remap = lambda c: base + c - 1  # noqa: E731
        f, thr, l, r, lf = sub[0]
        out[li] = (f, thr, remap(l), remap(r), lf) if f >= 0 else sub[0]
        for (f, thr, l, r, lf) in sub[1:]:
            out.append((f, thr, remap(l), remap(r), lf) if f >= 0 else (f, thr, 0, 0, lf))
    return out, acc1


def fit(path, seed=0, rows=None, cost_ordered=False):
    import warnings
    warnings.filterwarnings("ignore")
    rows = rows if rows is not None else load(path)
    result, report = {}, {}
    for dt in sorted({r["dtype"] for r in rows}):
        nodes, roots = [], []
        for fmt in range(4):
            sub = [r for r in rows if r["dtype"] == dt and r["fmt"] == fmt]
            X = np.asarray([r["feat"] for r in sub], np.float64)
            Y = np.asarray([labels(r["t"]) for r in sub], np.int64).reshape(-1, 5)
            for tree in range(5):
                cols = TREE_FEATURES[tree]
                if cost_ordered and fmt >= 2 and tree in LAZY_TREES and len(sub):
                    nodes_m, acc = _fit_cost_ordered(X, Y[:, tree], cols, seed)
                else:
                    clf, leaf, acc = _fit_one(X[:, cols] if len(sub) else X, Y[:, tree], seed)
                    nodes_m = export_tree(clf, cols) if clf is not None else [(-1, 0.0, 0, 0, leaf)]
                base = len(nodes)
                for (f, thr, l, r, lf) in nodes_m:
                    nodes.append((f, thr, l + base if f >= 0 else 0, r + base if f >= 0 else 0, lf))
                roots.append(base)
                report[f"{dt}/fmt{fmt}/tree{tree}"] = {"test_accuracy": round(acc, 4), "samples": len(sub),
                                                        "nodes": len(nodes_m)}
        result[dt] = {"nodes": nodes, "roots": roots}
    return result, report


def export_tree(clf, cols):
    t = clf.tree_
    out = []
    for i in range(t.node_count):
        if t.children_left[i] == -1:
            out.append((-1, 0.0, 0, 0, int(clf.classes_[int(np.argmax(t.value[i][0]))])))
        else:
            out.append((int(cols[t.feature[i]]), float(t.threshold[i]), int(t.children_left[i]),
                        int(t.children_right[i]), 0))
    return out


def predict(trees, dt, fmt, feat):
    T = trees[dt if dt in trees else "f32"]
    nodes, roots = T["nodes"], T["roots"]

    def walk(root):
        i = root
        while nodes[i][0] >= 0:
            f, thr, l, r, _ = nodes[i]
            i = l if feat[f] <= thr else r
        return nodes[i][4]
    r = roots[5 * fmt: 5 * fmt + 5]
    pat = min(max(walk(r[0]), 0), 2)
    dist = walk(r[1 + pat])
    wb = walk(r[4]) if pat == 0 else 0
    return kernel_id(pat, dist, wb)


def regret(path, trees, rows=None):
    rows = rows if rows is not None else load(path)
    out = {}
    for r in rows:
        k = predict(trees, r["dtype"], r["fmt"], r["feat"])
        best = min(r["t"])
        out.setdefault((r["dtype"], r["fmt"]), []).append(r["t"][k] / best)
    return {f"{dt}/fmt{f}": {"mean": round(float(np.mean(v)), 4), "p90": round(float(np.percentile(v, 90)), 4),
                             "max": round(float(np.max(v)), 4), "samples": len(v)}
            for (dt, f), v in sorted(out.items())}


def lazy_walk(trees, dt, fmt, feat):
    """The device's lazy decision for a listed x (Sec. VI-C): the kernel the
    trees pick from the cheap features alone, or None when the path needs
    nnz_s / m_sparsity or the kernel reads them (every push kernel but the
    warp push with atomics)."""
    if fmt < 2:
        return None
    T = trees[dt if dt in trees else "f32"]
    nodes, roots = T["nodes"], T["roots"]

    def walk(root):
        i = root
        while nodes[i][0] >= 0:
            f, thr, l, r, _ = nodes[i]
            if f not in CHEAP:
                return None
            i = l if feat[f] <= thr else r
        return nodes[i][4]
    r = roots[5 * fmt: 5 * fmt + 5]
    pat = walk(r[0])
    if pat is None:
        return None
    pat = min(max(pat, 0), 2)
    dist = walk(r[1 + pat])
    wb = walk(r[4]) if pat == 0 else 0
    if dist is None or wb is None:
        return None
    k = kernel_id(pat, dist, wb)
    return k if k <= 5 or k == 7 else None


def lazy_fraction(trees, rows):
    """Share of the listed-x samples the lazy walk decides, per value type."""
    out = {}
    for dt in sorted({r["dtype"] for r in rows}):
        sub = [r for r in rows if r["dtype"] == dt and r["fmt"] >= 2]
        got = [lazy_walk(trees, dt, r["fmt"], r["feat"]) is not None for r in sub]
        out[dt] = round(float(np.mean(got)), 4) if got else 0.0
    return out


def held_out(path, seed=0):
    """Regret on each corpus matrix with the trees fitted on the others."""
    rows = load(path)
    out = {}
    for mname in sorted({r["matrix"] for r in rows}):
        train = [r for r in rows if r["matrix"] != mname]
        test = [r for r in rows if r["matrix"] == mname]
        trees, _ = fit(None, seed, rows=train)
        reg = [r["t"][predict(trees, r["dtype"], r["fmt"], r["feat"])] / min(r["t"]) for r in test]
        out[mname] = {"mean": round(float(np.mean(reg)), 3), "max": round(float(np.max(reg)), 3)}
    return out


def emit(trees, path=None):
    """C header with one node table and 12 roots per value type."""
    path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc", "trees_default.h")
    lines = ["// Decision trees compiled into the library as its default selector,",
             "// trained on this GPU by paper_2006_16767_gb300/selector_train.py (do not edit).",
             "// Records: {feature, threshold, left, right, leaf_class}; feature < 0 = leaf.",
             "// Feature ids: 0 m, 1 n, 2 nnz, 3 max_row, 4 min_row, 5 avg_row,",
             "// 6 relative_range, 7 var_nnz_row, 8 gini, 9 nnz_x, 10 x_sparsity,",
             "// 11 nnz_s, 12 m_sparsity. Roots, five per call format -- pattern, distribution",
             "// after push / masked pull / pull, write-back -- for (x dense, y dense),",
             "// (x dense, y list), (x list, y dense), (x list, y list).",
             "#pragma once", "", "namespace asv {", ""]
    for dt in ("f32", "bool"):
        T = trees.get(dt) or trees["f32"]
        name = "F32" if dt == "f32" else "Bool"
        lines.append(f"static const int kTreeNodes{name} = {len(T['nodes'])};")
        lines.append(f"static const double kTrees{name}[][5] = {{")
        for (f, thr, l, r, leaf) in T["nodes"]:
            lines.append(f"    {{{f}, {thr!r}, {l}, {r}, {leaf}}},")
        lines.append("};")
        lines.append(f"static const int kTreeRoots{name}[20] = {{{', '.join(str(x) for x in T['roots'])}}};")
        lines.append("")
    lines += ["}  // namespace asv", ""]
    open(path, "w").write("\n".join(lines))
    return path


def compare(path, seed=0):
    """The model comparison of Sec. V-B / Table 2 on this corpus: decision
    trees (what the device walks) against SVM, random forest and gradient
    boosting, each per (value type, format, model), on the same 7:3 split.
    Reports test accuracy per model, the selection regret those predictions
    give on the test samples (time of the predicted kernel / fastest), and the
    host-side latency of predicting one sample."""
    import warnings
    warnings.filterwarnings("ignore")
    from sklearn.ensemble import GradientBoostingClassifier, RandomForestClassifier
    from sklearn.model_selection import train_test_split
    from sklearn.pipeline import make_pipeline
    from sklearn.preprocessing import FunctionTransformer, StandardScaler
    from sklearn.svm import SVC
    from sklearn.tree import DecisionTreeClassifier
    rows = load(path)
    log = FunctionTransformer(lambda X: np.log1p(np.abs(X)))
    families = {
        "decision_tree": lambda: DecisionTreeClassifier(random_state=seed, max_depth=8, max_leaf_nodes=24),
        "svm_rbf": lambda: make_pipeline(log, StandardScaler(), SVC(C=10.0, gamma="scale")),
        "random_forest": lambda: RandomForestClassifier(n_estimators=100, random_state=seed),
        "gradient_boosting": lambda: GradientBoostingClassifier(random_state=seed),
    }
    report = {}
    for dt in sorted({r["dtype"] for r in rows}):
        for fmt in range(4):
            sub = [r for r in rows if r["dtype"] == dt and r["fmt"] == fmt]
            X = np.asarray([r["feat"] for r in sub], np.float64)
            Y = np.asarray([labels(r["t"]) for r in sub], np.int64).reshape(-1, 5)
            T = np.asarray([[x if x is not None else np.inf for x in r["t"]] for r in sub])
            itr, ite = train_test_split(np.arange(len(sub)), test_size=0.3, random_state=seed)
            for fam, make in families.items():
                pred = np.zeros((len(ite), 5), np.int64)
                accs, lat = [], []
                for tree in range(5):
                    cols = list(TREE_FEATURES[tree])
                    y = Y[:, tree]
                    if len(set(y[itr].tolist())) < 2:
                        pred[:, tree] = int(np.bincount(y[itr]).argmax())
                        accs.append(float(np.mean(pred[:, tree] == y[ite])))
                        continue
                    clf = make().fit(X[itr][:, cols], y[itr])
                    pred[:, tree] = clf.predict(X[ite][:, cols])
                    accs.append(float(np.mean(pred[:, tree] == y[ite])))
                    one = X[ite[:1]][:, cols]
                    t0 = time.perf_counter()
                    for _ in range(50):
                        clf.predict(one)
                    lat.append((time.perf_counter() - t0) / 50)
                reg = []
                for q, i in enumerate(ite):
                    pat = int(pred[q, 0])
                    dist = int(pred[q, 1 + pat])
                    k = kernel_id(pat, dist, int(pred[q, 4]) if pat == 0 else 0)
                    reg.append(T[i, k] / np.min(T[i]))
                e = report.setdefault(fam, {"accuracy": [], "regret": [], "latency_us": []})
                e["accuracy"].append(accs)
                e["regret"] += reg
                e["latency_us"] += [x * 1e6 for x in lat]
    out = {}
    for fam, e in report.items():
        A = np.asarray(e["accuracy"])
        out[fam] = {"accuracy_pattern": round(float(A[:, 0].mean()), 4),
                    "accuracy_distribution": round(float(A[:, 1:4].mean()), 4),
                    "accuracy_writeback": round(float(A[:, 4].mean()), 4),
                    "regret_mean": round(float(np.mean(e["regret"])), 4),
                    "regret_p90": round(float(np.percentile(e["regret"], 90)), 4),
                    "host_predict_us_per_model": round(float(np.median(e["latency_us"])), 1)}
    return out


if __name__ == "__main__":
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    cmd = sys.argv[1]
    if cmd == "collect":
        collect(sys.argv[2], budget_s=float(sys.argv[3]) if len(sys.argv) > 3 else 900.0,
                only=sys.argv[4].split(",") if len(sys.argv) > 4 else None)
    elif cmd == "fit":
        trees, rep = fit(sys.argv[2], cost_ordered="--cost-ordered" in sys.argv)
        print(json.dumps(rep, indent=1))
        print(json.dumps(regret(sys.argv[2], trees), indent=1))
        print(json.dumps({"lazy_fraction": lazy_fraction(trees, load(sys.argv[2]))}))
        if "--held-out" in sys.argv:
            print(json.dumps(held_out(sys.argv[2]), indent=1))
        if "--emit" in sys.argv:
            print(emit(trees))
    elif cmd == "compare":
        print(json.dumps(compare(sys.argv[2]), indent=1))
