"""Planted mistakes in the oracle: each mutant of oracle.c must fail a pin.

Each case copies the oracle's C source, plants one plausible mistake (a
flipped sign, a dropped or shifted term, a wrong index or denominator, an
overwrite instead of an accumulation, a broken stable order) inside one
function, compiles the copy into a temporary library and runs the pin suite
(tests/test_oracle_pins.py and the C1 fixture check) against it in a child
process. A mutant that passes every pin shows a hole in the pins. Every
mutant keeps its memory accesses in bounds, so a pin fails by assertion,
not by a crash. CPU only; the repository's own oracle is not touched."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "oracle.c")

# (name, function whose body is changed, original text, planted text)
MUTANTS = [
    ("csr_pull sign", "void oracle_csr_pull(", "acc += p;", "acc -= p;"),
    ("csr_pull dropped last term", "void oracle_csr_pull(",
     "k < rowptr[i + 1]; ++k) {", "k < rowptr[i + 1] - 1; ++k) {"),
    ("csr_pull shifted column", "void oracle_csr_pull(",
     "double p = a * x[col[k]];", "double p = a * x[col[k] == 0 ? 0 : col[k] - 1];"),
    ("spmspv without validation", "void oracle_spmspv_rowmajor(", "if (!in[col[k]]) continue;", ""),
    ("csc_push overwrite", "void oracle_csc_push(", "y[rowidx[k]] += a * xj;", "y[rowidx[k]] = a * xj;"),
    ("csc_pull shifted row", "void oracle_csc_pull(",
     "* v[rowidx[k]];", "* v[rowidx[k] == 0 ? 0 : rowidx[k] - 1];"),
    ("transpose unstable", "void oracle_csr_to_csc(",
     "for (int64_t i = 0; i < m; ++i) {", "for (int64_t i = m - 1; i >= 0; --i) {"),
    ("compact NaN as zero", "int64_t oracle_compact(", "if (x[j] != 0.0) {", "if (fabs(x[j]) > 0.0) {"),
    ("relative_range over m", "void oracle_matrix_features(",
     "(double)(mx - mn) / (double)n", "(double)(mx - mn) / (double)m"),
    ("sample std", "void oracle_matrix_features(",
     "sqrt(ss / (double)m)", "sqrt(ss / (double)(m > 1 ? m - 1 : 1))"),
    ("gini weight", "void oracle_matrix_features(", "(2 * i - m - 1)", "(2 * i - m)"),
    ("nnz_s drops a column", "void oracle_vector_features(",
     "for (int64_t t = 0; t < nnz_x; ++t) s +=", "for (int64_t t = 1; t < nnz_x; ++t) s +="),
    ("bool skips first entry", "void oracle_bool_pull(",
     "if (x[col[k]]) { h = 1; break; }", "if (x[col[k]] && k > rowptr[i]) { h = 1; break; }"),
    ("i32 through doubles", "void oracle_i32_pull(",
     "acc += (uint32_t)(val ? val[k] : 1) * (uint32_t)x[col[k]];",
     "acc += (uint32_t)(int64_t)((double)(val ? val[k] : 1) * (double)x[col[k]]);"),
    ("bfs skips a level", "int32_t oracle_bfs(",
     "level[v] = level[u] + 1;", "level[v] = level[u] + (level[u] >= 2 ? 2 : 1);"),
    ("pagerank degree off by one", "void oracle_pagerank_step(",
     "r[j] / (double)deg", "r[j] / (double)(deg + 1)"),
    ("pagerank teleport over m", "void oracle_pagerank_step(",
     "(1.0 - d) / (double)N", "(1.0 - d) / (double)(N + 1)"),
    ("grad sign", "void oracle_grad_values(", "dA[k] = dy[i] * x[col[k]];", "dA[k] = -dy[i] * x[col[k]];"),
]

RUNNER = """
import sys
sys.path.insert(0, {root!r})
import oracle
oracle._SRC, oracle._SO, oracle._lib = {src!r}, {so!r}, None
import pytest
sys.exit(pytest.main(["-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu",
                      "tests/test_oracle_pins.py",
                      "tests/test_golden_c1.py::test_oracle_reproduces_the_c1_fixture"]))
"""


def plant(text, anchor, old, new):
    a = text.index(anchor)
    end = text.find("\n}\n", a)
    body = text[a:end]
    assert body.count(old) == 1, f"{old!r} must occur once in the body of {anchor!r}"
    return text[:a] + body.replace(old, new) + text[end:]


def test_every_planted_text_is_found_once():
    text = open(SRC).read()
    for name, anchor, old, new in MUTANTS:
        assert plant(text, anchor, old, new) != text, name


@pytest.mark.parametrize("name,anchor,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, name, anchor, old, new):
    src = tmp_path / "oracle_mutant.c"
    so = tmp_path / "liboracle_mutant.so"
    src.write_text(plant(open(SRC).read(), anchor, old, new))
    # compiled here, newer than its source, so the oracle loads it as is
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fno-fast-math", "-ffp-contract=off", "-shared", "-fPIC",
                    str(src), "-o", str(so), "-lm"], check=True, capture_output=True)
    r = subprocess.run([sys.executable, "-c", RUNNER.format(root=ROOT, src=str(src), so=str(so))], cwd=ROOT,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 1, f"mutant '{name}' passed every pin (exit {r.returncode}):\n{r.stdout[-2000:]}"
