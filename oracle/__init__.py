"""ORACLE -- TEST INFRASTRUCTURE ONLY.

Plain, serial, FP64 CPU statement of what the adaptive SpMV/SpMSpV path
computes, written from the paper (Li, Ao, Yang, arXiv 2006.16767). Only the
test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg
may import this package; the library's product path never does, and this
package imports nothing from the library. All arithmetic is in ``oracle.c``
(compiled on first use with the host C compiler); this file only marshals
numpy arrays (FP32 inputs are widened exactly to FP64 here).

Function -> passage:
  csr_pull           Sec. II problem statement; Sec. IV-A solution (3,6) "SpMV"
  spmspv_rowmajor    Sec. IV-A solution (3,5), effective nonzeros of Sec. II
  csc_push           Sec. IV-A solution (2,8), column-major SpMSpV
  csc_pull           adjoint A^T v through the CSC arrays (backward form)
  csr_to_csc         Sec. VI-A, both CSR and CSC stored
  compact            Sec. II vector formats; Sec. VI-A online conversion
  matrix_features    Table 1 (rows m .. G_c), Sec. V-A
  vector_features    Table 1 (rows nnz_x .. m_sparsity), Sec. V-A
  bool_pull, bfs     BFS application, Sec. I and Sec. VII
  i32_pull           integer (+, x) semiring, 32-bit wrap-around
  pagerank_step      PageRank application, Sec. VII (formula is a reading)
  grad_values        dA on A's pattern, dA_k = dy_row(k) * x_col(k)
  csr_pull_par, spmspv_rowmajor_par, csc_push_par
                     the same three products with their outer loop on all
                     host cores (oracle_omp.c), for the CPU baseline only

The kernel selector has no oracle (parity unpinned): the paper prints no
decision rules or thresholds (Sec. V-B, VI-B).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FEATURE_NAMES = ("m", "n", "nnz", "max_row", "min_row", "avg_row",
                 "relative_range", "var_nnz_row", "gini")
VECTOR_FEATURE_NAMES = ("nnz_x", "x_sparsity", "nnz_s", "m_sparsity")


def _elf_matches_host(path: str) -> bool:
    """True when the shared object at `path` was built for this machine."""
    import platform
    import struct
    want = {"x86_64": 0x3E, "aarch64": 0xB7, "arm64": 0xB7}.get(platform.machine())
    try:
        with open(path, "rb") as f:
            head = f.read(20)
    except OSError:
        return False
    if len(head) < 20 or head[:4] != b"\x7fELF":
        return False
    return want is None or struct.unpack("<H", head[18:20])[0] == want


def build(force: bool = False) -> str:
    """Compile oracle.c (serial, -O2, no fast-math) into liboracle.so."""
    if not force and _elf_matches_host(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fno-fast-math", "-ffp-contract=off",
                    "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _get():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            vp, i64 = ctypes.c_void_p, ctypes.c_int64
            lib.oracle_csr_pull.argtypes = [i64, vp, vp, vp, vp, vp, vp]
            lib.oracle_spmspv_rowmajor.argtypes = [i64, i64, vp, vp, vp, i64, vp, vp, vp, vp, vp]
            lib.oracle_csc_push.argtypes = [i64, vp, vp, vp, i64, vp, vp, vp, vp]
            lib.oracle_csc_pull.argtypes = [i64, vp, vp, vp, vp, vp, vp]
            lib.oracle_csr_to_csc.argtypes = [i64, i64, vp, vp, vp, vp, vp]
            lib.oracle_compact.argtypes = [i64, vp, vp, vp]
            lib.oracle_compact.restype = i64
            lib.oracle_matrix_features.argtypes = [i64, i64, vp, vp]
            lib.oracle_vector_features.argtypes = [i64, i64, vp, i64, vp, vp]
            lib.oracle_bool_pull.argtypes = [i64, vp, vp, vp, vp]
            lib.oracle_i32_pull.argtypes = [i64, vp, vp, vp, vp, vp]
            lib.oracle_bfs.argtypes = [i64, vp, vp, ctypes.c_int32, vp]
            lib.oracle_bfs.restype = ctypes.c_int32
            lib.oracle_pagerank_step.argtypes = [i64, vp, vp, vp, vp, ctypes.c_double, vp, vp, vp]
            lib.oracle_grad_values.argtypes = [i64, vp, vp, vp, vp, vp]
            _lib = lib
    return _lib


_SRC_PAR = os.path.join(_HERE, "oracle_omp.c")
_SO_PAR = os.path.join(_HERE, "liboracle_omp.so")
_lib_par = None


def build_par(force: bool = False) -> str:
    """Compile oracle_omp.c (the multi-threaded CPU-baseline forms) into
    liboracle_omp.so with OpenMP."""
    if not force and _elf_matches_host(_SO_PAR) and os.path.getmtime(_SO_PAR) >= os.path.getmtime(_SRC_PAR):
        return _SO_PAR
    tmp = _SO_PAR + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
                    "-shared", "-fPIC", _SRC_PAR, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _SO_PAR)
    return _SO_PAR


def _get_par():
    global _lib_par
    with _lock:
        if _lib_par is None:
            build_par()
            lib = ctypes.CDLL(_SO_PAR)
            vp, i64 = ctypes.c_void_p, ctypes.c_int64
            lib.oracle_par_threads.argtypes = []
            lib.oracle_par_threads.restype = ctypes.c_int
            lib.oracle_csr_pull_par.argtypes = [i64, vp, vp, vp, vp, vp, vp]
            lib.oracle_spmspv_rowmajor_par.argtypes = [i64, i64, vp, vp, vp, i64, vp, vp, vp, vp, vp]
            lib.oracle_csc_push_par.argtypes = [i64, vp, vp, vp, i64, vp, vp, vp, vp]
            _lib_par = lib
    return _lib_par


def par_threads() -> int:
    """Threads the multi-threaded forms use (OMP_NUM_THREADS or all cores)."""
    return int(_get_par().oracle_par_threads())


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def csr_pull(rowptr, col, val, x):
    """y = A x over CSR (val None = pattern). Returns (y, s) with s_i = sum|a x|."""
    rowptr, col, val, x = _i32(rowptr), _i32(col), _f64(val), _f64(x)
    m = len(rowptr) - 1
    y = np.empty(m, np.float64)
    s = np.empty(m, np.float64)
    _get().oracle_csr_pull(m, _p(rowptr), _p(col), _p(val), _p(x), _p(y), _p(s))
    return y, s


def spmspv_rowmajor(n, rowptr, col, val, xidx, xval):
    """Row-major SpMSpV with validation. Returns (y, s, hit[uint8])."""
    rowptr, col, val, xidx, xval = _i32(rowptr), _i32(col), _f64(val), _i32(xidx), _f64(xval)
    m = len(rowptr) - 1
    y = np.empty(m, np.float64)
    s = np.empty(m, np.float64)
    hit = np.empty(m, np.uint8)
    _get().oracle_spmspv_rowmajor(m, n, _p(rowptr), _p(col), _p(val), len(xidx), _p(xidx),
                                  _p(xval), _p(y), _p(s), _p(hit))
    return y, s, hit


def csr_pull_par(rowptr, col, val, x):
    """csr_pull on all host cores (rows divided among threads; identical result)."""
    rowptr, col, val, x = _i32(rowptr), _i32(col), _f64(val), _f64(x)
    m = len(rowptr) - 1
    y = np.empty(m, np.float64)
    s = np.empty(m, np.float64)
    _get_par().oracle_csr_pull_par(m, _p(rowptr), _p(col), _p(val), _p(x), _p(y), _p(s))
    return y, s


def spmspv_rowmajor_par(n, rowptr, col, val, xidx, xval):
    """spmspv_rowmajor on all host cores (rows divided among threads)."""
    rowptr, col, val, xidx, xval = _i32(rowptr), _i32(col), _f64(val), _i32(xidx), _f64(xval)
    m = len(rowptr) - 1
    y = np.empty(m, np.float64)
    s = np.empty(m, np.float64)
    hit = np.empty(m, np.uint8)
    _get_par().oracle_spmspv_rowmajor_par(m, n, _p(rowptr), _p(col), _p(val), len(xidx), _p(xidx),
                                          _p(xval), _p(y), _p(s), _p(hit))
    return y, s, hit


def csc_push_par(m, colptr, rowidx, val, xidx, xval):
    """csc_push on all host cores (listed columns divided among threads,
    atomic additions into y)."""
    colptr, rowidx, val, xidx, xval = _i32(colptr), _i32(rowidx), _f64(val), _i32(xidx), _f64(xval)
    y = np.empty(m, np.float64)
    touched = np.empty(m, np.uint8)
    _get_par().oracle_csc_push_par(m, _p(colptr), _p(rowidx), _p(val), len(xidx), _p(xidx), _p(xval),
                                   _p(y), _p(touched))
    return y, touched


def csc_push(m, colptr, rowidx, val, xidx, xval):
    """Column-major SpMSpV. Returns (y, touched[uint8])."""
    colptr, rowidx, val, xidx, xval = _i32(colptr), _i32(rowidx), _f64(val), _i32(xidx), _f64(xval)
    y = np.empty(m, np.float64)
    t = np.empty(m, np.uint8)
    _get().oracle_csc_push(m, _p(colptr), _p(rowidx), _p(val), len(xidx), _p(xidx), _p(xval),
                           _p(y), _p(t))
    return y, t


def csc_pull(colptr, rowidx, val, v):
    """A^T v through CSC arrays. Returns (out, s)."""
    colptr, rowidx, val, v = _i32(colptr), _i32(rowidx), _f64(val), _f64(v)
    n = len(colptr) - 1
    out = np.empty(n, np.float64)
    s = np.empty(n, np.float64)
    _get().oracle_csc_pull(n, _p(colptr), _p(rowidx), _p(val), _p(v), _p(out), _p(s))
    return out, s


def csr_to_csc(m, n, rowptr, col):
    """Stable counting-sort transpose. Returns (colptr, rowidx, perm)."""
    rowptr, col = _i32(rowptr), _i32(col)
    nnz = int(rowptr[m]) if m > 0 else 0
    colptr = np.empty(n + 1, np.int32)
    rowidx = np.empty(max(nnz, 1), np.int32)
    perm = np.empty(max(nnz, 1), np.int32)
    _get().oracle_csr_to_csc(m, n, _p(rowptr), _p(col), _p(colptr), _p(rowidx), _p(perm))
    return colptr, rowidx[:nnz], perm[:nnz]


def compact(x):
    """Ascending indices of x_j != 0 (IEEE) and their values (as float64)."""
    x = _f64(x)
    n = len(x)
    idx = np.empty(max(n, 1), np.int32)
    val = np.empty(max(n, 1), np.float64)
    c = _get().oracle_compact(n, _p(x), _p(idx), _p(val))
    return idx[:c].copy(), val[:c].copy()


def matrix_features(m, n, rowptr):
    rowptr = _i32(rowptr)
    out = np.empty(9, np.float64)
    _get().oracle_matrix_features(m, n, _p(rowptr), _p(out))
    return dict(zip(FEATURE_NAMES, out.tolist()))


def vector_features(n, nnz, colptr, xidx):
    colptr, xidx = _i32(colptr), _i32(xidx)
    out = np.empty(4, np.float64)
    _get().oracle_vector_features(n, nnz, _p(colptr), len(xidx), _p(xidx), _p(out))
    return dict(zip(VECTOR_FEATURE_NAMES, out.tolist()))


def bool_pull(rowptr, col, x):
    """(OR, AND) product over a pattern matrix; x, y as uint8 0/1."""
    rowptr, col = _i32(rowptr), _i32(col)
    x = np.ascontiguousarray(x, dtype=np.uint8)
    m = len(rowptr) - 1
    y = np.empty(m, np.uint8)
    _get().oracle_bool_pull(m, _p(rowptr), _p(col), _p(x), _p(y))
    return y


def i32_pull(rowptr, col, val, x):
    """Integer (+, x) product with 32-bit wrap-around."""
    rowptr, col, x = _i32(rowptr), _i32(col), _i32(x)
    val = None if val is None else _i32(val)
    m = len(rowptr) - 1
    y = np.empty(m, np.int32)
    _get().oracle_i32_pull(m, _p(rowptr), _p(col), _p(val), _p(x), _p(y))
    return y


def bfs(n, rowptr, col, root):
    """Queue BFS. Returns (level[int32], number_of_levels)."""
    rowptr, col = _i32(rowptr), _i32(col)
    level = np.empty(n, np.int32)
    L = _get().oracle_bfs(n, _p(rowptr), _p(col), int(root), _p(level))
    return level, int(L)


def frontiers(n, rowptr, col, root):
    """Successive BFS frontiers {v : level(v) = l}, each ascending (int32)."""
    level, L = bfs(n, rowptr, col, root)
    order = np.argsort(level, kind="stable")
    lv = level[order]
    out = []
    for l in range(L):
        lo, hi = np.searchsorted(lv, l, "left"), np.searchsorted(lv, l, "right")
        out.append(np.sort(order[lo:hi]).astype(np.int32))
    return out


def pagerank_step(N, rowptr, col, colptr, r, d=0.85):
    """One PageRank step. Returns (x, y, r_next)."""
    rowptr, col, colptr, r = _i32(rowptr), _i32(col), _i32(colptr), _f64(r)
    x = np.empty(N, np.float64)
    y = np.empty(N, np.float64)
    rn = np.empty(N, np.float64)
    _get().oracle_pagerank_step(N, _p(rowptr), _p(col), _p(colptr), _p(r), d, _p(x), _p(y), _p(rn))
    return x, y, rn


def pagerank_delta(n, rowptr, col, val, d, eps, max_iter):
    """Delta-form (incremental) PageRank, Sec. VII's incremental PageRank
    application read as: rank = sum of delta_k, delta_0 = (1 - d)/N on every
    vertex, delta_{k+1} = d A D^{-1} delta_k with D the column counts (a
    column with none contributes 0), entries with |delta| < eps dropped after
    each product. Each product is the oracle's row-major SpMSpV; the output
    set is the structural one. Returns (rank, products run, the smallest
    | |delta| - eps | / eps met, i.e. how far any keep/drop decision was
    from the threshold)."""
    rowptr, col = _i32(rowptr), _i32(col)
    val = None if val is None else _f64(val)
    deg = np.bincount(col, minlength=n).astype(np.float64)
    r = np.full(n, (1.0 - d) / n)
    idx = np.arange(n, dtype=np.int32)
    dv = r.copy()
    margin = np.inf
    it = 0
    for it in range(1, max_iter + 1):
        xv = np.where(deg[idx] > 0, dv / np.maximum(deg[idx], 1.0), 0.0)
        y, _, hit = spmspv_rowmajor(n, rowptr, col, val, idx, xv)
        rows = np.flatnonzero(hit).astype(np.int32)
        dnew = d * y[rows]
        r[rows] += dnew
        if eps > 0 and len(dnew):
            margin = min(margin, float(np.min(np.abs(np.abs(dnew) - eps)) / eps))
        keep = np.abs(dnew) >= eps
        idx, dv = rows[keep], dnew[keep]
        if len(idx) == 0:
            break
    else:
        it = max_iter
    return r, it, margin


def grad_values(rowptr, col, dy, x):
    """dA_k = dy[row(k)] * x[col_k] in CSR order."""
    rowptr, col, dy, x = _i32(rowptr), _i32(col), _f64(dy), _f64(x)
    m = len(rowptr) - 1
    nnz = int(rowptr[m]) if m > 0 else 0
    dA = np.empty(max(nnz, 1), np.float64)
    _get().oracle_grad_values(m, _p(rowptr), _p(col), _p(dy), _p(x), _p(dA))
    return dA[:nnz]
