"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module builds matrices and vectors only: it contains none of the method's
arithmetic. The heavy lifting is in ``gen.c`` (compiled on first use with the
host C compiler into ``libasvgen.so`` next to this file).

Workload recipes (stand-ins for the paper's datasets, Sec. VII Table 3, which
are not available here):

* ``laplace2d``     -- 2-D 5-point Laplacian (mesh / high-diameter class).
* ``stencil27``     -- 3-D 27-point stencil, diagonally dominant.
* ``rmat``          -- R-MAT graph, symmetrised and deduplicated (low-diameter class).
* ``lognormal_zipf``-- ML-style data matrix (lognormal row lengths, Zipf columns).
* ``bernoulli``     -- uniform random pattern with N(0, std) values (pruned layer).
* ``sparse_x``      -- input vectors with uniformly random nonzero positions.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_SO = os.path.join(_HERE, "libasvgen.so")
_lock = threading.Lock()
_lib = None

CONFIG_SEED_BASE = 20061676


def config_seed(k: int) -> int:
    """Base seed of workload configuration k (k = 1..5)."""
    return CONFIG_SEED_BASE + k


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
    """Compile gen.c into libasvgen.so (OpenMP if the compiler supports it)."""
    if not force and _elf_matches_host(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _get():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i32p = ctypes.POINTER(ctypes.c_int32)
            i32pp = ctypes.POINTER(i32p)
            f32pp = ctypes.POINTER(ctypes.POINTER(ctypes.c_float))
            vp = ctypes.c_void_p
            i64 = ctypes.c_int64
            u64 = ctypes.c_uint64
            d = ctypes.c_double
            lib.gen_laplace2d.argtypes = [ctypes.c_int32, vp, vp, vp]
            lib.gen_laplace2d.restype = i64
            lib.gen_stencil27_nnz.argtypes = [ctypes.c_int32]
            lib.gen_stencil27_nnz.restype = i64
            lib.gen_stencil27.argtypes = [ctypes.c_int32, u64, vp, vp, vp, vp]
            lib.gen_stencil27.restype = i64
            lib.gen_rmat.argtypes = [ctypes.c_int32, ctypes.c_int32, d, d, d, u64, i32pp, i32pp]
            lib.gen_rmat.restype = i64
            lib.gen_lognormal_zipf.argtypes = [i64, i64, d, d, d, u64, u64, i32pp, i32pp, f32pp]
            lib.gen_lognormal_zipf.restype = i64
            lib.gen_bernoulli.argtypes = [i64, i64, d, d, u64, i32pp, i32pp, f32pp]
            lib.gen_bernoulli.restype = i64
            lib.gen_uniform_f64.argtypes = [i64, d, d, u64, u64, vp]
            lib.gen_uniform_f32.argtypes = [i64, d, d, u64, u64, vp]
            lib.gen_halfnormal_f32.argtypes = [i64, d, u64, u64, vp]
            lib.gen_small_ints_f64.argtypes = [i64, ctypes.c_int32, ctypes.c_int32, d, u64, u64, vp]
            lib.gen_sample_positions.argtypes = [i64, i64, u64, u64, vp]
            lib.gen_randint.argtypes = [i64, i64, u64, u64, vp]
            lib.gen_free.argtypes = [vp]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _take(p, count, dtype):
    """Copy a malloc'ed C array into numpy and free it."""
    if count > 0:
        arr = np.ctypeslib.as_array(p, shape=(count,)).astype(dtype, copy=True)
    else:
        arr = np.zeros(0, dtype=dtype)
    _get().gen_free(ctypes.cast(p, ctypes.c_void_p))
    return arr


# ------------------------------------------------------------------ matrices
def laplace2d(g: int):
    """5-point Laplacian on a g x g grid: (rowptr, col, val[f64]); m = n = g*g."""
    m = g * g
    nnz = 5 * g * g - 4 * g if g > 0 else 0
    rowptr = np.zeros(m + 1, np.int32)
    col = np.zeros(max(nnz, 1), np.int32)
    val = np.zeros(max(nnz, 1), np.float64)
    got = _get().gen_laplace2d(g, _ptr(rowptr), _ptr(col), _ptr(val))
    assert got == nnz
    return rowptr, col[:nnz], val[:nnz]


def stencil27(g: int, seed: int):
    """27-point stencil on a g^3 grid: (rowptr, col, val[f32], rowsum[f64])."""
    lib = _get()
    m = g * g * g
    nnz = lib.gen_stencil27_nnz(g)
    rowptr = np.empty(m + 1, np.int32)
    col = np.empty(nnz, np.int32)
    val = np.empty(nnz, np.float32)
    rowsum = np.empty(m, np.float64)
    got = lib.gen_stencil27(g, seed, _ptr(rowptr), _ptr(col), _ptr(val), _ptr(rowsum))
    assert got == nnz
    return rowptr, col, val, rowsum


def rmat(scale: int, edge_factor: int, seed: int, a=0.57, b=0.19, c=0.19):
    """Symmetrised, deduplicated R-MAT graph without self-loops: (rowptr, col)."""
    lib = _get()
    rp = ctypes.POINTER(ctypes.c_int32)()
    cp = ctypes.POINTER(ctypes.c_int32)()
    nnz = lib.gen_rmat(scale, edge_factor, a, b, c, seed, ctypes.byref(rp), ctypes.byref(cp))
    n = 1 << scale
    return _take(rp, n + 1, np.int32), _take(cp, nnz, np.int32)


def lognormal_zipf(m: int, n: int, mu: float, sigma: float, s: float, seed: int, perm_seed: int | None = None):
    """Rows of lognormal length, Zipf(s) column ids: (rowptr, col, val[f32]).
    perm_seed fixes the rank -> column-id map (default: seed); matrices over
    the same feature space share it."""
    lib = _get()
    rp = ctypes.POINTER(ctypes.c_int32)()
    cp = ctypes.POINTER(ctypes.c_int32)()
    vp = ctypes.POINTER(ctypes.c_float)()
    ps = seed if perm_seed is None else perm_seed
    nnz = lib.gen_lognormal_zipf(m, n, mu, sigma, s, seed, ps, ctypes.byref(rp), ctypes.byref(cp), ctypes.byref(vp))
    return _take(rp, m + 1, np.int32), _take(cp, nnz, np.int32), _take(vp, nnz, np.float32)


def bernoulli(m: int, n: int, p: float, std: float, seed: int):
    """Uniform random pattern (each cell kept w.p. p), N(0, std) values."""
    lib = _get()
    rp = ctypes.POINTER(ctypes.c_int32)()
    cp = ctypes.POINTER(ctypes.c_int32)()
    vp = ctypes.POINTER(ctypes.c_float)()
    nnz = lib.gen_bernoulli(m, n, p, std, seed, ctypes.byref(rp), ctypes.byref(cp), ctypes.byref(vp))
    return _take(rp, m + 1, np.int32), _take(cp, nnz, np.int32), _take(vp, nnz, np.float32)


# ------------------------------------------------------------------ values / positions
def uniform(count: int, lo: float, hi: float, seed: int, stream: int = 0, dtype=np.float64):
    out = np.empty(count, dtype)
    if count:
        fn = _get().gen_uniform_f64 if np.dtype(dtype) == np.float64 else _get().gen_uniform_f32
        assert np.dtype(dtype) in (np.float64, np.float32)
        fn(count, lo, hi, seed, stream, _ptr(out))
    return out


def halfnormal(count: int, scale: float, seed: int, stream: int = 0):
    out = np.empty(count, np.float32)
    if count:
        _get().gen_halfnormal_f32(count, scale, seed, stream, _ptr(out))
    return out


def small_ints(count: int, lo: int, hi: int, den: float, seed: int, stream: int = 0):
    """Integers in [lo, hi] divided by den (float64); exactly representable."""
    out = np.empty(count, np.float64)
    if count:
        _get().gen_small_ints_f64(count, lo, hi, den, seed, stream, _ptr(out))
    return out


def sample_positions(n: int, count: int, seed: int, stream: int = 0):
    """`count` distinct ascending positions in [0, n)."""
    count = min(count, n)
    out = np.empty(count, np.int32)
    if count:
        _get().gen_sample_positions(n, count, seed, stream, _ptr(out))
    return out


def randint(count: int, n: int, seed: int, stream: int = 0):
    out = np.empty(count, np.int64)
    if count:
        _get().gen_randint(count, n, seed, stream, _ptr(out))
    return out


def sparse_x(n: int, nnz_x: int, seed: int, stream: int = 0, dtype=np.float64, lo=-1.0, hi=1.0):
    """Sparse vector: ascending distinct positions, values U(lo, hi)."""
    idx = sample_positions(n, nnz_x, seed, stream)
    val = uniform(len(idx), lo, hi, seed, stream + 17, dtype)
    return idx, val


def densify(n: int, idx, val, dtype=None):
    """Place (idx, val) into a zero vector of length n (input construction only)."""
    val = np.asarray(val)
    x = np.zeros(n, dtype or val.dtype)
    x[np.asarray(idx, np.int64)] = val
    return x


def random_csr(m: int, n: int, density: float, seed: int, values: str = "small", dtype=np.float64):
    """Small random CSR for tests. values='small' draws integers in {-2..2}/4
    (every product and partial sum exactly representable), 'uniform' U(-1, 1),
    'ones' all ones, 'none' returns no values (pattern only)."""
    rowptr, col, _ = bernoulli(m, n, density, 1.0, seed)
    nnz = len(col)
    if values == "small":
        val = small_ints(nnz, -2, 2, 4.0, seed, 1).astype(dtype)
    elif values == "uniform":
        val = uniform(nnz, -1.0, 1.0, seed, 2, np.float64).astype(dtype)
    elif values == "ones":
        val = np.ones(nnz, dtype)
    else:
        val = None
    return rowptr, col, val
