"""Python binding of the adaptive SpMV/SpMSpV library (C ABI in include/asv.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libasv.so (built by ``build.build()``). PyTorch supplies device
memory and streams; tensors are passed by ``data_ptr()`` and the current CUDA
stream is used unless one is given. There is no CPU fallback: if the shared
library is missing, importing the binding's functions raises.

The functions keep the C names (``asv_spmv``, ``asv_spmspv``, ...); ``Matrix``
is a small owner object that keeps the CSR tensors alive for a borrowed
handle and destroys the handle when collected (a transposed view keeps its
parent alive). ``spmv``, ``spmspv``, ``select``, ``spmspv_batched`` and
``transpose_view`` are the same calls in module form.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libasv.so")

# status codes and enums (mirrors include/asv.h)
ASV_OK, ASV_ERR_ARG, ASV_ERR_NONCANONICAL, ASV_ERR_OVERFLOW, ASV_ERR_CAPACITY = 0, 1, 2, 3, 4
ASV_ERR_TIMEOUT, ASV_ERR_CUDA, ASV_ERR_NOMEM, ASV_ERR_UNSUPPORTED = 5, 6, 8, 9  # 7 is reserved
ASV_F32, ASV_F64, ASV_BOOL, ASV_I32 = 0, 1, 2, 3
ASV_OUT_DENSE, ASV_OUT_SPARSE = 0, 1
ASV_BORROW, ASV_COPY, ASV_VALIDATE = 0, 1, 2
ASV_K_AUTO = -1
KERNELS = ("pull_thread", "pull_warp", "pull_bal", "mpull_thread", "mpull_warp", "mpull_bal",
           "push_thread_atom", "push_warp_atom", "push_bal_atom",
           "push_thread_sort", "push_warp_sort", "push_bal_sort",
           "push_thread_priv", "push_warp_priv", "push_bal_priv")
K = {name: i for i, name in enumerate(KERNELS)}
ASV_K_COUNT = len(KERNELS)
MATRIX_FEATURES = ("m", "n", "nnz", "max_row", "min_row", "avg_row", "relative_range",
                   "var_nnz_row", "gini")

_DT = {torch.float32: ASV_F32, torch.float64: ASV_F64, torch.int32: ASV_I32,
       torch.uint8: ASV_BOOL, torch.bool: ASV_BOOL}
TORCH_DTYPE = {ASV_F32: torch.float32, ASV_F64: torch.float64, ASV_I32: torch.int32, ASV_BOOL: torch.uint8}


class AsvError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} (status {status}, "
                         f"cuda error {lib().asv_last_cuda_error()})")


class AsvTune(ctypes.Structure):
    _fields_ = [("rows_per_tile", ctypes.c_int32), ("vectors_per_group", ctypes.c_int32),
                ("hot_columns", ctypes.c_int32)]


class AsvPullTune(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_int32), ("unroll", ctypes.c_int32), ("tma", ctypes.c_int32)]


class _MFeat(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("max_row", ctypes.c_int64), ("min_row", ctypes.c_int64),
                ("avg_row", ctypes.c_double), ("relative_range", ctypes.c_double),
                ("var_nnz_row", ctypes.c_double), ("gini", ctypes.c_double)]


class _VFeat(ctypes.Structure):
    _fields_ = [("nnz_x", ctypes.c_int64), ("nnz_s", ctypes.c_int64),
                ("x_sparsity", ctypes.c_double), ("m_sparsity", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libasv.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"libasv.so not built at {LIB_PATH}; run paper_2006_16767_gb300.build.build()")
            L = ctypes.CDLL(LIB_PATH)
            vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
            P = ctypes.POINTER
            L.asv_matrix_create_csr.argtypes = [P(vp), i64, i64, i64, vp, vp, vp, i32, ctypes.c_uint32, vp]
            L.asv_matrix_destroy.argtypes = [vp]
            L.asv_matrix_transpose_view.argtypes = [vp, P(vp), vp]
            L.asv_matrix_features.argtypes = [vp, P(_MFeat)]
            L.asv_matrix_arrays.argtypes = [vp] + [P(vp)] * 7
            L.asv_matrix_copy_csc.argtypes = [vp, vp, vp, vp, vp, vp]
            L.asv_spmv.argtypes = [vp, vp, vp, i32, vp]
            L.asv_matrix_update_values.argtypes = [vp, vp, vp]
            L.asv_spmspv_batched.argtypes = [vp, i32, i64, vp, vp, vp, vp, vp, P(AsvTune), vp]
            L.asv_autotune_batched.argtypes = [vp, i32, i64, vp, vp, vp, vp, vp, ctypes.c_char_p, P(AsvTune), vp]
            L.asv_spmspv_backward.argtypes = [vp, i32, vp, vp, vp, vp, vp]
            L.asv_spmv_noalloc_f32.argtypes = [i64, i64, i64, vp, vp, vp, vp, vp, vp]
            L.asv_spmspv.argtypes = [vp, vp, vp, vp, vp, i32, vp, vp, vp, vp, i64, i32, vp]
            L.asv_spmspv_masked.argtypes = [vp, vp, vp, vp, vp, vp, i32, vp, vp, vp, vp, i64, i32, vp]
            L.asv_bfs.argtypes = [vp, i32, vp, i32, P(i32), vp]
            L.asv_pagerank.argtypes = [vp, ctypes.c_double, ctypes.c_double, i32, vp, i32, P(i32), vp]
            L.asv_select.argtypes = [vp, vp, vp, vp, vp, i32, P(i32), P(_VFeat), vp]
            L.asv_last_kernel.argtypes = [vp, P(i32), vp]
            L.asv_compact.argtypes = [vp, vp, vp, vp, vp, vp]
            L.asv_set_trees.argtypes = [vp, vp, i32, vp, vp]
            L.asv_get_status.argtypes = [vp, vp]
            L.asv_last_cuda_error.argtypes = []
            L.asv_status_string.argtypes = [i32]
            L.asv_status_string.restype = ctypes.c_char_p
            L.asv_version.argtypes = []
            L.asv_spmspv_backward_list.argtypes = [vp, i32, vp, vp, vp, vp, vp, vp, vp]
            L.asv_spmspv_backward_list.restype = i32
            L.asv_autotune.argtypes = [vp, ctypes.c_char_p, ctypes.c_uint32, P(AsvPullTune), vp]
            L.asv_autotune.restype = i32
            L.asv_pull_tuning.argtypes = [vp, P(AsvPullTune)]
            L.asv_pull_tuning.restype = i32
            L.asv_debug_set_wait_limit.argtypes = [vp, ctypes.c_uint32]
            L.asv_debug_set_wait_limit.restype = i32
            L.asv_debug_fail_alloc.argtypes = [i32]
            L.asv_debug_fail_alloc.restype = None
            for name in ("asv_matrix_create_csr", "asv_matrix_destroy", "asv_matrix_features",
                         "asv_matrix_arrays", "asv_matrix_copy_csc", "asv_spmv", "asv_spmspv", "asv_select", "asv_last_kernel",
                         "asv_compact", "asv_set_trees", "asv_get_status", "asv_last_cuda_error",
                         "asv_version", "asv_matrix_update_values", "asv_spmspv_batched", "asv_autotune_batched",
                         "asv_spmspv_backward", "asv_spmv_noalloc_f32", "asv_spmspv_masked", "asv_bfs",
                         "asv_pagerank"):
                getattr(L, name).restype = i32
            _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().asv_status_string(int(s)).decode()


def _check(st: int, where: str):
    if st != ASV_OK:
        raise AsvError(st, where)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _kernel_id(kernel) -> int:
    if kernel is None or kernel == "auto":
        return ASV_K_AUTO
    if isinstance(kernel, str):
        return K[kernel]
    return int(kernel)


def _dev(t, dtype=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return t


# ---------------------------------------------------------------- C-named functions
def asv_matrix_create_csr(m, n, rowptr, col, val, dtype=None, flags=ASV_BORROW, stream=None):
    """Create a handle; returns the raw handle (c_void_p). Tensors must stay alive (ASV_BORROW)."""
    _dev(rowptr, torch.int32, "rowptr")
    _dev(col, torch.int32, "col")
    if dtype is None:
        dtype = ASV_BOOL if val is None else _DT[val.dtype]
    if val is not None:
        _dev(val, TORCH_DTYPE[dtype] if dtype != ASV_BOOL else None, "val")
    h = ctypes.c_void_p()
    nnz = col.numel()
    _check(lib().asv_matrix_create_csr(ctypes.byref(h), int(m), int(n), int(nnz), _ptr(rowptr), _ptr(col),
                                       _ptr(val), int(dtype), int(flags), _stream(stream)),
           "asv_matrix_create_csr")
    return h


def asv_matrix_transpose_view(h, stream=None):
    """Raw handle of A^T borrowing A's arrays; A must be destroyed after it."""
    t = ctypes.c_void_p()
    _check(lib().asv_matrix_transpose_view(h, ctypes.byref(t), _stream(stream)), "asv_matrix_transpose_view")
    return t


def asv_matrix_destroy(h):
    _check(lib().asv_matrix_destroy(h), "asv_matrix_destroy")


def asv_matrix_features(h) -> dict:
    f = _MFeat()
    _check(lib().asv_matrix_features(h, ctypes.byref(f)), "asv_matrix_features")
    return {k: getattr(f, k) for k in MATRIX_FEATURES}


def asv_matrix_arrays(h) -> dict:
    ptrs = [ctypes.c_void_p() for _ in range(7)]
    _check(lib().asv_matrix_arrays(h, *[ctypes.byref(p) for p in ptrs]), "asv_matrix_arrays")
    names = ("rowptr", "col", "val", "colptr", "rowidx", "val_csc", "perm")
    return {k: p.value for k, p in zip(names, ptrs)}


def asv_matrix_copy_csc(h, colptr=None, rowidx=None, val_csc=None, perm=None, stream=None):
    _check(lib().asv_matrix_copy_csc(h, _ptr(colptr), _ptr(rowidx), _ptr(val_csc), _ptr(perm), _stream(stream)),
           "asv_matrix_copy_csc")


def asv_matrix_update_values(h, val=None, stream=None):
    _check(lib().asv_matrix_update_values(h, _ptr(val), _stream(stream)), "asv_matrix_update_values")


def asv_spmspv_batched(h, B, max_entries=0, xptr=None, xidx=None, xval=None, X_dense=None, Y=None, tune=None,
                       stream=None):
    t = None if tune is None else ctypes.byref(AsvTune(int(tune[0]), int(tune[1]),
                                                      int(tune[2]) if len(tune) > 2 else 0))
    _check(lib().asv_spmspv_batched(h, int(B), int(max_entries), _ptr(xptr), _ptr(xidx), _ptr(xval), _ptr(X_dense),
                                    _ptr(Y), t, _stream(stream)), "asv_spmspv_batched")


def asv_autotune_batched(h, B, max_entries=0, xptr=None, xidx=None, xval=None, X_dense=None, Y=None,
                         cache_path=None, stream=None):
    best = AsvTune()
    cp = None if cache_path is None else str(cache_path).encode()
    _check(lib().asv_autotune_batched(h, int(B), int(max_entries), _ptr(xptr), _ptr(xidx), _ptr(xval),
                                      _ptr(X_dense), _ptr(Y), cp, ctypes.byref(best), _stream(stream)),
           "asv_autotune_batched")
    return best.rows_per_tile, best.vectors_per_group, best.hot_columns


def asv_spmspv_backward(h, B, X, dY, dX=None, dA=None, stream=None):
    _check(lib().asv_spmspv_backward(h, int(B), _ptr(X), _ptr(dY), _ptr(dX), _ptr(dA), _stream(stream)),
           "asv_spmspv_backward")


def asv_spmspv_backward_list(h, B, xptr, xidx, xval, dY, dX=None, dA=None, stream=None):
    _check(lib().asv_spmspv_backward_list(h, int(B), _ptr(xptr), _ptr(xidx), _ptr(xval), _ptr(dY), _ptr(dX),
                                          _ptr(dA), _stream(stream)), "asv_spmspv_backward_list")


def asv_autotune(h, cache_path=None, budget_ms=2000, stream=None):
    """Tunes the handle's pull launch shape; returns (lanes, unroll, tma)."""
    t = AsvPullTune()
    cp = None if cache_path is None else str(cache_path).encode()
    _check(lib().asv_autotune(h, cp, int(budget_ms), ctypes.byref(t), _stream(stream)), "asv_autotune")
    return t.lanes, t.unroll, t.tma


def asv_pull_tuning(h):
    t = AsvPullTune()
    _check(lib().asv_pull_tuning(h, ctypes.byref(t)), "asv_pull_tuning")
    return t.lanes, t.unroll, t.tma


def asv_spmv_noalloc_f32(m, n, rowptr, col, val, x, y, stream=None):
    """y = A x (FP32) on caller-owned CSR tensors with no device allocation and
    no handle (for callers that cannot allocate on their call path)."""
    _check(lib().asv_spmv_noalloc_f32(int(m), int(n), int(col.numel()), _ptr(rowptr), _ptr(col), _ptr(val),
                                      _ptr(x), _ptr(y), _stream(stream)), "asv_spmv_noalloc_f32")


def asv_spmv(h, x, y, kernel="auto", stream=None):
    _check(lib().asv_spmv(h, _ptr(x), _ptr(y), _kernel_id(kernel), _stream(stream)), "asv_spmv")


def asv_spmspv(h, nnz_x=None, xidx=None, xval=None, x_dense=None, out_mode=ASV_OUT_DENSE, y=None,
               yidx=None, yval=None, nnz_y=None, y_cap=0, kernel="auto", stream=None):
    _check(lib().asv_spmspv(h, _ptr(nnz_x), _ptr(xidx), _ptr(xval), _ptr(x_dense), int(out_mode), _ptr(y),
                            _ptr(yidx), _ptr(yval), _ptr(nnz_y), int(y_cap), _kernel_id(kernel),
                            _stream(stream)), "asv_spmspv")


def asv_spmspv_masked(h, ymask, nnz_x=None, xidx=None, xval=None, x_dense=None, out_mode=ASV_OUT_DENSE, y=None,
                      yidx=None, yval=None, nnz_y=None, y_cap=0, kernel="auto", stream=None):
    _check(lib().asv_spmspv_masked(h, _ptr(ymask), _ptr(nnz_x), _ptr(xidx), _ptr(xval), _ptr(x_dense),
                                   int(out_mode), _ptr(y), _ptr(yidx), _ptr(yval), _ptr(nnz_y), int(y_cap),
                                   _kernel_id(kernel), _stream(stream)), "asv_spmspv_masked")


def asv_bfs(h, source, level, kernel="auto", stream=None, wait=True):
    """Number of levels (waits for the search), or None with wait=False
    (the search is only enqueued on `stream`)."""
    depth = ctypes.c_int32()
    _check(lib().asv_bfs(h, int(source), _ptr(level), _kernel_id(kernel), ctypes.byref(depth) if wait else None,
                         _stream(stream)), "asv_bfs")
    return depth.value if wait else None


def asv_pagerank(h, damping, eps, max_iter, rank, kernel="auto", stream=None, wait=True):
    """Number of products run (waits), or None with wait=False (enqueued only)."""
    iters = ctypes.c_int32()
    _check(lib().asv_pagerank(h, float(damping), float(eps), int(max_iter), _ptr(rank), _kernel_id(kernel),
                              ctypes.byref(iters) if wait else None, _stream(stream)), "asv_pagerank")
    return iters.value if wait else None


def asv_select(h, nnz_x=None, xidx=None, xval=None, x_dense=None, out_mode=ASV_OUT_DENSE, stream=None):
    k = ctypes.c_int32()
    f = _VFeat()
    _check(lib().asv_select(h, _ptr(nnz_x), _ptr(xidx), _ptr(xval), _ptr(x_dense), int(out_mode), ctypes.byref(k),
                            ctypes.byref(f), _stream(stream)), "asv_select")
    return k.value, {"nnz_x": f.nnz_x, "nnz_s": f.nnz_s, "x_sparsity": f.x_sparsity,
                     "m_sparsity": f.m_sparsity}


def asv_last_kernel(h, stream=None) -> int:
    k = ctypes.c_int32()
    _check(lib().asv_last_kernel(h, ctypes.byref(k), _stream(stream)), "asv_last_kernel")
    return k.value


def asv_compact(h, x_dense, idx, val, count, stream=None):
    _check(lib().asv_compact(h, _ptr(x_dense), _ptr(idx), _ptr(val), _ptr(count), _stream(stream)),
           "asv_compact")


def asv_set_trees(h, nodes, roots, stream=None):
    """nodes: (feature, threshold, left, right, leaf) records; roots: 20 node indices, five per
    call format (pattern; distribution after push / masked pull / pull; write-back). Five
    roots are repeated for all four formats."""
    import numpy as np
    arr = np.ascontiguousarray(np.asarray(nodes, np.float64).reshape(-1, 5))
    r = np.ascontiguousarray(np.asarray(roots, np.int32).reshape(-1))
    if r.size == 5:
        r = np.tile(r, 4)
    _check(lib().asv_set_trees(h, arr.ctypes.data_as(ctypes.c_void_p), len(arr),
                               r.ctypes.data_as(ctypes.c_void_p), _stream(stream)), "asv_set_trees")


def asv_get_status(h, stream=None) -> int:
    return int(lib().asv_get_status(h, _stream(stream)))


ASV_WAIT_LIMIT_DEFAULT = 1 << 24


def asv_debug_set_wait_limit(h, polls):
    """Testing hook: polls of the first bounded TMA wait of the handle's
    staged kernels (0 makes it give up at once and latch ASV_ERR_TIMEOUT)."""
    _check(lib().asv_debug_set_wait_limit(h, int(polls)), "asv_debug_set_wait_limit")


def asv_debug_fail_alloc(countdown):
    """Testing hook: the countdown-th handle allocation from now on fails
    with ASV_ERR_NOMEM (0 disarms)."""
    lib().asv_debug_fail_alloc(int(countdown))


def asv_version() -> int:
    return int(lib().asv_version())


# ---------------------------------------------------------------- owner object
class Matrix:
    """A CSR matrix handle on the current CUDA device (CSR + CSC resident).

    ``rowptr``/``col``/``val`` are CUDA tensors (int32, int32, value dtype or
    None for the Boolean pattern). The tensors are kept alive by this object.
    """

    def __init__(self, m, n, rowptr, col, val=None, dtype=None, validate=False, copy=False, stream=None):
        self.m, self.n = int(m), int(n)
        self.rowptr, self.col, self.val = rowptr, col, val
        self.device = rowptr.device
        self.parent = None
        self.dtype = (ASV_BOOL if val is None else _DT[val.dtype]) if dtype is None else dtype
        flags = (ASV_VALIDATE if validate else 0) | (ASV_COPY if copy else 0)
        self.handle = asv_matrix_create_csr(m, n, rowptr, col, val, self.dtype, flags, stream)
        self.nnz = int(col.numel())
        self.tdtype = TORCH_DTYPE[self.dtype]

    def close(self):
        if getattr(self, "handle", None) is not None:
            asv_matrix_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def transpose_view(self, stream=None) -> "Matrix":
        """A^T as an n x m handle over this matrix's CSC and CSR (nothing copied).

        The view keeps this matrix alive; its ``rowptr``/``col``/``val`` are
        None because the arrays belong to this matrix's handle."""
        t = Matrix.__new__(Matrix)
        t.m, t.n, t.nnz = self.n, self.m, self.nnz
        t.dtype, t.tdtype, t.device = self.dtype, self.tdtype, self.device
        t.rowptr = t.col = t.val = None
        t.parent = self
        t.handle = asv_matrix_transpose_view(self.handle, stream)
        return t

    def features(self) -> dict:
        return asv_matrix_features(self.handle)

    def csc(self):
        """(colptr, rowidx, val_csc, perm) as CUDA tensors (copies of the handle's arrays)."""
        dev = self.device
        colptr = torch.empty(self.n + 1, dtype=torch.int32, device=dev)
        rowidx = torch.empty(max(self.nnz, 1), dtype=torch.int32, device=dev)
        perm = torch.empty(max(self.nnz, 1), dtype=torch.int32, device=dev)
        valc = None if self.dtype == ASV_BOOL else torch.empty(max(self.nnz, 1), dtype=self.tdtype, device=dev)
        asv_matrix_copy_csc(self.handle, colptr, rowidx, valc, perm)
        nz = self.nnz
        return colptr, rowidx[:nz], (valc[:nz] if valc is not None else None), perm[:nz]

    def spmv(self, x, y=None, kernel="auto", stream=None):
        if y is None:
            y = torch.empty(self.m, dtype=self.tdtype, device=x.device)
        asv_spmv(self.handle, x, y, kernel, stream)
        return y

    def spmspv(self, xidx=None, xval=None, nnz_x=None, x_dense=None, sparse_out=False, y=None, y_cap=None,
               kernel="auto", ymask=None, stream=None):
        """y = A x. x sparse (xidx[, xval]) or dense (x_dense). Returns y (dense) or
        (yidx, yval, nnz_y) views (sparse output). ymask: optional int32 bitmap of
        (m + 31) // 32 words; rows whose bit is set are excluded from y."""
        dev = (x_dense if x_dense is not None else xidx).device
        if x_dense is None and nnz_x is None:
            nnz_x = torch.tensor([xidx.numel()], dtype=torch.int64, device=dev)

        def call(*a):
            if ymask is None:
                asv_spmspv(self.handle, *a)
            else:
                asv_spmspv_masked(self.handle, ymask, *a)
        if not sparse_out:
            if y is None:
                y = torch.empty(self.m, dtype=self.tdtype, device=dev)
            call(nnz_x, xidx, xval, x_dense, ASV_OUT_DENSE, y, None, None, None, 0, kernel, stream)
            return y
        cap = self.m if y_cap is None else int(y_cap)
        yidx = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
        yval = torch.empty(max(cap, 1), dtype=self.tdtype, device=dev)
        nnz_y = torch.zeros(1, dtype=torch.int64, device=dev)
        call(nnz_x, xidx, xval, x_dense, ASV_OUT_SPARSE, None, yidx, yval, nnz_y, cap, kernel, stream)
        return yidx, yval, nnz_y

    def pagerank(self, damping=0.85, eps=1e-10, max_iter=100, kernel="auto", rank=None, stream=None, wait=True):
        """Delta-form PageRank (rank vector of the handle's value type, number of
        products run -- None with wait=False); deltas below eps are dropped
        after every product. The iterations run on the device."""
        if rank is None:
            rank = torch.empty(self.n, dtype=self.tdtype, device=self.device)
        iters = asv_pagerank(self.handle, damping, eps, max_iter, rank, kernel, stream, wait)
        return rank, iters

    def bfs(self, source, kernel="auto", level=None, stream=None, wait=True):
        """Breadth-first search levels from `source` (int32 [n], -1 = unreached)
        and the number of levels (None with wait=False); each level is one
        masked product, and the levels run on the device."""
        if level is None:
            level = torch.empty(self.n, dtype=torch.int32, device=self.device)
        depth = asv_bfs(self.handle, source, level, kernel, stream, wait)
        return level, depth

    def select(self, xidx=None, xval=None, nnz_x=None, x_dense=None, sparse_out=False, stream=None):
        dev = (x_dense if x_dense is not None else xidx).device
        if x_dense is None and nnz_x is None:
            nnz_x = torch.tensor([xidx.numel()], dtype=torch.int64, device=dev)
        return asv_select(self.handle, nnz_x, xidx, xval, x_dense, ASV_OUT_SPARSE if sparse_out else ASV_OUT_DENSE,
                          stream)

    def update_values(self, val=None, stream=None):
        asv_matrix_update_values(self.handle, val, stream)

    def spmspv_batched(self, xptr=None, xidx=None, xval=None, X_dense=None, Y=None, tune=None, stream=None):
        """Y[b,:] = A x_b. The batch is a CSR of vectors (xptr int64[B+1], xidx, xval) or dense [B][n]."""
        if X_dense is not None:
            B = X_dense.shape[0]
            dev = X_dense.device
        else:
            B = xptr.numel() - 1
            dev = xptr.device
        if Y is None:
            Y = torch.empty((B, self.m), dtype=torch.float32, device=dev)
        cap = 0 if xidx is None else xidx.numel()
        asv_spmspv_batched(self.handle, B, cap, xptr, xidx, xval, X_dense, Y, tune, stream)
        return Y

    def autotune_batched(self, xptr=None, xidx=None, xval=None, X_dense=None, cache_path=None, stream=None):
        B = X_dense.shape[0] if X_dense is not None else xptr.numel() - 1
        dev = (X_dense if X_dense is not None else xptr).device
        Y = torch.empty((B, self.m), dtype=torch.float32, device=dev)
        cap = 0 if xidx is None else xidx.numel()
        return asv_autotune_batched(self.handle, B, cap, xptr, xidx, xval, X_dense, Y, cache_path, stream)

    def backward(self, X, dY, need_dx=True, need_da=True, stream=None):
        """(dX [B][n] or None, dA [nnz] or None) for Y = X A^T row by row."""
        B = dY.shape[0]
        dX = torch.empty((B, self.n), dtype=torch.float32, device=dY.device) if need_dx else None
        dA = torch.empty(self.nnz, dtype=torch.float32, device=dY.device) if need_da else None
        asv_spmspv_backward(self.handle, B, X, dY, dX, dA, stream)
        return dX, dA

    def backward_list(self, xptr, xidx, xval, dY, need_dx=True, need_da=True, stream=None):
        """backward() with the batch listed (xptr int64[B+1], xidx, xval or None)."""
        B = dY.shape[0]
        dX = torch.empty((B, self.n), dtype=torch.float32, device=dY.device) if need_dx else None
        dA = torch.empty(self.nnz, dtype=torch.float32, device=dY.device) if need_da else None
        asv_spmspv_backward_list(self.handle, B, xptr, xidx, xval, dY, dX, dA, stream)
        return dX, dA

    def autotune(self, cache_path=None, budget_ms=2000, stream=None):
        """Tune the pull kernels' launch shape for this matrix; (lanes, unroll, tma)."""
        return asv_autotune(self.handle, cache_path, budget_ms, stream)

    def pull_tuning(self):
        return asv_pull_tuning(self.handle)

    def last_kernel(self, stream=None) -> int:
        return asv_last_kernel(self.handle, stream)

    def status(self, stream=None) -> int:
        return asv_get_status(self.handle, stream)

    def set_trees(self, nodes, roots, stream=None):
        asv_set_trees(self.handle, nodes, roots, stream)


class SpMSpVFunction(torch.autograd.Function):
    """Differentiable y_b = A x_b for a batch X [B][n] (FP32), A given by its
    pattern (a Matrix handle) and its stored values `values` [nnz] (CSR order).

    forward:  Y [B][m] through the batched product;
    backward: dX = dY A (dx_b = A^T dy_b) and dvalues_k = sum_b dy_b[row(k)] x_b[col(k)],
              the gradient on A's pattern, from one fused pass per view.
    The handle must read `values` in place (created with ASV_BORROW on it);
    its CSC copy is refreshed at every forward.
    """

    @staticmethod
    def forward(ctx, values, X, A):
        A.update_values()
        Xc = X.contiguous()
        Y = A.spmspv_batched(X_dense=Xc)
        ctx.save_for_backward(Xc)
        ctx.A = A
        return Y

    @staticmethod
    def backward(ctx, dY):
        (X,) = ctx.saved_tensors
        need_dv, need_dx = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        dX, dA = ctx.A.backward(X, dY.contiguous(), need_dx=need_dx, need_da=need_dv)
        return dA, dX, None


# ---------------------------------------------------------------- module-level forms
def spmv(A: Matrix, x, y=None, kernel="auto", stream=None):
    """y = A x for a dense x (selector-driven unless `kernel` forces a candidate)."""
    return A.spmv(x, y, kernel=kernel, stream=stream)


def spmspv(A: Matrix, **kw):
    """y = A x for a listed (xidx, xval[, nnz_x]) or dense (x_dense) x; see Matrix.spmspv."""
    return A.spmspv(**kw)


def select(A: Matrix, **kw):
    """(kernel id, vector features) the selector picks for this x; synchronises."""
    return A.select(**kw)


def spmspv_batched(A: Matrix, **kw):
    """Y[b] = A x_b for a batch of sparse (xptr, xidx, xval) or dense (X_dense) vectors."""
    return A.spmspv_batched(**kw)


def transpose_view(A: Matrix, stream=None) -> Matrix:
    """A^T over A's arrays (nothing copied); see Matrix.transpose_view."""
    return A.transpose_view(stream=stream)
