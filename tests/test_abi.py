"""CPU checks of the C ABI: the library builds for sm_103a, loads without a GPU,
and exports every entry point that include/asv.h declares."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "asv.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(asv_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2006_16767_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for want in ("asv_matrix_create_csr", "asv_matrix_destroy", "asv_spmv", "asv_spmspv", "asv_select",
                 "asv_compact", "asv_matrix_features", "asv_get_status", "asv_status_string"):
        assert want in syms


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (asv_\w+)", out))
    assert set(declared_symbols()) <= exported


def test_library_targets_sm103a_only(libpath):
    out = subprocess.run(["/usr/local/cuda/bin/cuobjdump", "--list-elf", libpath], capture_output=True,
                         text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    arches = set(re.findall(r"sm_(\d+a?)", out.stdout))
    assert arches == {"103a"}, arches


def test_status_strings_and_version(libpath):
    import paper_2006_16767_gb300 as asv
    assert asv.asv_version() >= 100
    assert asv.status_string(asv.ASV_OK) == "ok"
    assert "capacity" in asv.status_string(asv.ASV_ERR_CAPACITY) or "y_cap" in asv.status_string(4)
    assert asv.status_string(12345) == "unknown status"


def test_argument_errors_are_caught_on_the_host(libpath):
    import paper_2006_16767_gb300 as asv
    L = asv.lib()
    h = ctypes.c_void_p()
    assert L.asv_matrix_create_csr(None, 1, 1, 0, None, None, None, 0, 0, None) == asv.ASV_ERR_ARG
    assert L.asv_matrix_create_csr(ctypes.byref(h), -1, 1, 0, None, None, None, 0, 0, None) == asv.ASV_ERR_ARG
    assert L.asv_matrix_create_csr(ctypes.byref(h), 1, 1, 0, None, None, None, 9, 0, None) == asv.ASV_ERR_ARG
    assert L.asv_matrix_create_csr(ctypes.byref(h), 2**31, 1, 0, ctypes.c_void_p(16), None, None, 0, 0,
                                   None) == asv.ASV_ERR_OVERFLOW
    assert L.asv_spmv(None, None, None, 0, None) == asv.ASV_ERR_ARG
    assert L.asv_spmspv(None, None, None, None, None, 0, None, None, None, None, 0, 0, None) == asv.ASV_ERR_ARG
    assert L.asv_matrix_destroy(None) == asv.ASV_ERR_ARG
    h.value = 1
    assert L.asv_matrix_transpose_view(None, ctypes.byref(h), None) == asv.ASV_ERR_ARG
    assert h.value is None  # the out-handle is cleared before the argument check fails
    assert L.asv_matrix_transpose_view(None, None, None) == asv.ASV_ERR_ARG


def test_python_names_of_the_boundary():
    import paper_2006_16767_gb300 as asv
    for name in ("Matrix", "SpMSpVFunction", "spmv", "spmspv", "select", "spmspv_batched", "transpose_view"):
        assert callable(getattr(asv, name)), name
    for name in ("spmv", "spmspv", "select", "spmspv_batched", "transpose_view", "bfs", "pagerank", "backward"):
        assert callable(getattr(asv.Matrix, name)), name


def test_no_cpu_fallback_without_the_library(tmp_path, monkeypatch):
    import importlib

    import paper_2006_16767_gb300 as asv
    monkeypatch.setattr(asv, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(asv, "_lib", None)
    with pytest.raises(ImportError):
        asv.lib()
    importlib.reload(asv)
