"""The C ABI: the library builds for sm_103a, loads without a GPU, and exports
every entry point include/boba.h declares (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "boba.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(boba_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2306_10410_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("boba_reorder", "boba_reorder_ex", "boba_reorder_workspace_bytes",
                 "boba_reorder_batched", "boba_coo_to_csr", "boba_spmv_csr",
                 "boba_stream_status", "boba_status_string"):
        assert name in syms


def test_every_declared_symbol_is_exported(lib):
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_binding_mirrors_header():
    from paper_2306_10410_gb300 import _lib
    assert set(_lib.SIGNATURES) == set(declared_symbols())


def test_host_only_entry_points(lib):
    """Calls that touch no device: sizes, strings."""
    lib.boba_reorder_workspace_bytes.restype = ctypes.c_size_t
    lib.boba_reorder_workspace_bytes.argtypes = [ctypes.c_int64, ctypes.c_int64]
    assert lib.boba_reorder_workspace_bytes(1 << 28, 1 << 24) > 4 * (1 << 24)
    assert lib.boba_reorder_workspace_bytes(-1, 5) == 0
    assert lib.boba_reorder_workspace_bytes(1 << 31, 5) == 0
    lib.boba_status_string.restype = ctypes.c_char_p
    lib.boba_status_string.argtypes = [ctypes.c_int]
    assert lib.boba_status_string(2) == b"BOBA_ERR_ID_OUT_OF_RANGE"
    lib.boba_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.boba_version()


def test_argument_validation_without_gpu(lib):
    """Invalid sizes are refused before any CUDA call."""
    f = lib.boba_reorder_ex
    P, I = ctypes.c_void_p, ctypes.c_int64
    f.argtypes = [P, P, I, I, P, P, P, P, P, ctypes.c_size_t, P]
    f.restype = ctypes.c_int
    assert f(None, None, -1, 4, None, None, None, None, None, 0, None) == 1
    assert f(None, None, 1 << 31, 4, None, None, None, None, None, 0, None) == 3
    assert f(None, None, 3, 0, None, None, None, None, None, 0, None) == 1
    assert f(None, None, 0, 0, None, None, None, None, None, 0, None) == 0


def test_no_oracle_in_product():
    """The CUDA package never imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_2306_10410_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".hpp", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "boba_oracle" not in text and "liboracle" not in text, f


def test_python_binding_has_every_entry_point():
    """Every C entry point has a same-name Python function (the tuning/timing/server
    families through their helpers or the serve module)."""
    import paper_2306_10410_gb300 as pkg
    from paper_2306_10410_gb300 import serve
    missing = []
    for name in declared_symbols():
        if hasattr(pkg, name):
            continue
        method = {"create": "__init__", "destroy": "close"}.get(name[len("boba_server_"):],
                                                               name[len("boba_server_"):])
        if name.startswith("boba_server_") and hasattr(serve.Server, method):
            continue
        if name.startswith(("boba_timing_", "boba_tune_reorder", "boba_tune_batched",
                            "boba_tune_spmv", "boba_tune_csr")):
            continue                 # wrapped by kernel_timing() and tune_*()
        missing.append(name)
    assert not missing, missing
