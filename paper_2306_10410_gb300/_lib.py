"""ctypes loader for libboba.so (the C ABI of include/boba.h).

Argument marshalling only: every computation runs in the CUDA kernels of the
library.  There is no CPU fallback; if the library is missing, loading fails.
"""
from __future__ import annotations

import ctypes
import os
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libboba.so")

BOBA_OK = 0
STATUS_NAMES = {
    0: "BOBA_OK",
    1: "BOBA_ERR_INVALID_ARG",
    2: "BOBA_ERR_ID_OUT_OF_RANGE",
    3: "BOBA_ERR_TOO_LARGE",
    4: "BOBA_ERR_WORKSPACE",
    5: "BOBA_ERR_TIMEOUT",
    6: "BOBA_ERR_CUDA",
}

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_SZ = ctypes.c_size_t
_ST = ctypes.c_int

# name -> (restype, argtypes); mirrors include/boba.h
SIGNATURES = {
    "boba_reorder": (_ST, [_P, _P, _I64, _I64, _P, _P, _P, _P]),
    "boba_reorder_workspace_bytes": (_SZ, [_I64, _I64]),
    "boba_reorder_ex": (_ST, [_P, _P, _I64, _I64, _P, _P, _P, _P, _P, _SZ, _P]),
    "boba_reorder_host": (_ST, [_P, _P, _I64, _I64, _P, _P, _P, _P, _SZ, _P]),
    "boba_reorder_host_workspace_bytes": (_SZ, [_I64, _I64]),
    "boba_reorder_variant": (_ST, [_P, _P, _I64, _I64, _P, _P, _P, ctypes.c_int, _P, _SZ, _P]),
    "boba_first_keys": (_ST, [_P, _P, _I64, _I64, _I64, _I64, _P, ctypes.c_int, _P]),
    "boba_labels_workspace_bytes": (_SZ, [_I64, _I64]),
    "boba_labels_from_keys": (_ST, [_P, _I64, _I64, _P, _P, _P, _SZ, _P]),
    "boba_relabel": (_ST, [_P, _P, _I64, _I64, _P, _P, _P, _P]),
    "boba_reorder_static": (_ST, [_P, _P, _I64, _I64, _P, _P, _P, _P, _P]),
    "boba_reorder_batched": (_ST, [_P, _P, _P, _P, _I64, _I64, _I64, _I64, _I64, _P, _P, _P,
                                   _P, _SZ, _P]),
    "boba_reorder_batched_workspace_bytes": (_SZ, [_I64, _I64, _I64, _I64, _I64]),
    "boba_batched_set_mode": (None, [ctypes.c_int]),
    "boba_coo_to_csr": (_ST, [_P, _P, _I64, _I64, _P, _P, _P, _P, _SZ, _P]),
    "boba_coo_to_csr_workspace_bytes": (_SZ, [_I64, _I64]),
    "boba_spmv_csr": (_ST, [_P, _P, _P, _P, _P, _I64, _I64, _P, _SZ, _P]),
    "boba_spmv_workspace_bytes": (_SZ, [_I64, _I64]),
    "boba_pagerank": (_ST, [_P, _P, _P, _I64, _I64, ctypes.c_double, _I64, ctypes.c_double, _P,
                            _P, _P, _P, _SZ, _P]),
    "boba_pagerank_workspace_bytes": (_SZ, [_I64, _I64]),
    "boba_sort_by_dst": (_ST, [_P, _P, _I64, _I64, _P, _P, ctypes.c_int, _P, _SZ, _P]),
    "boba_sort_by_dst_workspace_bytes": (_SZ, [_I64, _I64]),
    "boba_nbr": (_ST, [_P, _P, _I64, _I64, _I64, _P, _P, _P, _SZ, _P]),
    "boba_nbr_workspace_bytes": (_SZ, [_I64, _I64]),
    "boba_stream_status": (_ST, [_P]),
    "boba_selftest_wait_timeout": (_ST, [ctypes.c_uint64, _P, _P]),
    "boba_probe_gather": (_ST, [ctypes.c_int, _P, _I64, _I64, ctypes.c_int, _P, _I64, _P, _P]),
    "boba_status_string": (ctypes.c_char_p, [_ST]),
    "boba_version": (ctypes.c_char_p, []),
    "boba_server_create": (_P, [_SZ, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "boba_server_submit": (_I64, [_P, _P, _P, _I64, _I64, _P, _P, _P]),
    "boba_server_poll": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int]),
    "boba_server_drain": (_ST, [_P]),
    "boba_server_cancel": (_ST, [_P, _I64]),
    "boba_server_stats": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "boba_server_destroy": (None, [_P]),
    "boba_tune_reorder": (_ST, [_P, _P, _I64, _I64, _P, _P, _P, _P, _SZ, ctypes.c_int, _P, _P]),
    "boba_tune_batched": (_ST, [_P, _P, _P, _P, _I64, _I64, _I64, _I64, _I64, _P, _P, _P, _P,
                                _SZ, ctypes.c_int, _P, _P]),
    "boba_tune_spmv": (_ST, [_P, _P, _P, _P, _P, _I64, _I64, _P, _SZ, ctypes.c_int, _P, _P]),
    "boba_tune_csr": (_ST, [_P, _P, _I64, _I64, _P, _P, _P, _P, _SZ, ctypes.c_int, _P, _P]),
    "boba_tune_get": (ctypes.c_int, [ctypes.c_int, _I64]),
    "boba_tune_set": (None, [ctypes.c_int, _I64, ctypes.c_int]),
    "boba_tune_save": (_ST, [ctypes.c_char_p]),
    "boba_tune_load": (_ST, [ctypes.c_char_p]),
    "boba_tune_reset": (None, []),
    "boba_timing_enable": (None, [ctypes.c_int]),
    "boba_timing_collect": (ctypes.c_int, []),
    "boba_timing_name": (ctypes.c_char_p, [ctypes.c_int]),
    "boba_timing_total_ms": (ctypes.c_double, [ctypes.c_int]),
    "boba_timing_launches": (_I64, [ctypes.c_int]),
    "boba_timing_reset": (None, []),
}


class BobaError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {STATUS_NAMES.get(code, code)}" if what else
                         STATUS_NAMES.get(code, str(code)))


_lock = threading.Lock()
_lib = None


def load() -> ctypes.CDLL:
    """Load libboba.so from the package directory (raises if it was never built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build the CUDA library first "
                    "(python -c 'import __graft_entry__ as g; g.build()')")
            lib = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def check(code: int, what: str = "") -> None:
    if code != BOBA_OK:
        raise BobaError(code, what)
