"""BOBA oracle -- TEST INFRASTRUCTURE ONLY.

A plain, slow CPU restatement of the BOBA hot path (arXiv 2306.10410), used to
prove the CUDA library right.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  It shares no
code with ``paper_2306_10410_gb300`` and never imports it.

The arithmetic lives in ``boba_oracle.c`` (single-threaded C, compiled here with
gcc); this module only marshals numpy arrays.  Every function cites the passage
of the paper it follows:

* :func:`first_keys`   -- Algorithm 2's key r with an AtomicMin update (Sec. 4.4)
* :func:`boba_perm`    -- Algorithm 1, Sequential BOBA (Sec. 4.3), plus the
                          isolated-vertex tail (ascending original ID)
* :func:`boba_perm_interleaved` -- the interleaved flattening drawn in Fig. 1
* :func:`relabel`      -- rewriting the COO through the permutation (Sec. 5.3)
* :func:`coo_to_csr`   -- stable pull CSR for Algorithm 3 (Sec. 1.2.2), values
                          fp32(1/outdeg(source))
* :func:`spmv_f64`     -- Algorithm 3 in fp64
* :func:`nbr`          -- the NBR line metric (Sec. 5.2)
* :func:`sort_by_dst`  -- the edge list stably sorted or binned by destination,
                          the remedy for random edge order (Sec. 5.6)
* :func:`pagerank`     -- the PR application of Sec. 5.1, power iteration in
                          fp64 with the standard damping and dangling terms

Parity status: every function here is pinned by ``tests/test_oracle_pins.py``
(paper worked examples, brute force, closed forms, invariants).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "boba_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

SENT = 0xFFFFFFFF


def build(force: bool = False) -> str:
    """Compile ``boba_oracle.c`` into ``liboracle.so`` (gcc, -O2, no fast-math)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11",
                           "-fno-fast-math", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            p = ctypes.c_void_p
            i64 = ctypes.c_int64
            for name, args in {
                "oracle_first_keys": [p, p, i64, i64, p],
                "oracle_boba_perm": [p, p, i64, i64, p, p],
                "oracle_boba_perm_interleaved": [p, p, i64, i64, p, p],
                "oracle_relabel": [p, p, i64, i64, p, p, p],
                "oracle_coo_to_csr": [p, p, i64, i64, p, p, p],
                "oracle_spmv_f64": [p, p, p, p, i64, p],
            }.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = ctypes.c_int
            lib.oracle_pagerank.argtypes = [p, p, i64, i64, ctypes.c_double, i64,
                                             ctypes.c_double, p, p, p]
            lib.oracle_pagerank.restype = ctypes.c_int
            lib.oracle_nbr.argtypes = [p, p, i64, i64, p]
            lib.oracle_nbr.restype = ctypes.c_double
            _lib = lib
    return _lib


class OracleError(ValueError):
    pass


def _i32(a) -> np.ndarray:
    a = np.ascontiguousarray(a)
    if a.dtype != np.int32:
        a = a.astype(np.int32)
    return a


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _check(rc: int, what: str):
    if rc == 1:
        raise OracleError(f"{what}: invalid argument")
    if rc == 2:
        raise OracleError(f"{what}: vertex ID outside [0, n)")
    if rc != 0:
        raise OracleError(f"{what}: error {rc}")


def first_keys(I, J, n: int) -> np.ndarray:
    """key[v] = lowest position of v in I ++ J, SENT if v is on no edge (Alg. 2 with AtomicMin)."""
    I, J = _i32(I), _i32(J)
    m = I.shape[0]
    key = np.empty(n, dtype=np.uint32)
    _check(_load().oracle_first_keys(_ptr(I), _ptr(J), m, n, _ptr(key)), "first_keys")
    return key


def boba_perm(I, J, n: int):
    """(perm, label) of Algorithm 1 with isolated vertices appended by ascending ID."""
    I, J = _i32(I), _i32(J)
    m = I.shape[0]
    perm = np.empty(n, dtype=np.int32)
    label = np.empty(n, dtype=np.int32)
    _check(_load().oracle_boba_perm(_ptr(I), _ptr(J), m, n, _ptr(perm), _ptr(label)),
           "boba_perm")
    return perm, label


def boba_perm_interleaved(I, J, n: int):
    """(perm, label) for the interleaved flattening I(0) J(0) I(1) J(1) ... of Fig. 1."""
    I, J = _i32(I), _i32(J)
    m = I.shape[0]
    perm = np.empty(n, dtype=np.int32)
    label = np.empty(n, dtype=np.int32)
    _check(_load().oracle_boba_perm_interleaved(_ptr(I), _ptr(J), m, n, _ptr(perm),
                                                _ptr(label)), "boba_perm_interleaved")
    return perm, label


def relabel(I, J, label, n: int):
    """(I_out, J_out) = (label[I], label[J]) with edge order kept (Sec. 5.3)."""
    I, J, label = _i32(I), _i32(J), _i32(label)
    m = I.shape[0]
    Io = np.empty(m, dtype=np.int32)
    Jo = np.empty(m, dtype=np.int32)
    _check(_load().oracle_relabel(_ptr(I), _ptr(J), m, n, _ptr(label), _ptr(Io), _ptr(Jo)),
           "relabel")
    return Io, Jo


def reorder(I, J, n: int):
    """The full BOBA reorder: (perm, I_out, J_out)."""
    perm, label = boba_perm(I, J, n)
    Io, Jo = relabel(I, J, label, n)
    return perm, Io, Jo


def coo_to_csr(I, J, n: int):
    """Stable pull CSR (row = J, col = I), val = fp32(1/outdeg(I)).  Returns (row_ptr, col, val)."""
    I, J = _i32(I), _i32(J)
    m = I.shape[0]
    row_ptr = np.empty(n + 1, dtype=np.int64)
    col = np.empty(m, dtype=np.int32)
    val = np.empty(m, dtype=np.float32)
    _check(_load().oracle_coo_to_csr(_ptr(I), _ptr(J), m, n, _ptr(row_ptr), _ptr(col),
                                     _ptr(val)), "coo_to_csr")
    return row_ptr, col, val


def spmv_f64(row_ptr, col, val, x) -> np.ndarray:
    """y = A x accumulated in fp64 (Algorithm 3)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = _i32(col)
    val = np.ascontiguousarray(val, dtype=np.float32)
    x = np.ascontiguousarray(x, dtype=np.float32)
    n_rows = row_ptr.shape[0] - 1
    y = np.empty(n_rows, dtype=np.float64)
    _check(_load().oracle_spmv_f64(_ptr(row_ptr), _ptr(col), _ptr(val), _ptr(x), n_rows,
                                   _ptr(y)), "spmv_f64")
    return y


def nbr(row_ptr, col, ids_per_line: int = 32):
    """(NBR, rows counted) of the CSR (Sec. 5.2); lines of ``ids_per_line`` vertex IDs."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = _i32(col)
    counted = ctypes.c_int64(0)
    v = _load().oracle_nbr(_ptr(row_ptr), _ptr(col), row_ptr.shape[0] - 1, ids_per_line,
                           ctypes.byref(counted))
    if counted.value < 0:
        raise OracleError("nbr: out of memory")
    return float(v), int(counted.value)


def sort_by_dst(I, J, n: int, top_digit_only: bool = False):
    """Edges stably sorted by destination (Sec. 5.6); or, with top_digit_only,
    stably binned by the top 8 bits of the ceil(log2 n)-bit destination."""
    I, J = _i32(I), _i32(J)
    bits = 1
    while bits < 31 and (1 << bits) < n:
        bits += 1
    key = J.astype(np.int64)
    if top_digit_only:
        key = (key >> max(0, bits - 8)) & 255
    order = np.argsort(key, kind="stable")
    return I[order], J[order]


def pagerank(I, J, n: int, damping: float = 0.85, max_iters: int = 100, tol: float = 0.0):
    """(pr, steps, residual): PageRank of the edge list by fp64 power iteration
    (Sec. 5.1 applications; standard damping and uniform dangling mass)."""
    I, J = _i32(I), _i32(J)
    m = I.shape[0]
    pr = np.empty(max(n, 0), dtype=np.float64)
    it = ctypes.c_int64(0)
    res = ctypes.c_double(0.0)
    _check(_load().oracle_pagerank(_ptr(I), _ptr(J), m, n, float(damping), int(max_iters),
                                   float(tol), _ptr(pr), ctypes.byref(it), ctypes.byref(res)),
           "pagerank")
    return pr, int(it.value), float(res.value)
