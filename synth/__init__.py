"""Seeded synthetic workloads (inputs only; no part of the BOBA method lives here).

The generators are counter based (SplitMix64 draws, Feistel permutations), so
the same seed gives the same arrays on every machine and with any thread count.
The tests, the oracle checks and ``bench.py`` all take their inputs from here.

The workloads stand in for the paper's SuiteSparse/SNAP datasets (Table 2,
Sec. 5.1), which are not used: R-MAT with the Graph500 initiator stands in for
``kron_g500``-style scale-free graphs, the 2D grid for road/Delaunay-style
meshes, and Erdos-Renyi for a graph with no structure at all.  Every workload
relabels vertices with a random permutation and shuffles the edge order, the
regime of the paper's randomised-edge-order experiment (Sec. 5.6, Table 3).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

RMAT_ABC = (0.57, 0.19, 0.19)   # d = 0.05
SEED_BASE = 0xB0BA0000


def build(force: bool = False) -> str:
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=gnu11", "-pthread",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            u64, i64, p, ci, d = (ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p,
                                  ctypes.c_int, ctypes.c_double)
            lib.synth_rmat.argtypes = [u64, ci, i64, i64, d, d, d, ci, ci, i64, i64, p, p, ci]
            lib.synth_grid.argtypes = [u64, i64, ci, ci, i64, i64, p, p, ci]
            lib.synth_er.argtypes = [u64, i64, i64, ci, ci, i64, i64, p, p, ci]
            lib.synth_permutation.argtypes = [u64, u64, i64, p]
            lib.synth_uniform_f32.argtypes = [u64, u64, i64, p]
            lib.synth_draws.argtypes = [u64, u64, i64, p]
            for f in (lib.synth_rmat, lib.synth_grid, lib.synth_er, lib.synth_permutation,
                      lib.synth_uniform_f32, lib.synth_draws):
                f.restype = ci
            _lib = lib
    return _lib


def _threads() -> int:
    return max(1, min(64, os.cpu_count() or 1))


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _alloc(m: int, out=None):
    if out is not None:
        src, dst = out
        assert src.dtype == np.int32 and dst.dtype == np.int32
        assert src.shape[0] >= m and dst.shape[0] >= m
        return src[:m], dst[:m]
    return np.empty(m, dtype=np.int32), np.empty(m, dtype=np.int32)


def _range(m, rng):
    lo, hi = (0, m) if rng is None else (int(rng[0]), int(rng[1]))
    if not 0 <= lo <= hi <= m:
        raise ValueError("edge range outside [0, m]")
    return lo, hi


def rmat(scale: int, m: int, seed: int, n: int | None = None, abc=RMAT_ABC,
         shuffle: bool = True, relabel: bool = True, out=None, edge_range=None):
    """Directed R-MAT COO (src, dst) int32 with ``n`` (default 2^scale) vertices.

    Duplicate edges and self-loops are kept.  ``out`` may pass preallocated
    (e.g. pinned) int32 arrays.  ``edge_range=(lo, hi)`` produces only edges
    [lo, hi) of the m-edge list (a prefix of the shuffled list is a uniform
    sample of its edges).
    """
    n = (1 << scale) if n is None else int(n)
    lo, hi = _range(m, edge_range)
    src, dst = _alloc(hi - lo, out)
    rc = _load().synth_rmat(seed, scale, n, m, abc[0], abc[1], abc[2], int(shuffle),
                            int(relabel), lo, hi, _ptr(src), _ptr(dst), _threads())
    if rc:
        raise ValueError("synth.rmat: bad arguments")
    return src, dst


def grid(side: int, seed: int, shuffle: bool = True, relabel: bool = True, out=None,
         edge_range=None):
    """4-neighbour side x side grid with both edge directions: m = 4 side (side-1)."""
    m = 4 * side * (side - 1)
    lo, hi = _range(m, edge_range)
    src, dst = _alloc(hi - lo, out)
    rc = _load().synth_grid(seed, side, int(shuffle), int(relabel), lo, hi, _ptr(src),
                            _ptr(dst), _threads())
    if rc:
        raise ValueError("synth.grid: bad arguments")
    return src, dst


def er(n: int, m: int, seed: int, shuffle: bool = True, relabel: bool = True, out=None,
       edge_range=None):
    """m edges with independent uniform endpoints in [0, n)."""
    lo, hi = _range(m, edge_range)
    src, dst = _alloc(hi - lo, out)
    rc = _load().synth_er(seed, n, m, int(shuffle), int(relabel), lo, hi, _ptr(src), _ptr(dst),
                          _threads())
    if rc:
        raise ValueError("synth.er: bad arguments")
    return src, dst


def permutation(N: int, seed: int, stream: int = 7) -> np.ndarray:
    out = np.empty(N, dtype=np.int64)
    if _load().synth_permutation(seed, stream, N, _ptr(out)):
        raise ValueError("synth.permutation: bad arguments")
    return out


def uniform_f32(n: int, seed: int, stream: int = 4) -> np.ndarray:
    """x ~ U[0, 1) as fp32 with 24 random bits."""
    out = np.empty(n, dtype=np.float32)
    _load().synth_uniform_f32(seed, stream, n, _ptr(out))
    return out


def draws(n: int, seed: int, stream: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint64)
    _load().synth_draws(seed, stream, n, _ptr(out))
    return out


# --------------------------------------------------------------------------
# Named workloads (sizes as specified for the evaluation)
# --------------------------------------------------------------------------

@dataclass(frozen=True)
class Workload:
    name: str
    kind: str          # "rmat" | "grid" | "er"
    n: int
    m: int
    seed: int
    scale: int = 0
    side: int = 0

    def generate(self, out=None, edge_range=None):
        if self.kind == "rmat":
            return rmat(self.scale, self.m, self.seed, n=self.n, out=out, edge_range=edge_range)
        if self.kind == "grid":
            return grid(self.side, self.seed, out=out, edge_range=edge_range)
        if self.kind == "er":
            return er(self.n, self.m, self.seed, out=out, edge_range=edge_range)
        raise ValueError(self.kind)


def rmat_workload(scale: int, m: int, seed: int, name: str | None = None) -> Workload:
    return Workload(name or f"rmat{scale}_m{m}", "rmat", 1 << scale, m, seed, scale=scale)


# R-MAT scale 14, edge factor 16 (262,144 edges): small enough for the oracle.
RMAT14 = Workload("rmat14_ef16", "rmat", 1 << 14, 1 << 18, SEED_BASE + 0, scale=14)
# R-MAT scale 24, 2^28 edges: the single-large-graph workload.
RMAT24 = Workload("rmat24_m2^28", "rmat", 1 << 24, 1 << 28, SEED_BASE + 1, scale=24)
# Low-skew structure: a 4096 x 4096 grid and an ER graph with n = 2^24, m = 2^27.
GRID4096 = Workload("grid4096", "grid", 4096 * 4096, 4 * 4096 * 4095, SEED_BASE + 2,
                    side=4096)
ER24 = Workload("er24_m2^27", "er", 1 << 24, 1 << 27, SEED_BASE + 12)
# A quarter-size R-MAT scale 24 (2^26 edges, 512 MiB of input > L2) for profiling captures.
RMAT24_SMALL = Workload("rmat24_m2^26", "rmat", 1 << 24, 1 << 26, SEED_BASE + 1, scale=24)

WORKLOADS = {w.name: w for w in (RMAT14, RMAT24, GRID4096, ER24, RMAT24_SMALL)}


def batch_sizes(G: int, seed: int, log2_lo: float = 8.0, log2_hi: float = 18.0,
                ef_lo: int = 4, ef_hi: int = 32):
    """Per-graph (n_g, m_g): n_g = floor(2^U(lo, hi)), edge factor uniform in {ef_lo..ef_hi}."""
    d = draws(2 * G, seed, stream=11)
    u = (d[0::2] >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    n = np.floor(np.exp2(log2_lo + (log2_hi - log2_lo) * u)).astype(np.int64)
    ef = (ef_lo + (d[1::2] % np.uint64(ef_hi - ef_lo + 1))).astype(np.int64)
    return n, n * ef


def rmat_batch(G: int, seed: int, log2_lo: float = 8.0, log2_hi: float = 18.0,
               ef_lo: int = 4, ef_hi: int = 32, out=None):
    """G independent R-MAT graphs packed back to back.

    Returns (src, dst, edge_off, vert_off): graph g owns edges
    [edge_off[g], edge_off[g+1]) and vertices [0, vert_off[g+1]-vert_off[g]) in
    its own local ID space.
    """
    n, m = batch_sizes(G, seed, log2_lo, log2_hi, ef_lo, ef_hi)
    edge_off = np.zeros(G + 1, dtype=np.int64)
    vert_off = np.zeros(G + 1, dtype=np.int64)
    edge_off[1:] = np.cumsum(m)
    vert_off[1:] = np.cumsum(n)
    src, dst = _alloc(int(edge_off[-1]), out)
    for g in range(G):
        scale = max(1, int(math.ceil(math.log2(int(n[g])))))
        lo, hi = int(edge_off[g]), int(edge_off[g + 1])
        rmat(scale, hi - lo, seed * 1000003 + g, n=int(n[g]), out=(src[lo:hi], dst[lo:hi]))
    return src, dst, edge_off, vert_off
