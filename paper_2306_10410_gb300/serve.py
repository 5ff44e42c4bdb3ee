"""Serving: a Poisson stream of reorder + CSR + SpMV requests under an HBM budget.

``Server`` wraps the native runtime of ``boba_server_*`` (include/boba.h):
admission by HBM budget, waves of admitted requests reordered by one batched
launch, per-request streams for CSR and SpMV, latency accounting.  This module
only marshals arguments and drives arrivals.

``serve_workload`` builds the request mix (R-MAT or 2D grid graphs, m
log-uniform in [1e4, 1e8], n = m/16 rounded to a power of two for R-MAT, a
side of about sqrt(m/4) for the grid), calibrates the mean service time with
each graph run alone, sets the Poisson arrival rate to a target device load,
and replays the arrivals in real time.
"""
from __future__ import annotations

import ctypes
import math
import time

import numpy as np
import torch

from ._lib import BobaError, load


class Server:
    def __init__(self, budget_bytes: int = 120 << 30, max_active: int = 64, spmv_iters: int = 10,
                 n_streams: int = 16):
        self.lib = load()
        self.h = self.lib.boba_server_create(budget_bytes, max_active, spmv_iters, n_streams)
        if not self.h:
            raise BobaError(6, "boba_server_create")
        self.spmv_iters = spmv_iters

    @staticmethod
    def _ptr(t):
        if t is None:
            return None
        if isinstance(t, np.ndarray):
            return ctypes.c_void_p(t.ctypes.data)
        assert not t.is_cuda and t.is_contiguous()
        return ctypes.c_void_p(t.data_ptr())

    def submit(self, src, dst, n: int, x=None, y=None, perm=None) -> int:
        """Enqueue one request (host buffers, pinned for asynchronous copies)."""
        m = len(src)
        rid = self.lib.boba_server_submit(self.h, self._ptr(src), self._ptr(dst), m, n,
                                          self._ptr(x), self._ptr(y), self._ptr(perm))
        if rid == -2:
            raise BobaError(4, "request does not fit in the HBM budget")
        if rid < 0:
            raise BobaError(1, "boba_server_submit")
        return int(rid)

    def poll(self, cap: int = 4096):
        ids = (ctypes.c_int64 * cap)()
        lat = (ctypes.c_double * cap)()
        st = (ctypes.c_int * cap)()
        k = self.lib.boba_server_poll(self.h, ids, lat, st, cap)
        return [(int(ids[i]), float(lat[i]), int(st[i])) for i in range(max(k, 0))]

    def cancel(self, rid: int) -> bool:
        """Withdraw a request still waiting for admission; False if it was already
        admitted (it then completes) or is unknown."""
        return self.lib.boba_server_cancel(self.h, int(rid)) == 0

    def drain(self):
        rc = self.lib.boba_server_drain(self.h)
        if rc != 0:
            raise BobaError(rc, "boba_server_drain")

    def stats(self) -> dict:
        out = (ctypes.c_double * 8)()
        self.lib.boba_server_stats(self.h, out, 8)
        return {"p50_ms": out[0], "p99_ms": out[1], "gedges_s": out[2],
                "requests": int(out[3]), "edges": int(out[4]), "peak_pool_bytes": int(out[5]),
                "span_s": out[6]}

    def close(self):
        if self.h:
            self.lib.boba_server_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
        return False


# ---------------------------------------------------------------------------
# the request mix and the Poisson driver
# ---------------------------------------------------------------------------

def request_pool(k: int, seed: int, m_lo: float = 1e4, m_hi: float = 1e8, pinned: bool = True):
    """k request graphs: (kind, src, dst, n, x) with m log-uniform in [m_lo, m_hi]."""
    import synth
    d = synth.draws(3 * k, seed, stream=21)
    out = []
    for i in range(k):
        u = float(d[3 * i] >> np.uint64(11)) / 9007199254740992.0
        m = int(round(math.exp(math.log(m_lo) + u * (math.log(m_hi) - math.log(m_lo)))))
        if int(d[3 * i + 1]) & 1:
            side = max(2, int(round(math.sqrt(m / 4.0))))
            kind, n, m = "grid", side * side, 4 * side * (side - 1)
        else:
            scale = max(1, int(round(math.log2(max(2, m / 16)))))
            kind, n = "rmat", 1 << scale
        alloc = (lambda sz, dt: torch.empty(sz, dtype=dt, pin_memory=True)) if pinned else \
                (lambda sz, dt: torch.empty(sz, dtype=dt))
        src, dst = alloc(m, torch.int32), alloc(m, torch.int32)
        gseed = seed * 7919 + i
        if kind == "grid":
            synth.grid(side, gseed, out=(src.numpy(), dst.numpy()))
        else:
            synth.rmat(scale, m, gseed, out=(src.numpy(), dst.numpy()))
        x = alloc(n, torch.float32)
        x.numpy()[:] = synth.uniform_f32(n, seed=gseed)
        out.append({"kind": kind, "src": src, "dst": dst, "n": n, "m": m, "x": x})
    return out


def _pinned_out(n):
    return torch.empty(n, dtype=torch.float32, pin_memory=True)


def calibrate(server: Server, pool) -> list:
    """Service time (ms) of each pool graph run alone."""
    times = []
    for g in pool:
        y = _pinned_out(g["n"])
        server.submit(g["src"], g["dst"], g["n"], g["x"], y)      # warm the path
        server.drain()
        server.poll()
        t0 = time.perf_counter()
        server.submit(g["src"], g["dst"], g["n"], g["x"], y)
        server.drain()
        times.append((time.perf_counter() - t0) * 1e3)
        server.poll()
    return times


def serve_workload(n_requests: int = 400, pool_size: int = 32, load: float = 0.8,
                   seed: int = 0xB0BA0004, budget_bytes: int = 120 << 30, spmv_iters: int = 10,
                   max_active: int = 64, m_lo: float = 1e4, m_hi: float = 1e8):
    """Replay a Poisson stream of requests in real time; return the server's statistics."""
    import synth
    pool = request_pool(pool_size, seed, m_lo, m_hi)
    with Server(budget_bytes, max_active, spmv_iters) as srv:
        svc = calibrate(srv, pool)
    mean_svc_s = float(np.mean(svc)) / 1e3
    rate = load / mean_svc_s                                     # requests per second
    d = synth.draws(2 * n_requests, seed, stream=22)
    u = (d[0::2] >> np.uint64(11)).astype(np.float64) / 9007199254740992.0
    arrivals = np.cumsum(-np.log1p(-u) / rate)
    which = (d[1::2] % np.uint64(pool_size)).astype(np.int64)
    # output buffers allocated up front (a ring per pool graph; the timing does not
    # depend on which earlier request's y a buffer last held)
    ring = 4
    ybufs = [[_pinned_out(g["n"]) for _ in range(ring)] for g in pool]
    used = [0] * pool_size
    statuses = []
    with Server(budget_bytes, max_active, spmv_iters) as srv:
        t0 = time.perf_counter()
        for i in range(n_requests):
            while time.perf_counter() - t0 < arrivals[i]:
                statuses += [st for _, _, st in srv.poll()]
                time.sleep(20e-6)
            k = int(which[i])
            g = pool[k]
            y = ybufs[k][used[k] % ring]
            used[k] += 1
            srv.submit(g["src"], g["dst"], g["n"], g["x"], y)
        srv.drain()
        statuses += [st for _, _, st in srv.poll()]
        st = srv.stats()
    if any(s != 0 for s in statuses):
        raise BobaError(next(s for s in statuses if s != 0), "served request")
    st.update({"offered_load": load, "rate_per_s": rate, "mean_service_ms": mean_svc_s * 1e3,
               "n_requests": n_requests, "pool_size": pool_size,
               "pool_edges_mean": float(np.mean([g["m"] for g in pool])),
               "spmv_iters": spmv_iters, "budget_bytes": budget_bytes})
    return st
