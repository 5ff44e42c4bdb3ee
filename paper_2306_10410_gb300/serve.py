"""Serving: a Poisson stream of reorder + CSR + SpMV requests under an HBM budget.

``Server`` wraps the native runtime of ``boba_server_*`` (include/boba.h):
admission by HBM budget, waves of admitted requests reordered by one batched
launch, per-request streams for CSR and SpMV, latency accounting.  This module
only marshals arguments and drives arrivals.

``serve_workload`` builds the request mix (R-MAT or 2D grid graphs, m
log-uniform in [1e4, 1e8], n = m/16 rounded to a power of two for R-MAT, a
side of about sqrt(m/4) for the grid), calibrates the mean service time with
each graph run alone, sets the Poisson arrival rate to a target device load,
and replays the arrivals in real time.  ``serve_vs_sequential`` runs a request
list at saturation through the server and one request at a time through the
per-graph entry points, and compares the outputs bit for bit.
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
        out = (ctypes.c_double * 13)()
        self.lib.boba_server_stats(self.h, out, 13)
        return {"p50_ms": out[0], "p99_ms": out[1], "gedges_s": out[2],
                "requests": int(out[3]), "edges": int(out[4]), "peak_pool_bytes": int(out[5]),
                "span_s": out[6], "peak_active": int(out[7]), "joined_while_busy": int(out[8]),
                "peak_device_overlap": int(out[9]), "p50_queue_ms": out[10],
                "p99_queue_ms": out[11], "p99_service_ms": out[12]}

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
                   max_active: int = 64, m_lo: float = 1e4, m_hi: float = 1e8, pool=None):
    """Replay a Poisson stream of requests in real time; return the server's statistics."""
    import synth
    pool = request_pool(pool_size, seed, m_lo, m_hi) if pool is None else pool
    pool_size = len(pool)
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


# ---------------------------------------------------------------------------
# saturation: the server against one request at a time, at identical output
# ---------------------------------------------------------------------------

def request_order(n_requests: int, pool_size: int, seed: int) -> np.ndarray:
    """Which pool graph each request of a closed-loop run uses (seeded)."""
    import synth
    d = synth.draws(n_requests, seed, stream=23)
    return (d % np.uint64(pool_size)).astype(np.int64)


def run_saturated(pool, order, budget_bytes: int = 120 << 30, spmv_iters: int = 10,
                  max_active: int = 64):
    """Every request submitted at once (the server is never idle): throughput at
    saturation.  Returns (stats, ys, perms) with one host output per request."""
    ys = [_pinned_out(pool[k]["n"]) for k in order]
    perms = [torch.empty(pool[k]["n"], dtype=torch.int32, pin_memory=True) for k in order]
    with Server(budget_bytes, max_active, spmv_iters) as srv:
        g = pool[int(order[0])]                          # warm the path once
        srv.submit(g["src"], g["dst"], g["n"], g["x"], _pinned_out(g["n"]))
        srv.drain()
        srv.poll()
    with Server(budget_bytes, max_active, spmv_iters) as srv:
        t0 = time.perf_counter()
        for i, k in enumerate(order):
            g = pool[int(k)]
            srv.submit(g["src"], g["dst"], g["n"], g["x"], ys[i], perms[i])
        srv.drain()
        t1 = time.perf_counter()
        done = srv.poll()
        st = srv.stats()
    bad = [s for _, _, s in done if s != 0]
    if bad or len(done) != len(order):
        raise BobaError(bad[0] if bad else 6, "saturated run")
    edges = sum(pool[int(k)]["m"] for k in order)
    st.update({"wall_s": t1 - t0, "gedges_s_wall": edges / (t1 - t0) / 1e9,
               "requests_submitted": len(order)})
    return st, ys, perms


def run_sequential(pool, order, spmv_iters: int = 10):
    """The same requests one after another through the per-graph entry points on
    one stream, as a caller without the server would run them: copy the edges
    and x in, boba_reorder_ex, boba_coo_to_csr, spmv_iters x boba_spmv_csr, copy
    y and perm out.  Device buffers are sized once for the largest request.
    Returns (stats, ys, perms)."""
    from . import (boba_coo_to_csr, boba_coo_to_csr_workspace_bytes, boba_reorder_ex,
                   boba_reorder_workspace_bytes, boba_spmv_csr, boba_spmv_workspace_bytes, check,
                   stream_status)
    dev = torch.device("cuda")
    M = max(pool[int(k)]["m"] for k in order)
    N = max(pool[int(k)]["n"] for k in order)
    i32, f32 = torch.int32, torch.float32
    src, dst, so, do = (torch.empty(M, dtype=i32, device=dev) for _ in range(4))
    col, val = torch.empty(M, dtype=i32, device=dev), torch.empty(M, dtype=f32, device=dev)
    perm = torch.empty(N, dtype=i32, device=dev)
    row_ptr = torch.empty(N + 1, dtype=torch.int64, device=dev)
    x, y = torch.empty(N, dtype=f32, device=dev), torch.empty(N, dtype=f32, device=dev)
    wr = torch.empty(max(boba_reorder_workspace_bytes(pool[int(k)]["m"], pool[int(k)]["n"])
                         for k in order), dtype=torch.uint8, device=dev)
    wc = torch.empty(max(boba_coo_to_csr_workspace_bytes(pool[int(k)]["m"], pool[int(k)]["n"])
                         for k in order), dtype=torch.uint8, device=dev)
    wsp = torch.empty(max(256, max(boba_spmv_workspace_bytes(pool[int(k)]["n"], pool[int(k)]["m"])
                                   for k in order)), dtype=torch.uint8, device=dev)
    ys = [_pinned_out(pool[int(k)]["n"]) for k in order]
    perms = [torch.empty(pool[int(k)]["n"], dtype=i32, pin_memory=True) for k in order]
    s = torch.cuda.current_stream()

    def one(i, k):
        g = pool[int(k)]
        m, n = g["m"], g["n"]
        src[:m].copy_(g["src"], non_blocking=True)
        dst[:m].copy_(g["dst"], non_blocking=True)
        x[:n].copy_(g["x"], non_blocking=True)
        check(boba_reorder_ex(src[:m], dst[:m], m, n, perm[:n], so[:m], do[:m], None, wr,
                              wr.numel(), s), "reorder")
        check(boba_coo_to_csr(so[:m], do[:m], m, n, row_ptr[:n + 1], col[:m], val[:m], wc,
                              wc.numel(), s), "csr")
        for _ in range(spmv_iters):
            check(boba_spmv_csr(row_ptr[:n + 1], col[:m], val[:m], x[:n], y[:n], n, m, wsp,
                                wsp.numel(), s), "spmv")
        ys[i].copy_(y[:n], non_blocking=True)
        perms[i].copy_(perm[:n], non_blocking=True)

    one(0, order[0])                                     # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, k in enumerate(order):
        one(i, k)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    stream_status(s)
    edges = sum(pool[int(k)]["m"] for k in order)
    return {"wall_s": t1 - t0, "gedges_s_wall": edges / (t1 - t0) / 1e9,
            "requests": len(order)}, ys, perms


def serve_vs_sequential(n_requests: int = 48, pool_size: int = 24, seed: int = 0xB0BA0004,
                        budget_bytes: int = 120 << 30, spmv_iters: int = 10,
                        max_active: int = 64, m_lo: float = 1e4, m_hi: float = 1e8, pool=None,
                        rounds: int = 3):
    """Saturated serving against the same request list run one request at a time
    through the per-graph entry points; outputs compared bit for bit.

    Both forms copy every request's data in and its results out over the host
    link, which other work on the machine can slow for a while.  So the two
    run in `rounds` alternating pairs: the speedup is the median of the
    paired ratios, and the reported runs are the median rounds of each form."""
    pool = request_pool(pool_size, seed, m_lo, m_hi) if pool is None else pool
    order = request_order(n_requests, len(pool), seed)
    sats, seqs, ratios = [], [], []
    identical = True
    for _ in range(max(1, rounds)):
        sat, ys_a, perms_a = run_saturated(pool, order, budget_bytes, spmv_iters, max_active)
        seq, ys_b, perms_b = run_sequential(pool, order, spmv_iters)
        identical = identical and \
            all(torch.equal(a, b) for a, b in zip(ys_a, ys_b)) and \
            all(torch.equal(a, b) for a, b in zip(perms_a, perms_b))
        sats.append(sat)
        seqs.append(seq)
        ratios.append(sat["gedges_s_wall"] / seq["gedges_s_wall"])
        del ys_a, perms_a, ys_b, perms_b

    def median_run(runs):
        return sorted(runs, key=lambda r: r["gedges_s_wall"])[len(runs) // 2]

    return {"saturated": median_run(sats), "sequential": median_run(seqs),
            "identical": bool(identical),
            "speedup_served_vs_sequential": sorted(ratios)[len(ratios) // 2],
            "rounds_gedges_s": {"saturated": [r["gedges_s_wall"] for r in sats],
                                "sequential": [r["gedges_s_wall"] for r in seqs]},
            "n_requests": int(n_requests), "edges": int(sum(pool[int(k)]["m"] for k in order))}
