"""BOBA (Batched Order By Attachment, arXiv 2306.10410) on the NVIDIA GB300.

Thin Python binding over the C ABI of ``include/boba.h`` (``libboba.so``).
PyTorch supplies device memory and streams; every step of the computation runs
in the library's CUDA kernels.  The functions named ``boba_*`` mirror the C
entry points one to one (tensors in, argument marshalling only); the
lower-case helpers allocate outputs and workspaces for convenience.
"""
from __future__ import annotations

import torch

from ._lib import BobaError, STATUS_NAMES, check, load

__all__ = [
    "BobaError", "load", "reorder", "reorder_perm", "reorder_batched", "coo_to_csr", "spmv", "stream_status",
    "boba_reorder", "boba_reorder_ex", "boba_reorder_workspace_bytes", "boba_reorder_static", "boba_reorder_batched",
    "boba_reorder_batched_workspace_bytes", "boba_batched_set_mode", "boba_coo_to_csr", "boba_coo_to_csr_workspace_bytes",
    "boba_spmv_csr", "boba_spmv_workspace_bytes", "boba_stream_status", "boba_status_string",
    "boba_pagerank", "boba_pagerank_workspace_bytes", "pagerank",
    "Workspace", "kernel_timing", "nbr", "reorder_variant", "reorder_host", "sort_by_dst", "tune_reorder", "tune_batched", "tune_spmv", "tune_save",
    "tune_load", "tune_reset", "tune_csr", "TUNE_FIRST", "TUNE_RELABEL", "TUNE_BATCHED",
    "TUNE_SPMV", "TUNE_CSR",
]

TUNE_FIRST, TUNE_RELABEL, TUNE_BATCHED, TUNE_SPMV, TUNE_CSR = 0, 1, 2, 3, 4


def _p(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libboba takes device tensors only")
    if not t.is_contiguous():
        raise ValueError("libboba takes contiguous tensors only")
    return t.data_ptr()


def _s(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def _dt(t, dtype, name):
    if t is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")


# ---------------------------------------------------------------------------
# raw C entry points (same names, same argument order)
# ---------------------------------------------------------------------------

def boba_reorder(src, dst, m, n, perm_out, src_out, dst_out, stream=None):
    return load().boba_reorder(_p(src), _p(dst), m, n, _p(perm_out), _p(src_out), _p(dst_out),
                               _s(stream))


def boba_reorder_workspace_bytes(m, n):
    return load().boba_reorder_workspace_bytes(m, n)


def boba_reorder_ex(src, dst, m, n, perm_out, src_out, dst_out, label_out, ws, ws_bytes,
                    stream=None):
    return load().boba_reorder_ex(_p(src), _p(dst), m, n, _p(perm_out), _p(src_out),
                                  _p(dst_out), _p(label_out), _p(ws), ws_bytes, _s(stream))


def boba_reorder_static(src, dst, m, n, perm_out, src_out, dst_out, error_bits=None,
                        stream=None):
    """The allocation-free reorder (scratch in the library's static device array)."""
    return load().boba_reorder_static(_p(src), _p(dst), m, n, _p(perm_out), _p(src_out),
                                      _p(dst_out), _p(error_bits), _s(stream))


def boba_reorder_batched(src, dst, edge_off, vert_off, G, max_m, max_n, total_m, total_n,
                         perm_out, src_out, dst_out, ws, ws_bytes, stream=None):
    return load().boba_reorder_batched(_p(src), _p(dst), _p(edge_off), _p(vert_off), G, max_m,
                                       max_n, total_m, total_n, _p(perm_out), _p(src_out),
                                       _p(dst_out), _p(ws), ws_bytes, _s(stream))


def boba_reorder_batched_workspace_bytes(G, max_m, max_n, total_m, total_n):
    return load().boba_reorder_batched_workspace_bytes(G, max_m, max_n, total_m, total_n)


def boba_batched_set_mode(mode):
    load().boba_batched_set_mode(int(mode))


def boba_coo_to_csr(src, dst, m, n, row_ptr, col_out, val_out, ws, ws_bytes, stream=None):
    return load().boba_coo_to_csr(_p(src), _p(dst), m, n, _p(row_ptr), _p(col_out),
                                  _p(val_out), _p(ws), ws_bytes, _s(stream))


def boba_coo_to_csr_workspace_bytes(m, n):
    return load().boba_coo_to_csr_workspace_bytes(m, n)


def boba_spmv_csr(row_ptr, col, val, x, y, n_rows, nnz, ws, ws_bytes, stream=None):
    return load().boba_spmv_csr(_p(row_ptr), _p(col), _p(val), _p(x), _p(y), n_rows, nnz,
                                _p(ws), ws_bytes, _s(stream))


def boba_spmv_workspace_bytes(n_rows, nnz):
    return load().boba_spmv_workspace_bytes(n_rows, nnz)


def boba_pagerank(row_ptr, col, val, n, nnz, damping, max_iters, tol, pr, iters_out,
                  residual_out, ws, ws_bytes, stream=None):
    return load().boba_pagerank(_p(row_ptr), _p(col), _p(val), n, nnz, float(damping),
                                int(max_iters), float(tol), _p(pr), _p(iters_out),
                                _p(residual_out), _p(ws), ws_bytes, _s(stream))


def boba_pagerank_workspace_bytes(n, nnz):
    return load().boba_pagerank_workspace_bytes(n, nnz)


def _hp(t):
    """Host tensor/array pointer (CPU tensors only)."""
    if t is None:
        return None
    if hasattr(t, "is_cuda"):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("host buffers must be contiguous CPU tensors")
        return t.data_ptr()
    return t.ctypes.data


def boba_reorder_host(src, dst, m, n, perm_out, src_out, dst_out, ws, ws_bytes, stream=None):
    return load().boba_reorder_host(_hp(src), _hp(dst), m, n, _hp(perm_out), _hp(src_out),
                                    _hp(dst_out), _p(ws), ws_bytes, _s(stream))


def boba_reorder_host_workspace_bytes(m, n):
    return load().boba_reorder_host_workspace_bytes(m, n)


def reorder_host(src, dst, n, *, perm_out=None, src_out=None, dst_out=None, ws=None, stream=None,
                 device=None):
    """BOBA of a graph in (preferably pinned) host memory; outputs in host memory."""
    m = src.numel()
    perm_out = torch.empty(n, dtype=torch.int32, pin_memory=True) if perm_out is None else perm_out
    src_out = torch.empty(m, dtype=torch.int32, pin_memory=True) if src_out is None else src_out
    dst_out = torch.empty(m, dtype=torch.int32, pin_memory=True) if dst_out is None else dst_out
    dev = torch.device("cuda") if device is None else torch.device(device)
    buf = _ws(ws, boba_reorder_host_workspace_bytes(m, n), dev)
    check(boba_reorder_host(src, dst, m, n, perm_out, src_out, dst_out, buf, buf.numel(), stream),
          "boba_reorder_host")
    return perm_out, src_out, dst_out


def boba_reorder_variant(src, dst, m, n, perm_out, src_out, dst_out, variant, ws, ws_bytes,
                         stream=None):
    return load().boba_reorder_variant(_p(src), _p(dst), m, n, _p(perm_out), _p(src_out),
                                       _p(dst_out), int(variant), _p(ws), ws_bytes, _s(stream))


def reorder_variant(src, dst, n, variant, *, ws=None, stream=None):
    """(perm, src_out, dst_out) for a reading of the method: 0 I ++ J, 1 interleaved
    (Fig. 1), 2 racy store (Alg. 2 as printed)."""
    m = src.numel()
    perm = torch.empty(n, dtype=torch.int32, device=src.device)
    so, do = torch.empty_like(src), torch.empty_like(dst)
    buf = _ws(ws, boba_reorder_workspace_bytes(m, n), src.device)
    check(boba_reorder_variant(src, dst, m, n, perm, so, do, variant, buf, buf.numel(), stream),
          "boba_reorder_variant")
    return perm, so, do


def boba_first_keys(src, dst, m_local, pos_src, pos_dst, n, key, init, stream=None):
    return load().boba_first_keys(_p(src), _p(dst), m_local, pos_src, pos_dst, n, _p(key), init,
                                  _s(stream))


def boba_labels_workspace_bytes(m_total, n):
    return load().boba_labels_workspace_bytes(m_total, n)


def boba_labels_from_keys(key, m_total, n, perm_out, label_out, ws, ws_bytes, stream=None):
    return load().boba_labels_from_keys(_p(key), m_total, n, _p(perm_out), _p(label_out), _p(ws),
                                        ws_bytes, _s(stream))


def boba_relabel(src, dst, m, n, label, src_out, dst_out, stream=None):
    return load().boba_relabel(_p(src), _p(dst), m, n, _p(label), _p(src_out), _p(dst_out),
                               _s(stream))


def boba_sort_by_dst(src, dst, m, n, src_out, dst_out, top_digit_only, ws, ws_bytes, stream=None):
    return load().boba_sort_by_dst(_p(src), _p(dst), m, n, _p(src_out), _p(dst_out),
                                   int(top_digit_only), _p(ws), ws_bytes, _s(stream))


def boba_sort_by_dst_workspace_bytes(m, n):
    return load().boba_sort_by_dst_workspace_bytes(m, n)


def boba_nbr(row_ptr, col, n_rows, nnz, ids_per_line, nbr_out, rows_counted, ws, ws_bytes,
             stream=None):
    """nbr_out / rows_counted are ctypes host objects (c_double / c_int64) passed by reference."""
    import ctypes
    return load().boba_nbr(_p(row_ptr), _p(col), n_rows, nnz, ids_per_line, ctypes.byref(nbr_out),
                           None if rows_counted is None else ctypes.byref(rows_counted), _p(ws),
                           ws_bytes, _s(stream))


def boba_nbr_workspace_bytes(n_rows, nnz):
    return load().boba_nbr_workspace_bytes(n_rows, nnz)


def boba_tune_get(kernel, size):
    return load().boba_tune_get(kernel, size)


def boba_tune_set(kernel, size, variant):
    load().boba_tune_set(kernel, size, variant)


def boba_tune_save(path):
    return load().boba_tune_save(str(path).encode())


def boba_tune_load(path):
    return load().boba_tune_load(str(path).encode())


def boba_tune_reset():
    load().boba_tune_reset()


def boba_timing_enable(on):
    load().boba_timing_enable(int(on))


def boba_version():
    return load().boba_version().decode()


def boba_selftest_wait_timeout(timeout_ns, scratch, stream=None):
    return load().boba_selftest_wait_timeout(int(timeout_ns), _p(scratch), _s(stream))


def boba_probe_gather(mode, table, table_words, loads_per_thread, cluster, out, out_words,
                      loads_issued, stream=None):
    """loads_issued is a ctypes c_int64 (host), passed by reference."""
    import ctypes
    return load().boba_probe_gather(int(mode), _p(table), table_words, loads_per_thread,
                                    int(cluster), _p(out), out_words, ctypes.byref(loads_issued),
                                    _s(stream))


def boba_stream_status(stream=None):
    return load().boba_stream_status(_s(stream))


def boba_status_string(code):
    return load().boba_status_string(code).decode()


# ---------------------------------------------------------------------------
# convenience helpers
# ---------------------------------------------------------------------------

class Workspace:
    """A reusable device scratch buffer (256-byte aligned, grown on demand)."""

    def __init__(self, device=None):
        self.device = torch.device("cuda") if device is None else torch.device(device)
        self.buf = None

    def get(self, nbytes: int) -> torch.Tensor:
        nbytes = max(int(nbytes), 256)
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        return self.buf


_default_ws = {}


def _ws(ws, nbytes, device):
    if ws is None:
        key = (torch.device(device).index, torch.cuda.current_stream(device).cuda_stream)
        ws = _default_ws.setdefault(key, Workspace(device))
    return ws.get(nbytes)


def stream_status(stream=None):
    """Synchronise ``stream`` and raise BobaError if any kernel recorded an error."""
    check(boba_stream_status(stream), "device status")


def reorder(src, dst, n, *, perm_out=None, src_out=None, dst_out=None, label_out=None,
            ws=None, stream=None):
    """BOBA reorder of a COO graph on the GPU: returns (perm, src_out, dst_out).

    ``src``/``dst`` are int32 CUDA tensors of length m with IDs in [0, n).
    """
    _dt(src, torch.int32, "src"); _dt(dst, torch.int32, "dst")
    m = src.numel()
    if dst.numel() != m:
        raise ValueError("src and dst differ in length")
    dev = src.device
    perm_out = torch.empty(n, dtype=torch.int32, device=dev) if perm_out is None else perm_out
    src_out = torch.empty_like(src) if src_out is None else src_out
    dst_out = torch.empty_like(dst) if dst_out is None else dst_out
    nbytes = boba_reorder_workspace_bytes(m, n)
    buf = _ws(ws, nbytes, dev)
    check(boba_reorder_ex(src, dst, m, n, perm_out, src_out, dst_out, label_out, buf,
                          buf.numel(), stream), "boba_reorder_ex")
    return perm_out, src_out, dst_out


def reorder_perm(src, dst, n, *, perm_out=None, label_out=None, ws=None, stream=None):
    """The permutation alone (no edge rewrite): returns perm (and fills label_out if given)."""
    _dt(src, torch.int32, "src"); _dt(dst, torch.int32, "dst")
    m = src.numel()
    dev = src.device
    perm_out = torch.empty(n, dtype=torch.int32, device=dev) if perm_out is None else perm_out
    buf = _ws(ws, boba_reorder_workspace_bytes(m, n), dev)
    check(boba_reorder_ex(src, dst, m, n, perm_out, None, None, label_out, buf, buf.numel(),
                          stream), "boba_reorder_ex")
    return perm_out


def reorder_batched(src, dst, edge_off, vert_off, *, max_m=None, max_n=None, perm_out=None,
                    src_out=None, dst_out=None, ws=None, stream=None):
    """BOBA of G packed graphs in one launch: returns (perm, src_out, dst_out), packed.

    ``edge_off``/``vert_off`` are int64 offset arrays (length G+1) on the device;
    ``max_m``/``max_n`` bound one graph's size (computed on the host if omitted).
    """
    _dt(src, torch.int32, "src"); _dt(dst, torch.int32, "dst")
    _dt(edge_off, torch.int64, "edge_off"); _dt(vert_off, torch.int64, "vert_off")
    G = edge_off.numel() - 1
    if max_m is None or max_n is None:
        eo, vo = edge_off.cpu(), vert_off.cpu()
        max_m = int((eo[1:] - eo[:-1]).max()) if G > 0 else 0
        max_n = int((vo[1:] - vo[:-1]).max()) if G > 0 else 0
    total_m, total_n = src.numel(), int(vert_off[-1].item()) if perm_out is None else perm_out.numel()
    dev = src.device
    perm_out = torch.empty(total_n, dtype=torch.int32, device=dev) if perm_out is None else perm_out
    src_out = torch.empty_like(src) if src_out is None else src_out
    dst_out = torch.empty_like(dst) if dst_out is None else dst_out
    buf = _ws(ws, boba_reorder_batched_workspace_bytes(G, max_m, max_n, total_m, total_n), dev)
    check(boba_reorder_batched(src, dst, edge_off, vert_off, G, max_m, max_n, total_m, total_n,
                               perm_out, src_out, dst_out, buf, buf.numel(), stream),
          "boba_reorder_batched")
    return perm_out, src_out, dst_out


def coo_to_csr(src, dst, n, *, row_ptr=None, col_out=None, val_out=None, ws=None, stream=None):
    """Stable pull CSR (rows = dst, cols = src, val = 1/outdeg(src)): (row_ptr, col, val)."""
    _dt(src, torch.int32, "src"); _dt(dst, torch.int32, "dst")
    m = src.numel()
    dev = src.device
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device=dev) if row_ptr is None else row_ptr
    col_out = torch.empty(m, dtype=torch.int32, device=dev) if col_out is None else col_out
    val_out = torch.empty(m, dtype=torch.float32, device=dev) if val_out is None else val_out
    buf = _ws(ws, boba_coo_to_csr_workspace_bytes(m, n), dev)
    check(boba_coo_to_csr(src, dst, m, n, row_ptr, col_out, val_out, buf, buf.numel(), stream),
          "boba_coo_to_csr")
    return row_ptr, col_out, val_out


def spmv(row_ptr, col, val, x, *, y=None, nnz=None, ws=None, stream=None):
    """y = A x (fp32) for a CSR built by coo_to_csr."""
    n_rows = row_ptr.numel() - 1
    nnz = col.numel() if nnz is None else nnz
    y = torch.empty(n_rows, dtype=torch.float32, device=x.device) if y is None else y
    buf = _ws(ws, boba_spmv_workspace_bytes(n_rows, nnz), x.device)
    check(boba_spmv_csr(row_ptr, col, val, x, y, n_rows, nnz, buf, buf.numel(), stream),
          "boba_spmv_csr")
    return y


def pagerank(row_ptr, col, val, *, damping=0.85, max_iters=100, tol=1e-6, pr=None, nnz=None,
             ws=None, stream=None):
    """PageRank over a CSR built by coo_to_csr: (pr, steps, residual) with pr an fp32
    device tensor and steps / residual device tensors (int32[1], float64[1])."""
    n = row_ptr.numel() - 1
    nnz = col.numel() if nnz is None else nnz
    dev = row_ptr.device
    pr = torch.empty(n, dtype=torch.float32, device=dev) if pr is None else pr
    steps = torch.zeros(1, dtype=torch.int32, device=dev)
    residual = torch.zeros(1, dtype=torch.float64, device=dev)
    buf = _ws(ws, boba_pagerank_workspace_bytes(n, nnz), dev)
    check(boba_pagerank(row_ptr, col, val, n, nnz, damping, max_iters, tol, pr, steps, residual,
                        buf, buf.numel(), stream), "boba_pagerank")
    return pr, steps, residual


class kernel_timing:
    """Context manager: per-kernel device time of every libboba launch inside it.

    ``with kernel_timing() as kt: ...`` then ``kt.result`` maps kernel name ->
    (total_ms, launches).  Events are recorded on each kernel's own stream.
    """

    def __enter__(self):
        lib = load()
        lib.boba_timing_reset()
        lib.boba_timing_enable(1)
        self.result = {}
        return self

    def __exit__(self, *exc):
        lib = load()
        lib.boba_timing_enable(0)
        k = lib.boba_timing_collect()
        if k < 0:
            raise BobaError(6, "boba_timing_collect")
        self.result = {lib.boba_timing_name(i).decode(): (lib.boba_timing_total_ms(i),
                                                         int(lib.boba_timing_launches(i)))
                       for i in range(k)}
        lib.boba_timing_reset()
        return False


# ---------------------------------------------------------------------------
# autotuning
# ---------------------------------------------------------------------------

def _i2():
    import ctypes
    return (ctypes.c_int * 2)()


def tune_reorder(src, dst, n, *, reps=3, ws=None, stream=None):
    """Pick the fastest bit-identical first-occurrence / relabel variants for this size."""
    m = src.numel()
    perm = torch.empty(n, dtype=torch.int32, device=src.device)
    so, do = torch.empty_like(src), torch.empty_like(dst)
    buf = _ws(ws, boba_reorder_workspace_bytes(m, n), src.device)
    ch = _i2()
    check(load().boba_tune_reorder(_p(src), _p(dst), m, n, _p(perm), _p(so), _p(do), _p(buf),
                                   buf.numel(), reps, ch, _s(stream)), "boba_tune_reorder")
    return {"first": ch[0], "relabel": ch[1]}


def tune_batched(src, dst, edge_off, vert_off, max_m, max_n, *, reps=3, stream=None):
    G = edge_off.numel() - 1
    total_m, total_n = src.numel(), int(vert_off[-1].item())
    perm = torch.empty(total_n, dtype=torch.int32, device=src.device)
    so, do = torch.empty_like(src), torch.empty_like(dst)
    lib = load()
    sizes = []
    for mode in (0, 1):                       # scratch for whichever schedule is tried
        lib.boba_batched_set_mode(mode)
        sizes.append(lib.boba_reorder_batched_workspace_bytes(G, max_m, max_n, total_m, total_n))
    lib.boba_batched_set_mode(-1)
    nbytes = max(sizes)
    buf = torch.empty(nbytes, dtype=torch.uint8, device=src.device)
    ch = _i2()
    check(load().boba_tune_batched(_p(src), _p(dst), _p(edge_off), _p(vert_off), G, max_m, max_n,
                                   total_m, total_n, _p(perm), _p(so), _p(do), _p(buf), buf.numel(),
                                   reps, ch, _s(stream)), "boba_tune_batched")
    return {"batched": ch[0]}


def tune_spmv(row_ptr, col, val, x, *, reps=3, stream=None):
    n_rows, nnz = row_ptr.numel() - 1, col.numel()
    y = torch.empty(n_rows, dtype=torch.float32, device=x.device)
    buf = _ws(None, boba_spmv_workspace_bytes(n_rows, nnz), x.device)
    ch = _i2()
    check(load().boba_tune_spmv(_p(row_ptr), _p(col), _p(val), _p(x), _p(y), n_rows, nnz, _p(buf),
                                buf.numel(), reps, ch, _s(stream)), "boba_tune_spmv")
    return {"spmv": ch[0]}


def tune_csr(src, dst, n, *, reps=3, stream=None):
    m = src.numel()
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device=src.device)
    col = torch.empty(m, dtype=torch.int32, device=src.device)
    val = torch.empty(m, dtype=torch.float32, device=src.device)
    buf = _ws(None, boba_coo_to_csr_workspace_bytes(m, n), src.device)
    ch = _i2()
    check(load().boba_tune_csr(_p(src), _p(dst), m, n, _p(row_ptr), _p(col), _p(val), _p(buf),
                               buf.numel(), reps, ch, _s(stream)), "boba_tune_csr")
    return {"csr": ch[0]}


def tune_save(path):
    check(load().boba_tune_save(str(path).encode()), "boba_tune_save")


def tune_load(path):
    check(load().boba_tune_load(str(path).encode()), "boba_tune_load")


def tune_reset():
    load().boba_tune_reset()


def nbr(row_ptr, col, *, ids_per_line=32, ws=None, stream=None):
    """(NBR, rows counted) of a CSR on the GPU (Sec. 5.2)."""
    import ctypes
    n_rows, nnz = row_ptr.numel() - 1, col.numel()
    buf = _ws(ws, load().boba_nbr_workspace_bytes(n_rows, nnz), row_ptr.device)
    out = ctypes.c_double(0.0)
    cnt = ctypes.c_int64(0)
    check(load().boba_nbr(_p(row_ptr), _p(col), n_rows, nnz, ids_per_line, ctypes.byref(out),
                          ctypes.byref(cnt), _p(buf), buf.numel(), _s(stream)), "boba_nbr")
    return out.value, cnt.value


def sort_by_dst(src, dst, n, *, bin_only=False, src_out=None, dst_out=None, ws=None, stream=None):
    """COO stably sorted (or binned by the top 8 bits) by destination: (src_out, dst_out)."""
    m = src.numel()
    src_out = torch.empty_like(src) if src_out is None else src_out
    dst_out = torch.empty_like(dst) if dst_out is None else dst_out
    buf = _ws(ws, load().boba_sort_by_dst_workspace_bytes(m, n), src.device)
    check(load().boba_sort_by_dst(_p(src), _p(dst), m, n, _p(src_out), _p(dst_out), int(bin_only),
                                  _p(buf), buf.numel(), _s(stream)), "boba_sort_by_dst")
    return src_out, dst_out
