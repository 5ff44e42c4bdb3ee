"""boba_reorder_static, the reorder entry point that allocates nothing.

It serves callers that cannot call cudaMalloc where they need a reorder (all
device memory owned by a pool or arena, a host framework that forbids
allocation on its hot path, a loop that cannot afford an allocation's implicit
synchronisation).  Its scratch is a fixed array in the library's device image.

The test calls it through the C ABI (ctypes on libboba.so) several times in a
row, on graphs of different sizes, and checks each result bit for bit against
the workspace entry point boba_reorder_ex on the same input.  This file is
named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _call_static(lib, src, dst, n, err, stream):
    m = src.numel()
    perm = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    so = torch.full((m,), -7, dtype=torch.int32, device="cuda")
    do = torch.full((m,), -7, dtype=torch.int32, device="cuda")
    rc = lib.boba_reorder_static(_ptr(src), _ptr(dst), m, n, _ptr(perm), _ptr(so), _ptr(do),
                                 _ptr(err), ctypes.c_void_p(stream.cuda_stream))
    return rc, perm, so, do


def test_static_entry_matches_workspace_entry_on_calls_in_a_row():
    import paper_2306_10410_gb300 as boba
    lib = boba.load()
    stream = torch.cuda.current_stream()
    big = synth.er(1 << 20, 1 << 22, seed=41)                 # at both limits
    small = synth.RMAT14.generate()                          # 2^18 edges, 2^14 vertices
    odd = synth.rmat(17, 1_000_003, seed=42, n=100_003)      # ragged sizes, misses tiles
    cases = [(big, 1 << 20), (small, 1 << 14), (odd, 100_003), (big, 1 << 20)]
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    for (I, J), n in cases:
        src = torch.from_numpy(I).cuda()
        dst = torch.from_numpy(J).cuda()
        perm_ref, so_ref, do_ref = boba.reorder(src, dst, n)
        boba.stream_status()
        rc, perm, so, do = _call_static(lib, src, dst, n, err, stream)
        assert rc == 0, boba.boba_status_string(rc)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        assert torch.equal(perm, perm_ref)
        assert torch.equal(so, so_ref)
        assert torch.equal(do, do_ref)


def test_static_entry_limits_and_errors():
    import paper_2306_10410_gb300 as boba
    lib = boba.load()
    stream = torch.cuda.current_stream()
    src = torch.zeros(4, dtype=torch.int32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = ctypes.c_void_p(stream.cuda_stream)
    # beyond the stated maxima: refused before any launch
    assert lib.boba_reorder_static(_ptr(src), _ptr(src), (1 << 22) + 1, 16, _ptr(src), _ptr(src),
                                   _ptr(src), None, s) == 3
    assert lib.boba_reorder_static(_ptr(src), _ptr(src), 4, (1 << 20) + 1, _ptr(src), _ptr(src),
                                   _ptr(src), None, s) == 3
    # an ID outside [0, n) is reported through the caller's error word
    I = torch.tensor([0, 1, 9, 2], dtype=torch.int32, device="cuda")
    rc, perm, so, do = _call_static(lib, I, I, 5, err, stream)
    assert rc == 0
    torch.cuda.synchronize()
    assert int(err.item()) & (1 << 2)
    assert int(so[2].item()) == -1 and int(do[2].item()) == -1
    # and the next call is clean again
    err.zero_()
    J = torch.tensor([0, 1, 3, 2], dtype=torch.int32, device="cuda")
    rc, perm, so, do = _call_static(lib, J, J, 5, err, stream)
    torch.cuda.synchronize()
    assert rc == 0 and int(err.item()) == 0
    assert perm.cpu().tolist() == [0, 1, 3, 2, 4]


def test_static_entry_misaligned_views_and_no_edges():
    """Inputs one element into their buffers (not 16-byte aligned: the scalar
    first-occurrence and relabel kernels run), and a graph with no edges (only
    the key initialisation and the rank kernel run); each bit for bit equal to
    boba_reorder_ex, twice in a row."""
    import paper_2306_10410_gb300 as boba
    lib = boba.load()
    stream = torch.cuda.current_stream()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    I, J = synth.rmat(15, 300_001, seed=43, n=30_011)
    srcb = torch.from_numpy(np.concatenate([[0], I]).astype(np.int32)).cuda()
    dstb = torch.from_numpy(np.concatenate([[0], J]).astype(np.int32)).cuda()
    src, dst = srcb[1:], dstb[1:]
    assert src.data_ptr() % 16 != 0 and dst.data_ptr() % 16 != 0
    for _ in range(2):
        perm_ref, so_ref, do_ref = boba.reorder(src, dst, 30_011)
        boba.stream_status()
        rc, perm, so, do = _call_static(lib, src, dst, 30_011, err, stream)
        assert rc == 0, boba.boba_status_string(rc)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        assert torch.equal(perm, perm_ref)
        assert torch.equal(so, so_ref)
        assert torch.equal(do, do_ref)
    empty = torch.zeros(0, dtype=torch.int32, device="cuda")
    for _ in range(2):
        perm_ref, _, _ = boba.reorder(empty, empty, 7)
        boba.stream_status()
        rc, perm, so, do = _call_static(lib, empty, empty, 7, err, stream)
        assert rc == 0, boba.boba_status_string(rc)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        assert torch.equal(perm, perm_ref)
        assert perm.cpu().tolist() == list(range(7))
