"""Guard words around every output and workspace (the stand-in for a memory
checker): each buffer handed to the library is a view into a larger one whose
margins hold a known pattern, and the margins must be untouched afterwards.
Sizes are ragged so that vector paths meet heads and tails."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

PAD = 64                      # elements of guard on each side (256 bytes for 4-byte types)
PATTERN = 0x5A5A5A5A


@pytest.fixture(scope="module")
def boba():
    import paper_2306_10410_gb300 as b
    b.load()
    return b


class Guarded:
    """A device buffer of `numel` elements with PAD guard elements on both sides."""

    def __init__(self, numel, dtype, pinned=False):
        itemsize = torch.empty(0, dtype=dtype).element_size()
        words = (numel * itemsize + 3) // 4
        if pinned:
            self.raw = torch.full((words + 2 * PAD,), PATTERN, dtype=torch.int32).pin_memory()
        else:
            self.raw = torch.full((words + 2 * PAD,), PATTERN, dtype=torch.int32, device="cuda")
        self.words = words
        self.view = self.raw[PAD:PAD + words].view(dtype)[:numel]

    def intact(self):
        r = self.raw.cpu() if self.raw.is_cuda else self.raw
        return bool(torch.all(r[:PAD] == PATTERN) and torch.all(r[PAD + self.words:] == PATTERN))


def ws_guard(nbytes):
    return Guarded((nbytes + 3) // 4 * 4, torch.uint8)


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_reorder_outputs_and_workspace(boba):
    n, m = 70_001, 1_000_003
    I, J = synth.rmat(17, m, seed=41, n=n)
    src, dst = dev(I), dev(J)
    perm, so, do, lab = (Guarded(n, torch.int32), Guarded(m, torch.int32),
                         Guarded(m, torch.int32), Guarded(n, torch.int32))
    nb = boba.boba_reorder_workspace_bytes(m, n)
    ws = ws_guard(nb)
    boba.check(boba.boba_reorder_ex(src, dst, m, n, perm.view, so.view, do.view, lab.view, ws.view,
                                    nb), "reorder")
    boba.stream_status()
    for g in (perm, so, do, lab, ws):
        assert g.intact()
    operm, oso, odo = oracle.reorder(I, J, n)
    np.testing.assert_array_equal(perm.view.cpu().numpy(), operm)
    np.testing.assert_array_equal(so.view.cpu().numpy(), oso)


def test_csr_spmv_pagerank(boba):
    n, m = 70_001, 600_007
    I, J = synth.rmat(17, m, seed=42, n=n)
    src, dst = dev(I), dev(J)
    rp, col, val = Guarded(n + 1, torch.int64), Guarded(m, torch.int32), Guarded(m, torch.float32)
    nb = boba.boba_coo_to_csr_workspace_bytes(m, n)
    ws = ws_guard(nb)
    boba.check(boba.boba_coo_to_csr(src, dst, m, n, rp.view, col.view, val.view, ws.view, nb),
               "csr")
    boba.stream_status()
    for g in (rp, col, val, ws):
        assert g.intact()
    x = dev(synth.uniform_f32(n, seed=3))
    y = Guarded(n, torch.float32)
    for variant in (0, 11):
        boba.load().boba_tune_set(boba.TUNE_SPMV, m, variant)
        nb = boba.boba_spmv_workspace_bytes(n, m)
        ws2 = ws_guard(nb)
        boba.check(boba.boba_spmv_csr(rp.view, col.view, val.view, x, y.view, n, m, ws2.view, nb),
                   "spmv")
        boba.stream_status()
        assert y.intact() and ws2.intact(), variant
    boba.load().boba_tune_set(boba.TUNE_SPMV, m, -1)
    pr = Guarded(n, torch.float32)
    steps, res = Guarded(1, torch.int32), Guarded(1, torch.float64)
    nb = boba.boba_pagerank_workspace_bytes(n, m)
    ws3 = ws_guard(nb)
    boba.check(boba.boba_pagerank(rp.view, col.view, val.view, n, m, 0.85, 7, 0.0, pr.view,
                                  steps.view, res.view, ws3.view, nb), "pagerank")
    boba.stream_status()
    for g in (pr, steps, res, ws3):
        assert g.intact()


def test_batched(boba):
    src, dst, eo, vo = synth.rmat_batch(40, seed=43, log2_lo=8, log2_hi=17)
    G, E, V = 40, int(eo[-1]), int(vo[-1])
    max_m, max_n = int(np.diff(eo).max()), int(np.diff(vo).max())
    for mode in (1, 4):
        boba.boba_batched_set_mode(mode)
        perm, so, do = Guarded(V, torch.int32), Guarded(E, torch.int32), Guarded(E, torch.int32)
        nb = boba.boba_reorder_batched_workspace_bytes(G, max_m, max_n, E, V)
        ws = ws_guard(nb)
        boba.check(boba.boba_reorder_batched(dev(src), dev(dst), dev(eo), dev(vo), G, max_m, max_n,
                                             E, V, perm.view, so.view, do.view, ws.view, nb),
                   "batched")
        boba.stream_status()
        for g in (perm, so, do, ws):
            assert g.intact(), mode
    boba.boba_batched_set_mode(-1)


def test_host_buffers_and_sort(boba):
    n, m = 50_001, 300_005
    I, J = synth.rmat(16, m, seed=44, n=n)
    src_h, dst_h = torch.from_numpy(I).pin_memory(), torch.from_numpy(J).pin_memory()
    perm, so, do = (Guarded(n, torch.int32, pinned=True), Guarded(m, torch.int32, pinned=True),
                    Guarded(m, torch.int32, pinned=True))
    nb = boba.boba_reorder_host_workspace_bytes(m, n)
    ws = ws_guard(nb)
    boba.check(boba.boba_reorder_host(src_h, dst_h, m, n, perm.view, so.view, do.view, ws.view,
                                      nb), "reorder_host")
    boba.stream_status()
    torch.cuda.synchronize()
    for g in (perm, so, do, ws):
        assert g.intact()
    for top in (0, 1):
        s2, d2 = Guarded(m, torch.int32), Guarded(m, torch.int32)
        nb = boba.boba_sort_by_dst_workspace_bytes(m, n)
        ws2 = ws_guard(nb)
        boba.check(boba.boba_sort_by_dst(dev(I), dev(J), m, n, s2.view, d2.view, top, ws2.view,
                                         nb), "sort")
        boba.stream_status()
        for g in (s2, d2, ws2):
            assert g.intact(), top
