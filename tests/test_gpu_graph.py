"""The hot path inside a CUDA graph: once the workspaces are sized, reorder ->
CSR -> SpMV is captured as one graph, and every replay gives exactly what the
eager calls give (the calls never allocate and never wait on the host).
Sizes on both sides of 2^22 edges, where the radix passes switch from the
look-back to the reduce-then-scan offsets."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def boba():
    import paper_2306_10410_gb300 as b
    b.load()
    return b


@pytest.mark.parametrize("m", [300_007, (1 << 22) + 4_099])
def test_reorder_csr_spmv_replay_equals_eager(boba, m):
    n = 1 << 18
    I, J = synth.rmat(18, m, seed=61)
    src, dst = torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda()
    x = torch.from_numpy(synth.uniform_f32(n, seed=62)).cuda()
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    so, do = torch.empty_like(src), torch.empty_like(dst)
    rp = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(m, dtype=torch.int32, device="cuda")
    val = torch.empty(m, dtype=torch.float32, device="cuda")
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    ws_r = torch.empty(boba.boba_reorder_workspace_bytes(m, n), dtype=torch.uint8, device="cuda")
    ws_c = torch.empty(boba.boba_coo_to_csr_workspace_bytes(m, n), dtype=torch.uint8,
                       device="cuda")
    ws_s = torch.empty(max(256, boba.boba_spmv_workspace_bytes(n, m)), dtype=torch.uint8,
                       device="cuda")
    outs = (perm, so, do, rp, col, val, y)

    def path(s):
        boba.check(boba.boba_reorder_ex(src, dst, m, n, perm, so, do, None, ws_r, ws_r.numel(), s),
                   "reorder")
        boba.check(boba.boba_coo_to_csr(so, do, m, n, rp, col, val, ws_c, ws_c.numel(), s), "csr")
        boba.check(boba.boba_spmv_csr(rp, col, val, x, y, n, m, ws_s, ws_s.numel(), s), "spmv")

    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        path(side)                                   # eager, and the one-time setup
    side.synchronize()
    boba.stream_status(side)
    eager = [t.clone() for t in outs]
    operm, oso, odo = oracle.reorder(I, J, n)
    np.testing.assert_array_equal(eager[0].cpu().numpy(), operm)

    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        path(side)
    for _ in range(2):
        for t in outs:
            t.fill_(0)
        g.replay()
        torch.cuda.synchronize()
        boba.stream_status()
        for a, b in zip(outs, eager):
            assert torch.equal(a.view(torch.int32) if a.dtype == torch.float32 else a,
                               b.view(torch.int32) if b.dtype == torch.float32 else b)
