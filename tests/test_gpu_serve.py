"""Serving: requests admitted under an HBM budget and run concurrently give the
same results as the same requests run alone (bit for bit: every kernel treats
each request on its own), and match the oracle."""
import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu

SPMV_RTOL = 1e-5


@pytest.fixture(scope="module")
def serve():
    import paper_2306_10410_gb300 as b
    b.load()
    from paper_2306_10410_gb300 import serve as s
    return s


def test_mix_equals_alone_and_oracle(serve):
    pool = serve.request_pool(12, seed=77, m_lo=1e4, m_hi=3e5)
    # alone: one request at a time
    alone = []
    with serve.Server(budget_bytes=2 << 30, spmv_iters=10) as srv:
        for g in pool:
            y = serve._pinned_out(g["n"])
            p = torch.empty(g["n"], dtype=torch.int32, pin_memory=True)
            srv.submit(g["src"], g["dst"], g["n"], g["x"], y, p)
            srv.drain()
            assert all(st == 0 for _, _, st in srv.poll())
            alone.append((y.clone(), p.clone()))
    # mixed: 36 requests submitted back to back (several waves, overlapping streams)
    order = [i % len(pool) for i in range(36)]
    outs = []
    with serve.Server(budget_bytes=2 << 30, spmv_iters=10, max_active=16) as srv:
        for i in order:
            g = pool[i]
            y = serve._pinned_out(g["n"])
            p = torch.empty(g["n"], dtype=torch.int32, pin_memory=True)
            srv.submit(g["src"], g["dst"], g["n"], g["x"], y, p)
            outs.append((i, y, p))
        srv.drain()
        done = srv.poll()
        assert len(done) == 36 and all(st == 0 for _, _, st in done)
        st = srv.stats()
        assert st["requests"] == 36 and st["peak_pool_bytes"] <= 2 << 30
        # continuous batching: requests joined while others were on the GPU, and
        # the device work of several requests overlapped in time
        assert st["peak_active"] > 1, st
        assert st["joined_while_busy"] > 0, st
        assert st["peak_device_overlap"] > 1, st
    for i, y, p in outs:
        assert torch.equal(y, alone[i][0]), i
        assert torch.equal(p, alone[i][1]), i
    # against the oracle: perm, and y within the fp32 bound
    for i in (0, 5, 11):
        g = pool[i]
        I, J = g["src"].numpy(), g["dst"].numpy()
        operm, oI, oJ = oracle.reorder(I, J, g["n"])
        np.testing.assert_array_equal(alone[i][1].numpy(), operm)
        rp, col, val = oracle.coo_to_csr(oI, oJ, g["n"])
        y64 = oracle.spmv_f64(rp, col, val, g["x"].numpy())
        err = np.linalg.norm(alone[i][0].numpy() - y64) / max(np.linalg.norm(y64), 1e-30)
        assert err <= SPMV_RTOL, err


def test_budget_limits_residency(serve):
    pool = serve.request_pool(4, seed=78, m_lo=2e5, m_hi=3e5)
    budget = 96 << 20                      # room for only a few such requests at once
    with serve.Server(budget_bytes=budget, spmv_iters=2, max_active=64) as srv:
        for _ in range(3):
            for g in pool:
                srv.submit(g["src"], g["dst"], g["n"], g["x"], serve._pinned_out(g["n"]))
        srv.drain()
        done = srv.poll()
        st = srv.stats()
    assert len(done) == 12 and all(s == 0 for _, _, s in done)
    assert 0 < st["peak_pool_bytes"] <= budget


def test_cancel_waiting_requests(serve):
    """A request still queued can be withdrawn; the rest complete correctly."""
    pool = serve.request_pool(4, seed=80, m_lo=2e5, m_hi=3e5)
    with serve.Server(budget_bytes=64 << 20, spmv_iters=2, max_active=2) as srv:
        ids = []
        for _ in range(4):
            for g in pool:
                ids.append(srv.submit(g["src"], g["dst"], g["n"], g["x"],
                                      serve._pinned_out(g["n"])))
        cancelled = {rid for rid in ids[-6:] if srv.cancel(rid)}
        assert not srv.cancel(10 ** 9)                 # unknown id
        srv.drain()
        done = srv.poll()
    got = {rid for rid, _, st in done if st == 0}
    assert len(cancelled) > 0
    assert got == set(ids) - cancelled
    assert all(st == 0 for _, _, st in done)


def test_request_too_large_is_refused(serve):
    import paper_2306_10410_gb300 as b
    pool = serve.request_pool(1, seed=79, m_lo=1e6, m_hi=1e6)
    g = pool[0]
    with serve.Server(budget_bytes=8 << 20, spmv_iters=1) as srv:
        with pytest.raises(b.BobaError) as e:
            srv.submit(g["src"], g["dst"], g["n"], g["x"], serve._pinned_out(g["n"]))
        assert e.value.code == 4


@pytest.mark.slow
def test_poisson_stream_small(serve):
    st = serve.serve_workload(n_requests=60, pool_size=8, load=0.8, m_lo=1e4, m_hi=2e6,
                              budget_bytes=8 << 30, spmv_iters=10)
    assert st["requests"] == 60 and st["p99_ms"] >= st["p50_ms"] > 0 and st["gedges_s"] > 0


def test_saturated_server_equals_one_request_at_a_time(serve):
    """The served results at saturation equal, bit for bit, the same requests run
    one after another through boba_reorder_ex / boba_coo_to_csr / boba_spmv_csr."""
    res = serve.serve_vs_sequential(n_requests=20, pool_size=6, m_lo=1e4, m_hi=5e5,
                                    budget_bytes=4 << 30, spmv_iters=3, max_active=16)
    assert res["identical"]
    sat = res["saturated"]
    assert sat["requests"] == 20 and sat["peak_active"] > 1
    assert res["sequential"]["requests"] == 20
