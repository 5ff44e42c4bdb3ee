"""Several ranks (gloo on CPU, world size 2 and 3): the exchange step of a
sharded reorder -- the MIN merge of per-rank first-occurrence keys -- gives
the keys of the whole graph, and the timing reduction takes the slowest rank."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth

SENT = 0xFFFFFFFF


def local_keys(I, J, m_total, e0, n):
    """Keys of a shard, written from the definition (test-only, numpy)."""
    key = np.full(n, SENT, dtype=np.uint64)
    pos_src = e0 + np.arange(len(I), dtype=np.uint64)
    pos_dst = m_total + e0 + np.arange(len(J), dtype=np.uint64)
    np.minimum.at(key, I, pos_src)
    np.minimum.at(key, J, pos_dst)
    return key.astype(np.uint32)


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2306_10410_gb300 import dist as bd
        n = 1 << 11
        I, J = synth.rmat(11, 30011, seed=5)
        m = len(I)
        e0, e1 = bd.shard_bounds(m, rank, world)
        k = local_keys(I[e0:e1], J[e0:e1], m, e0, n)
        merged = bd.merge_keys_min(torch.from_numpy(k.view(np.int32).copy()))
        slowest = bd.max_over_ranks(float(rank + 1))
        q.put((rank, merged.numpy().view(np.uint32).copy(), slowest))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_keys_merge_to_whole_graph(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    I, J = synth.rmat(11, 30011, seed=5)
    want = oracle.first_keys(I, J, 1 << 11)
    for rank, merged, slowest in res:
        np.testing.assert_array_equal(merged, want)
        assert slowest == float(world)


def test_shard_bounds_partition():
    from paper_2306_10410_gb300 import dist as bd
    for total in (0, 1, 7, 1000):
        for world in (1, 2, 3, 8):
            b = [bd.shard_bounds(total, r, world) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == total
            assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))


def test_wire_order_preserves_unsigned_min():
    from paper_2306_10410_gb300 import dist as bd
    a = np.array([0, 1, 0x7FFFFFFF, 0x80000000, SENT - 1, SENT], dtype=np.uint32)
    w = bd.keys_to_wire(torch.from_numpy(a.view(np.int32).copy()))
    order = np.argsort(w.numpy(), kind="stable")
    assert np.array_equal(a[order], np.sort(a))
    assert np.array_equal(bd.wire_to_keys(w).numpy().view(np.uint32), a)
