"""The sharded reorder with the library's own kernels on several ranks: each
rank (a process) takes a contiguous share of the edges, computes its
first-occurrence keys with boba_first_keys, the ranks merge the key arrays
with an all-reduce MIN (gloo), and every rank derives the labels
(boba_labels_from_keys) and relabels its share (boba_relabel).  The ranks
share the one GPU; their kernels never wait on one another (the only
exchange is the collective on the host side), so this is an ordinary
multi-process run, not an emulation of several devices.  Every rank's perm
and the concatenated relabelled edges must equal the oracle's bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth

pytestmark = pytest.mark.gpu

N_SCALE, M_EDGES, SEED = 16, 1_000_003, 77


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
        torch.cuda.set_device(0)
        import paper_2306_10410_gb300 as boba
        from paper_2306_10410_gb300 import dist as bd
        boba.load()
        I, J = synth.rmat(N_SCALE, M_EDGES, seed=SEED)
        n, m = 1 << N_SCALE, len(I)
        e0, e1 = bd.shard_bounds(m, rank, world)
        src = torch.from_numpy(I[e0:e1].copy()).cuda()
        dst = torch.from_numpy(J[e0:e1].copy()).cuda()
        perm, so, do = bd.sharded_reorder(src, dst, m, n, e0)
        boba.stream_status()
        q.put((rank, e0, perm.cpu().numpy(), so.cpu().numpy(), do.cpu().numpy()))
    except Exception as exc:          # reported to the parent, never swallowed
        q.put((rank, -1, repr(exc), None, None))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_reorder_on_ranks_equals_oracle(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    errs = [r for r in res if r[1] < 0]
    assert not errs, errs
    I, J = synth.rmat(N_SCALE, M_EDGES, seed=SEED)
    n = 1 << N_SCALE
    operm, oso, odo = oracle.reorder(I, J, n)
    res.sort(key=lambda r: r[1])
    for _, _, perm, _, _ in res:
        np.testing.assert_array_equal(perm, operm)
    np.testing.assert_array_equal(np.concatenate([r[3] for r in res]), oso)
    np.testing.assert_array_equal(np.concatenate([r[4] for r in res]), odo)
