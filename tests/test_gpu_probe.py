"""boba_probe_gather, the random-load ceiling measurement: arguments are
validated before any launch, every mode runs, reports the loads it issued,
and the rates keep their order (an L1-resident table faster than an
L2-resident one, shared memory faster than L2)."""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def boba():
    import paper_2306_10410_gb300 as b
    b.load()
    return b


def run(boba, mode, words, cluster=0, per_thread=256, reps=3):
    table = torch.arange(1 << 22, dtype=torch.int32, device="cuda")
    out_words = 152 * 16 * 256
    out = torch.zeros(out_words, dtype=torch.int32, device="cuda")
    issued = ctypes.c_int64(0)
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rc = boba.boba_probe_gather(mode, table, words, per_thread, cluster, out, out_words,
                                    issued)
        e1.record()
        if rc != 0:
            return rc, None, None
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    boba.stream_status()
    assert int(out.abs().sum().item()) > 0          # the loads were not optimised away
    return 0, issued.value, issued.value / (min(times) * 1e-3)


def test_probe_modes_and_order(boba):
    rc, n_g, r_l2 = run(boba, 0, 1 << 20)              # 4 MiB: L2
    assert rc == 0 and n_g > 0 and n_g % 256 == 0
    rc, _, r_l1 = run(boba, 0, 1 << 13)                # 32 KiB: L1
    assert rc == 0
    rc, _, r_sh = run(boba, 1, 1 << 13)                # 32 KiB per block in shared memory
    assert rc == 0
    rc, n_c, r_cl = run(boba, 2, 1 << 16, cluster=4)   # 256 KiB over 4-block clusters
    assert rc == 0 and n_c > 0
    assert r_l1 > r_l2 and r_sh > r_l2, (r_l1, r_sh, r_l2)


def test_probe_rejects_bad_arguments(boba):
    t = torch.zeros(1 << 10, dtype=torch.int32, device="cuda")
    o = torch.zeros(256, dtype=torch.int32, device="cuda")
    n = ctypes.c_int64(0)
    assert boba.boba_probe_gather(3, t, 1 << 10, 8, 0, o, 256, n) == 1        # no such mode
    assert boba.boba_probe_gather(0, t, 1000, 8, 0, o, 256, n) == 1           # not a power of two
    assert boba.boba_probe_gather(0, t, 1 << 10, 7, 0, o, 256, n) == 1        # not a multiple of 8
    assert boba.boba_probe_gather(1, t, 1 << 16, 8, 0, o, 256, n) == 1        # 256 KiB > 227 KiB
    assert boba.boba_probe_gather(2, t, 1 << 10, 8, 3, o, 256, n) == 1        # cluster of 3
    assert n.value == 0
