"""Failure detection without a GPU fault: a bounded device wait that can never be
satisfied gives up, reports BOBA_ERR_TIMEOUT through the status word, and the
context stays usable (the next reorder is correct)."""
import time

import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


def test_wait_gives_up_and_reports_timeout():
    import paper_2306_10410_gb300 as boba
    scratch = torch.empty(4, dtype=torch.int64, device="cuda")
    t0 = time.perf_counter()
    assert boba.boba_selftest_wait_timeout(20_000_000, scratch) == 0      # 20 ms
    with pytest.raises(boba.BobaError) as e:
        boba.stream_status()
    elapsed = time.perf_counter() - t0
    assert e.value.code == 5                                             # BOBA_ERR_TIMEOUT
    assert elapsed < 5.0
    boba.stream_status()                                                 # word cleared
    I, J = synth.RMAT14.generate()                                       # context still fine
    perm, so, do = boba.reorder(torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda(),
                                synth.RMAT14.n)
    boba.stream_status()
    operm, _, _ = oracle.reorder(I, J, synth.RMAT14.n)
    np.testing.assert_array_equal(perm.cpu().numpy(), operm)


def test_selftest_argument_checks():
    import paper_2306_10410_gb300 as boba
    scratch = torch.empty(4, dtype=torch.int64, device="cuda")
    assert boba.boba_selftest_wait_timeout(0, scratch) == 1
    assert boba.boba_selftest_wait_timeout(3_000_000_000, scratch) == 1
    assert boba.boba_selftest_wait_timeout(1000, None) == 1
