"""GPU PageRank (the PR application of Sec. 5.1) against the fp64 oracle.

Tolerance: each step is one fp32 SpMV, whose relative error is within the SpMV
bound 1e-5, plus fp32 rounding of the ranks (6e-8).  The error e_t of the
iterate obeys e_{t+1} = d A e_t + delta_t with ||A||_1 <= 1, so it stays below
max ||delta|| / (1 - d) = 6.7e-5 for d = 0.85; the relative L1 bound is 1e-4.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

PR_RTOL = 1e-4
D = 0.85


@pytest.fixture(scope="module")
def boba():
    import paper_2306_10410_gb300 as b
    b.load()
    return b


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def graph(case):
    rng = np.random.default_rng(17)
    if case == "rmat14":
        w = synth.RMAT14
        I, J = w.generate()
        return I, J, w.n
    if case == "rmat14_boba":
        w = synth.RMAT14
        I, J = w.generate()
        _, I, J = oracle.reorder(I, J, w.n)
        return I, J, w.n
    if case == "ragged_dangling":                 # many vertices with no out-edge
        n = 70001
        I = rng.integers(0, n // 3, 150_001).astype(np.int32)
        J = rng.integers(0, n, 150_001).astype(np.int32)
        return I, J, n
    if case == "hubs":                            # rows crossing many merge-path tiles
        n = 3000
        I = rng.integers(0, n, 300_000).astype(np.int32)
        J = np.where(rng.random(300_000) < 0.5, 17, rng.integers(0, n, 300_000)).astype(np.int32)
        return I, J, n
    if case == "two_vertex":
        return np.array([0], np.int32), np.array([1], np.int32), 2
    if case == "n1":
        return np.zeros(5, np.int32), np.zeros(5, np.int32), 1
    if case == "no_edges":
        return np.zeros(0, np.int32), np.zeros(0, np.int32), 4097
    raise ValueError(case)


def rel_l1(a, b):
    return np.abs(np.asarray(a, np.float64) - b).sum() / np.abs(b).sum()


@pytest.mark.parametrize("case", ["rmat14", "rmat14_boba", "ragged_dangling", "hubs",
                                  "two_vertex", "n1", "no_edges"])
def test_fixed_steps_parity(boba, case):
    I, J, n = graph(case)
    csr = boba.coo_to_csr(dev(I), dev(J), n)
    pr, steps, res = boba.pagerank(*csr, damping=D, max_iters=30, tol=0.0)
    boba.stream_status()
    want, ost, ores = oracle.pagerank(I, J, n, D, 30, 0.0)
    assert int(steps.item()) == ost == 30
    got = pr.cpu().numpy()
    assert rel_l1(got, want) <= PR_RTOL, rel_l1(got, want)
    assert abs(float(res.item()) - ores) <= 1e-4 * max(ores, 1e-3) + 1e-6
    if case == "two_vertex":
        np.testing.assert_allclose(got, [1 / (2 + D), (1 + D) / (2 + D)], rtol=1e-6)


def test_converges_like_the_oracle(boba):
    I, J, n = graph("rmat14_boba")
    csr = boba.coo_to_csr(dev(I), dev(J), n)
    tol = 1e-7
    pr, steps, res = boba.pagerank(*csr, damping=D, max_iters=500, tol=tol)
    boba.stream_status()
    want, ost, ores = oracle.pagerank(I, J, n, D, 500, tol)
    assert ost < 500
    assert abs(int(steps.item()) - ost) <= 1          # the stop test is an fp decision
    assert float(res.item()) < tol
    assert rel_l1(pr.cpu().numpy(), want) <= PR_RTOL


def test_deterministic_and_stops_early(boba):
    """Two runs give the same bits; steps after convergence leave pr untouched."""
    I, J, n = graph("hubs")
    csr = boba.coo_to_csr(dev(I), dev(J), n)
    a, sa, _ = boba.pagerank(*csr, damping=D, max_iters=200, tol=1e-6)
    b, sb, _ = boba.pagerank(*csr, damping=D, max_iters=200, tol=1e-6)
    c, sc, _ = boba.pagerank(*csr, damping=D, max_iters=int(sa.item()), tol=0.0)
    boba.stream_status()
    assert torch.equal(a, b) and int(sa.item()) == int(sb.item()) < 200
    assert torch.equal(a, c)


@pytest.mark.parametrize("variant", list(range(5, 14)))
def test_every_merge_path_shape(boba, variant):
    I, J, n = graph("rmat14")
    csr = boba.coo_to_csr(dev(I), dev(J), n)
    boba.load().boba_tune_set(boba.TUNE_SPMV, csr[1].numel(), variant)
    try:
        pr, steps, _ = boba.pagerank(*csr, damping=D, max_iters=20, tol=0.0)
        boba.stream_status()
    finally:
        boba.load().boba_tune_set(boba.TUNE_SPMV, csr[1].numel(), -1)
    want, _, _ = oracle.pagerank(I, J, n, D, 20, 0.0)
    assert rel_l1(pr.cpu().numpy(), want) <= PR_RTOL


def test_edge_cases_and_errors(boba):
    I, J, n = graph("rmat14")
    csr = boba.coo_to_csr(dev(I), dev(J), n)
    pr, steps, res = boba.pagerank(*csr, max_iters=0)
    boba.stream_status()
    assert int(steps.item()) == 0
    assert torch.all(pr == np.float32(1.0 / n))
    with pytest.raises(boba.BobaError) as e:
        boba.pagerank(*csr, damping=1.0)
    assert e.value.code == 1
    with pytest.raises(boba.BobaError):
        boba.pagerank(*csr, tol=-1.0)
    # a column ID outside [0, n): recorded, and no step runs
    rp, col, val = csr
    bad = col.clone()
    bad[5] = n
    pr, steps, _ = boba.pagerank(rp, bad, val, max_iters=10)
    with pytest.raises(boba.BobaError) as e:
        boba.stream_status()
    assert e.value.code == 2
    assert int(steps.item()) == 0
    assert torch.all(pr == np.float32(1.0 / n))
    boba.stream_status()


@pytest.mark.slow
def test_full_size_rmat24_pagerank(boba):
    """R-MAT scale 24 with 2^28 edges in BOBA order, 5 steps, against the oracle."""
    w = synth.RMAT24
    I, J = w.generate()
    perm, so, do = boba.reorder(dev(I), dev(J), w.n)
    boba.stream_status()
    Io, Jo = so.cpu().numpy(), do.cpu().numpy()
    del I, J, perm
    csr = boba.coo_to_csr(so, do, w.n)
    del so, do
    pr, steps, _ = boba.pagerank(*csr, damping=D, max_iters=5, tol=0.0)
    boba.stream_status()
    want, _, _ = oracle.pagerank(Io, Jo, w.n, D, 5, 0.0)
    assert int(steps.item()) == 5
    assert rel_l1(pr.cpu().numpy(), want) <= PR_RTOL
