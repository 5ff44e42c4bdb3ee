"""GPU parity of the batched reorder: every graph of the batch equals the oracle
(and the single-graph entry point) bit for bit."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

KCAP = 54 * 1024          # vertices one CTA keeps in shared memory
TEAM_MAX = 8 * KCAP       # largest graph a cluster handles


@pytest.fixture(scope="module")
def boba():
    import paper_2306_10410_gb300 as b
    b.load()
    yield b
    b.boba_batched_set_mode(-1)


MODES = [pytest.param(0, id="cluster"), pytest.param(1, id="split"),
         pytest.param(2, id="sliced"), pytest.param(3, id="sliced_mixed"),
         pytest.param(4, id="global"), pytest.param(5, id="sliced_small"),
         pytest.param(6, id="relabel_runs"), pytest.param(7, id="runs"),
         pytest.param(8, id="runs_first")]


def pack(graphs):
    """graphs: list of (I, J, n) -> packed numpy arrays and offsets."""
    eo = np.zeros(len(graphs) + 1, np.int64)
    vo = np.zeros(len(graphs) + 1, np.int64)
    for g, (I, J, n) in enumerate(graphs):
        eo[g + 1] = eo[g] + len(I)
        vo[g + 1] = vo[g] + n
    src = np.concatenate([np.asarray(I, np.int32) for I, _, _ in graphs] or [np.zeros(0, np.int32)])
    dst = np.concatenate([np.asarray(J, np.int32) for _, J, _ in graphs] or [np.zeros(0, np.int32)])
    return src, dst, eo, vo


def run_batched(boba, src, dst, eo, vo):
    perm, so, do = boba.reorder_batched(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(),
                                        torch.from_numpy(eo).cuda(), torch.from_numpy(vo).cuda())
    boba.stream_status()
    return perm.cpu().numpy(), so.cpu().numpy(), do.cpu().numpy()


def check_against_oracle(graphs, perm, so, do, eo, vo, which=None):
    for g in (range(len(graphs)) if which is None else which):
        I, J, n = graphs[g]
        operm, oso, odo = oracle.reorder(I, J, n)
        np.testing.assert_array_equal(perm[vo[g]:vo[g + 1]], operm, err_msg=f"graph {g}")
        np.testing.assert_array_equal(so[eo[g]:eo[g + 1]], oso, err_msg=f"graph {g}")
        np.testing.assert_array_equal(do[eo[g]:eo[g + 1]], odo, err_msg=f"graph {g}")


@pytest.mark.parametrize("mode", MODES)
def test_mixed_small_batch(boba, mode):
    boba.boba_batched_set_mode(mode)
    rng = np.random.default_rng(0)
    graphs = []
    for g in range(60):
        kind = g % 6
        if kind == 0:
            n, m = 0, 0                                     # empty graph
        elif kind == 1:
            n, m = int(rng.integers(1, 50)), 0              # vertices only
        elif kind == 2:
            n, m = 1, int(rng.integers(1, 30))              # single vertex, self-loops
        else:
            n = int(rng.integers(2, 5000))
            m = int(rng.integers(1, 20 * n))
        I = rng.integers(0, max(n, 1), m).astype(np.int32)
        J = rng.integers(0, max(n, 1), m).astype(np.int32)
        graphs.append((I, J, n))
    src, dst, eo, vo = pack(graphs)
    perm, so, do = run_batched(boba, src, dst, eo, vo)
    check_against_oracle(graphs, perm, so, do, eo, vo)


@pytest.mark.parametrize("mode", MODES)
def test_large_graphs(boba, mode):
    """Graphs above one CTA's capacity: an 8-CTA cluster (distributed shared memory)
    or the phase-batched global-memory path."""
    boba.boba_batched_set_mode(mode)
    graphs = []
    for n, m, seed in ((KCAP + 1, 200_000, 1), (150_000, 2_400_000, 2), (TEAM_MAX, 3_000_000, 3),
                       (KCAP, 500_000, 4), (300, 9000, 5)):
        scale = int(np.ceil(np.log2(n)))
        I, J = synth.rmat(scale, m, seed=seed, n=n)
        graphs.append((I, J, n))
    src, dst, eo, vo = pack(graphs)
    perm, so, do = run_batched(boba, src, dst, eo, vo)
    check_against_oracle(graphs, perm, so, do, eo, vo)


@pytest.mark.parametrize("mode", MODES)
def test_rmat_batch_equals_single_graph_entry(boba, mode):
    """A batch drawn like the evaluation's (log-uniform sizes, edge factor 4..32),
    smaller: batched output == boba_reorder per graph == oracle (on a sample)."""
    boba.boba_batched_set_mode(mode)
    src, dst, eo, vo = synth.rmat_batch(300, seed=17, log2_lo=8, log2_hi=17)
    perm, so, do = run_batched(boba, src, dst, eo, vo)
    s_d, d_d = torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda()
    for g in range(300):
        n = int(vo[g + 1] - vo[g])
        p1, s1, d1 = boba.reorder(s_d[eo[g]:eo[g + 1]], d_d[eo[g]:eo[g + 1]], n)
        assert np.array_equal(p1.cpu().numpy(), perm[vo[g]:vo[g + 1]]), g
        assert np.array_equal(s1.cpu().numpy(), so[eo[g]:eo[g + 1]]), g
        assert np.array_equal(d1.cpu().numpy(), do[eo[g]:eo[g + 1]]), g
    boba.stream_status()
    graphs = [(src[eo[g]:eo[g + 1]], dst[eo[g]:eo[g + 1]], int(vo[g + 1] - vo[g]))
              for g in range(300)]
    check_against_oracle(graphs, perm, so, do, eo, vo, which=range(0, 300, 17))


@pytest.mark.parametrize("mode", MODES)
def test_bad_offsets_are_skipped_and_reported(boba, mode):
    boba.boba_batched_set_mode(mode)
    rng = np.random.default_rng(5)
    graphs = [(rng.integers(0, 100, 500).astype(np.int32), rng.integers(0, 100, 500).astype(np.int32),
               100) for _ in range(3)]
    src, dst, eo, vo = pack(graphs)
    eo_bad = eo.copy()
    eo_bad[2] = eo_bad[1] - 1                     # graph 1 has negative size
    perm = torch.full((int(vo[-1]),), -9, dtype=torch.int32, device="cuda")
    p, so, do = boba.reorder_batched(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(),
                                     torch.from_numpy(eo_bad).cuda(), torch.from_numpy(vo).cuda(),
                                     max_m=500, max_n=100, perm_out=perm)
    with pytest.raises(boba.BobaError) as e:
        boba.stream_status()
    assert e.value.code == 1
    operm, _, _ = oracle.reorder(*graphs[0])
    np.testing.assert_array_equal(p.cpu().numpy()[:100], operm)        # graph 0 still done
    assert np.all(p.cpu().numpy()[100:200] == -9)                       # graph 1 skipped


@pytest.mark.parametrize("mode", MODES)
def test_out_of_range_ids_reported(boba, mode):
    """An endpoint outside [0, n) of its own graph raises BOBA_ERR_ID_OUT_OF_RANGE
    and is written as -1; the other graphs of the batch come out unchanged.
    Graph 0 runs in one CTA; graph 1 has three slices, its bad IDs in
    several of them and at both ends of its endpoint stream.  Graph 0's odd
    edge count leaves graph 1's arrays off a 16-byte boundary, and graph 1's
    own count leaves a tail, so its first and last IDs are read one by one."""
    boba.boba_batched_set_mode(mode)
    graphs = []
    for n, m, seed in ((3000, 40_001, 31), (2 * KCAP + 100, 600_003, 32),
                       (3 * KCAP + 7, 900_000, 33), (5000, 60_000, 34)):
        I, J = synth.rmat(int(np.ceil(np.log2(n))), m, seed=seed, n=n)
        graphs.append((I.copy(), J.copy(), n))
    n0, n1 = graphs[0][2], graphs[1][2]
    m1 = len(graphs[1][0])
    bad = {0: [(0, 17, n0), (1, 5, -1)],
           1: [(0, 0, n1 + 7), (1, 999, -3), (0, 400_000, 1 << 30), (1, m1 - 1, n1),
               (0, m1 - 1, -2)]}
    for g, items in bad.items():
        for side, e, v in items:
            graphs[g][side][e] = v
    src, dst, eo, vo = pack(graphs)
    perm, so, do = boba.reorder_batched(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(),
                                        torch.from_numpy(eo).cuda(), torch.from_numpy(vo).cuda())
    with pytest.raises(boba.BobaError) as e:
        boba.stream_status()
    assert e.value.code == 2
    so, do = so.cpu().numpy(), do.cpu().numpy()
    for g, items in bad.items():
        for side, e_, _ in items:
            assert (so if side == 0 else do)[eo[g] + e_] == -1, (g, side, e_)
    check_against_oracle(graphs, perm.cpu().numpy(), so, do, eo, vo, which=[2, 3])
    boba.stream_status()                          # the word was cleared


def test_size_limits(boba):
    z = torch.zeros(8, dtype=torch.int64, device="cuda")
    i = torch.zeros(8, dtype=torch.int32, device="cuda")
    boba.boba_batched_set_mode(0)          # cluster mode: key array must fit a cluster
    assert boba.boba_reorder_batched(i, i, z, z, 1, 4, TEAM_MAX + 1, 4, 4, i, i, i, None, 0) == 3
    boba.boba_batched_set_mode(-1)
    assert boba.boba_reorder_batched_workspace_bytes(4096, 1 << 23, TEAM_MAX, 1 << 31, 1 << 28) > 0


@pytest.mark.parametrize("mode", [1, 2, 4, 6, 7, 8])
def test_split_mode_takes_graphs_beyond_cluster_capacity(boba, mode):
    boba.boba_batched_set_mode(mode)           # the largest go to the global phases
    graphs = []
    for n, m, seed in ((TEAM_MAX + 5000, 900_000, 21), (3000, 40_000, 22), (1 << 20, 3_000_000, 23),
                       (50_000, 2_500_000, 24)):                 # last: small n, many edges
        scale = int(np.ceil(np.log2(n)))
        I, J = synth.rmat(scale, m, seed=seed, n=n)
        graphs.append((I, J, n))
    src, dst, eo, vo = pack(graphs)
    perm, so, do = run_batched(boba, src, dst, eo, vo)
    check_against_oracle(graphs, perm, so, do, eo, vo)


@pytest.mark.slow
def test_full_batch_4096_graphs(boba):
    """The evaluation's batch: 4096 R-MAT graphs, n log-uniform in [2^8, 2^18),
    edge factor 4..32 (about 2.8e9 edges).  Every graph is compared with the
    single-graph entry point on the GPU; a sample of graphs with the oracle."""
    G = 4096
    src, dst, eo, vo = synth.rmat_batch(G, seed=synth.SEED_BASE + 3)
    s_d, d_d = torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda()
    eo_d, vo_d = torch.from_numpy(eo).cuda(), torch.from_numpy(vo).cuda()
    boba.boba_batched_set_mode(0)
    perm0, so0, do0 = boba.reorder_batched(s_d, d_d, eo_d, vo_d)
    boba.boba_batched_set_mode(4)            # global large phases only
    perm2, so2, do2 = boba.reorder_batched(s_d, d_d, eo_d, vo_d)
    boba.boba_batched_set_mode(1)
    perm, so, do = boba.reorder_batched(s_d, d_d, eo_d, vo_d)
    boba.stream_status()
    assert torch.equal(perm0, perm) and torch.equal(so0, so) and torch.equal(do0, do)
    assert torch.equal(perm2, perm) and torch.equal(so2, so) and torch.equal(do2, do)
    del perm0, so0, do0, perm2, so2, do2
    for g in range(G):
        n = int(vo[g + 1] - vo[g])
        p1, s1, d1 = boba.reorder(s_d[eo[g]:eo[g + 1]], d_d[eo[g]:eo[g + 1]], n)
        assert torch.equal(p1, perm[vo[g]:vo[g + 1]]), g
        assert torch.equal(s1, so[eo[g]:eo[g + 1]]), g
        assert torch.equal(d1, do[eo[g]:eo[g + 1]]), g
    boba.stream_status()
    perm_h, so_h, do_h = perm.cpu().numpy(), so.cpu().numpy(), do.cpu().numpy()
    for g in list(range(0, G, 257)) + [int(np.argmax(np.diff(eo)))]:
        I, J, n = src[eo[g]:eo[g + 1]], dst[eo[g]:eo[g + 1]], int(vo[g + 1] - vo[g])
        operm, oso, odo = oracle.reorder(I, J, n)
        np.testing.assert_array_equal(perm_h[vo[g]:vo[g + 1]], operm)
        np.testing.assert_array_equal(so_h[eo[g]:eo[g + 1]], oso)
        np.testing.assert_array_equal(do_h[eo[g]:eo[g + 1]], odo)
