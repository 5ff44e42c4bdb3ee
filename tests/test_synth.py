"""Sanity of the seeded workload generators (inputs only, no BOBA arithmetic)."""
import numpy as np

import synth


def test_deterministic_and_in_range():
    a = synth.rmat(12, 30000, seed=1)
    b = synth.rmat(12, 30000, seed=1)
    c = synth.rmat(12, 30000, seed=2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0])
    for arr in a:
        assert arr.min() >= 0 and arr.max() < 1 << 12


def test_thread_count_does_not_matter(monkeypatch):
    a = synth.rmat(14, 200000, seed=3)
    monkeypatch.setattr(synth, "_threads", lambda: 1)
    b = synth.rmat(14, 200000, seed=3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_rmat_quadrant_skew_without_relabel():
    s, d = synth.rmat(16, 400000, seed=4, relabel=False, shuffle=False)
    # the top bit of src is 0 with probability a + b = 0.76, of dst with a + c = 0.76
    assert abs(np.mean(s < (1 << 15)) - 0.76) < 0.01
    assert abs(np.mean(d < (1 << 15)) - 0.76) < 0.01
    # shuffling permutes the same edge multiset
    s2, d2 = synth.rmat(16, 400000, seed=4, relabel=False, shuffle=True)
    k1 = np.sort(s.astype(np.int64) << 32 | d)
    k2 = np.sort(s2.astype(np.int64) << 32 | d2)
    assert np.array_equal(k1, k2)


def test_rmat_non_power_of_two_n():
    s, d = synth.rmat(10, 5000, seed=5, n=700)
    assert s.max() < 700 and d.max() < 700


def test_grid_structure():
    side = 9
    s, d = synth.grid(side, seed=6, relabel=False, shuffle=False)
    assert len(s) == 4 * side * (side - 1)
    pairs = set(zip(s.tolist(), d.tolist()))
    assert len(pairs) == len(s)                          # no duplicates
    assert all((b, a) in pairs for a, b in pairs)        # both directions
    for a, b in pairs:
        ra, ca, rb, cb = a // side, a % side, b // side, b % side
        assert abs(ra - rb) + abs(ca - cb) == 1
    deg = np.bincount(s, minlength=side * side)
    assert deg.min() == 2 and deg.max() == 4


def test_permutation_is_bijection():
    for N in (1, 2, 3, 1000, 4096, 12345):
        p = synth.permutation(N, seed=7)
        assert np.array_equal(np.sort(p), np.arange(N))


def test_uniform_vector():
    x = synth.uniform_f32(100000, seed=8)
    assert x.min() >= 0.0 and x.max() < 1.0 and abs(x.mean() - 0.5) < 0.01


def test_batch_sizes_recipe():
    n, m = synth.batch_sizes(4096, seed=9)
    assert n.min() >= 256 and n.max() < (1 << 18)
    ef = m // n
    assert np.all(m == n * ef) and ef.min() == 4 and ef.max() == 32
    lg = np.log2(n)
    assert abs(lg.mean() - 13.0) < 0.2                  # log-uniform on [8, 18]
    s, d, eo, vo = synth.rmat_batch(6, seed=9, log2_hi=10)
    for g in range(6):
        ng = vo[g + 1] - vo[g]
        assert s[eo[g]:eo[g + 1]].max() < ng and d[eo[g]:eo[g + 1]].max() < ng


def test_edge_range_is_a_slice():
    full = synth.rmat(12, 100000, seed=10)
    part = synth.rmat(12, 100000, seed=10, edge_range=(30000, 70001))
    assert np.array_equal(part[0], full[0][30000:70001])
    assert np.array_equal(part[1], full[1][30000:70001])
    g = synth.grid(20, seed=3)
    gp = synth.grid(20, seed=3, edge_range=(5, 17))
    assert np.array_equal(gp[0], g[0][5:17])
