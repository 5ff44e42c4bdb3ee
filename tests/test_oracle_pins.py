"""Pins for the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: each check is a value printed in
the paper, a brute-force definition written independently in Python, a library
routine that solves a special case, or an invariant that must hold.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth

SENT = oracle.SENT


# --------------------------------------------------------------------------
# independent brute-force definitions (pure Python, tiny inputs only)
# --------------------------------------------------------------------------

def brute_keys(I, J, n):
    """key(v) = min{i : (I ++ J)[i] == v} by a double loop over vertices and positions."""
    stream = list(I) + list(J)
    keys = []
    for v in range(n):
        best = SENT
        for i, w in enumerate(stream):
            if w == v and i < best:
                best = i
        keys.append(best)
    return keys


def brute_perm(I, J, n):
    """Vertices sorted by (key, original id): the first-occurrence order with the isolated tail."""
    keys = brute_keys(I, J, n)
    return sorted(range(n), key=lambda v: (keys[v], v))


def letters_to_ids(tokens, alphabet):
    return [alphabet.index(t) for t in tokens]


# --------------------------------------------------------------------------
# worked examples printed in the paper
# --------------------------------------------------------------------------

def test_fig2_roads_printed_order(golden):
    """Fig. 2: the printed uniquified order T M R G C B V S N E L P D, labels 1..13."""
    g = golden("fig2_roads.txt")
    alphabet = sorted(set(g["I"]) | set(g["J"]))       # any integer naming works
    assert len(alphabet) == 13 and len(g["I"]) == len(g["J"]) == 24
    I = letters_to_ids(g["I"], alphabet)
    J = letters_to_ids(g["J"], alphabet)
    perm, label = oracle.boba_perm(I, J, len(alphabet))
    assert [alphabet[v] for v in perm] == g["order"]
    # labels printed 1-based under the order
    for name, lab in zip(g["order"], g["labels"]):
        assert label[alphabet.index(name)] + 1 == int(lab)


def test_fig2_relabel_invariant_to_naming(golden):
    """The new labels do not depend on how the letters are numbered."""
    g = golden("fig2_roads.txt")
    base = sorted(set(g["I"]))
    outs = []
    for alphabet in (base, base[::-1], base[3:] + base[:3]):
        I = letters_to_ids(g["I"], alphabet)
        J = letters_to_ids(g["J"], alphabet)
        perm, Io, Jo = oracle.reorder(I, J, 13)
        outs.append((Io.tolist(), Jo.tolist(), [alphabet[v] for v in perm]))
    assert outs[0] == outs[1] == outs[2]


def test_fig1_star_interleaved_row_is_printed(golden):
    """Fig. 1 prints the uniquification of the interleaved flattening."""
    g = golden("fig1_star.txt")
    alphabet = sorted(set(g["I"]) | set(g["J"]))
    flat = [t for pair in zip(g["I"], g["J"]) for t in pair]
    assert flat == g["flattened"]                       # the transcription is consistent
    I = letters_to_ids(g["I"], alphabet)
    J = letters_to_ids(g["J"], alphabet)
    perm, _ = oracle.boba_perm_interleaved(I, J, len(alphabet))
    assert [alphabet[v] for v in perm] == g["uniquified"]


def test_fig1_star_concatenated(golden):
    """Alg. 1 / Alg. 2 scan I ++ J: the star's order is I's own order."""
    g = golden("fig1_star.txt")
    alphabet = sorted(set(g["I"]) | set(g["J"]))
    I = letters_to_ids(g["I"], alphabet)
    J = letters_to_ids(g["J"], alphabet)
    perm, _ = oracle.boba_perm(I, J, len(alphabet))
    assert [alphabet[v] for v in perm] == g["concat_uniquified"]
    assert [alphabet[v] for v in perm] == g["I"]


# --------------------------------------------------------------------------
# brute force
# --------------------------------------------------------------------------

def _all_coos(n, m):
    for I in itertools.product(range(n), repeat=m):
        for J in itertools.product(range(n), repeat=m):
            yield list(I), list(J)


@pytest.mark.parametrize("n,m", [(1, 0), (1, 1), (2, 1), (2, 2), (3, 1), (3, 2), (3, 3), (4, 2)])
def test_exhaustive_small(n, m):
    for I, J in _all_coos(n, m):
        perm, label = oracle.boba_perm(I, J, n)
        assert perm.tolist() == brute_perm(I, J, n), (I, J)
        assert oracle.first_keys(I, J, n).tolist() == brute_keys(I, J, n), (I, J)
        assert label[perm].tolist() == list(range(n))


def test_random_small_brute_force():
    rng = np.random.default_rng(12345)
    for _ in range(3000):
        n = int(rng.integers(1, 9))
        m = int(rng.integers(0, 25))
        I = rng.integers(0, n, m).tolist()
        J = rng.integers(0, n, m).tolist()
        if rng.random() < 0.2 and m:                    # force self-loops
            J = list(I)
        perm, label = oracle.boba_perm(I, J, n)
        assert perm.tolist() == brute_perm(I, J, n)
        assert oracle.first_keys(I, J, n).tolist() == brute_keys(I, J, n)
        Io, Jo = oracle.relabel(I, J, label, n)
        assert Io.tolist() == [int(label[v]) for v in I]
        assert Jo.tolist() == [int(label[v]) for v in J]


# --------------------------------------------------------------------------
# invariants (any size)
# --------------------------------------------------------------------------

def check_invariants(I, J, n, perm, Io, Jo):
    I = np.asarray(I); J = np.asarray(J)
    m = I.shape[0]
    assert np.array_equal(np.sort(perm), np.arange(n))             # bijection
    assert np.array_equal(perm[Io], I) and np.array_equal(perm[Jo], J)   # edges kept in place
    keys = oracle.first_keys(I, J, n)
    kp = keys[perm].astype(np.int64)
    app = int((kp != SENT).sum())
    assert np.all(kp[:app] != SENT) and np.all(kp[app:] == SENT)
    assert np.all(np.diff(kp[:app]) > 0)                           # keys strictly increase
    assert np.all(np.diff(perm[app:]) > 0)                         # isolated tail ascending
    if m:
        assert Io[0] == 0


def test_invariants_rmat14():
    w = synth.RMAT14
    I, J = w.generate()
    perm, Io, Jo = oracle.reorder(I, J, w.n)
    check_invariants(I, J, w.n, perm, Io, Jo)
    # idempotence: BOBA of the output is the identity
    perm2, Io2, Jo2 = oracle.reorder(Io, Jo, w.n)
    assert np.array_equal(perm2, np.arange(w.n))
    assert np.array_equal(Io2, Io) and np.array_equal(Jo2, Jo)


def test_relabel_invariance_metamorphic():
    """Renaming the input vertices by any permutation pi leaves src_out/dst_out unchanged."""
    I, J = synth.rmat(10, 6000, seed=99)
    n = 1 << 10
    pi = synth.permutation(n, seed=5)
    perm, Io, Jo = oracle.reorder(I, J, n)
    perm_b, Io_b, Jo_b = oracle.reorder(pi[I], pi[J], n)
    assert np.array_equal(Io, Io_b) and np.array_equal(Jo, Jo_b)
    app = len(np.unique(np.concatenate([I, J])))
    assert np.array_equal(perm_b[:app], pi[perm[:app]])


@pytest.mark.parametrize("case", ["empty", "selfloops", "hub", "isolated_heavy", "n1"])
def test_special_cases(case):
    if case == "empty":
        I, J, n = [], [], 5
    elif case == "selfloops":
        I = [3, 1, 3, 0]; J = list(I); n = 5
    elif case == "hub":
        I = [2] * 50; J = [7] * 50; n = 9
    elif case == "isolated_heavy":
        I = [900, 3]; J = [3, 17]; n = 1000
    else:
        I = [0, 0]; J = [0, 0]; n = 1
    perm, Io, Jo = oracle.reorder(I, J, n)
    assert perm.tolist() == brute_perm(I, J, n)
    check_invariants(I, J, n, perm, Io, Jo)
    if case == "empty":
        assert perm.tolist() == list(range(n))
    if case == "hub":
        assert perm[:2].tolist() == [2, 7] and set(Io.tolist()) == {0} and set(Jo.tolist()) == {1}


def test_out_of_range_ids_rejected():
    with pytest.raises(oracle.OracleError):
        oracle.boba_perm([0, 5], [1, 1], 5)
    with pytest.raises(oracle.OracleError):
        oracle.boba_perm([0, -1], [1, 1], 5)
    with pytest.raises(oracle.OracleError):
        oracle.first_keys([0], [0], 0)


def test_planted_mistake_is_caught():
    """A plausible slip -- scanning J ++ I instead of I ++ J -- fails the Fig. 2 pin."""
    from conftest import read_golden
    g = read_golden("fig2_roads.txt")
    alphabet = sorted(set(g["I"]))
    I = letters_to_ids(g["I"], alphabet)
    J = letters_to_ids(g["J"], alphabet)
    perm_swapped, _ = oracle.boba_perm(J, I, 13)
    assert [alphabet[v] for v in perm_swapped] != g["order"]


# --------------------------------------------------------------------------
# CSR, SpMV, NBR
# --------------------------------------------------------------------------

def test_csr_equals_library_stable_sort():
    """A stable counting sort by row is np.argsort(kind='stable') on the row array."""
    I, J = synth.rmat(12, 40000, seed=3)
    n = 1 << 12
    row_ptr, col, val = oracle.coo_to_csr(I, J, n)
    order = np.argsort(J, kind="stable")
    assert np.array_equal(col, I[order])
    assert np.array_equal(row_ptr, np.concatenate([[0], np.cumsum(np.bincount(J, minlength=n))]))
    outdeg = np.bincount(I, minlength=n)
    assert np.array_equal(val, (1.0 / outdeg[I[order]]).astype(np.float32))


def test_csr_values_closed_form():
    """Column c holds outdeg(c) entries, each the fp32 value nearest 1/outdeg(c)."""
    I, J = synth.rmat(10, 9000, seed=8)
    n = 1 << 10
    row_ptr, col, val = oracle.coo_to_csr(I, J, n)
    outdeg = np.bincount(I, minlength=n)
    for c in np.unique(col)[:200]:
        vals = val[col == c]
        assert vals.shape[0] == outdeg[c]
        q = np.float32(1.0) / np.float32(outdeg[c])     # IEEE fp32 division
        assert np.all(vals == q)
        assert abs(float(vals.astype(np.float64).sum()) - 1.0) < 1e-6


def test_spmv_against_scipy_and_closed_forms():
    sp = pytest.importorskip("scipy.sparse")
    I, J = synth.rmat(12, 50000, seed=4)
    n = 1 << 12
    row_ptr, col, val = oracle.coo_to_csr(I, J, n)
    x = synth.uniform_f32(n, seed=4)
    y = oracle.spmv_f64(row_ptr, col, val, x)
    A = sp.csr_matrix((val.astype(np.float64), col, row_ptr), shape=(n, n))
    np.testing.assert_allclose(y, A @ x.astype(np.float64), rtol=1e-13, atol=1e-13)
    # y with x = 1 is the row sum of the values
    y1 = oracle.spmv_f64(row_ptr, col, val, np.ones(n, np.float32))
    np.testing.assert_allclose(y1, np.add.reduceat(np.r_[val.astype(np.float64), 0],
                                                   row_ptr[:-1])
                               * (np.diff(row_ptr) > 0), rtol=1e-12)
    # sum(y) = sum_c x_c * outdeg_c * val_c  (the matrix's column sums)
    outdeg = np.bincount(I, minlength=n).astype(np.float64)
    colval = np.zeros(n); colval[col] = val
    assert abs(y.sum() - float((x * outdeg * colval).sum())) < 1e-9 * max(1.0, y.sum())


def test_spmv_small_hand_example():
    # edges 0->1, 2->1, 1->0 : rows (dst) 0: [1], 1: [0, 2]
    row_ptr, col, val = oracle.coo_to_csr([0, 2, 1], [1, 1, 0], 3)
    assert row_ptr.tolist() == [0, 1, 3, 3] and col.tolist() == [1, 0, 2]
    y = oracle.spmv_f64(row_ptr, col, val, np.array([1.0, 2.0, 4.0], np.float32))
    assert y.tolist() == [2.0, 5.0, 0.0]


def brute_nbr(row_ptr, col, L):
    tot, cnt = 0.0, 0
    for r in range(len(row_ptr) - 1):
        nb = set(col[row_ptr[r]:row_ptr[r + 1]].tolist())
        if not nb:
            continue
        tot += len({u // L for u in nb}) / len(nb)
        cnt += 1
    return tot / cnt if cnt else 0.0, cnt


def test_nbr_hand_and_brute():
    # row 0: {0,1,2} one line -> 1/3 ; row 1: {0, 32} -> 2/2 ; row 2: {5,5} -> 1/1 ; row 3 empty
    row_ptr = np.array([0, 3, 5, 7, 7]); col = np.array([0, 1, 2, 0, 32, 5, 5])
    v, c = oracle.nbr(row_ptr, col, 32)
    assert c == 3 and abs(v - (1 / 3 + 1 + 1) / 3) < 1e-15
    I, J = synth.rmat(11, 20000, seed=6)
    for L in (1, 8, 32):
        rp, cl, _ = oracle.coo_to_csr(J, I, 1 << 11)     # out-neighbour rows
        v, c = oracle.nbr(rp, cl, L)
        bv, bc = brute_nbr(rp, cl, L)
        assert c == bc and abs(v - bv) < 1e-12
    v1, _ = oracle.nbr(rp, cl, 1)
    assert v1 == 1.0                                     # one ID per line: ratio is 1


def test_sort_by_dst_pins():
    """The full sort is the CSR's edge order; the binned order has non-decreasing
    top digits and keeps input order within a bin (brute force)."""
    I, J = synth.rmat(12, 30000, seed=13)
    n = 1 << 12
    Is, Js = oracle.sort_by_dst(I, J, n)
    rp, col, _ = oracle.coo_to_csr(I, J, n)
    assert np.array_equal(Is, col)
    assert np.array_equal(Js, np.repeat(np.arange(n), np.diff(rp)))
    Ib, Jb = oracle.sort_by_dst(I, J, n, top_digit_only=True)
    top = lambda j: j >> 4                                  # top 8 of 12 bits: 256 bins
    assert np.all(np.diff(top(Jb)) >= 0)
    for d in range(0, 256, 37):
        sel = top(J) == d
        assert np.array_equal(Ib[top(Jb) == d], I[sel]) and np.array_equal(Jb[top(Jb) == d], J[sel])


# --- PageRank (Sec. 5.1 applications) -------------------------------------------

def google_matrix(I, J, n, d):
    """The dense Google matrix, entry by entry: column u spreads pr(u) over u's
    out-edges (duplicates counted), or over all n vertices when u has none."""
    outdeg = np.bincount(np.asarray(I, dtype=np.int64), minlength=n)
    G = np.zeros((n, n))
    for u, v in zip(I, J):
        G[v, u] += 1.0 / outdeg[u]
    for u in range(n):
        if outdeg[u] == 0:
            G[:, u] = 1.0 / n
    return d * G + (1.0 - d) / n


def stationary(G):
    """The eigenvector of G for the eigenvalue nearest 1, scaled to sum 1."""
    w, V = np.linalg.eig(G)
    k = int(np.argmin(np.abs(w - 1.0)))
    assert abs(w[k] - 1.0) < 1e-9
    v = np.real(V[:, k])
    return v / v.sum()


def random_small_graph(rng, n, m):
    I = rng.integers(0, n, m).astype(np.int32)
    J = rng.integers(0, n, m).astype(np.int32)
    return I, J


@pytest.mark.parametrize("d", [0.0, 0.5, 0.85, 0.95])
def test_pagerank_two_vertex_closed_form(d):
    """One edge 0 -> 1 (vertex 1 dangling): pr = (1/(2+d), (1+d)/(2+d))."""
    pr, steps, res = oracle.pagerank([0], [1], 2, d, 10000, 1e-15)
    np.testing.assert_allclose(pr, [1 / (2 + d), (1 + d) / (2 + d)], rtol=0, atol=1e-13)
    assert res < 1e-15


def test_pagerank_cycle_is_uniform():
    n = 9
    I = np.arange(n, dtype=np.int32)
    J = (I + 1) % n
    pr, steps, res = oracle.pagerank(I, J, n, 0.85, 50)
    np.testing.assert_allclose(pr, np.full(n, 1 / n), rtol=0, atol=1e-15)
    assert steps == 50 and res < 1e-15


def test_pagerank_is_the_google_eigenvector():
    """Converged power iteration equals the stationary vector of the dense Google
    matrix, found by an eigen-decomposition (dangling vertices, duplicated edges
    and self-loops included)."""
    rng = np.random.default_rng(2024)
    for trial in range(40):
        n = int(rng.integers(1, 13))
        m = int(rng.integers(0, 3 * n + 1))
        I, J = random_small_graph(rng, n, m)
        d = float(rng.choice([0.3, 0.85, 0.9]))
        pr, steps, res = oracle.pagerank(I, J, n, d, 100000, 1e-15)
        np.testing.assert_allclose(pr, stationary(google_matrix(I, J, n, d)), rtol=0,
                                   atol=1e-11, err_msg=f"trial {trial}")


def test_pagerank_mass_and_special_cases():
    rng = np.random.default_rng(5)
    I, J = random_small_graph(rng, 30, 40)            # many dangling vertices
    for t in range(6):
        pr, steps, res = oracle.pagerank(I, J, 30, 0.85, t)
        assert steps == t
        assert abs(pr.sum() - 1.0) < 1e-13            # mass is conserved every step
        if t == 0:
            np.testing.assert_array_equal(pr, np.full(30, 1 / 30))
    pr, _, _ = oracle.pagerank(I, J, 30, 0.0, 1)      # no damping weight on edges
    np.testing.assert_allclose(pr, np.full(30, 1 / 30), rtol=0, atol=1e-16)
    pr, _, _ = oracle.pagerank([], [], 7, 0.85, 10)   # no edges: everything dangling
    np.testing.assert_allclose(pr, np.full(7, 1 / 7), rtol=0, atol=1e-16)
    pr, _, _ = oracle.pagerank([0, 0], [0, 0], 1, 0.85, 10)
    np.testing.assert_allclose(pr, [1.0], rtol=0, atol=1e-15)
    with pytest.raises(oracle.OracleError):
        oracle.pagerank([0], [2], 2, 0.85, 5)
    with pytest.raises(oracle.OracleError):
        oracle.pagerank([0], [1], 2, 1.0, 5)


def test_pagerank_planted_mistakes_fail_the_eigen_pin():
    """Plausible slips in a power iteration (dropped dangling term, normalising by
    in-degree, transposed edges) all miss the eigenvector pin."""
    rng = np.random.default_rng(11)
    n, d = 12, 0.85
    I, J = random_small_graph(rng, n, 20)
    I[0], J[0] = 3, 3
    want = stationary(google_matrix(I, J, n, d))

    def power(I, J, deg, dangling):
        pr = np.full(n, 1 / n)
        for _ in range(500):
            nxt = np.zeros(n)
            for u, v in zip(I, J):
                nxt[v] += pr[u] / deg[u]
            D = pr[deg == 0].sum() if dangling else 0.0
            pr = (1 - d) / n + d * (nxt + D / n)
        return pr

    outdeg = np.bincount(I, minlength=n)
    indeg = np.bincount(J, minlength=n)
    np.testing.assert_allclose(power(I, J, outdeg, True), want, atol=1e-11)
    assert np.abs(power(I, J, outdeg, False) - want).max() > 1e-3
    assert np.abs(power(I, J, np.maximum(indeg, 1), True) - want).max() > 1e-3
    assert np.abs(power(J, I, np.bincount(J, minlength=n), True) - want).max() > 1e-3


# --- theory of Sec. 4.1 and 4.4 (informational: they check the paper's claims) ---

def nscore(adj, p):
    """NScore(G, p) = sum over consecutive p_i, p_{i+1} of |N(p_i) & N(p_{i+1})| (Sec. 4.1)."""
    return sum(len(adj[p[i]] & adj[p[i + 1]]) for i in range(len(p) - 1))


def small_regular_graphs():
    """(name, undirected edges, n, d) for d-regular graphs with n <= 8."""
    out = [(f"C{n}", [(i, (i + 1) % n) for i in range(n)], n, 2) for n in range(5, 9)]
    out.append(("K4", [(a, b) for a in range(4) for b in range(a + 1, 4)], 4, 3))
    out.append(("K33", [(a, b) for a in range(3) for b in range(3, 6)], 6, 3))
    out.append(("Q3", [(a, a ^ (1 << k)) for a in range(8) for k in range(3) if a < a ^ (1 << k)],
                8, 3))
    out.append(("K5", [(a, b) for a in range(5) for b in range(a + 1, 5)], 5, 4))
    out.append(("K44", [(a, b) for a in range(4) for b in range(4, 8)], 8, 4))
    return out


def adjacency(edges, n):
    adj = [set() for _ in range(n)]
    for u, v in edges:
        adj[u].add(v)
        adj[v].add(u)
    return adj


def best_nscore(adj, n):
    return max(nscore(adj, p) for p in itertools.permutations(range(n)))


def test_lemma1_bound_is_the_degree_sum():
    """Lemma 1: NScore(G, p*) <= m.  The proof bounds the sum by the degree sum,
    which is 2|E| for an undirected graph (its COO lists both directions); with
    m = |E| the statement fails, e.g. on K3,3 (p* scores 12, |E| = 9)."""
    for name, edges, n, _ in small_regular_graphs():
        adj = adjacency(edges, n)
        best = best_nscore(adj, n)
        assert best <= sum(len(a) for a in adj), name
    k33 = [(a, b) for a in range(3) for b in range(3, 6)]
    assert best_nscore(adjacency(k33, 6), 6) == 12 > len(k33)


def test_prop1_regular_graph_sorted_by_destination():
    """Prop. 1: for a d-regular graph whose COO is sorted by destination, the
    BOBA order scores at least 1/(d+1) of the optimum (checked by brute force)."""
    for name, edges, n, d in small_regular_graphs():
        arcs = sorted([(u, v) for u, v in edges] + [(v, u) for u, v in edges],
                      key=lambda a: (a[1], a[0]))
        I = np.array([a[0] for a in arcs], np.int32)
        J = np.array([a[1] for a in arcs], np.int32)
        perm, _ = oracle.boba_perm(I, J, n)
        adj = adjacency(edges, n)
        assert (d + 1) * nscore(adj, list(perm)) >= best_nscore(adj, n), name
