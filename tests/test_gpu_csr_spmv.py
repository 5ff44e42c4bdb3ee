"""GPU parity of the measurement path (COO -> CSR, SpMV) against the oracle.

CSR (row_ptr, col, val) is compared bit for bit: the stable sort makes it
unique and val = fp32(1/outdeg) is correctly rounded on both sides.  SpMV is
fp32 against the fp64 oracle with the relative L2 bound 1e-5.
"""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu

SPMV_RTOL = 1e-5          # relative L2 error bound of the fp32 SpMV vs the fp64 oracle


@pytest.fixture(scope="module")
def boba():
    import paper_2306_10410_gb300 as b
    b.load()
    return b


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def check_csr(boba, I, J, n):
    rp, col, val = boba.coo_to_csr(dev(I), dev(J), n)
    boba.stream_status()
    orp, ocol, oval = oracle.coo_to_csr(I, J, n)
    np.testing.assert_array_equal(rp.cpu().numpy(), orp)
    np.testing.assert_array_equal(col.cpu().numpy(), ocol)
    np.testing.assert_array_equal(val.cpu().numpy().view(np.uint32), oval.view(np.uint32))
    return (rp, col, val), (orp, ocol, oval)


def check_spmv(boba, gpu_csr, ora_csr, x):
    rp, col, val = gpu_csr
    y = boba.spmv(rp, col, val, dev(x))
    boba.stream_status()
    y64 = oracle.spmv_f64(*ora_csr, x)
    y32 = y.cpu().numpy().astype(np.float64)
    nrm = np.linalg.norm(y64)
    err = np.linalg.norm(y32 - y64) / nrm if nrm > 0 else np.linalg.norm(y32)
    assert err <= SPMV_RTOL, err
    return y


@pytest.mark.parametrize("case", ["rmat14", "rmat14_reordered", "ragged", "isolated", "tiny",
                                  "n1", "wide_ids"])
def test_csr_and_spmv_parity(boba, case):
    if case.startswith("rmat14"):
        w = synth.RMAT14
        I, J = w.generate()
        n = w.n
        if case == "rmat14_reordered":
            _, I, J = oracle.reorder(I, J, n)
    elif case == "ragged":
        n = 70001
        I, J = synth.er(n, 123457, seed=5)
    elif case == "isolated":
        n = 300000
        I, J = synth.er(n, 5003, seed=6)
    elif case == "tiny":
        n, I, J = 3, np.array([0, 2, 1], np.int32), np.array([1, 1, 0], np.int32)
    elif case == "n1":
        n, I, J = 1, np.zeros(7, np.int32), np.zeros(7, np.int32)
    else:                                    # 3 radix passes (n > 2^16)
        n = (1 << 20) + 3
        I, J = synth.er(n, 400001, seed=7)
    g, o = check_csr(boba, I, J, n)
    x = synth.uniform_f32(n, seed=11)
    check_spmv(boba, g, o, x)


def test_empty_graph(boba):
    n = 1000
    e = np.zeros(0, np.int32)
    rp, col, val = boba.coo_to_csr(dev(e), dev(e), n)
    boba.stream_status()
    assert np.all(rp.cpu().numpy() == 0)
    y = boba.spmv(rp, col, val, dev(synth.uniform_f32(n, seed=1)))
    boba.stream_status()
    assert np.all(y.cpu().numpy() == 0)


def test_long_rows_are_chunked(boba):
    """Hub rows far longer than one chunk (in-degree 50k .. 300k)."""
    n = 5000
    rng = np.random.default_rng(3)
    parts_I, parts_J = [rng.integers(0, n, 200000)], [rng.integers(0, n, 200000)]
    for hub, deg in ((7, 300000), (4999, 50001), (123, 4097), (124, 4096)):
        parts_I.append(rng.integers(0, n, deg))
        parts_J.append(np.full(deg, hub))
    I = np.concatenate(parts_I).astype(np.int32)
    J = np.concatenate(parts_J).astype(np.int32)
    p = rng.permutation(len(I))
    I, J = I[p], J[p]
    g, o = check_csr(boba, I, J, n)
    check_spmv(boba, g, o, synth.uniform_f32(n, seed=2))


def test_spmv_deterministic_and_permutation_equivalent(boba):
    """With x_boba[label[u]] = x_rand[u], y_boba[label[v]] equals y_rand[v] bit for bit:
    both CSRs hold each row's entries in the same edge order."""
    w = synth.RMAT14
    I, J = w.generate()
    n = w.n
    src, dst = dev(I), dev(J)
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    perm, so, do = boba.reorder(src, dst, n, label_out=lab)
    x_rand = dev(synth.uniform_f32(n, seed=9))
    x_boba = torch.empty_like(x_rand)
    x_boba[lab.long()] = x_rand
    csr_r = boba.coo_to_csr(src, dst, n)
    csr_b = boba.coo_to_csr(so, do, n)
    y_r = boba.spmv(*csr_r, x_rand)
    y_r2 = boba.spmv(*csr_r, x_rand)
    y_b = boba.spmv(*csr_b, x_boba)
    boba.stream_status()
    assert torch.equal(y_r, y_r2)
    assert torch.equal(y_b[lab.long()], y_r)


@pytest.mark.slow
def test_full_size_rmat24_csr_spmv(boba):
    """R-MAT scale 24, 2^28 edges, as the benchmark runs it: BOBA reorder, CSR of
    the reordered graph, SpMV; CSR bit-exact and SpMV within 1e-5 of fp64."""
    w = synth.RMAT24
    I, J = w.generate()
    src, dst = dev(I), dev(J)
    perm, so, do = boba.reorder(src, dst, w.n)
    boba.stream_status()
    del src, dst
    Io, Jo = so.cpu().numpy(), do.cpu().numpy()
    operm, oIo, oJo = oracle.reorder(I, J, w.n)
    np.testing.assert_array_equal(Io, oIo)
    np.testing.assert_array_equal(Jo, oJo)
    del I, J, operm
    rp, col, val = boba.coo_to_csr(so, do, w.n)
    boba.stream_status()
    orp, ocol, oval = oracle.coo_to_csr(oIo, oJo, w.n)
    np.testing.assert_array_equal(rp.cpu().numpy(), orp)
    np.testing.assert_array_equal(col.cpu().numpy(), ocol)
    np.testing.assert_array_equal(val.cpu().numpy().view(np.uint32), oval.view(np.uint32))
    x = synth.uniform_f32(w.n, seed=w.seed)
    check_spmv(boba, (rp, col, val), (orp, ocol, oval), x)
    # every SpMV variant -- the lanes-per-row kernels and every merge-path shape,
    # among them the one the tuner picks for this graph -- on this CSR, within
    # the fp32 bound of the fp64 oracle
    check_spmv_all_variants(boba, (rp, col, val), (orp, ocol, oval), x, w.m)
    # the default above ran the reduce-then-scan passes (variant 8); the
    # look-back passes (1, 5) and the other reduce-then-scan ranking (9) too
    for v in (1, 5, 9):
        boba.load().boba_tune_set(boba.TUNE_CSR, w.m, v)
        rp, col, val = boba.coo_to_csr(so, do, w.n)
        boba.stream_status()
        np.testing.assert_array_equal(rp.cpu().numpy(), orp, err_msg=f"variant {v}")
        np.testing.assert_array_equal(col.cpu().numpy(), ocol, err_msg=f"variant {v}")
        np.testing.assert_array_equal(val.cpu().numpy().view(np.uint32), oval.view(np.uint32),
                                      err_msg=f"variant {v}")
    boba.load().boba_tune_set(boba.TUNE_CSR, w.m, -1)


N_SPMV_VARIANTS = 15


def check_spmv_all_variants(boba, gpu_csr, ora_csr, x, nnz):
    """y of every SpMV variant against one fp64 oracle product."""
    rp, col, val = gpu_csr
    y64 = oracle.spmv_f64(*ora_csr, x)
    nrm = np.linalg.norm(y64)
    xd = dev(x)
    errs = {}
    try:
        for v in range(N_SPMV_VARIANTS):
            boba.load().boba_tune_set(boba.TUNE_SPMV, nnz, v)
            y = boba.spmv(rp, col, val, xd)
            boba.stream_status()
            y32 = y.cpu().numpy().astype(np.float64)
            errs[v] = float(np.linalg.norm(y32 - y64) / nrm)
    finally:
        boba.load().boba_tune_set(boba.TUNE_SPMV, nnz, -1)
    bad = {v: e for v, e in errs.items() if not e <= SPMV_RTOL}
    assert not bad, bad
    return errs


@pytest.mark.slow
def test_full_size_rmat24_random_order_csr_spmv(boba):
    """The same graph in its input (random) order, the baseline the benchmark
    compares against: CSR bit-exact, every SpMV variant within 1e-5 of fp64."""
    w = synth.RMAT24
    I, J = w.generate()
    src, dst = dev(I), dev(J)
    rp, col, val = boba.coo_to_csr(src, dst, w.n)
    boba.stream_status()
    del src, dst
    orp, ocol, oval = oracle.coo_to_csr(I, J, w.n)
    del I, J
    np.testing.assert_array_equal(rp.cpu().numpy(), orp)
    np.testing.assert_array_equal(col.cpu().numpy(), ocol)
    np.testing.assert_array_equal(val.cpu().numpy().view(np.uint32), oval.view(np.uint32))
    check_spmv_all_variants(boba, (rp, col, val), (orp, ocol, oval),
                            synth.uniform_f32(w.n, seed=w.seed), w.m)


@pytest.mark.parametrize("variant", list(range(N_SPMV_VARIANTS)))
@pytest.mark.parametrize("case", ["rmat14", "hubs", "empty_rows", "one_row", "no_edges"])
def test_spmv_variants(boba, variant, case):
    """Every SpMV variant (lanes per row 4..32, merge path) within the fp32 bound,
    deterministic run to run; hub rows crossing many merge-path tiles."""
    rng = np.random.default_rng(9)
    if case == "rmat14":
        w = synth.RMAT14
        I, J = w.generate()
        n = w.n
    elif case == "hubs":
        n = 3000
        I = rng.integers(0, n, 400_000).astype(np.int32)
        J = np.where(rng.random(400_000) < 0.5, 17, rng.integers(0, n, 400_000)).astype(np.int32)
    elif case == "empty_rows":                      # most rows empty, trailing empty rows
        n = 100_000
        I = rng.integers(0, n, 20_000).astype(np.int32)
        J = rng.integers(0, 5_000, 20_000).astype(np.int32)
    elif case == "one_row":
        n = 1
        I = np.zeros(70_000, np.int32)
        J = np.zeros(70_000, np.int32)
    else:
        n = 777
        I = np.zeros(0, np.int32)
        J = np.zeros(0, np.int32)
    rp, col, val = boba.coo_to_csr(dev(I), dev(J), n)
    x = dev(synth.uniform_f32(n, seed=12))
    boba.load().boba_tune_set(boba.TUNE_SPMV, col.numel(), variant)
    try:
        y1 = boba.spmv(rp, col, val, x)
        y2 = boba.spmv(rp, col, val, x)
        boba.stream_status()
    finally:
        boba.load().boba_tune_set(boba.TUNE_SPMV, col.numel(), -1)
    assert torch.equal(y1, y2)
    orp, ocol, oval = oracle.coo_to_csr(I, J, n)
    y64 = oracle.spmv_f64(orp, ocol, oval, x.cpu().numpy())
    y32 = y1.cpu().numpy().astype(np.float64)
    nrm = np.linalg.norm(y64)
    err = np.linalg.norm(y32 - y64) / nrm if nrm > 0 else np.linalg.norm(y32)
    assert err <= SPMV_RTOL, err
