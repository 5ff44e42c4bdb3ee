"""Autotuner: every launch variant gives the same bits; the tuner only picks among
bit-identical variants; choices round-trip through the tune file."""
import numpy as np
import pytest
import torch

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def boba():
    import paper_2306_10410_gb300 as b
    b.load()
    yield b
    b.tune_reset()


def test_every_reorder_variant_is_bit_exact(boba):
    I, J = synth.rmat(16, 1_000_003, seed=31)
    n = 1 << 16
    operm, oso, odo = oracle.reorder(I, J, n)
    src, dst = torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda()
    # 0..5 launch shapes, 6 warp-aggregated lookups, 7 bulk-copied streams
    for kernel in (boba.TUNE_FIRST, boba.TUNE_RELABEL):
        for v in range(8):
            boba.tune_reset()
            boba.load().boba_tune_set(kernel, len(I), v)
            assert boba.load().boba_tune_get(kernel, len(I)) == v
            perm, so, do = boba.reorder(src, dst, n)
            boba.stream_status()
            np.testing.assert_array_equal(perm.cpu().numpy(), operm, err_msg=f"{kernel}/{v}")
            np.testing.assert_array_equal(so.cpu().numpy(), oso, err_msg=f"{kernel}/{v}")
            np.testing.assert_array_equal(do.cpu().numpy(), odo, err_msg=f"{kernel}/{v}")
    boba.tune_reset()


def test_tuner_picks_and_persists(boba, tmp_path):
    I, J = synth.rmat(18, 1 << 22, seed=32)
    n = 1 << 18
    src, dst = torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda()
    boba.tune_reset()
    ch = boba.tune_reorder(src, dst, n, reps=2)
    assert 0 <= ch["first"] < 8 and 0 <= ch["relabel"] < 8
    path = tmp_path / "tune.txt"
    boba.tune_save(path)
    boba.tune_reset()
    assert boba.load().boba_tune_get(boba.TUNE_FIRST, len(I)) == 0
    boba.tune_load(path)
    assert boba.load().boba_tune_get(boba.TUNE_FIRST, len(I)) == ch["first"]
    assert boba.load().boba_tune_get(boba.TUNE_RELABEL, len(I)) == ch["relabel"]
    perm, so, do = boba.reorder(src, dst, n)
    boba.stream_status()
    operm, oso, odo = oracle.reorder(I, J, n)
    np.testing.assert_array_equal(perm.cpu().numpy(), operm)
    np.testing.assert_array_equal(so.cpu().numpy(), oso)
    boba.tune_reset()


def test_tune_batched_and_spmv(boba):
    src, dst, eo, vo = synth.rmat_batch(64, seed=33, log2_lo=8, log2_hi=17)
    s_d, d_d = torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda()
    eo_d, vo_d = torch.from_numpy(eo).cuda(), torch.from_numpy(vo).cuda()
    ch = boba.tune_batched(s_d, d_d, eo_d, vo_d, int(np.diff(eo).max()), int(np.diff(vo).max()),
                           reps=2)
    assert 0 <= ch["batched"] < 9
    perm, so, do = boba.reorder_batched(s_d, d_d, eo_d, vo_d)
    boba.stream_status()
    for g in (0, 31, 63):
        operm, _, _ = oracle.reorder(src[eo[g]:eo[g + 1]], dst[eo[g]:eo[g + 1]], int(vo[g + 1] - vo[g]))
        np.testing.assert_array_equal(perm.cpu().numpy()[vo[g]:vo[g + 1]], operm)
    w = synth.RMAT14
    I, J = w.generate()
    rp, col, val = boba.coo_to_csr(torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda(), w.n)
    x = torch.from_numpy(synth.uniform_f32(w.n, seed=3)).cuda()
    ch = boba.tune_spmv(rp, col, val, x, reps=2)
    assert 0 <= ch["spmv"] < 15
    orp, ocol, oval = oracle.coo_to_csr(I, J, w.n)
    y64 = oracle.spmv_f64(orp, ocol, oval, x.cpu().numpy())
    for v in range(15):                      # every variant within the bound
        boba.load().boba_tune_set(boba.TUNE_SPMV, col.numel(), v)
        y = boba.spmv(rp, col, val, x)
        boba.stream_status()
        err = np.linalg.norm(y.cpu().numpy() - y64) / np.linalg.norm(y64)
        assert err <= 1e-5, (v, err)
    boba.tune_reset()


CSR_RANKINGS = tuple(range(10))       # ranking x tile shape x look-back or prescan


def test_csr_ranking_variants_bit_identical(boba):
    I, J = synth.rmat(17, 800_001, seed=35)
    n = 1 << 17
    # a second graph whose digits are mostly equal: one hub row takes half the
    # edges, so whole warps share a digit in every pass
    rng = np.random.default_rng(36)
    m2 = 300_017
    I2 = rng.integers(0, n, m2, dtype=np.int32)
    J2 = np.where(rng.random(m2) < 0.5, 70_000, rng.integers(0, n, m2)).astype(np.int32)
    for I_, J_ in ((I, J), (I2, J2)):
        orp, ocol, oval = oracle.coo_to_csr(I_, J_, n)
        for v in CSR_RANKINGS:
            boba.load().boba_tune_set(boba.TUNE_CSR, len(I_), v)
            rp, col, val = boba.coo_to_csr(torch.from_numpy(I_).cuda(), torch.from_numpy(J_).cuda(),
                                           n)
            boba.stream_status()
            np.testing.assert_array_equal(rp.cpu().numpy(), orp, err_msg=f"variant {v}")
            np.testing.assert_array_equal(col.cpu().numpy(), ocol, err_msg=f"variant {v}")
            np.testing.assert_array_equal(val.cpu().numpy(), oval, err_msg=f"variant {v}")
        boba.load().boba_tune_set(boba.TUNE_CSR, len(I_), -1)
    ch = boba.tune_csr(torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda(), n, reps=2)
    assert ch["csr"] in CSR_RANKINGS
    boba.tune_reset()


@pytest.mark.parametrize("n,m", [(1, 1_000), (256, 70_001), (257, 70_001), (65_537, 300_007),
                                 (200, (1 << 22) + 77)])
def test_csr_variants_across_pass_counts(boba, n, m):
    """Every radix variant on one pass (n <= 256: the run ends are found after
    the sort), two and three passes, and a tiny n under many edges (the
    reduce-then-scan default with a single pass), ragged m throughout."""
    rng = np.random.default_rng(n + m)
    I = rng.integers(0, n, m, dtype=np.int32)
    J = np.where(rng.random(m) < 0.3, n - 1, rng.integers(0, n, m)).astype(np.int32)
    orp, ocol, oval = oracle.coo_to_csr(I, J, n)
    src, dst = torch.from_numpy(I).cuda(), torch.from_numpy(J).cuda()
    for v in CSR_RANKINGS:
        boba.load().boba_tune_set(boba.TUNE_CSR, m, v)
        rp, col, val = boba.coo_to_csr(src, dst, n)
        boba.stream_status()
        np.testing.assert_array_equal(rp.cpu().numpy(), orp, err_msg=f"variant {v}")
        np.testing.assert_array_equal(col.cpu().numpy(), ocol, err_msg=f"variant {v}")
        np.testing.assert_array_equal(val.cpu().numpy().view(np.uint32), oval.view(np.uint32),
                                      err_msg=f"variant {v}")
    boba.load().boba_tune_set(boba.TUNE_CSR, m, -1)
