"""Host-side pieces of bench.py (no GPU): the algorithmic bytes per kernel,
the relative L2 error, the DRAM traffic read from the committed ncu
summaries, and the lookup roofline built from the probe's figures."""
import json
import os

import numpy as np

import bench


def test_algorithmic_bytes_of_the_reorder_and_spmv():
    m, n = 1 << 28, 1 << 24
    a = bench.algorithmic_bytes(m, n, m)
    assert a["reorder.first"] == 8 * m + 4 * n
    assert a["reorder.relabel"] == 16 * m + 4 * n
    assert a["spmv"] == 8 * m + 16 * n
    # three 8-bit passes for 24-bit keys: two of 16m, the last 12m + 4n
    assert a["csr.pass"] == (2 * 16 * m + 12 * m + 4 * n) // 3


def test_rel_l2():
    y64 = np.array([3.0, 4.0])
    assert bench.rel_l2(y64, y64) == 0.0
    assert abs(bench.rel_l2(np.array([3.0, 4.5]), y64) - 0.1) < 1e-15
    assert bench.rel_l2(np.array([1.0, 0.0]), np.zeros(2)) == 1.0     # zero reference


def test_spmv_errors_from_futures():
    class Done:
        def __init__(self, v):
            self.v = v

        def result(self, timeout=None):
            return self.v

    class Failed:
        def result(self, timeout=None):
            raise RuntimeError("boom")

    futs = {("w", "boba"): Done(np.ones(4)), ("w", "random"): Failed()}
    out = bench.spmv_errors(futs, "w", {"boba": np.ones(4, np.float32), "random": np.ones(4)})
    assert out["boba"] == 0.0
    assert out["random"].startswith("oracle failed")
    assert bench.spmv_errors({}, "w", {"boba": None}) == {"boba": None}


def test_reorder_traffic_from_the_committed_summary():
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        d = json.load(f)["rmat24_m2^28"]
    t = bench.reorder_dram_traffic("rmat24_m2^28", 1 << 28, 1 << 24)
    assert t["reorder.first"]["dram_bytes"] == d["reorder.first"]
    assert t["reorder.relabel"]["alg_bytes"] == 16 * (1 << 28) + 4 * (1 << 24)
    assert t["reorder.first"]["ratio"] > 1.0                 # misses above the compulsory bytes
    assert bench.reorder_dram_traffic("no_such_workload", 1, 1) is None


def test_lookup_roofline():
    g = {"probe": {"global_64MiB": {"loads_per_s": 3.0e11}},
         "reorder_lookups_per_s": {"reorder.first": 2.7e11},
         "lookups_frac_of_ceiling": {"reorder.first": 0.9}}
    r = bench.lookup_roofline(g)
    assert r["peak"] == 3.0e11 and r["frac"]["reorder.first"] == 0.9
    assert bench.lookup_roofline(None) is None


def test_paper_reported_context():
    p = bench.PAPER_REPORTED
    k = p["kron_g500-logn20"]
    assert abs(k["edges"] / (k["ms"] * 1e-3) / 1e9 - k["gedges_s"]) < 0.1
    a = p["arabic-2005"]
    assert abs(a["edges"] / (a["ms"] * 1e-3) / 1e9 - a["gedges_s"]) < 0.1
