"""Host logic of the served-vs-sequential comparison (no GPU): the two forms
run in alternating pairs, the speedup is the median of the paired ratios,
the reported runs are each form's median round, and any round whose outputs
differ makes the comparison non-identical."""
import itertools

import pytest
import torch

import paper_2306_10410_gb300.serve as serve


def fake_runs(monkeypatch, sat_rates, seq_rates, differ_round=None):
    """Replace the GPU legs by runs with the given throughputs (one per round)."""
    calls = []
    sat_it, seq_it = iter(sat_rates), iter(seq_rates)
    rounds = itertools.count()

    def run_saturated(pool, order, budget, iters, max_active):
        r = next(sat_it)
        calls.append(("sat", r))
        return {"gedges_s_wall": r, "tag": "sat%g" % r}, [torch.ones(3)], [torch.arange(3)]

    def run_sequential(pool, order, iters):
        r = next(seq_it)
        k = next(rounds)
        calls.append(("seq", r))
        y = torch.ones(3) if k != differ_round else torch.zeros(3)
        return {"gedges_s_wall": r, "tag": "seq%g" % r}, [y], [torch.arange(3)]

    monkeypatch.setattr(serve, "run_saturated", run_saturated)
    monkeypatch.setattr(serve, "run_sequential", run_sequential)
    monkeypatch.setattr(serve, "request_order", lambda n, p, seed: list(range(n)))
    return calls


POOL = [{"m": 10}, {"m": 20}]


def test_pairs_alternate_and_median_of_ratios(monkeypatch):
    calls = fake_runs(monkeypatch, [6.0, 3.0, 5.0], [4.0, 3.0, 2.0])
    res = serve.serve_vs_sequential(n_requests=2, pool=POOL, rounds=3)
    assert [c[0] for c in calls] == ["sat", "seq"] * 3          # alternating pairs
    # paired ratios 1.5, 1.0, 2.5 -> median 1.5 (not 5.0 / 3.0 from the medians)
    assert res["speedup_served_vs_sequential"] == pytest.approx(1.5)
    assert res["saturated"]["tag"] == "sat5" and res["sequential"]["tag"] == "seq3"
    assert res["rounds_gedges_s"] == {"saturated": [6.0, 3.0, 5.0], "sequential": [4.0, 3.0, 2.0]}
    assert res["identical"] is True
    assert res["edges"] == 30 and res["n_requests"] == 2


def test_any_differing_round_is_reported(monkeypatch):
    fake_runs(monkeypatch, [5.0, 5.0, 5.0], [4.0, 4.0, 4.0], differ_round=2)
    res = serve.serve_vs_sequential(n_requests=2, pool=POOL, rounds=3)
    assert res["identical"] is False


def test_one_round_is_a_single_pair(monkeypatch):
    calls = fake_runs(monkeypatch, [5.0], [4.0])
    res = serve.serve_vs_sequential(n_requests=1, pool=POOL, rounds=1)
    assert len(calls) == 2
    assert res["speedup_served_vs_sequential"] == pytest.approx(1.25)
