"""Host logic of the push-shape autotuner and of the many-graph workload (no GPU)."""

import json
import math

import numpy as np
import pytest

from paper_2306_08967_gb300.autotune import (blocks_for, choose, fleet_signature, measured_weights, plan, tune_grids,
                                             tune_shares)
from synth import FLEETS


def test_blocks_for_rule():
    assert blocks_for(10_000, 0, 304) == 304          # 0: the full grid
    assert blocks_for(10_000, 2048, 304) == 5         # ceil(10000 / 2048)
    assert blocks_for(1, 2048, 304) == 1              # at least one CTA
    assert blocks_for(10 ** 9, 512, 304) == 304       # at most the resident grid
    assert plan([100, 5000], 1000, 8, 4) == [(1, 4), (5, 4)]


def test_choose_keeps_fastest_and_first_of_ties():
    best, table = choose([3, 1, 2], lambda c: {3: 5.0, 1: 2.0, 2: 2.0}[c])
    assert best == 1 and table == {3: 5.0, 1: 2.0, 2: 2.0}
    calls = []

    def noisy(c):
        calls.append(c)
        return 10.0 - len(calls)      # later measurements read faster: min over repeats
    best, table = choose(["a", "b"], noisy, repeats=3)
    assert calls == ["a"] * 3 + ["b"] * 3 and best == "b" and table["a"] == 7.0
    with pytest.raises(ValueError):
        choose([], lambda c: 0.0)


class FakeGraph:
    def __init__(self, n, max_blocks):
        self.n, self.max_blocks = n, max_blocks
        self.blocks, self.chunks = 0, -1

    def set_tuning(self, push_blocks=0, push_direct_chunks=-1):
        self.blocks, self.chunks = push_blocks, push_direct_chunks

    def tuning(self):
        b = self.blocks if 0 < self.blocks < self.max_blocks else self.max_blocks
        return {"push_blocks": b, "push_direct_chunks": 8 if self.chunks < 0 else self.chunks}


def test_tune_grids_finds_the_best_rule_and_leaves_it_set():
    graphs = [FakeGraph(n, 304) for n in (1000, 20_000, 400_000)]

    # a made-up cost: each graph's push wants about n / 4096 CTAs; grids above the SM share
    # cost time, as do fewer CTAs than the work wants; hub threshold 16 is best
    def step_ms():
        ms = 0.0
        for g in graphs:
            want = max(1.0, g.n / 4096)
            b = g.tuning()["push_blocks"]
            ms += abs(math.log(b / want))
        ms += {4: 0.5, 8: 0.3, 16: 0.0}[graphs[0].tuning()["push_direct_chunks"]]
        return ms

    res = tune_grids(graphs, step_ms, rows_per_cta=(0, 32768, 4096, 512), direct_chunks=(-1, 4, 16))
    assert res["rows_per_cta"] == 4096 and res["push_direct_chunks"] == 16 and res["max_blocks"] == 304
    assert [g.blocks for g in graphs] == [1, 5, 98]
    assert all(g.chunks == 16 for g in graphs)
    assert set(res["table_rules"]) == {"0", "32768", "4096", "512"}


def test_fleet_members_follow_the_workload():
    fw = FLEETS["C4"]
    m = fw.members()
    assert len(m) == 256
    n = np.array([x.n for x in m])
    assert n.min() >= fw.n_lo and n.max() <= fw.n_hi
    # log-uniform: the median is near the geometric mean of the ends
    assert abs(math.log(np.median(n)) - 0.5 * (math.log(fw.n_lo) + math.log(fw.n_hi))) < 0.5
    deg = np.array([x.avg_deg for x in m])
    assert deg.min() >= 4.0 and deg.max() <= 32.0
    assert {x.d for x in m} == {32, 64, 128}
    assert len({x.seed for x in m}) == 256
    assert [x.n for x in fw.members()] == list(n)      # seeded
    assert all(x.p_node == 0.0 and x.k_hi == 128 for x in m)


class FakeFleet:
    def __init__(self, graphs, maxb=304):
        self.graphs, self.maxb = graphs, maxb
        self.p = 1.0
        self.snap = None

    def set_shares(self, blocks=None, exponent=1.0):
        self.p = exponent
        self.w = None
        self.snap = [g.chunks for g in self.graphs]     # the fleet snapshots the hub threshold

    def set_weights(self, w):
        self.w = list(w)

    def shares(self):
        w = self.w if self.w is not None else [g.n ** self.p for g in self.graphs]
        return [max(1, int(self.maxb * x / sum(w))) for x in w], 1


def test_tune_shares_picks_exponent_then_hub_threshold():
    graphs = [FakeGraph(n, 304) for n in (1000, 20_000, 400_000)]
    fleet = FakeFleet(graphs)

    def step_ms():   # best at p = 0.75, then chunks 4 (as snapshotted by the fleet)
        return abs(fleet.p - 0.75) * 10 + {-1: 1.0, 4: 0.0, 16: 2.0}[fleet.snap[0]]

    res = tune_shares(fleet, graphs, step_ms)
    assert res["exponent"] == 0.75 and res["push_direct_chunks"] == 4
    assert fleet.p == 0.75 and fleet.snap == [4, 4, 4]
    assert res["ms_per_step"] == 0.0 and res["shares"]["launches"] == 1
    assert set(res["table_exponents"]) == {"0.5", "0.75", "1.0", "1.25"}


def test_measured_weights():
    assert measured_weights([10.0, 4.0, 0.0], [3, 0, 1]) == [30.0, 4.0, 30.0 * 1e-6]


def test_tune_shares_rebalances_on_measured_work():
    # true work per graph is not its size: graph 0 is slow for its size. Time per step is the
    # slowest graph's work / CTAs; measured rebalancing must find shares near the work ratio
    graphs = [FakeGraph(n, 304) for n in (1000, 20_000, 400_000)]
    work = [900.0, 100.0, 3000.0]
    fleet = FakeFleet(graphs)

    def times():
        return [wk / b for wk, b in zip(work, fleet.shares()[0])]

    def step_ms():
        return max(times())

    res = tune_shares(fleet, graphs, step_ms, exponents=(0.5, 1.0), direct_chunks=(-1,), push_times=times,
                      rebalance_rounds=2)
    assert res["chosen"] == "measured"
    b = fleet.shares()[0]
    assert abs(b[0] / b[2] - 900.0 / 3000.0) < 0.05
    assert res["ms_per_step"] < min(res["table_exponents"].values())


def test_tuning_cache_skips_measuring_the_same_fleet(tmp_path):
    graphs = [FakeGraph(n, 304) for n in (1000, 20_000, 400_000)]
    fleet = FakeFleet(graphs)
    calls = []

    def step_ms():
        calls.append(1)
        return abs(fleet.p - 0.75) * 10 + {-1: 1.0, 4: 0.0, 16: 2.0}[fleet.snap[0]]

    cache = str(tmp_path / "tune.json")
    first = tune_shares(fleet, graphs, step_ms, cache=cache)
    assert first["cached"] is False and len(calls) > 0
    n_calls = len(calls)
    fleet2 = FakeFleet([FakeGraph(n, 304) for n in (1000, 20_000, 400_000)])
    again = tune_shares(fleet2, fleet2.graphs, step_ms, cache=cache)
    assert again["cached"] is True and len(calls) == n_calls          # nothing measured
    assert fleet2.p == 0.75 and fleet2.snap == [4, 4, 4]               # the cached shape applied
    other = FakeFleet([FakeGraph(n, 304) for n in (1000, 30_000)])      # another fleet: measured
    third = tune_shares(other, other.graphs, step_ms, cache=cache)
    assert third["cached"] is False and len(calls) > n_calls


def test_a_damaged_tuning_cache_means_tuning_afresh(tmp_path):
    graphs = [FakeGraph(n, 304) for n in (1000, 20_000, 400_000)]
    calls = []

    def step_ms():
        calls.append(1)
        return abs(fleet.p - 0.75) * 10 + {-1: 1.0, 4: 0.0, 16: 2.0}[fleet.snap[0]]

    sig = fleet_signature(graphs)
    for content in ("not json", "[1, 2, 3]", json.dumps({sig: {"exponent": 0.5}}),
                    json.dumps({sig: {"push_direct_chunks": 4, "weights": [1.0, -2.0, 3.0]}}),
                    json.dumps({sig: {"push_direct_chunks": 4, "weights": [1.0, 2.0]}})):
        cache = tmp_path / "tune.json"
        cache.write_text(content)
        fleet = FakeFleet(graphs)
        calls.clear()
        out = tune_shares(fleet, graphs, step_ms, cache=str(cache))
        assert out["cached"] is False and calls, content
        assert fleet.p == 0.75
        # and the file now holds a usable entry for this fleet
        again = tune_shares(FakeFleet(graphs), graphs, step_ms, cache=str(cache))
        assert again["cached"] is True
