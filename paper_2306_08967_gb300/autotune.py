"""Autotuner of the PPR push launch shape for many graphs that share one GPU.

A fleet (damf_fleet_*) pushes all its graphs in one grouped cooperative launch in which each
graph owns a share of the resident CTAs. How the CTAs are best split depends on the graphs
(rows, adjacency size, rank) and on the mix, so it is measured rather than guessed:

* a share rule gives graph i CTAs in proportion to (d_i (n_i + m_i))^p, at least one each;
  the tuner times whole fleet steps (the caller's `measure` callback runs real steps and
  returns milliseconds per step) for each exponent p and keeps the fastest;
* under that rule it then tries the hub threshold (push_direct_chunks: how many in-edge
  chunks a row task scatters itself before its row is split into items);
* then it measures each graph's push time in the grouped launch and re-plans the shares in
  proportion to the measured work (time x CTAs), for a few rounds, keeping the fastest;
* the result can be kept in a JSON cache file keyed by the fleet's graphs, so that the same
  fleet is not measured again.

For graphs pushed one launch each (damf_step_multi), tune_grids picks the push grid per graph
by a rows-per-CTA rule instead. Tuning changes only launch shapes: every result stays within
the push bound.
"""

from __future__ import annotations

import hashlib
import json
import math
import os
from typing import Callable, Dict, Iterable, List, Sequence, Tuple

DEFAULT_ROWS_PER_CTA = (0, 32768, 8192, 2048, 512)
DEFAULT_EXPONENTS = (0.5, 0.75, 1.0, 1.25)
DEFAULT_DIRECT_CHUNKS = (-1, 4, 16)


def blocks_for(n: int, rows_per_cta: int, max_blocks: int) -> int:
    """Push CTAs for a graph of n rows under a rule (0: the full grid, max_blocks)."""
    if rows_per_cta <= 0:
        return int(max_blocks)
    return int(max(1, min(max_blocks, math.ceil(n / rows_per_cta))))


def plan(sizes: Sequence[int], rows_per_cta: int, max_blocks: int, direct_chunks: int = -1) -> List[Tuple[int, int]]:
    """(push_blocks, push_direct_chunks) for each graph of the given row counts."""
    return [(blocks_for(n, rows_per_cta, max_blocks), int(direct_chunks)) for n in sizes]


def choose(candidates: Iterable, measure: Callable[[object], float], repeats: int = 1) -> Tuple[object, Dict]:
    """The candidate with the least measured time (min over `repeats` measurements each);
    ties keep the earlier candidate. Returns (best, {candidate: ms})."""
    table = {}
    best, best_ms = None, math.inf
    for cand in candidates:
        ms = min(float(measure(cand)) for _ in range(max(1, repeats)))
        table[cand] = ms
        if ms < best_ms:
            best, best_ms = cand, ms
    if best is None:
        raise ValueError("no candidates")
    return best, table


def tune_grids(graphs, measure_step_ms: Callable[[], float], rows_per_cta: Sequence[int] = DEFAULT_ROWS_PER_CTA,
               direct_chunks: Sequence[int] = DEFAULT_DIRECT_CHUNKS, repeats: int = 1) -> Dict:
    """Tunes the push shape of every graph of a fleet by timing fleet steps.

    graphs: objects with .n (rows), .set_tuning(push_blocks, push_direct_chunks) and .tuning()
    (DamfGraph). measure_step_ms(): runs a few real fleet steps under the tunings set and
    returns ms per step (it must rebuild any captured launch first). Leaves the best tuning
    set on every graph and returns {"rows_per_cta", "push_direct_chunks", "table_rules",
    "table_chunks", "ms_per_step"}."""
    graphs = list(graphs)
    if not graphs:
        raise ValueError("no graphs")
    for g in graphs:
        g.set_tuning(0, -1)
    max_blocks = max(int(g.tuning()["push_blocks"]) for g in graphs)
    sizes = [int(g.n) for g in graphs]

    def apply(rule, chunks):
        for g, (b, c) in zip(graphs, plan(sizes, rule, max_blocks, chunks)):
            g.set_tuning(b, c)

    def by_rule(rule):
        apply(rule, -1)
        return measure_step_ms()

    rule, t_rules = choose(rows_per_cta, by_rule, repeats)

    def by_chunks(chunks):
        apply(rule, chunks)
        return measure_step_ms()

    chunks, t_chunks = choose(direct_chunks, by_chunks, repeats)
    apply(rule, chunks)
    return {"rows_per_cta": rule, "push_direct_chunks": chunks, "max_blocks": max_blocks,
            "table_rules": {str(k): v for k, v in t_rules.items()},
            "table_chunks": {str(k): v for k, v in t_chunks.items()},
            "ms_per_step": t_chunks[chunks]}


def measured_weights(push_ns: Sequence[float], blocks: Sequence[int]) -> List[float]:
    """Work of each graph's push from one grouped launch: its push time times the CTAs it ran
    on (one for a graph sharing a CTA); a floor keeps every weight positive."""
    w = [float(t) * max(int(b), 1) for t, b in zip(push_ns, blocks)]
    floor = max(max(w) * 1e-6, 1e-9) if w else 1.0
    return [max(x, floor) for x in w]


def fleet_signature(graphs) -> str:
    """Key of a fleet in a tuning cache: its graphs' rows and ranks in fleet order."""
    desc = [[int(g.n), int(getattr(g, "d", 0))] for g in graphs]
    return hashlib.sha1(json.dumps(desc).encode()).hexdigest()


def _load_cache(path: str) -> Dict:
    """The cache file's entries; an absent, unreadable or malformed file counts as empty."""
    try:
        with open(path) as f:
            data = json.load(f)
    except (OSError, ValueError):
        return {}
    return data if isinstance(data, dict) else {}


def _usable(entry, ngraphs: int) -> bool:
    """A cache entry that _apply can set on a fleet of ngraphs graphs."""
    if not isinstance(entry, dict) or not isinstance(entry.get("push_direct_chunks"), int):
        return False
    w = entry.get("weights")
    if w:
        return isinstance(w, list) and len(w) == ngraphs and all(isinstance(x, (int, float)) and x > 0 for x in w)
    return isinstance(entry.get("exponent"), (int, float))


def _apply(fleet, graphs, entry: Dict):
    for g in graphs:
        g.set_tuning(0, int(entry["push_direct_chunks"]))
    if entry.get("weights"):
        fleet.set_weights(entry["weights"])
    else:
        fleet.set_shares(exponent=float(entry["exponent"]))


def tune_shares(fleet, graphs, measure_step_ms: Callable[[], float],
                exponents: Sequence[float] = DEFAULT_EXPONENTS,
                direct_chunks: Sequence[int] = DEFAULT_DIRECT_CHUNKS, repeats: int = 1,
                push_times: Callable[[], Sequence[float]] = None, rebalance_rounds: int = 3,
                cache: str = None) -> Dict:
    """Tunes a fleet's grouped push by timing fleet steps.

    fleet: .set_shares(blocks=None, exponent=p), .set_weights(w) and .shares() (DamfFleet).
    graphs: the fleet's graphs with .set_tuning(push_blocks, push_direct_chunks) (DamfGraph).
    measure_step_ms(): runs a few real fleet steps under the current shape and returns ms per
    step (it must rebuild any captured launch first). push_times(): each graph's push time
    per step (any unit) over the steps since its previous call; with it, after the exponent
    and hub-threshold searches, `rebalance_rounds` rounds set the shares from the measured
    work (push time x CTAs) of the previous round. Leaves the fastest shape seen set and
    returns {"exponent", "push_direct_chunks", "table_exponents", "table_chunks",
    "rebalance_ms", "chosen", "ms_per_step", "shares"}. With `cache` (a JSON file), a fleet of
    the same signature (fleet_signature) tuned before gets that shape without measuring
    ("cached": True); a new result is added to the file."""
    graphs = list(graphs)
    sig = fleet_signature(graphs)
    if cache:
        entry = _load_cache(cache).get(sig)
        if _usable(entry, len(graphs)):   # otherwise (damaged or foreign) the fleet is tuned afresh
            _apply(fleet, graphs, entry)
            blocks, launches = fleet.shares()
            return dict(entry, cached=True, shares={"min": min(blocks), "max": max(blocks), "launches": launches})
    for g in graphs:
        g.set_tuning(0, -1)

    def by_exponent(p):
        fleet.set_shares(exponent=p)
        return measure_step_ms()

    p, t_exp = choose(exponents, by_exponent, repeats)

    def by_chunks(c):
        for g in graphs:
            g.set_tuning(0, c)
        fleet.set_shares(exponent=p)     # the fleet takes the graphs' hub threshold here
        return measure_step_ms()

    c, t_chunks = choose(direct_chunks, by_chunks, repeats)
    for g in graphs:
        g.set_tuning(0, c)
    fleet.set_shares(exponent=p)
    best_ms, best_w, chosen = t_chunks[c], None, "exponent"
    reb = []
    if push_times is not None and rebalance_rounds > 0:
        push_times()                                   # start counting under the exponent rule
        ms = measure_step_ms()
        for _ in range(rebalance_rounds):
            w = measured_weights(push_times(), fleet.shares()[0])
            fleet.set_weights(w)
            ms = min(measure_step_ms() for _ in range(max(1, repeats)))
            reb.append(ms)
            if ms < best_ms:
                best_ms, best_w, chosen = ms, w, "measured"
        if best_w is None:
            fleet.set_shares(exponent=p)
        else:
            fleet.set_weights(best_w)
    blocks, launches = fleet.shares()
    out = {"exponent": p, "push_direct_chunks": c, "table_exponents": {str(k): v for k, v in t_exp.items()},
           "table_chunks": {str(k): v for k, v in t_chunks.items()}, "rebalance_ms": reb, "chosen": chosen,
           "ms_per_step": best_ms, "cached": False,
           "shares": {"min": min(blocks), "max": max(blocks), "launches": launches}}
    if cache:
        entries = _load_cache(cache)
        entries[sig] = {"exponent": p, "push_direct_chunks": c, "weights": list(best_w) if best_w else None,
                        "chosen": chosen, "ms_per_step": best_ms}
        tmp = cache + ".tmp%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(entries, f)
        os.replace(tmp, cache)
    return out
