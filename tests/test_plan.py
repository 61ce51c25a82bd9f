"""The grouped push's CTA plan (damf_plan_slots), on the host: every graph in exactly one slot,
the CTAs within the resident budget, owners at least their floor share, small graphs packed
onto one-CTA slots of total share <= 1, and the result deterministic."""

import numpy as np
import pytest

from paper_2306_08967_gb300.api import DamfError, plan_slots


def _check(w, maxb):
    w = np.asarray(w, np.float64)
    slot_of, ctas = plan_slots(w, maxb)
    S = len(ctas)
    assert S >= 1 and (ctas >= 1).all() and ctas.sum() <= maxb
    assert slot_of.min() >= 0 and slot_of.max() < S
    members = [np.flatnonzero(slot_of == s) for s in range(S)]
    assert all(len(m) >= 1 for m in members)            # no empty slot
    x = maxb * w / w.sum()                                # fair shares
    cap = max(1.0, max(x[m].sum() for m in members if len(m) > 1) if any(len(m) > 1 for m in members) else 1.0)
    for s, m in enumerate(members):
        if len(m) > 1:
            assert ctas[s] == 1                           # a shared slot has one CTA
            assert x[m].sum() <= cap + 1e-9
        else:
            g = m[0]
            if x[g] >= cap:                               # an owner: at least its floor share
                assert ctas[s] >= np.floor(x[g])
    return slot_of, ctas, x


def test_equal_weights_split_evenly():
    slot_of, ctas, _ = _check([1.0] * 4, 10)
    assert list(slot_of) == [0, 1, 2, 3] and sorted(ctas) == [2, 2, 3, 3]
    slot_of, ctas, _ = _check([1.0] * 304, 304)
    assert (ctas == 1).all() and len(ctas) == 304


def test_owners_take_all_ctas_and_small_graphs_share():
    w = [1000.0, 300.0, 1.0, 0.7, 0.5, 0.2]
    slot_of, ctas, x = _check(w, 64)
    assert ctas.sum() == 64                               # owners absorb the leftover CTAs
    assert slot_of[2] == slot_of[3] or slot_of[3] == slot_of[4]   # the small ones share
    assert ctas[slot_of[0]] > ctas[slot_of[1]] > 1


def test_more_graphs_than_ctas_still_fit():
    rng = np.random.default_rng(3)
    w = np.exp(rng.uniform(np.log(1e3), np.log(5e5), size=1000))   # log-uniform sizes
    slot_of, ctas, _ = _check(w, 304)
    assert len(ctas) <= 304 and ctas.sum() <= 304
    # the largest graph owns the most CTAs
    assert ctas[slot_of[int(np.argmax(w))]] == ctas.max()


def test_deterministic_and_validated():
    w = [5.0, 3.0, 0.1, 0.1, 0.1]
    a = plan_slots(w, 16)
    b = plan_slots(w, 16)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for bad in ([1.0, 0.0], [1.0, -2.0], [float("nan")]):
        with pytest.raises(DamfError):
            plan_slots(bad, 16)
    with pytest.raises(DamfError):
        plan_slots([1.0], 0)


def test_one_graph_gets_everything():
    slot_of, ctas, _ = _check([7.0], 608)
    assert list(ctas) == [608]


@pytest.mark.parametrize("seed", range(20))
def test_random_fleets_keep_the_plan_invariants(seed):
    rng = np.random.default_rng(seed)
    g = int(rng.integers(1, 700))
    maxb = int(rng.choice([1, 2, 7, 152, 304, 608]))
    w = np.exp(rng.uniform(0.0, float(rng.choice([0.1, 3.0, 12.0])), size=g))
    slot_of, ctas, x = _check(w, maxb)
    # every CTA of the budget goes to some slot unless there are fewer graphs than CTAs to give
    assert ctas.sum() == maxb or len(ctas) == g
    assert len(ctas) <= maxb


def test_a_large_fleet_plans_quickly():
    import time
    rng = np.random.default_rng(9)
    w = np.exp(rng.uniform(0.0, 6.0, size=5000))
    t = time.perf_counter()
    slot_of, ctas, _ = _check(w, 608)
    assert time.perf_counter() - t < 5.0
    assert ctas.sum() == 608 and len(ctas) <= 608
