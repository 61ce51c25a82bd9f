"""Many graphs through the C ABI: device-counted batches, damf_step_multi, captured fleet
steps and the push launch shape (damf_set_tuning).

Each graph's result must not depend on the company it keeps: its factors (Ub, Vb, PU, PV,
sigma) and adjacency are bit-identical to the same batches applied to it alone (every
factor kernel is deterministic), and its PPR state keeps the push bound
|Zb - Pi Xb| <= eps against the exact Pi of the graph it ends with (the push's order of
floating-point adds depends on timing, so Zb itself is compared through the bound).
"""

import numpy as np
import pytest
import torch

from oracle.ppr import ppr_matrix_dense
from tests.gpu_util import dense_adj, make_pair

pytestmark = pytest.mark.gpu

SEED = 0xDA3F0000 + 400
FACTORS = ("Ub", "Vb", "PU", "PV", "sigma")


def _events(rng, n, k, p_del=0.2):
    src, dst, op = [], [], []
    while len(src) < k:
        u, v = rng.integers(0, n, 2)
        if u != v:
            src.append(u), dst.append(v), op.append(-1 if rng.random() < p_del else 1)
    return np.array(src, np.int32), np.array(dst, np.int32), np.array(op, np.int8)


def _padded(ev, kmax):
    # events in buffers of kmax entries; the tail holds junk a counted call must ignore
    # (ids that would fail validation if they were read as events)
    src = np.full(kmax, -7, np.int32)
    dst = np.full(kmax, -7, np.int32)
    op = np.full(kmax, 3, np.int8)
    k = ev[0].shape[0]
    src[:k], dst[:k], op[:k] = ev
    return torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), torch.from_numpy(op).cuda()


def _same_factors(a, b):
    sa, sb = a.state(), b.state()
    for key in FACTORS:
        assert torch.equal(sa[key], sb[key]), key
    ra, ca = a.adjacency()
    rb, cb = b.adjacency()
    assert np.array_equal(ra, rb)
    for u in range(a.n):   # rows hold the same set (the order within a row is the edit order)
        assert np.array_equal(np.sort(ca[ra[u]:ra[u + 1]]), np.sort(cb[rb[u]:rb[u + 1]]))


def _push_bound(g, alpha, eps):
    st = g.state()
    Xb = (st["Ub"] * st["s0"]).double().cpu().numpy()
    Zb = st["Zb"].double().cpu().numpy()
    r = st["r"].double().cpu().numpy()
    rp, col = g.adjacency()
    exact = ppr_matrix_dense(dense_adj(rp, col, g.n), alpha) @ Xb
    assert np.abs(r).max() <= eps
    assert np.abs(Zb - exact).max() <= eps * (1 + 1e-3) + 2e-6 * np.abs(Xb).max()


@pytest.mark.parametrize("k,k_live", [(128, 0), (128, 1), (128, 64), (128, 65), (128, 100), (128, 128),
                                      (100, 250), (64, -5)])
def test_counted_apply_equals_plain_apply(k, k_live):
    # the live count (clamped to [0, k_max]) decides which events apply, across update
    # boundaries (64 events per update); the junk beyond it is never read
    rng = np.random.default_rng(7 + k_live % 97)
    n, d = 700, 32
    a, _, _ = make_pair(n, 8.0, 2.5, d, 0.15, 1e-5, SEED + 1, oracle=False)
    b, _, _ = make_pair(n, 8.0, 2.5, d, 0.15, 1e-5, SEED + 1, oracle=False)
    live = min(max(k_live, 0), k)
    ev = _events(rng, n, k)
    a.apply_edges(ev[0][:live], ev[1][:live], ev[2][:live])
    a.ppr_refresh()
    s, t, o = _padded(tuple(x[:live] for x in ev), k) if live < k else _padded(ev, k)
    kd = torch.tensor([k_live], dtype=torch.int32, device="cuda")
    b.apply_edges_counted(s, t, o, kd)
    b.ppr_refresh()
    a.check()
    b.check()
    _same_factors(a, b)
    assert a.stats()["edges_applied"] == b.stats()["edges_applied"]
    a.close()
    b.close()


def _fleet(specs, seed):
    gs, twins = [], []
    for i, (n, deg, d) in enumerate(specs):
        g, _, _ = make_pair(n, deg, 2.4, d, 0.15, 1e-5, seed + 17 * i, oracle=False)
        t, _, _ = make_pair(n, deg, 2.4, d, 0.15, 1e-5, seed + 17 * i, oracle=False)
        gs.append(g)
        twins.append(t)
    return gs, twins


SPECS = [(400, 6.0, 32), (1200, 10.0, 64), (2500, 8.0, 128), (900, 20.0, 32), (1800, 5.0, 128)]


def test_step_multi_equals_each_graph_alone():
    from paper_2306_08967_gb300 import step_multi
    rng = np.random.default_rng(21)
    gs, twins = _fleet(SPECS, SEED + 50)
    # uneven push grids: the graphs' pushes then share the SMs
    for g, blocks in zip(gs, [4, 16, 64, 8, 0]):
        g.set_tuning(blocks)
    for step in range(4):
        evs = [_events(rng, g.n, int(rng.integers(1, 129))) for g in gs]
        step_multi([(g, *ev) for g, ev in zip(gs, evs)])
        for t, ev in zip(twins, evs):
            t.apply_edges(*ev)
            t.ppr_refresh()
    torch.cuda.synchronize()
    for g, t in zip(gs, twins):
        g.check()
        t.check()
        _same_factors(g, t)
        _push_bound(g, 0.15, 1e-5)
        g.close()
        t.close()


def test_step_multi_rejects_a_repeated_graph():
    from paper_2306_08967_gb300 import DamfError, step_multi
    gs, twins = _fleet(SPECS[:2], SEED + 60)
    ev = _events(np.random.default_rng(3), 400, 10)
    with pytest.raises(DamfError):
        step_multi([(gs[0], *ev), (gs[0], *ev)])
    # nothing was enqueued and the context stays usable
    step_multi([(gs[0], *ev)])
    twins[0].apply_edges(*ev)
    twins[0].ppr_refresh()
    _same_factors(gs[0], twins[0])
    for g in gs + twins:
        g.close()


def test_captured_step_multi_replays_like_direct_calls():
    # one CUDA graph holds the whole damf_step_multi step (every graph's update and push);
    # replays with new events and new counts written into fixed buffers equal direct calls
    from paper_2306_08967_gb300 import _lib
    from paper_2306_08967_gb300.api import batch_array
    rng = np.random.default_rng(33)
    gs, twins = _fleet(SPECS, SEED + 70)
    for g, blocks in zip(gs, [8, 8, 32, 8, 16]):
        g.set_tuning(blocks)
    kmax = 128
    bufs = [(torch.zeros(kmax, dtype=torch.int32, device="cuda"), torch.zeros(kmax, dtype=torch.int32, device="cuda"),
             torch.zeros(kmax, dtype=torch.int8, device="cuda"), torch.zeros(1, dtype=torch.int32, device="cuda"))
            for _ in gs]
    stream = torch.cuda.Stream()
    lib = _lib.load()
    arr = batch_array([(g, b[0], b[1], b[2], 0, b[3]) for g, b in zip(gs, bufs)])
    import ctypes
    sptr = ctypes.c_void_p(stream.cuda_stream)
    with torch.cuda.stream(stream):
        for g in gs:
            g.join(stream)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
        assert lib.damf_step_multi(arr, len(gs), sptr) == 0
    # the capture ran nothing: the twins stay at the initial state too
    for step in range(5):
        evs = []
        for g, (s, t, o, kd) in zip(gs, bufs):
            k = int(rng.integers(0, kmax + 1)) if step else kmax
            ev = _events(rng, g.n, k) if k else (np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int8))
            ps, pt, po = _padded(ev, kmax)
            s.copy_(ps), t.copy_(pt), o.copy_(po)
            kd.fill_(k)
            evs.append(ev)
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        for tw, ev in zip(twins, evs):
            tw.apply_edges(*ev)
            tw.ppr_refresh()
    for g, t in zip(gs, twins):
        g.check()
        t.check()
        _same_factors(g, t)
        _push_bound(g, 0.15, 1e-5)
    del graph
    for g in gs + twins:
        g.close()


def test_tuning_round_trip_and_bounds():
    g, _, _ = make_pair(1500, 10.0, 2.4, 64, 0.15, 1e-5, SEED + 90, oracle=False)
    full = g.tuning()
    assert full["push_blocks"] >= 1 and full["push_direct_chunks"] == 8
    g.set_tuning(5, 3)
    assert g.tuning() == {"push_blocks": 5, "push_direct_chunks": 3}
    g.set_tuning(10 ** 6, -1)                   # clamped to the push's own occupancy (4 per SM)
    big = g.tuning()["push_blocks"]
    assert full["push_blocks"] <= big <= 2 * full["push_blocks"]
    from paper_2306_08967_gb300 import DamfError
    with pytest.raises(DamfError):
        g.set_tuning(-1, -1)
    with pytest.raises(DamfError):
        g.set_tuning(1, 5000)
    assert g.tuning()["push_blocks"] == big     # a rejected call changes nothing
    rng = np.random.default_rng(5)
    # the whole occupancy, then one CTA with a low hub threshold: both reach the bound
    for blocks, chunks in ((big, -1), (1, 1)):
        g.set_tuning(blocks, chunks)
        for _ in range(3):
            g.apply_edges(*_events(rng, g.n, 90))
            g.ppr_refresh()
        g.check()
        _push_bound(g, 0.15, 1e-5)
    g.close()


def _degree_bound(g, eps):
    st = g.state()
    r = st["r"].double().cpu().numpy()
    rp, _ = g.adjacency()
    deg = np.maximum(np.diff(rp), 1)
    assert (np.abs(r).max(axis=1) <= eps * deg * (1 + 1e-6)).all()


def test_fleet_step_equals_each_graph_alone():
    # the grouped push (one launch, each graph on its share of CTAs) leaves every graph as its
    # own update and push would; one graph with the degree-scaled threshold makes a second launch
    from paper_2306_08967_gb300 import DamfFleet
    rng = np.random.default_rng(41)
    specs = SPECS + [(120, 5.0, 32), (150, 4.0, 32), (200, 5.0, 64)]
    gs, twins = _fleet(specs, SEED + 110)
    g6, _, _ = make_pair(1500, 9.0, 2.4, 64, 0.15, 1e-5, SEED + 119, oracle=False, threshold="degree")
    t6, _, _ = make_pair(1500, 9.0, 2.4, 64, 0.15, 1e-5, SEED + 119, oracle=False, threshold="degree")
    gs.append(g6)
    twins.append(t6)
    nabs = len(specs)
    fleet = DamfFleet(gs)
    blocks, nl = fleet.shares()
    assert nl == 2 and min(blocks) >= 1
    # larger graphs get at least as many CTAs as smaller ones of the same rank
    assert blocks[2] >= blocks[1] >= blocks[0]
    fleet.set_timing(True)
    for step in range(7):
        evs = [_events(rng, g.n, int(rng.integers(0, 129))) for g in gs]
        fleet.step(evs)
        for t, ev in zip(twins, evs):
            t.apply_edges(*ev)
            t.ppr_refresh()
        if step == 2:
            fleet.set_shares(exponent=0.0)            # equal shares
            sh = fleet.shares()[0][:nabs]
            assert max(sh) - min(sh) <= 1
        if step == 4:
            # shares by the square of the size: the small graphs share CTAs, pushed in turn
            fleet.set_shares(exponent=2.0)
            sh = fleet.shares()[0][:nabs]
            assert sh[5] == sh[6] == sh[7] == 0 and sh[2] > 1
    torch.cuda.synchronize()
    assert fleet.launches == 2 * 2 * 7
    tm = fleet.timing()
    assert tm["steps"] == 7 and tm["update_ms"] > 0 and tm["push_ms"] > 0
    for i, (g, t) in enumerate(zip(gs, twins)):
        g.check()
        t.check()
        _same_factors(g, t)
        if i < nabs:
            _push_bound(g, 0.15, 1e-5)
        else:
            _degree_bound(g, 1e-5)
    fleet.close()
    for g in gs + twins:
        g.close()


def test_fleet_shares_are_validated():
    from paper_2306_08967_gb300 import DamfError, DamfFleet
    gs, twins = _fleet(SPECS[:3], SEED + 130)
    fleet = DamfFleet(gs)
    before = fleet.shares()
    with pytest.raises(DamfError):
        fleet.set_shares([1, 0, 1])                   # a graph without a CTA
    with pytest.raises(DamfError):
        fleet.set_shares([10 ** 6, 1, 1])             # more than stay resident
    with pytest.raises(DamfError):
        fleet.set_shares(exponent=-1.0)
    assert fleet.shares() == before                   # rejected calls change nothing
    fleet.set_shares([1, 2, 3])
    assert fleet.shares() == ([1, 2, 3], 1)
    # a context appears once per fleet
    with pytest.raises(DamfError):
        DamfFleet([gs[0], gs[0]])
    # one CTA per graph still reaches the bound
    rng = np.random.default_rng(2)
    for _ in range(3):
        evs = [_events(rng, g.n, 60) for g in gs]
        fleet.step(evs)
        for t, ev in zip(twins, evs):
            t.apply_edges(*ev)
            t.ppr_refresh()
    torch.cuda.synchronize()
    for g, t in zip(gs, twins):
        _same_factors(g, t)
        _push_bound(g, 0.15, 1e-5)
    # a step whose second batch the host checks reject (node capacity) enqueues nothing for
    # any graph: the others stay where their twins are and go on alone; the second is poisoned
    evs = [_events(rng, g.n, 40) for g in gs]
    evs[1] = evs[1] + (10 ** 6,)
    with pytest.raises(DamfError):
        fleet.step(evs)
    torch.cuda.synchronize()
    for i in (0, 2):
        _same_factors(gs[i], twins[i])
        gs[i].apply_edges(*evs[i])
        gs[i].ppr_refresh()
        twins[i].apply_edges(*evs[i])
        twins[i].ppr_refresh()
        gs[i].check()
        _same_factors(gs[i], twins[i])
        _push_bound(gs[i], 0.15, 1e-5)
    with pytest.raises(DamfError):
        gs[1].check()
    fleet.close()
    for g in gs + twins:
        g.close()


def test_captured_fleet_step_replays_like_direct_calls():
    # the whole fleet step (updates and the grouped push) as one CUDA graph; each replay reads
    # new events and counts from fixed buffers
    from paper_2306_08967_gb300 import DamfFleet
    from paper_2306_08967_gb300.api import batch_array
    rng = np.random.default_rng(43)
    gs, twins = _fleet(SPECS, SEED + 150)
    fleet = DamfFleet(gs)
    kmax = 128
    bufs = [(torch.zeros(kmax, dtype=torch.int32, device="cuda"), torch.zeros(kmax, dtype=torch.int32, device="cuda"),
             torch.zeros(kmax, dtype=torch.int8, device="cuda"), torch.zeros(1, dtype=torch.int32, device="cuda"))
            for _ in gs]
    arr = batch_array([(g, b[0], b[1], b[2], 0, b[3]) for g, b in zip(gs, bufs)])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for g in gs:
            g.join(stream)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
        fleet.step_array(arr, stream)
    for step in range(6):
        evs = []
        for g, (s, t, o, kd) in zip(gs, bufs):
            k = int(rng.integers(0, kmax + 1))
            ev = _events(rng, g.n, k) if k else (np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int8))
            ps, pt, po = _padded(ev, kmax)
            s.copy_(ps), t.copy_(pt), o.copy_(po)
            kd.fill_(k)
            evs.append(ev)
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        for tw, ev in zip(twins, evs):
            tw.apply_edges(*ev)
            tw.ppr_refresh()
    for g, t in zip(gs, twins):
        g.check()
        t.check()
        _same_factors(g, t)
        _push_bound(g, 0.15, 1e-5)
    del graph
    fleet.close()
    for g in gs + twins:
        g.close()


def test_captured_step_after_new_shares_reports_instead_of_running():
    # a captured grouped push carries its plan; after the shares change it must not run on the
    # new tables: every CTA returns at once and the contexts report DAMF_ERR_INVALID
    from paper_2306_08967_gb300 import DamfFleet
    from paper_2306_08967_gb300.api import batch_array
    gs, twins = _fleet(SPECS[:3], SEED + 170)
    fleet = DamfFleet(gs)
    kmax = 64
    bufs = [(torch.zeros(kmax, dtype=torch.int32, device="cuda"), torch.zeros(kmax, dtype=torch.int32, device="cuda"),
             torch.zeros(kmax, dtype=torch.int8, device="cuda"), torch.zeros(1, dtype=torch.int32, device="cuda"))
            for _ in gs]
    arr = batch_array([(g, b[0], b[1], b[2], 0, b[3]) for g, b in zip(gs, bufs)])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for g in gs:
            g.join(stream)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
        fleet.step_array(arr, stream)
    graph.replay()                          # the plan it was captured with: fine
    torch.cuda.synchronize()
    assert all(g.sync_status() == 0 for g in gs)
    fleet.set_shares(exponent=0.0)          # a new plan
    graph.replay()
    torch.cuda.synchronize()
    assert all(g.sync_status() == 1 for g in gs)   # DAMF_ERR_INVALID
    del graph
    fleet.close()
    for g in gs + twins:
        g.close()
