"""Serving through the library: sessions admitted by device memory, continuous batching of
their requests into fleet steps, release as sessions close. Each graph's result in the mix
must be its result alone: factors and adjacency bit-identical to the same requests applied
to a twin one by one, and the PPR state within the push bound of the graph it ends with."""

import numpy as np
import pytest
import torch

from oracle.ppr import ppr_matrix_dense
from synth import chung_lu_graph, gaussian_test_matrix
from tests.gpu_util import dense_adj

pytestmark = pytest.mark.gpu

SEED = 0xDA3F0000 + 500
SPECS = [(600, 8.0, 32), (1500, 6.0, 64), (900, 12.0, 128), (2000, 5.0, 32), (700, 9.0, 64)]


def _spec(i, n, deg, d):
    from paper_2306_08967_gb300 import make_config, rsvd_width
    ip, ix, _ = chung_lu_graph(n, deg, 2.4, seed=SEED + 31 * i)
    cfg = make_config(n, d, 0.15, 1e-5, nnz=len(ix))
    return ip, ix, cfg, gaussian_test_matrix(n, rsvd_width(cfg), seed=SEED + 31 * i + 2)


def _events(rng, n, k):
    src, dst, op = [], [], []
    while len(src) < k:
        u, v = rng.integers(0, n, 2)
        if u != v:
            src.append(u), dst.append(v), op.append(-1 if rng.random() < 0.2 else 1)
    return np.array(src, np.int32), np.array(dst, np.int32), np.array(op, np.int8)


def _snapshot(g):
    st = g.state()
    rp, col = g.adjacency()
    rows = [np.sort(col[rp[u]:rp[u + 1]]) for u in range(g.n)]
    return {k: st[k].cpu() for k in ("Ub", "Vb", "PU", "PV", "sigma", "Zb", "r", "s0")}, rp, col, rows


def _bound_ok(snap, alpha=0.15, eps=1e-5):
    st, rp, col, _ = snap
    Xb = (st["Ub"] * st["s0"]).double().numpy()
    exact = ppr_matrix_dense(dense_adj(rp, col, len(rp) - 1), alpha) @ Xb
    return (np.abs(st["r"].double().numpy()).max() <= eps and
            np.abs(st["Zb"].double().numpy() - exact).max() <= eps * (1 + 1e-3) + 2e-6 * np.abs(Xb).max())


def test_each_result_is_the_same_alone_and_in_the_mix():
    from paper_2306_08967_gb300 import DamfGraph, bytes_required
    from paper_2306_08967_gb300.serving import Server
    rng = np.random.default_rng(9)
    specs = [_spec(i, *s) for i, s in enumerate(SPECS)]
    need = [bytes_required(sp[2]) for sp in specs]
    budget = need[0] + need[1] + need[2]            # sessions 3 and 4 wait for memory
    released = {}
    used_max = [0]

    def on_release(sid, g):
        released[sid] = _snapshot(g)

    srv = Server(budget, max_events=256, run_ahead=2, on_release=on_release)
    for i, sp in enumerate(specs):
        srv.open(i, *sp)
    reqs = {i: [_events(rng, SPECS[i][0], int(rng.integers(1, 257))) for _ in range(int(rng.integers(3, 7)))]
            for i in range(len(SPECS))}
    order = [i for i in reqs for _ in reqs[i]]
    rng.shuffle(order)
    nxt = {i: 0 for i in reqs}
    rid = 0
    for i in order:
        srv.submit(rid, i, *reqs[i][nxt[i]])
        rid += 1
        nxt[i] += 1
        if nxt[i] == len(reqs[i]):
            srv.close(i)
        srv.poll()
        used_max[0] = max(used_max[0], srv.sched.used)
        assert srv.sched.used <= budget
    srv.drain()
    srv.shutdown()
    assert sorted(released) == list(range(len(SPECS)))
    # 3 and 4 came in only after memory was freed by closed sessions
    sess = srv.sched.sessions
    assert all(sess[i].state == "freed" for i in sess)
    assert used_max[0] <= budget
    assert len(srv.completed) == rid and all(r.t_done is not None and r.t_done >= r.t_arrive for r in srv.completed)
    for i, sp in enumerate(specs):
        twin = DamfGraph(*sp)
        for ev in reqs[i]:
            twin.apply_edges(*ev)
            twin.ppr_refresh()
        twin.check()
        mine = _snapshot(twin)
        got = released[i]
        for key in ("Ub", "Vb", "PU", "PV", "sigma"):
            assert torch.equal(got[0][key], mine[0][key]), (i, key)
        assert np.array_equal(got[1], mine[1])
        assert all(np.array_equal(a, b) for a, b in zip(got[3], mine[3]))
        assert _bound_ok(got), i
        twin.close()


def _snapshot_any(x):
    # a released graph, or the checkpoint of a graph that closed while evicted
    if isinstance(x, dict):
        rp, col = x["indptr"].astype(np.int64), x["indices"]
        rows = [np.sort(col[rp[u]:rp[u + 1]]) for u in range(len(rp) - 1)]
        return {k: v.cpu() for k, v in x["state"].items()}, rp, col, rows
    return _snapshot(x)


def test_evicted_graphs_come_back_where_they_left_off():
    # a budget for two of four graphs: idle graphs are checkpointed to host memory and freed to
    # admit others, and restored when a request comes for them; every graph still ends exactly
    # where its requests applied alone take it
    from paper_2306_08967_gb300 import DamfGraph, bytes_required
    from paper_2306_08967_gb300.serving import Server
    rng = np.random.default_rng(19)
    specs = [_spec(10 + i, *s) for i, s in enumerate(SPECS[:4])]
    need = sorted(bytes_required(sp[2]) for sp in specs)
    budget = need[-1] + need[-2]
    final = {}
    srv = Server(budget, max_events=128, run_ahead=2, on_release=lambda sid, g: final.update({sid: _snapshot_any(g)}))
    for i, sp in enumerate(specs):
        srv.open(i, *sp)
    reqs = {i: [] for i in range(4)}
    rid = 0
    for rnd in range(5):                      # round robin: every graph is asked again and again
        for i in range(4):
            ev = _events(rng, SPECS[i][0], int(rng.integers(1, 129)))
            reqs[i].append(ev)
            srv.submit(rid, i, *ev)
            rid += 1
            srv.drain()                       # serve it before the next graph's request
            assert srv.sched.used <= budget
    for i in range(4):
        srv.close(i)
    srv.drain()
    srv.shutdown()
    evictions = sum(s.evictions for s in srv.sched.sessions.values())
    assert evictions >= 4                     # graphs really left and came back
    assert sorted(final) == [0, 1, 2, 3]
    for i, sp in enumerate(specs):
        twin = DamfGraph(*sp)
        for ev in reqs[i]:
            twin.apply_edges(*ev)
            twin.ppr_refresh()
        twin.check()
        mine = _snapshot(twin)
        got = final[i]
        for key in ("Ub", "Vb", "PU", "PV", "sigma"):
            assert torch.equal(got[0][key], mine[0][key]), (i, key)
        assert np.array_equal(got[1], mine[1])
        assert all(np.array_equal(a, b) for a, b in zip(got[3], mine[3]))
        assert _bound_ok(got), i
        twin.close()
