"""The seeded input generators against the recipe they state: Chung-Lu weights and graphs
(power law, expected degrees, valid CSR), edge-event streams (batch sizes, event mix, node
arrivals, deletions of existing edges) and the paper's node-arrival protocol."""

import numpy as np
import pytest

from synth import chung_lu_graph, edge_stream, gaussian_test_matrix
from synth.chung_lu import chung_lu_weights, csr_from_edges, node_arrival_stream


def _edges(ip, ix):
    rows = np.repeat(np.arange(len(ip) - 1), np.diff(ip.astype(np.int64)))
    return rows, ix.astype(np.int64)


def test_weights_follow_the_power_law_and_the_cap():
    n, m, gamma = 50_000, 250_000, 2.2
    w = chung_lu_weights(n, m, gamma)
    cap = w.max()
    i = np.arange(n, dtype=np.float64)
    free = w < cap
    # uncapped weights lie on a line of slope -1/(gamma-1) in log-log
    slope = np.polyfit(np.log(i[free] + 1.0), np.log(w[free]), 1)[0]
    assert abs(slope + 1.0 / (gamma - 1.0)) < 1e-9
    # the cap is the square root of the uncapped total 2m, so capping only lowers the sum
    assert w.sum() <= 2 * m + 1e-6 and np.isclose(cap ** 2, 2 * m, rtol=1e-9) and (~free).sum() >= 1
    assert np.all(np.diff(w) <= 0)


@pytest.mark.parametrize("directed", [False, True])
def test_graph_is_a_valid_csr_with_the_requested_shape(directed):
    n, deg, gamma = 20_000, 10.0, 2.2
    ip, ix, w = chung_lu_graph(n, deg, gamma, seed=7, directed=directed)
    ip2, ix2, w2 = chung_lu_graph(n, deg, gamma, seed=7, directed=directed)
    assert np.array_equal(ip, ip2) and np.array_equal(ix, ix2) and np.array_equal(w, w2)   # seeded
    assert ip.dtype == np.int32 and ix.dtype == np.int32 and ip[0] == 0 and ip[-1] == len(ix)
    assert np.all(np.diff(ip) >= 0) and ix.min() >= 0 and ix.max() < n
    rows, cols = _edges(ip, ix)
    assert not np.any(rows == cols)                                   # no self-loops
    for u in range(0, n, 997):                                         # rows sorted, no duplicates
        assert np.all(np.diff(ix[ip[u]:ip[u + 1]]) > 0)
    key = rows * n + cols
    if not directed:                                                  # both directions stored
        assert np.array_equal(np.sort(key), np.sort(cols * n + rows))
    # realised mean degree a little below the target (duplicates and self-loops dropped)
    mean = len(ix) / n
    assert 0.8 * deg <= mean <= deg
    # degrees follow the weights; hubs exist (heavy tail)
    d = np.diff(ip.astype(np.int64)) + (np.bincount(ix, minlength=n) if directed else 0)
    rd = np.argsort(np.argsort(d))
    rw = np.argsort(np.argsort(w))
    assert np.corrcoef(rd, rw)[0, 1] > 0.7                           # rank correlation (Poisson noise at low degree)
    assert d.max() > 20 * d.mean()
    # ids are a random permutation of the weights: the heaviest nodes are not the lowest ids
    top = np.argsort(-w)[:100]
    assert top.mean() > 0.2 * n


def test_csr_from_edges_sorts_rows_by_column():
    ip, ix = csr_from_edges(4, np.array([2, 0, 2, 1, 0]), np.array([1, 3, 0, 2, 1]))
    assert list(ip) == [0, 2, 3, 5, 5] and list(ix) == [1, 3, 2, 0, 1]


def test_edge_stream_follows_its_recipe():
    n = 5000
    ip, ix, w = chung_lu_graph(n, 8.0, 2.2, seed=11)
    st = edge_stream(ip, ix, w, 400, 1, 64, p_node=0.05, p_del=0.10, seed=12)
    st2 = edge_stream(ip, ix, w, 400, 1, 64, p_node=0.05, p_del=0.10, seed=12)
    assert all(np.array_equal(a.src, b.src) and np.array_equal(a.op, b.op) for a, b in zip(st.batches, st2.batches))
    existing = set(zip(*[x.tolist() for x in _edges(ip, ix)]))
    deleted = set()
    n_cur = n
    n_del = n_ins = n_arr = 0
    for b in st.batches:
        assert 1 <= b.k <= 64                                          # k ~ U[1, 64] events per batch
        assert b.src.dtype == np.int32 and b.op.dtype == np.int8 and set(np.unique(b.op)) <= {-1, 1}
        n_after = n_cur + b.new_nodes
        assert b.src.min() >= 0 and b.dst.min() >= 0 and max(b.src.max(), b.dst.max()) < n_after
        assert not np.any(b.src == b.dst)
        new = b.src >= n_cur
        # a node arrival's edges come from the new node to existing nodes, inserted
        assert np.all(b.op[new] == 1) and np.all(b.dst[new] < n_cur)
        assert len(np.unique(b.src[new])) == b.new_nodes
        if b.new_nodes:
            assert set(np.unique(b.src[new]).tolist()) == set(range(n_cur, n_after))
        for s, t, o in zip(b.src[~new], b.dst[~new], b.op[~new]):
            if o == -1:                                                # deletions: initial edges, once each
                assert s < t and (int(s), int(t)) in existing and (s, t) not in deleted
                deleted.add((s, t))
                n_del += 1
            else:
                n_ins += 1
        n_arr += b.new_nodes
        n_cur = n_after
    assert st.n_final == n_cur
    ev = n_del + n_ins + n_arr
    # event mix: about 10% deletions and 5% arrivals among the draws
    assert abs(n_del / ev - 0.10) < 0.02 and abs(n_arr / ev - 0.05) < 0.02


def test_log_sizes_and_forced_arrivals():
    ip, ix, w = chung_lu_graph(3000, 8.0, 2.2, seed=21)
    st = edge_stream(ip, ix, w, 2000, 1, 1024, 0.0, 0.0, seed=22, log_sizes=True)
    ks = np.array([b.k for b in st.batches])
    assert ks.min() >= 1 and ks.max() <= 1024
    # log-uniform: about as many batches in [1, 32) as in [32, 1024]
    assert 0.4 < (ks < 32).mean() < 0.6
    st = edge_stream(ip, ix, w, 50, 5, 5, 0.0, 0.0, seed=23, nodes_per_batch=2, max_new_degree=4)
    n_cur = st.n0
    for b in st.batches:
        assert b.new_nodes == 2
        arr = int((b.src >= n_cur).sum())
        assert 2 <= arr <= 8 and b.k == arr + 5          # the forced arrivals' edges, then k events
        n_cur += b.new_nodes


def test_gaussian_test_matrix():
    a = gaussian_test_matrix(20_000, 32, seed=5)
    assert a.shape == (20_000, 32) and a.dtype == np.float32 and a.flags.c_contiguous
    assert np.array_equal(a, gaussian_test_matrix(20_000, 32, seed=5))
    assert not np.array_equal(a, gaussian_test_matrix(20_000, 32, seed=6))
    assert abs(a.mean()) < 0.01 and abs(a.std() - 1.0) < 0.01


@pytest.mark.parametrize("directed", [False, True])
def test_node_arrivals_rebuild_the_graph(directed):
    n, n0 = 3000, 1000
    ip, ix, _ = chung_lu_graph(n, 8.0, 2.2, seed=31, directed=directed)
    ip0, ix0, st = node_arrival_stream(ip, ix, n0, directed=directed)
    assert len(ip0) == n0 + 1 and len(st.batches) == n - n0 and st.n_final == n
    rows, cols = _edges(ip0, ix0)
    assert rows.max(initial=0) < n0 and cols.max(initial=0) < n0
    got = set(zip(rows.tolist(), cols.tolist()))
    for i, b in enumerate(st.batches):
        v = n0 + i
        assert b.new_nodes == 1 and np.all(b.op == 1)
        # every event touches the arriving node, and only nodes already present besides it
        assert np.all((b.src == v) | (b.dst == v))
        assert np.all(np.maximum(b.src, b.dst) == v)
        for s, t in zip(b.src.tolist(), b.dst.tolist()):
            got.add((s, t))
            if not directed:
                got.add((t, s))
    want = set(zip(*[x.tolist() for x in _edges(ip, ix)]))
    assert got == want


def test_serving_workload_sessions_and_arrivals():
    from synth import SERVING
    sw = SERVING["C5"]
    big = sw.big()
    assert big.directed and big.n == sw.big_n and big.d == 128
    smalls = [sw.small(i) for i in range(400)]
    n = np.array([s.n for s in smalls])
    assert n.min() >= sw.small_lo and n.max() <= sw.small_hi and all(s.directed for s in smalls)
    # log-uniform sizes: the median near the geometric mean of the ends
    assert abs(np.log(np.median(n)) - 0.5 * (np.log(sw.small_lo) + np.log(sw.small_hi))) < 0.15
    assert [sw.small(i).n for i in range(5)] == list(n[:5]) and len({s.seed for s in smalls}) == 400
    # Poisson arrivals: increasing times in [0, T), count and mean gap as the rate says
    rate, T = 200.0, 50.0
    t = sw.arrivals(rate, T, seed=3)
    assert np.all(np.diff(t) > 0) and t.min() >= 0 and t.max() < T
    assert abs(len(t) - rate * T) < 4 * np.sqrt(rate * T)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / rate) < 0.05 / rate and abs(gaps.std() / gaps.mean() - 1.0) < 0.05


def test_fleet_inputs_in_spawned_workers_equal_the_inputs_made_here():
    # the many-graph inputs are generated in spawned processes (safe beside a GPU context);
    # each graph's inputs must not depend on where they were made
    import dataclasses
    from synth import FLEETS
    from synth.configs import fleet_inputs
    members = [dataclasses.replace(m, n=min(m.n, 3000)) for m in FLEETS["C4"].members()[:3]]
    here = fleet_inputs(members, 5, workers=1)
    there = fleet_inputs(members, 5, workers=2)
    for (c1, ip1, ix1, st1), (c2, ip2, ix2, st2) in zip(here, there):
        assert c1 == c2 and np.array_equal(ip1, ip2) and np.array_equal(ix1, ix2)
        assert all(np.array_equal(a.src, b.src) and np.array_equal(a.dst, b.dst) and np.array_equal(a.op, b.op)
                   for a, b in zip(st1.batches, st2.batches))
