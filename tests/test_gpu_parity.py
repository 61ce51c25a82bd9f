"""CUDA path (through the C ABI) against the FP64 oracle and the paper's definitions.

Tolerances (from the FP32 device arithmetic: unit roundoff 6e-8 grown over the d-term sums and sweeps):
  * integer work (adjacency, touched sets S/T): bit-exact
  * one update vs the brute-force t-SVD of (previous product + dA) (Theorem 2):
    sigma rel 2e-4, X Y^T rel Frobenius 2e-4
  * PPR: |Zb - Pi Xb|_max <= eps (1 + 1e-3) + 2e-6 |Xb|_max  (push bound plus FP32 rounding)
  * whole-stream runs vs the FP64 oracle: sigma rel 1e-4, X Y^T rel Frobenius 1e-4 (the FP32
    tolerance after 1,000 updates; these streams are shorter; 1e-3 for the node-arrival stream
    on a few hundred nodes, whose small gap at the cut amplifies rounding); Z Y^T rel Frobenius 1e-3, since
    Z is PPR(X) only within the push's eps and two push orders land at different points of it
"""

import numpy as np
import pytest
import torch

from oracle.ppr import ppr_matrix_dense
from oracle.tsvd import brute_force_update
from synth import CONFIGS, chung_lu_graph, edge_stream
from tests.gpu_util import dense_adj, gpu_xy, make_pair, rel_fro

pytestmark = pytest.mark.gpu

SEED = 0xDA3F0000 + 200
STREAM_TOL = 1e-4


def _stream_close(tag, sg, Xg, Yg, orc, xy_tol=STREAM_TOL):
    es = float(np.max(np.abs(sg - orc.sigma) / orc.sigma))
    ex = rel_fro(Xg @ Yg.T, orc.X() @ orc.Y().T)
    print("%s: sigma rel %.2e, X Y^T rel %.2e" % (tag, es, ex))
    assert es <= STREAM_TOL, (tag, es)
    assert ex <= xy_tol, (tag, ex)


def _events(rng, n, k, p_del=0.25):
    src, dst, op = [], [], []
    while len(src) < k:
        u, v = rng.integers(0, n, 2)
        if u != v:
            src.append(u), dst.append(v), op.append(-1 if rng.random() < p_del else 1)
    return np.array(src, np.int32), np.array(dst, np.int32), np.array(op, np.int8)


@pytest.mark.parametrize("d,n", [(16, 1500), (64, 3000)])
def test_init_matches_oracle(d, n):
    g, orc, _ = make_pair(n, 10.0, 2.5, d, 0.15, 1e-4, SEED + d, propagate=False)
    X, Y, s = gpu_xy(g)
    np.testing.assert_allclose(s, orc.sigma, rtol=1e-3)
    assert rel_fro(X @ Y.T, orc.X() @ orc.Y().T) < 1e-3
    U = X / np.sqrt(s)
    assert np.abs(U.T @ U - np.eye(d)).max() < 1e-4
    g.close()


@pytest.mark.parametrize("directed", [False, True])
def test_init_with_rows_longer_than_a_chunk_matches_oracle(directed):
    # hub rows of 2,500, 1,800 and 2,000 entries: the initialisation's SpMM cuts rows of more than
    # 1,024 entries into chunks whose partial sums it adds per row; against the FP64 oracle's
    # randomized t-SVD with the same test matrix
    from oracle.damf import DamfOracle
    from paper_2306_08967_gb300 import DamfGraph, make_config, rsvd_width
    from synth import gaussian_test_matrix
    n, d = 3000, 32
    ip, ix, _ = chung_lu_graph(n, 8.0, 2.5, seed=SEED + 520, directed=directed)
    rows = np.repeat(np.arange(n), np.diff(ip))
    # out-rows of nodes 0 and 7, and the in-row of node 11 (2,000 entries)
    hub_u = np.concatenate([np.zeros(2500, np.int64), np.full(1800, 7), np.arange(100, 2100)])
    hub_v = np.concatenate([np.arange(1, 2501), np.arange(1000, 2800), np.full(2000, 11)])
    u = np.concatenate([rows, hub_u] + ([] if directed else [hub_v]))
    v = np.concatenate([ix, hub_v] + ([] if directed else [hub_u]))
    keep = u != v
    key = np.unique(u[keep].astype(np.int64) * n + v[keep])
    u, v = key // n, key % n
    ip2 = np.concatenate([[0], np.cumsum(np.bincount(u, minlength=n))]).astype(np.int32)
    ix2 = v.astype(np.int32)
    assert np.diff(ip2).max() > 1024
    cfg = make_config(n, d, 0.15, 1e-4, n_capacity=n + 8, nnz=len(ix2), directed=directed)
    om = gaussian_test_matrix(n, rsvd_width(cfg), seed=SEED + 521)
    g = DamfGraph(ip2, ix2, cfg, om)
    orc = DamfOracle(ip2, ix2, d, 0.15, 1e-4, n_cap=n + 8, directed=directed, Omega=om, propagate=False)
    X, Y, sg = gpu_xy(g)
    np.testing.assert_allclose(sg, orc.sigma, rtol=1e-3)
    assert rel_fro(X @ Y.T, orc.X() @ orc.Y().T) < 1e-3
    g.close()


@pytest.mark.parametrize("directed", [False, True])
def test_each_update_equals_bruteforce_tsvd(directed):
    rng = np.random.default_rng(7)
    n, d = 400, 16
    g, _, (ip, ix, _) = make_pair(n, 8.0, 2.5, d, 0.15, 1e-4, SEED + 3, directed=directed, oracle=False)
    checked = 0
    for step in range(30):
        X1, Y1, _ = gpu_xy(g)
        rp0, col0 = g.adjacency()
        nn = 1 if step % 7 == 3 else 0
        src, dst, op = _events(rng, g.n + nn, int(rng.integers(1, 40)))
        if nn:
            src[0], dst[0], op[0] = g.n, int(rng.integers(0, g.n)), 1
        g.apply_edges(src, dst, op, new_nodes=nn)
        g.check()
        n1 = g.n
        rp1, col1 = g.adjacency()
        dA = dense_adj(rp1, col1, n1)
        A0 = np.zeros((n1, n1))
        A0[: n1 - nn, : n1 - nn] = dense_adj(rp0, col0, n1 - nn)
        dA -= A0
        Xp = np.vstack([X1, np.zeros((nn, d))])
        Yp = np.vstack([Y1, np.zeros((nn, d))])
        target = Xp @ Yp.T + dA
        sv = np.linalg.svd(target, compute_uv=False)
        if (sv[d - 1] - sv[d]) / sv[0] < 1e-3:
            continue
        X2, Y2, s2 = brute_force_update(Xp, Yp, dA, d)
        Xg, Yg, sg = gpu_xy(g)
        np.testing.assert_allclose(sg, s2, rtol=2e-4)
        assert rel_fro(Xg @ Yg.T, X2 @ Y2.T) < 2e-4
        checked += 1
    assert checked >= 15
    g.close()


@pytest.mark.parametrize("directed", [False, True])
def test_node_deletion(directed):
    # deleting a node = zeroing its row and column of A; a node of degree <= 48 goes in one
    # update, which must equal the brute-force t-SVD of (previous product + that change)
    # (Theorem 2); a hub goes in several updates; the adjacency loses exactly its edges
    n, d = 400, 16
    g, _, (ip, ix, _) = make_pair(n, 8.0, 2.5, d, 0.15, 1e-4, SEED + 70, directed=directed, oracle=False)
    rp, col = g.adjacency()
    A = dense_adj(rp, col, n)
    deg = A.sum(axis=1) + A.sum(axis=0)
    small = int(np.argmax(np.where((deg >= 8) & (deg <= 40), deg, -1)))
    checked = 0
    for u in (small, int(np.argmax(deg))):
        X1, Y1, _ = gpu_xy(g)
        rp0, col0 = g.adjacency()
        A0 = dense_adj(rp0, col0, n)
        g.delete_nodes([u])
        g.ppr_refresh()
        g.check()
        rp1, col1 = g.adjacency()
        A1 = dense_adj(rp1, col1, n)
        want = A0.copy()
        want[u, :] = 0.0
        want[:, u] = 0.0
        assert np.array_equal(A1, want)
        if u == small:
            dA = A1 - A0
            target = X1 @ Y1.T + dA
            sv = np.linalg.svd(target, compute_uv=False)
            if (sv[d - 1] - sv[d]) / sv[0] > 1e-3:
                X2, Y2, s2 = brute_force_update(X1, Y1, dA, d)
                Xg, Yg, sg = gpu_xy(g)
                np.testing.assert_allclose(sg, s2, rtol=2e-4)
                assert rel_fro(Xg @ Yg.T, X2 @ Y2.T) < 2e-4
                checked += 1
    assert checked == 1
    from paper_2306_08967_gb300 import DamfError
    with pytest.raises(DamfError):
        g.delete_nodes([n + 5])
    g.check()                      # a rejected id leaves the context usable
    g.close()


@pytest.mark.parametrize("directed", [False, True])
def test_adjacency_and_touched_sets_bit_exact(directed):
    from oracle.graph import DynGraph
    rng = np.random.default_rng(9)
    n, d = 600, 16
    g, _, (ip, ix, _) = make_pair(n, 6.0, 2.3, d, 0.15, 1e-4, SEED + 5, directed=directed, oracle=False)
    og = DynGraph(ip, ix, n + 64, directed=directed)
    for step in range(40):
        k = int(rng.integers(1, 49))
        src, dst, op = _events(rng, n, k, p_del=0.4)
        if step % 5 == 0:    # repeat events inside one update: the last one decides
            src[-1], dst[-1], op[-1] = src[0], dst[0], -op[0]
        g.apply_edges(src, dst, op)
        ch = og.apply(src, dst, op)
        S, T = g.last_touched()
        if ch.empty:
            assert len(S) == 0 and len(T) == 0
        else:
            assert S.tolist() == ch.S.tolist() and T.tolist() == ch.T.tolist()
    g.check()
    for outgoing in (True, False):
        rp, col = g.adjacency(outgoing)
        adj = og.out if outgoing else og.inn
        for u in range(n):
            assert sorted(col[rp[u]:rp[u + 1]].tolist()) == sorted(adj.row(u).tolist()), u
    g.close()


@pytest.mark.parametrize("directed", [False, True])
def test_ppr_within_eps_of_exact(directed):
    rng = np.random.default_rng(11)
    n, d, alpha, eps = 500, 16, 0.15, 1e-5
    g, _, _ = make_pair(n, 8.0, 2.5, d, alpha, eps, SEED + 7, directed=directed, oracle=False)
    for step in range(6):
        if step:
            src, dst, op = _events(rng, n, 20)
            g.apply_edges(src, dst, op)
            g.ppr_refresh()
        g.check()
        st = g.state()
        Xb = (st["Ub"] * st["s0"]).double().cpu().numpy()
        Zb = st["Zb"].double().cpu().numpy()
        r = st["r"].double().cpu().numpy()
        rp, col = g.adjacency()
        A = dense_adj(rp, col, g.n)
        exact = ppr_matrix_dense(A, alpha) @ Xb
        assert np.abs(r).max() <= eps
        assert np.abs(Zb - exact).max() <= eps * (1 + 1e-3) + 2e-6 * np.abs(Xb).max()
    g.close()


@pytest.mark.parametrize("directed", [False, True])
def test_ppr_bound_with_hub_rows(directed):
    # d = 128 and a heavy-tailed graph: rows with more than 64 in-edges are pushed as hub
    # items (rho slot + chunk tasks), rows with fewer directly; both must keep the eps bound
    rng = np.random.default_rng(13)
    n, d, alpha, eps = 2500, 128, 0.15, 1e-5
    g, _, (ip, ix, _) = make_pair(n, 12.0, 2.05, d, alpha, eps, SEED + 27, directed=directed, oracle=False)
    assert np.diff(ip).max() > 150                      # the graph has hubs
    for step in range(4):
        if step:
            src, dst, op = _events(rng, n, 30)
            g.apply_edges(src, dst, op)
            g.ppr_refresh()
        g.check()
        st = g.state()
        Xb = (st["Ub"] * st["s0"]).double().cpu().numpy()
        Zb = st["Zb"].double().cpu().numpy()
        r = st["r"].double().cpu().numpy()
        rp, col = g.adjacency()
        A = dense_adj(rp, col, g.n)
        exact = ppr_matrix_dense(A, alpha) @ Xb
        assert np.abs(r).max() <= eps
        assert np.abs(Zb - exact).max() <= eps * (1 + 1e-3) + 2e-6 * np.abs(Xb).max()
    g.close()


def test_ppr_bound_when_the_queue_overflows(monkeypatch):
    # a 2048-position work queue: the initial push (every row seeded) and the larger updates
    # overflow it, so rows and hub items miss the queue; the rows are found again by the rescan
    # that ends each phase and the hub items are scattered there, so the eps bound must hold
    monkeypatch.setenv("DAMF_PUSH_QUEUE_CAP", "2048")
    rng = np.random.default_rng(15)
    n, d, alpha, eps = 1500, 128, 0.15, 1e-5
    g, _, (ip, ix, _) = make_pair(n, 12.0, 2.05, d, alpha, eps, SEED + 29, oracle=False)
    assert np.diff(ip).max() > 100
    for step in range(3):
        if step:
            src, dst, op = _events(rng, n, 30)
            g.apply_edges(src, dst, op)
            g.ppr_refresh()
        g.check()
        st = g.state()
        Xb = (st["Ub"] * st["s0"]).double().cpu().numpy()
        Zb = st["Zb"].double().cpu().numpy()
        r = st["r"].double().cpu().numpy()
        rp, col = g.adjacency()
        A = dense_adj(rp, col, g.n)
        exact = ppr_matrix_dense(A, alpha) @ Xb
        assert np.abs(r).max() <= eps
        assert np.abs(Zb - exact).max() <= eps * (1 + 1e-3) + 2e-6 * np.abs(Xb).max()
    assert g.stats()["push_rounds"] > 3           # the pushes took several phases
    g.close()


@pytest.mark.parametrize("directed", [False, True])
def test_degree_scaled_threshold_bound(directed):
    # threshold eps * max(deg(u), 1): every residual ends below its own threshold and
    # |Zb - Pi Xb|[i] <= (Pi t)[i] for the thresholds t (FP32 slack as in the absolute test)
    rng = np.random.default_rng(21)
    n, d, alpha, eps = 500, 16, 0.15, 1e-4
    g, _, _ = make_pair(n, 8.0, 2.5, d, alpha, eps, SEED + 17, directed=directed, oracle=False,
                        threshold="degree")
    above_eps = False
    for step in range(5):
        if step:
            src, dst, op = _events(rng, n, 20)
            g.apply_edges(src, dst, op)
            g.ppr_refresh()
        g.check()
        st = g.state()
        Xb = (st["Ub"] * st["s0"]).double().cpu().numpy()
        Zb = st["Zb"].double().cpu().numpy()
        r = st["r"].double().cpu().numpy()
        rp, col = g.adjacency()
        A = dense_adj(rp, col, g.n)
        thr = eps * np.maximum(A.sum(axis=1), 1.0)
        rmax = np.abs(r[: g.n]).max(axis=1)
        assert np.all(rmax <= thr * (1 + 1e-6))
        above_eps |= bool(np.any(rmax > eps))
        Pi = ppr_matrix_dense(A, alpha)
        err = np.abs(Zb - Pi @ Xb).max(axis=1)
        assert np.all(err <= (Pi @ thr) * (1 + 1e-3) + 2e-6 * np.abs(Xb).max())
    assert above_eps
    g.close()


def test_apply_edges_multi_equals_each_graph_alone():
    # graphs of uneven size and rank in one call: every graph's factor state must be the same,
    # bit for bit, as when its batch is applied alone (the push order is free, so Z_b and r are
    # compared through the eps bound elsewhere)
    from paper_2306_08967_gb300 import apply_edges_multi
    rng = np.random.default_rng(23)
    specs = [(400, 16, False), (900, 32, True), (650, 64, False)]
    mix = [make_pair(n, 8.0, 2.5, d, 0.15, 1e-5, SEED + 40 + i, directed=dr, oracle=False)[0]
           for i, (n, d, dr) in enumerate(specs)]
    alone = [make_pair(n, 8.0, 2.5, d, 0.15, 1e-5, SEED + 40 + i, directed=dr, oracle=False)[0]
             for i, (n, d, dr) in enumerate(specs)]
    for step in range(4):
        batches = []
        for (n, d, dr), gm, ga in zip(specs, mix, alone):
            src, dst, op = _events(rng, n, int(rng.integers(1, 70)))
            batches.append((gm, src, dst, op))
            ga.apply_edges(src, dst, op)
            ga.ppr_refresh()
        apply_edges_multi(batches)
        for gm in mix:
            gm.ppr_refresh()
    for i, (gm, ga) in enumerate(zip(mix, alone)):
        gm.check()
        ga.check()
        a, b = gm.state(), ga.state()
        for k in ("Ub", "Vb", "PU", "PV", "sigma"):
            assert torch.equal(a[k], b[k]), (i, k)
        ra, ca = gm.adjacency()
        rb, cb = ga.adjacency()
        assert np.array_equal(ra, rb)
        for u in range(len(ra) - 1):
            assert sorted(ca[ra[u]:ra[u + 1]].tolist()) == sorted(cb[rb[u]:rb[u + 1]].tolist())
        gm.close()
        ga.close()


def test_captured_step_replays_like_direct_calls():
    # one step (apply a 40-event batch, push, join) captured in a CUDA graph and replayed with
    # new events written into its input buffers must leave the same factor state, bit for bit,
    # as the same batches applied by direct calls to a twin context
    from paper_2306_08967_gb300 import DamfGraph
    rng = np.random.default_rng(31)
    n, k = 500, 40
    g, _, _ = make_pair(n, 8.0, 2.5, 32, 0.15, 1e-5, SEED + 120, oracle=False)
    twin, _, _ = make_pair(n, 8.0, 2.5, 32, 0.15, 1e-5, SEED + 120, oracle=False)
    batches = [_events(rng, n, k) for _ in range(6)]
    src = torch.empty(k, dtype=torch.int32, device="cuda")
    dst = torch.empty(k, dtype=torch.int32, device="cuda")
    op = torch.empty(k, dtype=torch.int8, device="cuda")
    stream = torch.cuda.Stream()
    lib, h = g.lib, g.h
    sp = __import__("ctypes").c_void_p
    sptr = sp(stream.cuda_stream)

    def step_calls():
        assert lib.damf_apply_edges(h, sp(src.data_ptr()), sp(dst.data_ptr()), sp(op.data_ptr()), k, 0, sptr) == 0
        assert lib.damf_ppr_refresh(h, sptr) == 0
        assert lib.damf_join(h, sptr) == 0

    def load(b):
        src.copy_(torch.from_numpy(b[0]))
        dst.copy_(torch.from_numpy(b[1]))
        op.copy_(torch.from_numpy(b[2]))

    # the first batch by direct calls on both, then capture
    load(batches[0])
    with torch.cuda.stream(stream):
        assert lib.damf_join(h, sptr) == 0
        step_calls()
    stream.synchronize()
    twin.apply_edges(*batches[0])
    twin.ppr_refresh()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
        step_calls()
    for b in batches[1:]:
        load(b)
        graph.replay()
        torch.cuda.synchronize()
        twin.apply_edges(*b)
        twin.ppr_refresh()
    g.check()
    twin.check()
    a, b = g.state(), twin.state()
    for key in ("Ub", "Vb", "PU", "PV", "sigma"):
        assert torch.equal(a[key], b[key]), key
    ra, ca = g.adjacency()
    rb, cb = twin.adjacency()
    assert np.array_equal(ra, rb)
    g.close()
    twin.close()


def test_alpha_one_gives_z_equal_x():
    # the paper's ablation: alpha = 1 means Z = X
    g, _, _ = make_pair(300, 8.0, 2.5, 16, 1.0, 1e-6, SEED + 9, oracle=False)
    g.apply_edges(np.array([1, 2], np.int32), np.array([5, 9], np.int32), np.array([1, 1], np.int8))
    g.ppr_refresh()
    e = g.embeddings()
    np.testing.assert_allclose(e["Z"].cpu().numpy(), e["X"].cpu().numpy(), atol=2e-6)
    g.close()


def test_c1_stream_against_oracle():
    c = CONFIGS["C1"]
    ip, ix, w = chung_lu_graph(c.n, c.avg_deg, c.gamma, seed=c.seed)
    stream = edge_stream(ip, ix, w, c.n_batches, c.k_lo, c.k_hi, c.p_node, c.p_del, c.seed + 1,
                         max_new_degree=c.max_new_degree, nodes_per_batch=c.nodes_per_batch)
    from oracle.damf import DamfOracle
    from paper_2306_08967_gb300 import DamfGraph, make_config, rsvd_width
    from synth import gaussian_test_matrix
    cfg = make_config(c.n, c.d, c.alpha, c.eps, n_capacity=stream.n_final, nnz=len(ix))
    om = gaussian_test_matrix(c.n, rsvd_width(cfg), seed=c.seed + 2)
    g = DamfGraph(ip, ix, cfg, om)
    orc = DamfOracle(ip, ix, c.d, c.alpha, c.eps, n_cap=stream.n_final, Omega=om)
    for b in stream.batches:
        g.apply_edges(b.src, b.dst, b.op, b.new_nodes)
        g.ppr_refresh()
        orc.apply_edges(b.src, b.dst, b.op, b.new_nodes)
        orc.ppr_refresh()
    g.check()
    Xg, Yg, sg = gpu_xy(g)
    _stream_close("C1 stream", sg, Xg, Yg, orc)
    # Z is PPR(X); columns of X, Y, Z carry a common sign (or rotation within a repeated
    # singular value), so compare the invariant product Z Y^T = PPR(X Y^T)
    Zg = g.embeddings()["Z"].double().cpu().numpy()
    assert rel_fro(Zg @ Yg.T, orc.Z() @ orc.Y().T) < 1e-3
    g.close()


@pytest.mark.parametrize("directed", [False, True])
def test_node_arrival_stream_against_oracle(directed):
    # the paper's protocol (Sec. 5.1): an initial induced graph, then nodes arrive one at a time
    # with their edges to the nodes already present; one call (and one push) per node event
    from oracle.damf import DamfOracle
    from paper_2306_08967_gb300 import DamfGraph, make_config, rsvd_width
    from synth import gaussian_test_matrix, node_arrival_stream
    n, n0, d = 520, 220, 16
    ip, ix, _ = chung_lu_graph(n, 8.0, 2.5, seed=SEED + 60, directed=directed)
    ip0, ix0, stream = node_arrival_stream(ip, ix, n0, directed=directed)
    # 300 FP32 updates: with the periodic fold (re-orthonormalisation, as in the bench) the
    # drift stays bounded; the fold leaves U Sigma V^T unchanged, so the FP64 oracle needs none
    cfg = make_config(n0, d, 0.15, 1e-4, n_capacity=n, nnz=len(ix0), directed=directed, refold_every=100)
    om = gaussian_test_matrix(n0, rsvd_width(cfg), seed=SEED + 61)
    g = DamfGraph(ip0, ix0, cfg, om)
    orc = DamfOracle(ip0, ix0, d, 0.15, 1e-4, n_cap=n, directed=directed, Omega=om)
    for b in stream.batches:
        g.apply_edges(b.src, b.dst, b.op, b.new_nodes)
        g.ppr_refresh()
        orc.apply_edges(b.src, b.dst, b.op, b.new_nodes)
        orc.ppr_refresh()
    g.check()
    assert g.n == n
    Xg, Yg, sg = gpu_xy(g)
    # X Y^T to 1e-3 here: on this 220-520 node graph the gap at the rank-16 cut falls to
    # 5.5e-3 sigma_1, and each update near such a gap turns rounding of the FP32 state into a
    # lasting difference in which direction is truncated (an FP32 emulation of the same steps
    # with an LAPACK core SVD reaches 7.6e-5 after the 300 arrivals, the device 5.3e-4);
    # sigma stays within 1e-4
    _stream_close("node arrivals, directed=%s" % directed, sg, Xg, Yg, orc, xy_tol=1e-3)
    Zg = g.embeddings()["Z"].double().cpu().numpy()
    assert rel_fro(Zg @ Yg.T, orc.Z() @ orc.Y().T) < 1e-3
    # the final graph is the full graph
    rp, col = g.adjacency()
    A = dense_adj(rp, col, n)
    assert np.array_equal(A, dense_adj(ip, ix, n))
    g.close()


def test_c3_shaped_stream_against_oracle():
    # the C3 shape at a checkable size: gamma 2.1, mean degree 40, calls of up to 256 events
    # (up to four updates each), node arrivals and deletions, the fold every 256 updates
    from oracle.damf import DamfOracle
    from paper_2306_08967_gb300 import DamfGraph, make_config, rsvd_width
    from synth import gaussian_test_matrix
    n, d = 3000, 32
    ip, ix, w = chung_lu_graph(n, 40.0, 2.1, seed=SEED + 80)
    st = edge_stream(ip, ix, w, 24, 1, 256, 0.05, 0.10, SEED + 81)
    cfg = make_config(n, d, 0.15, 1e-4, n_capacity=st.n_final, nnz=len(ix), refold_every=256)
    om = gaussian_test_matrix(n, rsvd_width(cfg), seed=SEED + 82)
    g = DamfGraph(ip, ix, cfg, om)
    orc = DamfOracle(ip, ix, d, 0.15, 1e-4, n_cap=st.n_final, Omega=om)
    for b in st.batches:
        g.apply_edges(b.src, b.dst, b.op, b.new_nodes)
        g.ppr_refresh()
        orc.apply_edges(b.src, b.dst, b.op, b.new_nodes)
        orc.ppr_refresh()
    g.check()
    assert g.stats()["updates"] > len(st.batches)     # calls above 64 events took several updates
    Xg, Yg, sg = gpu_xy(g)
    _stream_close("C3 shape", sg, Xg, Yg, orc)
    Zg = g.embeddings()["Z"].double().cpu().numpy()
    assert rel_fro(Zg @ Yg.T, orc.Z() @ orc.Y().T) < 1e-3
    g.close()


def test_c4_shaped_graphs_in_one_call_against_oracles():
    # the C4 shape at a checkable size: graphs of log-uniform n, mean degree U[4, 32] and
    # d in {32, 64, 128}, one batch of U[1, 128] events per graph per damf_apply_edges_multi
    # call; each graph against its own FP64 oracle
    from oracle.damf import DamfOracle
    from paper_2306_08967_gb300 import DamfGraph, apply_edges_multi, make_config, rsvd_width
    from synth import gaussian_test_matrix
    rng = np.random.default_rng(SEED + 90)
    graphs = []
    for i in range(6):
        n = int(np.exp(rng.uniform(np.log(300), np.log(2500))))
        d = int(rng.choice([32, 64, 128]))
        if d >= n // 4:
            d = 32
        ip, ix, w = chung_lu_graph(n, float(rng.uniform(4, 32)), 2.3, seed=SEED + 91 + i)
        st = edge_stream(ip, ix, w, 8, 1, 128, 0.05, 0.10, SEED + 101 + i)
        cfg = make_config(n, d, 0.15, 1e-4, n_capacity=st.n_final, nnz=len(ix))
        om = gaussian_test_matrix(n, rsvd_width(cfg), seed=SEED + 111 + i)
        graphs.append((DamfGraph(ip, ix, cfg, om), DamfOracle(ip, ix, d, 0.15, 1e-4, n_cap=st.n_final, Omega=om), st))
    for t in range(8):
        apply_edges_multi([(g, st.batches[t].src, st.batches[t].dst, st.batches[t].op, st.batches[t].new_nodes)
                           for g, _, st in graphs])
        for g, orc, st in graphs:
            b = st.batches[t]
            g.ppr_refresh()
            orc.apply_edges(b.src, b.dst, b.op, b.new_nodes)
            orc.ppr_refresh()
    for g, orc, _ in graphs:
        g.check()
        Xg, Yg, sg = gpu_xy(g)
        _stream_close("C4 shape, n=%d d=%d" % (g.n, g.d), sg, Xg, Yg, orc)
        Zg = g.embeddings()["Z"].double().cpu().numpy()
        assert rel_fro(Zg @ Yg.T, orc.Z() @ orc.Y().T) < 1e-3
        g.close()


def test_edge_cases():
    from paper_2306_08967_gb300 import DamfError
    g, _, _ = make_pair(200, 6.0, 2.5, 16, 0.2, 1e-4, SEED + 11, n_extra=4, oracle=False)
    s0 = gpu_xy(g)[2]
    g.apply_edges(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int8))   # empty call
    rp, col = g.adjacency()
    u = 0
    v = int(col[rp[0]])
    g.apply_edges(np.array([u], np.int32), np.array([v], np.int32), np.array([1], np.int8))  # existing edge
    g.check()
    np.testing.assert_array_equal(gpu_xy(g)[2], s0)
    g.apply_edges(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int8), new_nodes=1)  # lone node
    assert g.n == 201
    # 130 events: three consecutive updates in one call
    rng = np.random.default_rng(3)
    src, dst, op = _events(rng, 201, 130)
    g.apply_edges(src, dst, op)
    g.ppr_refresh()
    g.check()
    with pytest.raises(DamfError):
        g.apply_edges(np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int8), new_nodes=10)
    g.close()
    # device-side validation: a self-loop poisons the context, nothing is written
    g, _, _ = make_pair(200, 6.0, 2.5, 16, 0.2, 1e-4, SEED + 13, oracle=False)
    g.apply_edges(np.array([3], np.int32), np.array([3], np.int32), np.array([1], np.int8))
    assert g.sync_status() == 1
    g.close()
    # adjacency capacity exhaustion is reported before any write
    from paper_2306_08967_gb300 import DamfGraph, make_config, rsvd_width
    from synth import gaussian_test_matrix
    ip, ix, _ = chung_lu_graph(200, 6.0, 2.5, seed=SEED + 15)
    cfg = make_config(200, 16, 0.2, 1e-4, nnz=len(ix), m_capacity=int(len(ix) * 1.3) + 1200)
    g = DamfGraph(ip, ix, cfg, gaussian_test_matrix(200, rsvd_width(cfg), SEED + 17))
    status = 0
    for i in range(200):
        src = np.arange(0, 40, dtype=np.int32) + (i % 4) * 40
        dst = (src + 1 + i) % 200
        g.apply_edges(src.astype(np.int32), dst.astype(np.int32), np.ones(40, np.int8))
        status = g.sync_status()
        if status:
            break
    assert status == 2
    g.close()


@pytest.mark.parametrize("d,r", [(16, 5), (64, 40), (128, 96), (128, 128)])
def test_core_svd_against_numpy(d, r):
    # Step 2 alone: the top-d SVD of diag(sigma, 0) + L R^T for random cores shaped like
    # the update's (W blocks small, R blocks O(1))
    from paper_2306_08967_gb300 import core_svd
    rng = np.random.default_rng(d + r)
    sigma = np.sort(rng.uniform(2.0, 40.0, d))[::-1]
    L = np.vstack([0.05 * rng.standard_normal((d, r)), np.triu(rng.standard_normal((r, r))) + np.eye(r)])
    R = np.vstack([0.05 * rng.standard_normal((d, r)), np.triu(rng.standard_normal((r, r))) + np.eye(r)])
    M = np.zeros((d + r, d + r))
    M[:d, :d] = np.diag(sigma)
    M += L @ R.T
    U, s, Vt = np.linalg.svd(M)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    E, H, th = core_svd(sigma.astype(np.float32), L.astype(np.float32), R.astype(np.float32), status=status)
    E, H, th = E.double().cpu().numpy(), H.double().cpu().numpy(), th.double().cpu().numpy()
    assert int(status.item()) == 0          # converged, finite
    np.testing.assert_allclose(th, s[:d], rtol=1e-4, atol=1e-5 * s[0])
    top = (U[:, :d] * s[:d]) @ Vt[:d]
    assert rel_fro((E * th) @ H.T, top) < 1e-4
    # E comes from orthogonalised columns (Jacobi tolerance 1e-6); H = M^T E Theta^{-1}
    # inherits FP32 rounding amplified by sigma_1 / sigma_d (20 here) and sqrt(d + r)
    assert np.abs(E.T @ E - np.eye(d)).max() < 2e-5
    assert np.abs(H.T @ H - np.eye(d)).max() < 5e-4


def _run_stream(precision, refold_every, n_batches=30, d=32, seed=SEED + 21):
    from paper_2306_08967_gb300 import DamfGraph, make_config, rsvd_width
    from synth import gaussian_test_matrix
    ip, ix, w = chung_lu_graph(1500, 10.0, 2.5, seed=seed)
    st = edge_stream(ip, ix, w, n_batches, 1, 40, 0.05, 0.1, seed + 1)
    cfg = make_config(1500, d, 0.15, 1e-5, n_capacity=st.n_final, nnz=len(ix), refold_every=refold_every,
                      precision=precision)
    g = DamfGraph(ip, ix, cfg, gaussian_test_matrix(1500, rsvd_width(cfg), seed + 2))
    for b in st.batches:
        g.apply_edges(b.src, b.dst, b.op, b.new_nodes)
        g.ppr_refresh()
    g.check()
    X, Y, s = gpu_xy(g)
    Z = g.embeddings()["Z"].double().cpu().numpy()
    folds = g.stats()["folds"]
    g.close()
    return X, Y, Z, s, folds, (ip, ix, st)


def test_fold_preserves_the_factorisation():
    # the periodic fold re-bases U_b, V_b and resets P to I; U Sigma V^T must not change
    X0, Y0, Z0, s0, f0, _ = _run_stream("fp32", 0)
    X1, Y1, Z1, s1, f1, (ip, ix, st) = _run_stream("fp32", 4)
    assert f0 == 0 and f1 >= 7
    np.testing.assert_allclose(s1, s0, rtol=2e-5)
    assert rel_fro(X1 @ Y1.T, X0 @ Y0.T) < 2e-5
    assert rel_fro(Z1 @ Y1.T, Z0 @ Y0.T) < 1e-3      # both within eps of PPR of the same X
    # and against the FP64 oracle on the same stream
    from oracle.damf import DamfOracle
    from synth import gaussian_test_matrix
    from paper_2306_08967_gb300 import make_config, rsvd_width
    cfg = make_config(1500, 32, 0.15, 1e-5)
    orc = DamfOracle(ip, ix, 32, 0.15, 1e-5, n_cap=st.n_final, Omega=gaussian_test_matrix(1500, rsvd_width(cfg), SEED + 23),
                     propagate=False)
    for b in st.batches:
        orc.apply_edges(b.src, b.dst, b.op, b.new_nodes)
    _stream_close("folded stream", s1, X1, Y1, orc)


def test_mixed_precision_matches_plain_fp32():
    # tensor-core GEMMs (TF32 with a three-term split) in the fold, init and query give
    # the FP32 results within FP32-level differences
    Xm, Ym, Zm, sm, fm, _ = _run_stream("mixed", 4)
    Xp, Yp, Zp, sp, fp, _ = _run_stream("fp32", 4)
    assert fm == fp and fm >= 7
    np.testing.assert_allclose(sm, sp, rtol=2e-5)
    assert rel_fro(Xm @ Ym.T, Xp @ Yp.T) < 2e-5
    assert rel_fro(Zm @ Ym.T, Zp @ Yp.T) < 1e-3


def test_factor_reads_do_not_depend_on_the_push():
    # X, Y and sigma are final when the update's work on the caller's stream is; reading them
    # right after damf_ppr_refresh (the push possibly still running) gives what a read after
    # the push gives, and Z (which waits for the push) is the push's result
    rng = np.random.default_rng(61)
    g, _, _ = make_pair(3000, 10.0, 2.2, 64, 0.15, 1e-5, SEED + 140, oracle=False)
    for _ in range(4):
        g.apply_edges(*_events(rng, g.n, 60))
        g.ppr_refresh()
        early = g.embeddings(want=("X", "Y", "sigma"))
        g.join()
        torch.cuda.synchronize()
        late = g.embeddings(want=("X", "Y", "Z", "sigma"))
        for k in ("X", "Y", "sigma"):
            assert torch.equal(early[k], late[k]), k
        st = g.state()
        Z = ((st["Zb"].double() / st["s0"].double()) @ st["PU"].double()) * st["sigma"].double().sqrt()
        assert torch.allclose(late["Z"].double(), Z, rtol=1e-4, atol=1e-6)
    g.check()
    g.close()


def test_inputs_are_staged_on_the_given_stream():
    # host events handed over with stream=s are copied to the device on s: a long kernel queued
    # on torch's current stream must not hold the copies back past the library's reads on s,
    # and a twin stepped on the current stream ends with bit-identical factors
    rng = np.random.default_rng(71)
    a, _, _ = make_pair(2000, 8.0, 2.2, 32, 0.15, 1e-5, SEED + 150, oracle=False)
    b, _, _ = make_pair(2000, 8.0, 2.2, 32, 0.15, 1e-5, SEED + 150, oracle=False)
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    for _ in range(5):
        ev = _events(rng, a.n, 50)
        torch.cuda._sleep(20_000_000)         # about 10 ms of spinning on the current stream
        a.apply_edges(*ev, stream=s)
        a.ppr_refresh(stream=s)
        b.apply_edges(*ev)
        b.ppr_refresh()
    ea = a.embeddings(want=("X", "Y", "sigma"), stream=s)
    s.synchronize()
    eb = b.embeddings(want=("X", "Y", "sigma"))
    torch.cuda.synchronize()
    for k in ("X", "Y", "sigma"):
        assert torch.equal(ea[k], eb[k]), k
    a.check()
    b.check()
    a.close()
    b.close()


@pytest.mark.parametrize("d,n", [(32, 203), (64, 1000), (128, 1300)])
def test_full_table_query_on_tensor_cores_matches_row_query(d, n):
    # mixed precision answers a full-table query (rows = NULL) with the TMA-fed tcgen05 GEMM
    # (three-term TF32 split) and a row list with the SIMT kernel: the two must agree to FP32
    # accuracy; n is not a multiple of the 128-row tile, and 203 and 1300 end in a partial
    # group of 8 rows, which the tensor map leaves out and the kernel reads with plain loads
    g, _, _ = make_pair(n, 10.0, 2.5, d, 0.15, 1e-4, SEED + 500 + d, oracle=False)
    full = g.embeddings()
    rows = g.embeddings(rows=np.arange(g.n, dtype=np.int32))
    for k in ("X", "Y", "Z"):
        a, b = full[k].double().cpu().numpy(), rows[k].double().cpu().numpy()
        scale = np.abs(b).max()
        assert np.abs(a - b).max() <= 2e-6 * scale, (k, np.abs(a - b).max() / scale)
    g.close()
