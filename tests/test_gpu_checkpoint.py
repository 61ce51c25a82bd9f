"""Checkpoint and resume through the C ABI (damf_save_state, damf_export_adjacency,
damf_restore): a context restored from a checkpoint continues the original exactly — the same
further calls (node arrivals, deletions, a fold) give bit-identical factors and adjacency, and
its PPR state keeps the eps bound of the graph it ends with."""

import numpy as np
import pytest
import torch

from oracle.ppr import ppr_matrix_dense
from tests.gpu_util import dense_adj, make_pair

pytestmark = pytest.mark.gpu

SEED = 0xDA3F0000 + 700
FACTORS = ("Ub", "Vb", "PU", "PV", "sigma")


def _events(rng, n, k, p_del=0.2):
    src, dst, op = [], [], []
    while len(src) < k:
        u, v = rng.integers(0, n, 2)
        if u != v:
            src.append(u), dst.append(v), op.append(-1 if rng.random() < p_del else 1)
    return np.array(src, np.int32), np.array(dst, np.int32), np.array(op, np.int8)


def _same(a, b, directed):
    sa, sb = a.state(), b.state()
    for key in FACTORS:
        assert torch.equal(sa[key], sb[key]), key
    for outgoing in ([True, False] if directed else [True]):
        ra, ca = a.adjacency(outgoing=outgoing)
        rb, cb = b.adjacency(outgoing=outgoing)
        assert np.array_equal(ra, rb)
        for u in range(a.n):
            assert np.array_equal(np.sort(ca[ra[u]:ra[u + 1]]), np.sort(cb[rb[u]:rb[u + 1]]))


@pytest.mark.parametrize("directed", [False, True])
def test_restore_continues_the_original(directed):
    from paper_2306_08967_gb300 import DamfGraph
    rng = np.random.default_rng(71 + directed)
    g, _, _ = make_pair(700, 8.0, 2.4, 32, 0.15, 1e-5, SEED + directed, directed=directed, refold_every=4,
                      oracle=False)
    for i in range(5):
        n = g.n
        nn = i % 2
        ev = _events(rng, n + nn, 40)
        if nn:   # the arriving node's first edge
            ev = (np.append(ev[0], n).astype(np.int32), np.append(ev[1], 3).astype(np.int32),
                  np.append(ev[2], 1).astype(np.int8))
        g.apply_edges(*ev, new_nodes=nn)
        g.ppr_refresh()
    ck = g.save()
    torch.cuda.synchronize()
    h = DamfGraph.restore(ck)
    assert h.n == g.n
    _same(g, h, directed)
    st_g, st_h = g.state(), h.state()
    assert torch.equal(st_g["Zb"], st_h["Zb"]) and torch.equal(st_g["r"], st_h["r"])
    for i in range(6):   # the fold comes at the 8th update since the start
        n = g.n
        nn = 1 if i == 2 else 0
        ev = _events(rng, n + nn, 50)
        if nn:
            ev = (np.append(ev[0], n).astype(np.int32), np.append(ev[1], 5).astype(np.int32),
                  np.append(ev[2], 1).astype(np.int8))
        for x in (g, h):
            x.apply_edges(*ev, new_nodes=nn)
            x.ppr_refresh()
    g.check()
    h.check()
    assert g.stats()["folds"] >= 1 and h.stats()["folds"] >= 1
    _same(g, h, directed)
    st = h.state()
    Xb = (st["Ub"] * st["s0"]).double().cpu().numpy()
    rp, col = h.adjacency()
    exact = ppr_matrix_dense(dense_adj(rp, col, h.n), 0.15) @ Xb
    assert np.abs(st["r"].double().cpu().numpy()).max() <= 1e-5
    assert np.abs(st["Zb"].double().cpu().numpy() - exact).max() <= 1e-5 * (1 + 1e-3) + 2e-6 * np.abs(Xb).max()
    g.close()
    h.close()
