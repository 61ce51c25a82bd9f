"""Long FP32 streams against the FP64 oracle: the stated tolerance after 1,000 updates.

The target is relative error <= 1e-4 for the FP32 device path after 1,000 updates: sigma
elementwise and X Y^T in relative Frobenius norm (X Y^T = U Sigma V^T is invariant to the
signs and rotations of the singular vectors, Thm 2).  Two workloads, each 1,000 batches
that are one update each (<= 64 events):
  * the C1 shape (d = 16, n = 2,000, gamma 2.5, 10 insertions plus one node arrival per batch);
  * the C2 shape at a checkable size (d = 128, n = 3,000, gamma 2.2, mean degree 10, batches
    of U[1, 64] events with 5% node arrivals and 10% deletions).
Both device precisions (plain FP32 and mixed) step in lockstep against one oracle run, the
fold every 256 updates as in the bench.  The oracle pushes nothing (the factors do not
depend on the push); the device pushes after every batch, so the factor chain runs beside
its pushes as in production.
"""

import numpy as np
import pytest

from synth import chung_lu_graph, edge_stream, gaussian_test_matrix
from tests.gpu_util import gpu_xy, rel_fro

pytestmark = pytest.mark.gpu

TOL = 1e-4
UPDATES = 1000


def _run(n, avg_deg, gamma, d, k_lo, k_hi, p_node, p_del, nodes_per_batch, eps, seed):
    from oracle.damf import DamfOracle
    from paper_2306_08967_gb300 import DamfGraph, make_config, rsvd_width
    ip, ix, w = chung_lu_graph(n, avg_deg, gamma, seed=seed)
    st = edge_stream(ip, ix, w, UPDATES, k_lo, k_hi, p_node, p_del, seed + 1, nodes_per_batch=nodes_per_batch)
    assert all(b.k <= 64 for b in st.batches)        # one update per batch
    graphs = {}
    for prec in ("mixed", "fp32"):
        cfg = make_config(n, d, 0.15, eps, n_capacity=st.n_final, nnz=len(ix), refold_every=256, precision=prec)
        om = gaussian_test_matrix(n, rsvd_width(cfg), seed=seed + 2)
        graphs[prec] = DamfGraph(ip, ix, cfg, om)
    orc = DamfOracle(ip, ix, d, 0.15, eps, n_cap=st.n_final, Omega=om, propagate=False)
    gaps = []
    for b in st.batches:
        for g in graphs.values():
            g.apply_edges(b.src, b.dst, b.op, b.new_nodes)
            g.ppr_refresh()
        orc.apply_edges(b.src, b.dst, b.op, b.new_nodes)
        sv = orc.last_core_sv
        if sv is not None and len(sv) > d:
            gaps.append((sv[d - 1] - sv[d]) / sv[0])
    assert orc.stats_updates >= UPDATES - 10          # a batch whose events cancel is no update
    P = orc.X() @ orc.Y().T
    out = {}
    for prec, g in graphs.items():
        g.check()
        assert g.stats()["updates"] == orc.stats_updates
        X, Y, s = gpu_xy(g)
        out[prec] = (float(np.max(np.abs(s - orc.sigma) / orc.sigma)), rel_fro(X @ Y.T, P))
        g.close()
    return out, min(gaps)


def test_c1_shape_1000_updates_within_1e4():
    out, gap = _run(2000, 10.0, 2.5, 16, 10, 10, 0.0, 0.0, 1, 1e-4, 0xDA3F0000 + 300)
    print("C1 shape, 1000 updates: %s (smallest relative gap at the cut %.2e)" % (out, gap))
    for prec, (es, ex) in out.items():
        assert es <= TOL, (prec, es)
        assert ex <= TOL, (prec, ex)


def test_c2_shape_d128_1000_updates_within_1e4():
    out, gap = _run(3000, 10.0, 2.2, 128, 1, 64, 0.05, 0.10, 0, 1e-4, 0xDA3F0000 + 310)
    print("C2 shape d=128, 1000 updates: %s (smallest relative gap at the cut %.2e)" % (out, gap))
    for prec, (es, ex) in out.items():
        assert es <= TOL, (prec, es)
        assert ex <= TOL, (prec, ex)
