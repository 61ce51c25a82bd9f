"""Pins for the oracle's PPR pieces (Sec. 4.4, Eq. "ppr")."""

import numpy as np
import pytest

from oracle.damf import DamfOracle
from oracle.graph import DynGraph
from oracle.ppr import (graph_change_fixup, ppr_matrix_dense, ppr_power_iteration, ppr_series_dense,
                        push)
from tests.helpers import csr_of_dense, random_graph_dense


def _graph_with_dangling(rng, n, directed):
    A = random_graph_dense(n, 0.08, rng, directed=directed)
    A[3, :] = 0.0          # node 3 has no out-edge (dangling) ...
    if not directed:
        A[:, 3] = 0.0      # ... and in the undirected case it is isolated
    return A


@pytest.mark.parametrize("directed", [False, True])
def test_closed_form_equals_literal_series(directed):
    rng = np.random.default_rng(2)
    A = _graph_with_dangling(rng, 40, directed)
    X = rng.standard_normal((40, 3))
    alpha = 0.15
    Z_closed = ppr_matrix_dense(A, alpha) @ X
    Z_series = ppr_series_dense(A, X, alpha, terms=400)   # (1-alpha)^400 ~ 5e-29
    np.testing.assert_allclose(Z_closed, Z_series, atol=1e-12)
    indptr, indices = csr_of_dense(A)
    np.testing.assert_allclose(ppr_power_iteration(indptr, indices, X, alpha), Z_closed, atol=1e-11)


def test_pi_is_row_stochastic_without_dangling_nodes():
    # a constant signal is a fixed point: Pi 1 = 1 when every node has an out-edge
    rng = np.random.default_rng(4)
    A = random_graph_dense(30, 0.2, rng)
    assert A.sum(axis=1).min() > 0
    Pi = ppr_matrix_dense(A, 0.3)
    np.testing.assert_allclose(Pi @ np.ones(30), np.ones(30), atol=1e-13)
    assert Pi.min() >= 0.0


@pytest.mark.parametrize("directed", [False, True])
def test_push_within_eps_of_exact(directed):
    rng = np.random.default_rng(8)
    A = _graph_with_dangling(rng, 60, directed)
    indptr, indices = csr_of_dense(A)
    g = DynGraph(indptr, indices, 60, directed=directed)
    X = rng.standard_normal((60, 4))
    eps, alpha = 1e-5, 0.15
    Z = np.zeros_like(X)
    r = X.copy()
    k = push(g, Z, r, alpha, eps)
    assert k > 0 and np.abs(r).max() <= eps
    exact = ppr_matrix_dense(A, alpha) @ X
    assert np.abs(Z - exact).max() <= eps * (1 + 1e-9)
    # invariant Pi X = Z + Pi r holds exactly (up to rounding)
    Pi = ppr_matrix_dense(A, alpha)
    np.testing.assert_allclose(Z + Pi @ r, exact, atol=1e-12)


@pytest.mark.parametrize("directed", [False, True])
def test_degree_scaled_push_bound(directed):
    # threshold eps * max(deg(u), 1): every residual ends below its own threshold, the
    # invariant Pi X = Z + Pi r still holds, so |Z - Pi X|[i] <= (Pi t)[i] with t the thresholds
    rng = np.random.default_rng(18)
    A = _graph_with_dangling(rng, 60, directed)
    indptr, indices = csr_of_dense(A)
    g = DynGraph(indptr, indices, 60, directed=directed)
    X = rng.standard_normal((60, 4))
    eps, alpha = 1e-4, 0.15
    Z = np.zeros_like(X)
    r = X.copy()
    k = push(g, Z, r, alpha, eps, degree_scaled=True)
    thr = eps * np.maximum(A.sum(axis=1), 1.0)
    assert k > 0 and np.all(np.abs(r).max(axis=1) <= thr)
    assert np.any(np.abs(r).max(axis=1) > eps)          # the scaled threshold was used somewhere
    Pi = ppr_matrix_dense(A, alpha)
    np.testing.assert_allclose(Z + Pi @ r, Pi @ X, atol=1e-12)
    assert np.all(np.abs(Z - Pi @ X).max(axis=1) <= (Pi @ thr) * (1 + 1e-9))


def test_degree_scaled_push_is_absolute_push_at_constant_out_degree():
    # every node has out-degree 2 (in-degrees vary): the scaled push with eps / 2 takes the same
    # decisions in the same order as the absolute push with eps, so the results are identical
    rng = np.random.default_rng(19)
    n = 40
    A = np.zeros((n, n))
    for u in range(n):
        A[u, rng.choice([v for v in range(n) if v != u], size=2, replace=False)] = 1.0
    assert len(set(A.sum(axis=0))) > 1
    indptr, indices = csr_of_dense(A)
    X = rng.standard_normal((n, 3))
    out = []
    for eps, scaled in ((1e-5, False), (0.5e-5, True)):
        g = DynGraph(indptr, indices, n, directed=True)
        Z, r = np.zeros_like(X), X.copy()
        k = push(g, Z, r, 0.2, eps, degree_scaled=scaled)
        out.append((k, Z, r))
    assert out[0][0] == out[1][0]
    np.testing.assert_array_equal(out[0][1], out[1][1])
    np.testing.assert_array_equal(out[0][2], out[1][2])


def test_alpha_one_gives_identity():
    # the paper's ablation (Sec. 5.6): alpha = 1 means no enhancement, Z = X exactly
    rng = np.random.default_rng(9)
    A = random_graph_dense(25, 0.2, rng)
    indptr, indices = csr_of_dense(A)
    g = DynGraph(indptr, indices, 25)
    X = rng.standard_normal((25, 3))
    Z = np.zeros_like(X)
    r = X.copy()
    push(g, Z, r, 1.0, 1e-9)
    assert np.array_equal(Z, X)


@pytest.mark.parametrize("directed", [False, True])
def test_graph_change_fixup_keeps_invariant(directed):
    rng = np.random.default_rng(12)
    n = 45
    A = _graph_with_dangling(rng, n, directed)
    indptr, indices = csr_of_dense(A)
    g = DynGraph(indptr, indices, n, directed=directed)
    X = rng.standard_normal((n, 3))
    alpha = 0.2
    Z, r = np.zeros_like(X), X.copy()
    push(g, Z, r, alpha, 1e-3)
    # a change touching the dangling node 3 and some deletions
    src = np.array([3, 0, 5, 7], np.int32)
    dst = np.array([9, 1, 6, 8], np.int32)
    op = np.array([1, -1, 1, -1], np.int8)
    touched = set(src.tolist()) | (set() if directed else set(dst.tolist()))
    old = {u: g.out.row(u) for u in touched}
    ch = g.apply(src, dst, op)
    new = {int(u): g.out.row(int(u)) for u in ch.S}
    graph_change_fixup(r, Z, {int(u): old[int(u)] for u in ch.S}, new, alpha)
    indptr2, indices2 = g.out.csr()
    A2 = np.zeros((n, n))
    for u in range(n):
        A2[u, indices2[indptr2[u]:indptr2[u + 1]]] = 1.0
    np.testing.assert_array_equal(A2 - A, ch.dense(n))
    Pi2 = ppr_matrix_dense(A2, alpha)
    np.testing.assert_allclose(Z + Pi2 @ r, Pi2 @ X, atol=1e-12)


def test_dynamic_enhancement_bound_after_updates():
    rng = np.random.default_rng(14)
    n0, d = 50, 5
    A = random_graph_dense(n0, 0.12, rng)
    indptr, indices = csr_of_dense(A)
    eps = 1e-6
    orc = DamfOracle(indptr, indices, d, alpha=0.15, eps=eps, n_cap=n0 + 5, exact_init=True)
    for step in range(6):
        src = rng.integers(0, orc.n, 4).astype(np.int32)
        dst = rng.integers(0, orc.n, 4).astype(np.int32)
        keep = src != dst
        orc.apply_edges(src[keep], dst[keep], np.ones(keep.sum(), np.int8))
        orc.ppr_refresh()
        indptr2, indices2 = orc.graph.out.csr()
        An = np.zeros((orc.n, orc.n))
        for u in range(orc.n):
            An[u, indices2[indptr2[u]:indptr2[u + 1]]] = 1.0
        exact = ppr_matrix_dense(An, 0.15) @ orc.Xb[: orc.n]
        assert np.abs(orc.Zb[: orc.n] - exact).max() <= eps * (1 + 1e-8)
