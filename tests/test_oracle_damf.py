"""Pins for the oracle's incremental update (Algorithms 1-2) against Theorem 2.

Theorem 2 (Sec. 4.3) states that after an update the embedding is exactly the rank-d
t-SVD embedding of (previous low-rank product + dA).  The brute force computes that
definition with a dense SVD of the n x n matrix, independently of the incremental
formulas, so a dropped term, a wrong sign or a transposed factor in the oracle fails
these tests.
"""

import numpy as np
import pytest

from oracle.damf import DamfOracle
from oracle.tsvd import brute_force_update
from tests.helpers import csr_of_dense, random_graph_dense, rel_fro


def _random_events(rng, n, k, directed, p_del=0.3):
    src, dst, op = [], [], []
    while len(src) < k:
        u, v = rng.integers(0, n, size=2)
        if u == v:
            continue
        src.append(u), dst.append(v), op.append(-1 if rng.random() < p_del else 1)
    return np.array(src, np.int32), np.array(dst, np.int32), np.array(op, np.int8)


def _gap_ok(A_dense, d):
    s = np.linalg.svd(A_dense, compute_uv=False)
    return (s[d - 1] - s[d]) / s[0] > 1e-6


@pytest.mark.parametrize("directed", [False, True])
def test_incremental_update_equals_brute_force(directed):
    rng = np.random.default_rng(11 if directed else 7)
    n0, d = 40, 6
    A = random_graph_dense(n0, 0.15, rng, directed=directed)
    indptr, indices = csr_of_dense(A)
    orc = DamfOracle(indptr, indices, d, alpha=0.15, eps=1e-4, n_cap=n0 + 20, directed=directed,
                     exact_init=True, propagate=False)
    checked = 0
    for step in range(25):
        new_nodes = 1 if step % 5 == 2 else 0
        n_before = orc.n
        X1 = np.zeros((n_before + new_nodes, d))
        Y1 = np.zeros((n_before + new_nodes, d))
        X1[:n_before], Y1[:n_before] = orc.X(), orc.Y()
        src, dst, op = _random_events(rng, n_before + new_nodes, int(rng.integers(1, 6)), directed)
        if new_nodes:  # connect the arriving node
            src[0] = n_before
            dst[0] = int(rng.integers(0, n_before))
            op[0] = 1
        Xb_before = orc.Xb.copy()
        (ch,) = orc.apply_edges(src, dst, op, new_nodes)
        if ch.empty:
            continue
        dA = ch.dense(orc.n)
        target = X1 @ Y1.T + dA
        if not _gap_ok(target, d):
            continue
        X2, Y2, s2 = brute_force_update(X1, Y1, dA, d)
        np.testing.assert_allclose(orc.sigma, s2, rtol=1e-10, atol=1e-12)
        assert rel_fro(orc.X() @ orc.Y().T, X2 @ Y2.T) < 1e-10
        # orthonormal effective bases: U = X Sigma^{-1/2}
        U = orc.X() / np.sqrt(orc.sigma)
        V = orc.Y() / np.sqrt(orc.sigma)
        np.testing.assert_allclose(U.T @ U, np.eye(d), atol=1e-10)
        np.testing.assert_allclose(V.T @ V, np.eye(d), atol=1e-10)
        # Lemma 1 / Eq. "update": base rows outside S are not rewritten
        untouched = np.setdiff1d(np.arange(orc.n), ch.S)
        assert np.array_equal(orc.Xb[untouched], Xb_before[untouched])
        checked += 1
    assert checked >= 10


def test_noop_update_leaves_state_unchanged():
    rng = np.random.default_rng(5)
    A = random_graph_dense(30, 0.2, rng)
    indptr, indices = csr_of_dense(A)
    orc = DamfOracle(indptr, indices, 5, alpha=0.2, eps=1e-4, exact_init=True, propagate=False)
    u, v = np.argwhere(A > 0)[0]
    state = (orc.Xb.copy(), orc.PX.copy(), orc.sigma.copy())
    # inserting an existing edge and deleting an absent one are no-ops (set semantics)
    w = next(int(x) for x in np.nonzero(A[u] == 0)[0] if x != u)
    (ch,) = orc.apply_edges(np.array([u, u], np.int32), np.array([v, w], np.int32), np.array([1, -1], np.int8))
    assert ch.empty
    assert np.array_equal(orc.Xb, state[0]) and np.array_equal(orc.PX, state[1])
    assert np.array_equal(orc.sigma, state[2])


def test_node_arrival_matches_theorem_1():
    # Thm 1: adding a column B to A~ gives the t-SVD of [A~, B].  With the node-arrival
    # reading (zero row and column appended, then edges), the directed update of the
    # column entries (u, new) must equal that definition on the first n columns.
    rng = np.random.default_rng(21)
    n0, d = 35, 5
    A = random_graph_dense(n0, 0.2, rng, directed=True)
    indptr, indices = csr_of_dense(A)
    orc = DamfOracle(indptr, indices, d, alpha=0.15, eps=1e-4, n_cap=n0 + 1, directed=True,
                     exact_init=True, propagate=False)
    X1, Y1 = orc.X(), orc.Y()
    rows = rng.choice(n0, size=4, replace=False)
    Bcol = np.zeros(n0)
    Bcol[rows] = 1.0
    (ch,) = orc.apply_edges(rows.astype(np.int32), np.full(4, n0, np.int32), np.ones(4, np.int8), 1)
    # Thm 1's target: t-SVD of [X1 Y1^T, B] (n0 x (n0+1))
    U, s, Vt = np.linalg.svd(np.hstack([X1 @ Y1.T, Bcol[:, None]]), full_matrices=False)
    np.testing.assert_allclose(orc.sigma, s[:d], rtol=1e-10)
    target = (U[:, :d] * s[:d]) @ Vt[:d]
    got = orc.X() @ orc.Y().T
    assert rel_fro(got[:n0, :], target) < 1e-10
    assert np.abs(got[n0, :]).max() < 1e-12          # the new row stays zero


def test_residual_factor_of_a_block_partly_in_the_span():
    # Prop. 1 for a block: the residual (I - U U^T) B factors as Q R with R^T R = B^T B - W^T W,
    # W = U^T B. Columns inside span(U) add nothing to the residual: two of three columns in the
    # span leave R with one row, all three in the span leave R empty (R_B = 0, the
    # rank-deficient branch), and the factor's pseudo-inverse inverts it on its row space.
    from oracle.damf import _sqrt_factor
    rng = np.random.default_rng(17)
    n, d = 60, 6
    U, _ = np.linalg.qr(rng.standard_normal((n, d)))
    inside = U @ rng.standard_normal((d, 2))
    outside = rng.standard_normal((n, 1))
    for B, rank in ((np.hstack([inside, outside]), 1), (np.hstack([inside, U[:, :1]]), 0),
                    (rng.standard_normal((n, 3)), 3)):
        W = U.T @ B
        R, Rp = _sqrt_factor(B.T @ B - W.T @ W)
        assert R.shape == (rank, B.shape[1]) and Rp.shape == (B.shape[1], rank)
        np.testing.assert_allclose(R.T @ R, B.T @ B - W.T @ W, atol=1e-10)
        np.testing.assert_allclose(R @ Rp, np.eye(rank), atol=1e-10)
        resid = B - U @ W
        if rank:
            Q = resid @ Rp                              # orthonormal residual directions
            np.testing.assert_allclose(Q.T @ Q, np.eye(rank), atol=1e-10)
            np.testing.assert_allclose(Q @ R, resid, atol=1e-10)
        else:
            assert np.abs(resid).max() < 1e-12
