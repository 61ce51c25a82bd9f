"""Pins for the oracle's link-prediction scores and top-k ranking (Sec. 5)."""

import numpy as np
import pytest

from oracle.scoring import link_scores, score_rows, top_k
from oracle.tsvd import embedding_from_tsvd, t_svd


def test_scores_equal_explicit_sums():
    rng = np.random.default_rng(31)
    C, Y = rng.standard_normal((9, 4)), rng.standard_normal((9, 4))
    src, dst = [0, 3, 8, 5, 5], [1, 3, 2, 7, 0]
    for sym in (False, True):
        got = link_scores(C, Y, src, dst, sym)
        for i, (u, v) in enumerate(zip(src, dst)):
            a = sum(C[u][j] * Y[v][j] for j in range(4))
            b = sum(C[v][j] * Y[u][j] for j in range(4))
            assert got[i] == pytest.approx(max(a, b) if sym else a, abs=1e-14)


def test_top_k_equals_sorting_all_pairs():
    rng = np.random.default_rng(32)
    n = 12
    C, Y = rng.standard_normal((n, 3)), rng.standard_normal((n, 3))
    C[5] = C[4]                      # ties: nodes 4 and 5 score alike against every query
    Y[5] = Y[4]
    rows = [0, 4, 11]
    for sym in (False, True):
        ids, sc = top_k(C, Y, rows, 7, sym)
        for i, u in enumerate(rows):
            cand = []
            for v in range(n):
                if v == u:
                    continue
                s = float(C[u] @ Y[v])
                if sym:
                    s = max(s, float(C[v] @ Y[u]))
                cand.append((-s, v))
            cand.sort()
            assert [v for _, v in cand[:7]] == ids[i].tolist()
            np.testing.assert_allclose(sc[i], [-s for s, _ in cand[:7]], atol=1e-14)
    # more k than candidates: padded
    ids, sc = top_k(C, Y, [2], n + 3, False)
    assert (ids[0, n - 1:] == -1).all() and np.isneginf(sc[0, n - 1:]).all()
    assert sorted(ids[0, : n - 1].tolist()) == [v for v in range(n) if v != 2]


def test_symmetric_scores_are_symmetric():
    rng = np.random.default_rng(33)
    C, Y = rng.standard_normal((20, 5)), rng.standard_normal((20, 5))
    S = score_rows(C, Y, np.arange(20), True)
    off = ~np.eye(20, dtype=bool)
    np.testing.assert_array_equal(S[off], S.T[off])


def test_disjoint_cliques_closed_form():
    # cliques of sizes 5, 4, 3: the rank-3 t-SVD keeps each clique's Perron pair, sigma = k - 1,
    # u = v = 1/sqrt(k) on the clique, so X Y^T = (k - 1)/k inside clique k and 0 across
    sizes = [5, 4, 3]
    n = sum(sizes)
    A = np.zeros((n, n))
    o = 0
    label = []
    for i, k in enumerate(sizes):
        A[o:o + k, o:o + k] = 1.0 - np.eye(k)
        label += [i] * k
        o += k
    U, s, V = t_svd(A, 3)
    np.testing.assert_allclose(s, [4.0, 3.0, 2.0], atol=1e-12)
    X, Y = embedding_from_tsvd(U, s, V)
    S = score_rows(X, Y, np.arange(n), False)
    for u in range(n):
        for v in range(n):
            if u == v:
                continue
            want = (sizes[label[u]] - 1) / sizes[label[u]] if label[u] == label[v] else 0.0
            assert S[u, v] == pytest.approx(want, abs=1e-12)
    ids, sc = top_k(X, Y, [6], 4, True)     # node 6 is in the clique {5, 6, 7, 8}
    assert ids[0, :3].tolist() == [5, 7, 8]
    np.testing.assert_allclose(sc[0, :3], 0.75, atol=1e-12)
    assert abs(sc[0, 3]) < 1e-12                      # then a node of another clique (score 0)
