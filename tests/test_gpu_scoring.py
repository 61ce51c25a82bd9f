"""Link-prediction scores and top-k (Sec. 5) through the C ABI against the FP64 scoring oracle.

The oracle scores the embeddings the library itself returns (damf_get_embeddings), so the
check isolates the scoring kernels, which work from the base state through G = PU Sigma PV^T.
Tolerance: FP32 sums over d products, |score error| <= 2e-5 |C[u]| |Y[v]| (plus the same
for the other direction when symmetric).
"""

import numpy as np
import pytest

from oracle.scoring import link_scores, score_rows, top_k
from tests.gpu_util import make_pair

pytestmark = pytest.mark.gpu

SEED = 0xDA3F0000 + 300


def _events(rng, n, k):
    src, dst = [], []
    while len(src) < k:
        u, v = rng.integers(0, n, 2)
        if u != v:
            src.append(u), dst.append(v)
    return np.array(src, np.int32), np.array(dst, np.int32), np.ones(k, np.int8)


def _graph(n, d, directed, seed):
    g, _, _ = make_pair(n, 8.0, 2.5, d, 0.15, 1e-5, seed, directed=directed, oracle=False)
    rng = np.random.default_rng(seed)
    for _ in range(3):
        g.apply_edges(*_events(rng, n, 12))
        g.ppr_refresh()
    g.check()
    e = g.embeddings()
    return g, {k: e[k].double().cpu().numpy() for k in ("X", "Y", "Z")}


def _tol(C, Y, u, v, sym):
    t = 2e-5 * np.linalg.norm(C[u], axis=-1) * np.linalg.norm(Y[v], axis=-1)
    if sym:
        t = t + 2e-5 * np.linalg.norm(C[v], axis=-1) * np.linalg.norm(Y[u], axis=-1)
    return t + 1e-7


@pytest.mark.parametrize("d,directed", [(16, False), (64, True), (128, False)])
def test_score_pairs_match_oracle(d, directed):
    n = 700
    g, E = _graph(n, d, directed, SEED + d)
    rng = np.random.default_rng(5)
    src = rng.integers(0, n, 3001).astype(np.int32)       # ragged count, duplicates, u == v pairs
    dst = rng.integers(0, n, 3001).astype(np.int32)
    dst[:7] = src[:7]
    for context in ("Z", "X"):
        for sym in (False, True):
            got = g.score_pairs(src, dst, context=context, symmetric=sym).double().cpu().numpy()
            want = link_scores(E[context], E["Y"], src, dst, sym)
            assert np.all(np.abs(got - want) <= _tol(E[context], E["Y"], src, dst, sym))
    assert g.score_pairs(src[:0], dst[:0]).numel() == 0
    g.check()
    g.close()


@pytest.mark.parametrize("d,k,directed", [(16, 10, False), (64, 64, True), (128, 17, False)])
def test_topk_is_a_valid_top_k(d, k, directed):
    n = 900
    g, E = _graph(n, d, directed, SEED + 10 + d)
    rng = np.random.default_rng(6)
    rows = rng.integers(0, n, 37).astype(np.int32)        # two passes of 32 queries, ragged
    rows[1] = rows[0]                                      # a repeated query
    for context in ("Z", "X"):
        sym = not directed
        ids, sc = g.topk(rows, k, context=context, symmetric=sym)
        ids, sc = ids.cpu().numpy(), sc.double().cpu().numpy()
        S = score_rows(E[context], E["Y"], rows, sym)
        want_ids, want_sc = top_k(E[context], E["Y"], rows, k, sym)
        for i, u in enumerate(rows):
            tol = float(_tol(E[context], E["Y"], np.full(n, u), np.arange(n), sym).max())
            got = ids[i]
            assert len(set(got.tolist())) == k and u not in got and got.min() >= 0
            assert np.all(np.diff(sc[i]) <= 0)                               # decreasing
            np.testing.assert_allclose(sc[i], S[i, got], atol=tol)           # the right scores
            kth = want_sc[i, -1]
            assert sc[i, -1] >= kth - 2 * tol                                 # nothing better left out
            must = np.where(S[i] > kth + 2 * tol)[0]
            assert set(must.tolist()) <= set(got.tolist())
            # away from near-ties the order is unique and must match exactly
            gaps = np.diff(want_sc[i])
            clear = np.ones(k, bool)
            clear[1:] &= np.abs(gaps) > 2 * tol
            clear[:-1] &= np.abs(gaps) > 2 * tol
            assert np.array_equal(got[clear], want_ids[i][clear])
        np.testing.assert_array_equal(ids[0], ids[1])
    g.close()


def test_topk_pads_when_fewer_candidates_than_k():
    n = 40
    g, E = _graph(n, 16, False, SEED + 50)
    ids, sc = g.topk(np.array([3, 39], np.int32), 64)
    ids, sc = ids.cpu().numpy(), sc.cpu().numpy()
    for i, u in enumerate((3, 39)):
        assert sorted(ids[i, : n - 1].tolist()) == [v for v in range(n) if v != u]
        assert (ids[i, n - 1:] == -1).all() and np.isneginf(sc[i, n - 1:]).all()
    from paper_2306_08967_gb300 import DamfError
    with pytest.raises(DamfError):
        g.topk(np.array([0], np.int32), 65)
    g.check()                                   # a rejected argument leaves the context usable
    assert g.topk(np.array([0], np.int32), 5)[0].shape == (1, 5)
    g.close()
