"""Pins for the oracle's graph store: set semantics against an independent dense replay."""

import numpy as np
import pytest

from oracle.graph import DynGraph, split_updates
from tests.helpers import csr_of_dense, random_graph_dense


@pytest.mark.parametrize("directed", [False, True])
def test_set_semantics_against_dense_replay(directed):
    rng = np.random.default_rng(31)
    n = 30
    A = random_graph_dense(n, 0.1, rng, directed=directed)
    indptr, indices = csr_of_dense(A)
    g = DynGraph(indptr, indices, n, directed=directed)
    ref = A.copy()
    for _ in range(40):
        k = int(rng.integers(1, 12))
        src = rng.integers(0, n, k).astype(np.int32)
        dst = rng.integers(0, n, k).astype(np.int32)
        keep = src != dst
        src, dst = src[keep], dst[keep]
        op = np.where(rng.random(len(src)) < 0.4, -1, 1).astype(np.int8)
        before = ref.copy()
        for u, v, o in zip(src, dst, op):      # event-by-event replay
            ref[u, v] = 1.0 if o == 1 else 0.0
            if not directed:
                ref[v, u] = ref[u, v]
        ch = g.apply(src, dst, op)
        np.testing.assert_array_equal(ch.dense(n), ref - before)
        # touched sets: non-zero rows / columns of dA (Lemma 1's row set)
        dA = ref - before
        assert ch.S.tolist() == np.nonzero(np.abs(dA).sum(axis=1))[0].tolist()
        assert ch.T.tolist() == np.nonzero(np.abs(dA).sum(axis=0))[0].tolist()
        ip, ix = g.out.csr()
        got = np.zeros((n, n))
        for u in range(n):
            got[u, ix[ip[u]:ip[u + 1]]] = 1.0
        np.testing.assert_array_equal(got, ref)
        if directed:
            ip, ix = g.inn.csr()
            gin = np.zeros((n, n))
            for u in range(n):
                gin[u, ix[ip[u]:ip[u + 1]]] = 1.0
            np.testing.assert_array_equal(gin, ref.T)


def test_validation_rejects_bad_events():
    g = DynGraph(np.array([0, 1, 2], np.int32), np.array([1, 0], np.int32), 4)
    with pytest.raises(ValueError):
        g.validate(np.array([0], np.int32), np.array([0], np.int32), np.array([1], np.int8), 0)
    with pytest.raises(ValueError):
        g.validate(np.array([0], np.int32), np.array([2], np.int32), np.array([1], np.int8), 0)
    g.validate(np.array([0], np.int32), np.array([2], np.int32), np.array([1], np.int8), 1)
    with pytest.raises(ValueError):
        g.validate(np.array([0], np.int32), np.array([1], np.int32), np.array([0], np.int8), 0)


def test_split_updates():
    assert split_updates(0, 64) == []
    assert split_updates(5, 64) == [(0, 5)]
    assert split_updates(64, 64) == [(0, 64)]
    assert split_updates(65, 64) == [(0, 64), (64, 65)]
    assert split_updates(3, 1) == [(0, 1), (1, 2), (2, 3)]
    with pytest.raises(ValueError):
        split_updates(3, 0)
