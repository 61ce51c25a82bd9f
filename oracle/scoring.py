"""Oracle: link-prediction scores and the top-k ranking (FP64).  Test infrastructure only.

Sec. 5 ("Link Prediction") and the appendix "Additional Details of Link Prediction": the
score of the node pair (u, v) is the inner product of u's context vector with v's content
vector; for an undirected graph both directions are scored and the larger one is kept.
Graph reconstruction (Sec. 5) ranks node pairs by that same score (precision@K).
The context vector is Z (the PPR-enhanced embedding) or X; the content vector is Y.
"""

from __future__ import annotations

import numpy as np


def link_scores(C: np.ndarray, Yc: np.ndarray, src, dst, symmetric: bool) -> np.ndarray:
    """score(u, v) = C[u] . Yc[v] for every pair (src[i], dst[i]); symmetric keeps
    max(score(u, v), score(v, u))."""
    C = np.asarray(C, dtype=np.float64)
    Yc = np.asarray(Yc, dtype=np.float64)
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    s = np.einsum("ij,ij->i", C[src], Yc[dst])
    if symmetric:
        s = np.maximum(s, np.einsum("ij,ij->i", C[dst], Yc[src]))
    return s


def score_rows(C: np.ndarray, Yc: np.ndarray, rows, symmetric: bool) -> np.ndarray:
    """Every node's score against each query u in rows (len(rows) x n), self-pairs at -inf."""
    C = np.asarray(C, dtype=np.float64)
    Yc = np.asarray(Yc, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    S = C[rows] @ Yc.T                       # score(u, v) for all v
    if symmetric:
        S = np.maximum(S, Yc[rows] @ C.T)    # score(v, u) = C[v] . Yc[u]
    S[np.arange(len(rows)), rows] = -np.inf
    return S


def top_k(C: np.ndarray, Yc: np.ndarray, rows, k: int, symmetric: bool):
    """The k nodes v != u of largest score(u, v) per query u, decreasing score, equal
    scores by increasing id; (ids, scores) of shape len(rows) x k, padded with -1 / -inf."""
    S = score_rows(C, Yc, rows, symmetric)
    n = S.shape[1]
    ids = np.full((len(S), k), -1, dtype=np.int64)
    sc = np.full((len(S), k), -np.inf)
    ar = np.arange(n)
    for i, row in enumerate(S):
        order = np.lexsort((ar, -row))       # primary: score descending; then id ascending
        order = order[np.isfinite(row[order])][:k]
        ids[i, : len(order)] = order
        sc[i, : len(order)] = row[order]
    return ids, sc
