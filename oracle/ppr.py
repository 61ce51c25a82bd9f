"""Oracle: Personalized PageRank of an n x d signal (Sec. 4.4, Eq. "ppr"), FP64.

Test infrastructure only.

PPR(X) = sum_{i>=0} alpha (1-alpha)^i (D^{-1} A)^i X, D the diagonal out-degree matrix.
With P = D^{-1} A (a node with no out-edge has a zero row of P) the series sums to
Pi X with Pi = alpha (I - (1-alpha) P)^{-1}.

The dynamic enhancement (Sec. 4.4, Step 4 of Sec. 4.5) keeps (Z_b, r) with the
invariant Pi X_b = Z_b + Pi r.  Three operations keep it:
  * signal change  X_b += dX_b            ->  r += dX_b
  * graph change   P -> P'                ->  r += ((1-alpha)/alpha) (P' - P) Z_b
    (from r = X_b - Pi^{-1} Z_b and Pi^{-1} = (I - (1-alpha) P) / alpha; only the
    rows u whose out-row changed are touched)
  * push (oracle/c/oracle_graph.c) until max |r| <= eps, giving |Z_b - Pi X_b| <= eps.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .graph import DynGraph, _load, _ptr


def transition_dense(A: np.ndarray) -> np.ndarray:
    """P = D^{-1} A with zero rows for nodes without out-edges."""
    deg = A.sum(axis=1)
    P = np.zeros_like(A, dtype=np.float64)
    nz = deg > 0
    P[nz] = A[nz] / deg[nz, None]
    return P


def ppr_matrix_dense(A: np.ndarray, alpha: float) -> np.ndarray:
    """Pi = alpha (I - (1-alpha) D^{-1} A)^{-1}, by a dense solve."""
    n = A.shape[0]
    P = transition_dense(A)
    return alpha * np.linalg.solve(np.eye(n) - (1.0 - alpha) * P, np.eye(n))


def ppr_series_dense(A: np.ndarray, X: np.ndarray, alpha: float, terms: int) -> np.ndarray:
    """Eq. "ppr" summed literally for `terms` terms."""
    P = transition_dense(A)
    out = np.zeros_like(X, dtype=np.float64)
    T = np.array(X, dtype=np.float64)
    for i in range(terms):
        out += alpha * (1.0 - alpha) ** i * T
        T = P @ T
    return out


def transition_sparse(indptr, indices, n: int) -> sp.csr_matrix:
    indptr = np.asarray(indptr, dtype=np.int64)
    indices = np.asarray(indices, dtype=np.int64)
    deg = np.diff(indptr).astype(np.float64)
    vals = np.repeat(np.where(deg > 0, 1.0 / np.maximum(deg, 1.0), 0.0), np.diff(indptr))
    return sp.csr_matrix((vals, indices, indptr), shape=(n, n))


def ppr_power_iteration(indptr, indices, X: np.ndarray, alpha: float, tol: float = 1e-13,
                        max_iter: int = 10000) -> np.ndarray:
    """Z = Pi X as the fixed point of Z = alpha X + (1-alpha) P Z, iterated until the
    max-norm change is below tol."""
    n = X.shape[0]
    P = transition_sparse(indptr, indices, n)
    X = np.asarray(X, dtype=np.float64)
    Z = alpha * X
    for _ in range(max_iter):
        Zn = alpha * X + (1.0 - alpha) * (P @ Z)
        if np.max(np.abs(Zn - Z)) < tol:
            return Zn
        Z = Zn
    return Z


def graph_change_fixup(r: np.ndarray, Z: np.ndarray, rows_old: dict, rows_new: dict, alpha: float):
    """r[u] += ((1-alpha)/alpha) (P'[u] - P[u]) Z for each u in rows_old/rows_new
    (dicts node -> neighbour array before/after the change)."""
    c = (1.0 - alpha) / alpha
    for u in rows_new:
        old = rows_old[u]
        new = rows_new[u]
        p_new = Z[new].sum(axis=0) / len(new) if len(new) else 0.0
        p_old = Z[old].sum(axis=0) / len(old) if len(old) else 0.0
        r[u] += c * (p_new - p_old)


def push(graph: DynGraph, Z: np.ndarray, r: np.ndarray, alpha: float, eps: float,
         max_pushes: int = 1 << 40, degree_scaled: bool = False) -> int:
    """Sequential FIFO push in place (plain C); returns the number of pushes.

    Node u is pushed while max_j |r[u][j]| exceeds its threshold: eps, or with degree_scaled
    eps * max(deg(u), 1) with deg the out-degree (the degree factor c in the push cost of
    Sec. 4.5, as in the push of InstantGNN that the paper builds on).
    """
    assert Z.dtype == np.float64 and r.dtype == np.float64
    assert Z.flags.c_contiguous and r.flags.c_contiguous
    assert Z.shape[0] >= graph.n and r.shape[0] >= graph.n
    lib = _load()
    d = Z.shape[1]
    k = lib.og_push(graph.inn.h, graph.out.h, d, _ptr(Z), _ptr(r), alpha, eps, max_pushes, int(degree_scaled))
    if k < 0:
        raise RuntimeError("push did not converge within max_pushes")
    return int(k)
