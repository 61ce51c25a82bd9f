"""Oracle: truncated SVD, the brute-force update, and the randomized t-SVD (FP64).

Test infrastructure only.
"""

from __future__ import annotations

import numpy as np


def t_svd(A: np.ndarray, d: int):
    """Rank-d truncated SVD (Sec. 4.1, Eq. "ne"): U (n x d), sigma (d), V (m x d),
    singular values in non-increasing order.  A library SVD is the step."""
    U, s, Vt = np.linalg.svd(np.asarray(A, dtype=np.float64), full_matrices=False)
    return U[:, :d], s[:d], Vt[:d].T


def embedding_from_tsvd(U, s, V):
    """X = U sqrt(Sigma), Y = V sqrt(Sigma) (Sec. 4.1, Eq. "ne")."""
    r = np.sqrt(s)
    return U * r, V * r


def brute_force_update(X1: np.ndarray, Y1: np.ndarray, dA: np.ndarray, d: int):
    """The definition the update must reach (Thm 2, Eqs. "node_target1", "svd_edge_2"):
    the rank-d t-SVD embedding of X1 Y1^T + dA.  Returns (X2, Y2, sigma2)."""
    U, s, V = t_svd(X1 @ Y1.T + dA, d)
    X2, Y2 = embedding_from_tsvd(U, s, V)
    return X2, Y2, s


def _orth(Y: np.ndarray) -> np.ndarray:
    Q, _ = np.linalg.qr(Y)
    return Q


def randomized_tsvd(A, Omega: np.ndarray, d: int, power_iters: int):
    """Randomized t-SVD (Halko, Martinsson and Tropp 2011, randomized subspace
    iteration), the initial factorisation of Appendix A, Algorithm 3.

    A may be a dense array or a scipy.sparse matrix; Omega is the n x l Gaussian test
    matrix (l >= d), supplied by the caller.  Steps: Q = orth(A Omega); then
    power_iters times: Q' = orth(A^T Q), Q = orth(A Q'); finally the SVD of the small
    l x n matrix Q^T A gives U = Q U~, Sigma, V.  Returns (U, sigma, V), rank d."""
    Om = np.asarray(Omega, dtype=np.float64)
    Q = _orth(A @ Om)
    for _ in range(power_iters):
        Qt = _orth(A.T @ Q)
        Q = _orth(A @ Qt)
    Bt = A.T @ Q                        # (Q^T A)^T, n x l
    Ub, s, Vbt = np.linalg.svd(np.asarray(Bt).T, full_matrices=False)
    U = Q @ Ub[:, :d]
    V = Vbt[:d].T
    return U, s[:d], V

