"""Oracle: incremental DAMF in the paper's own X-form, FP64 (Secs. 4.1-4.5, Algs. 1-3).

Test infrastructure only.

State (Algorithm 2 inputs): base embeddings X_b, Y_b (n x d), accumulated space
projections P_X, P_Y (d x d) and their inverses, singular values Sigma, the enhanced
embedding Z_b and the PPR residual r (n x d) in base space, and the graph.

One update with net change dA = B C^T follows Algorithm 1 ("UpdateEmbeddingE"),
generalised from rank one to rank rho:
  Step 1  U = X_b P_X Sigma^{-1/2}, V = Y_b P_Y Sigma^{-1/2} (only rows of B, C);
          W_B = U^T B, W_C = V^T C; the residual (I - U U^T) B = Q_B R_B where
          R_B^T R_B = B^T B - W_B^T W_B (Prop. 1 for a block of columns), same for C.
  Step 2  M = [[Sigma, 0], [0, 0]] + [W_B; R_B] [W_C; R_C]^T, E Theta H^T = t-SVD(M, d)
          (Eq. "svd_small_edge").
  Step 3  F = Sigma^{-1/2} (E[:d] - W_B R_B^+ E[d:]) Theta^{1/2}            (Eq. "f_edge")
          G = Sigma^{-1/2} (H[:d] - W_C R_C^+ H[d:]) Theta^{1/2}            (Eq. "g_edge")
          dX = B R_B^+ E[d:] Theta^{1/2},  dY = C R_C^+ H[d:] Theta^{1/2}   (Eqs. "x_edge", "y_edge")
          P_X <- P_X F, X_b <- X_b + dX P_X^{-1} (new P_X), same for Y      (Eq. "update")
  Step 4  PPR: the base-signal change dX P_X^{-1} and the graph change enter r, then push.

R_B is a square-root factor of the residual Gram (eigen-decomposition based, rank
revealing; R^+ its pseudo-inverse), which equals the paper's scalar R_B = sqrt(|B|^2 -
|W_B|^2) for one column.  B and C come from the thin SVD of the small net-change
matrix N (dA = I_S N I_T^T): B = I_S P_N diag(nu), C = I_T Q_N, so rho = rank(N).
Node arrival: zero rows are appended (the padding of Sec. 4.2 reduced to edges).
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .graph import DynGraph, split_updates
from .ppr import graph_change_fixup, push
from .tsvd import randomized_tsvd, t_svd


def _sqrt_factor(G: np.ndarray, tol: float = 1e-12):
    """R with R^T R = G (R has full row rank) and its pseudo-inverse R^+ (R R^+ = I)."""
    G = 0.5 * (G + G.T)
    lam, Q = np.linalg.eigh(G)
    scale = max(float(np.max(np.abs(lam))) if lam.size else 0.0, 1.0)
    keep = lam > tol * scale
    lam, Q = lam[keep], Q[:, keep]
    R = np.sqrt(lam)[:, None] * Q.T
    Rp = Q / np.sqrt(lam)[None, :]
    return R, Rp


class DamfOracle:
    def __init__(self, indptr, indices, d: int, alpha: float, eps: float, n_cap: int = None,
                 directed: bool = False, Omega: np.ndarray = None, power_iters: int = 4,
                 exact_init: bool = False, propagate: bool = True, degree_scaled: bool = False,
                 edges_per_update: int = 64):
        """edges_per_update: a call's events are applied as consecutive updates of at most this
        many events each (the batched reading of Algorithm 2: one rank-r update per group of
        events; 1 gives the paper's one event per update)."""
        n = int(len(indptr) - 1)
        self.edges_per_update = int(edges_per_update)
        self.stats_updates = 0          # non-empty updates applied
        self.last_core_sv = None        # full spectrum of the most recent update's core M
        n_cap = n if n_cap is None else n_cap
        self.d, self.alpha, self.eps, self.directed = d, alpha, eps, directed
        self.degree_scaled = degree_scaled
        self.graph = DynGraph(indptr, indices, n_cap, directed=directed)
        A = sp.csr_matrix((np.ones(len(indices)), np.asarray(indices, dtype=np.int64),
                           np.asarray(indptr, dtype=np.int64)), shape=(n, n))
        # Algorithm 3, line 1: t-SVD of the initial adjacency matrix
        if exact_init:
            U, s, V = t_svd(A.toarray(), d)
        else:
            U, s, V = randomized_tsvd(A, Omega[:n], d, power_iters)
        # line 2-4
        self.Xb = np.zeros((n_cap, d))
        self.Yb = np.zeros((n_cap, d))
        self.Xb[:n] = U * np.sqrt(s)
        self.Yb[:n] = V * np.sqrt(s)
        self.sigma = s.copy()
        self.PX = np.eye(d)
        self.PY = np.eye(d)
        self.PXi = np.eye(d)
        self.PYi = np.eye(d)
        self.r = self.Xb.copy()
        self.Zb = np.zeros((n_cap, d))
        self.pushes = 0
        # line 5: propagation
        if propagate:
            self.pushes += push(self.graph, self.Zb, self.r, alpha, eps, degree_scaled=degree_scaled)

    @property
    def n(self) -> int:
        return self.graph.n

    # ---- queries (Sec. 4.6, "Time Complexity of Query Node's Embedding") ----
    def X(self):
        return self.Xb[: self.n] @ self.PX

    def Y(self):
        return self.Yb[: self.n] @ self.PY

    def Z(self):
        return self.Zb[: self.n] @ self.PX

    # ---- Algorithm 2 ----
    def apply_edges(self, src, dst, op, new_nodes: int = 0):
        src, dst, op = np.asarray(src), np.asarray(dst), np.asarray(op)
        self.graph.validate(src, dst, op, new_nodes)
        self.graph.add_nodes(new_nodes)
        changes = []
        for lo, hi in split_updates(len(src), self.edges_per_update):
            changes.append(self.apply_update(src[lo:hi], dst[lo:hi], op[lo:hi]))
        return changes

    def apply_update(self, src, dst, op):
        """One update: graph edit, Steps 1-3, and the PPR residual changes of Step 4."""
        touched = set(np.asarray(src).tolist())
        if not self.directed:
            touched |= set(np.asarray(dst).tolist())
        rows_old = {u: self.graph.out.row(u) for u in touched}
        ch = self.graph.apply(src, dst, op)
        if ch.empty:
            self.last_core_sv = None
            return ch
        self.stats_updates += 1
        rows_new = {int(u): self.graph.out.row(int(u)) for u in ch.S}
        rows_old = {int(u): rows_old[int(u)] for u in ch.S}
        dXb_S = self._factor_update(ch)
        self.r[ch.S] += dXb_S
        graph_change_fixup(self.r, self.Zb, rows_old, rows_new, self.alpha)
        return ch

    def _factor_update(self, ch):
        d, S, T = self.d, ch.S, ch.T
        sig = self.sigma
        Pn, nu, Qnt = np.linalg.svd(ch.N, full_matrices=False)
        keep = nu > 1e-12 * nu.max()
        B_S = Pn[:, keep] * nu[keep]          # rows S of B
        C_T = Qnt[keep].T                     # rows T of C
        # Step 1: orthogonalization
        isq = 1.0 / np.sqrt(sig)
        U_S = (self.Xb[S] @ self.PX) * isq
        V_T = (self.Yb[T] @ self.PY) * isq
        W_B = U_S.T @ B_S
        W_C = V_T.T @ C_T
        R_B, R_Bp = _sqrt_factor(B_S.T @ B_S - W_B.T @ W_B)
        R_C, R_Cp = _sqrt_factor(C_T.T @ C_T - W_C.T @ W_C)
        # Step 2: rediagonalization
        kb, kc = R_B.shape[0], R_C.shape[0]
        M = np.zeros((d + kb, d + kc))
        M[:d, :d] = np.diag(sig)
        M += np.vstack([W_B, R_B]) @ np.vstack([W_C, R_C]).T
        E, theta, Ht = np.linalg.svd(M, full_matrices=False)
        self.last_core_sv = theta.copy()
        E, theta, H = E[:, :d], theta[:d], Ht[:d].T
        # Step 3: space projection
        sq2 = np.sqrt(theta)
        RBE = R_Bp @ E[d:]
        RCH = R_Cp @ H[d:]
        F = (isq[:, None] * (E[:d] - W_B @ RBE)) * sq2[None, :]
        G = (isq[:, None] * (H[:d] - W_C @ RCH)) * sq2[None, :]
        dX_S = (B_S @ RBE) * sq2[None, :]
        dY_T = (C_T @ RCH) * sq2[None, :]
        self.PX = self.PX @ F
        self.PY = self.PY @ G
        self.PXi = np.linalg.solve(F, self.PXi)
        self.PYi = np.linalg.solve(G, self.PYi)
        dXb_S = dX_S @ self.PXi
        dYb_T = dY_T @ self.PYi
        self.Xb[S] += dXb_S
        self.Yb[T] += dYb_T
        self.sigma = theta
        return dXb_S

    def ppr_refresh(self, max_pushes: int = 1 << 40) -> int:
        k = push(self.graph, self.Zb, self.r, self.alpha, self.eps, max_pushes, self.degree_scaled)
        self.pushes += k
        return k
