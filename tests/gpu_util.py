"""Shared setup for the GPU parity tests: the same seeded inputs for both sides."""

import numpy as np

from synth import chung_lu_graph, gaussian_test_matrix


def make_pair(n, avg_deg, gamma, d, alpha, eps, seed, n_extra=64, directed=False, oracle=True, propagate=True,
              refold_every=0, power_iters=4, threshold="absolute"):
    from oracle.damf import DamfOracle
    from paper_2306_08967_gb300 import DamfGraph, make_config, rsvd_width
    indptr, indices, w = chung_lu_graph(n, avg_deg, gamma, seed=seed, directed=directed)
    cfg = make_config(n, d, alpha, eps, n_capacity=n + n_extra, nnz=len(indices), directed=directed,
                      refold_every=refold_every, rsvd_power_iters=power_iters, threshold=threshold)
    om = gaussian_test_matrix(n, rsvd_width(cfg), seed=seed + 2)
    g = DamfGraph(indptr, indices, cfg, om)
    orc = None
    if oracle:
        orc = DamfOracle(indptr, indices, d, alpha, eps, n_cap=n + n_extra, directed=directed, Omega=om,
                         power_iters=power_iters, propagate=propagate, degree_scaled=threshold == "degree")
    return g, orc, (indptr, indices, w)


def dense_adj(rp, col, n):
    A = np.zeros((n, n))
    for u in range(n):
        A[u, col[rp[u]:rp[u + 1]]] = 1.0
    return A


def gpu_xy(g):
    e = g.embeddings()
    return e["X"].double().cpu().numpy(), e["Y"].double().cpu().numpy(), e["sigma"].double().cpu().numpy()


def rel_fro(A, B):
    return float(np.linalg.norm(A - B) / max(np.linalg.norm(B), 1e-300))
