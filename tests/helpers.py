"""Small shared test helpers (no method arithmetic)."""

import os

import numpy as np

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_closed_form_spectra():
    out = []
    with open(os.path.join(GOLDEN, "closed_form_spectra.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, edges, sv = [x.strip() for x in line.split("|")]
            pairs = [tuple(int(t) for t in e.split("-")) for e in edges.split()]
            out.append((name, pairs, np.array([float(x) for x in sv.split()])))
    return out


def dense_from_pairs(pairs, n=None):
    n = n or (max(max(p) for p in pairs) + 1)
    A = np.zeros((n, n))
    for u, v in pairs:
        A[u, v] = A[v, u] = 1.0
    return A


def csr_of_dense(A):
    n = A.shape[0]
    indptr = [0]
    indices = []
    for u in range(n):
        nz = np.nonzero(A[u])[0]
        indices.extend(nz.tolist())
        indptr.append(len(indices))
    return np.array(indptr, dtype=np.int32), np.array(indices, dtype=np.int32)


def random_graph_dense(n, p, rng, directed=False):
    A = (rng.random((n, n)) < p).astype(np.float64)
    np.fill_diagonal(A, 0.0)
    if not directed:
        A = np.triu(A, 1)
        A = A + A.T
    return A


def rel_fro(A, B):
    return np.linalg.norm(A - B) / max(np.linalg.norm(B), 1e-300)
