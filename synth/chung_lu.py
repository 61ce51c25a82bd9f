"""Chung-Lu graphs, edge-event streams and Gaussian test matrices (seeded).

Recipe (stated once here; every caller uses it):

* weights  w_i = (i + i0)^(-1/(gamma-1)),  i = 0..n-1, scaled so that sum(w) = 2m,
  then capped at sqrt(sum(w)) (the Chung-Lu admissibility bound); node ids are
  randomly permuted so hubs are not clustered at low ids.
* edges    m endpoint pairs drawn independently with P(i) proportional to w_i;
  self-loops and duplicates are dropped (so the realised m is a little lower).
  Undirected graphs store both (u, v) and (v, u) in CSR.
* events   a batch first holds `nodes_per_batch` forced node arrivals, then k more
  edges, k ~ U[k_lo, k_hi], drawn event by event: with probability p_node a node arrival (a fresh node id,
  degree drawn from the weight law, min 1, clipped to the remaining budget,
  endpoints proportional to w among existing nodes), with probability p_del a
  deletion (an edge of the initial graph, drawn uniformly without replacement),
  otherwise an insertion (both endpoints proportional to w).  Insertions may hit
  an existing edge; under set semantics that is a no-op.
* RNG      numpy PCG64 seeded with 0xDA3F0000 + config index (graph) and
  seed + 1 (event stream), seed + 2 (Gaussian test matrix).
"""

from __future__ import annotations

import dataclasses
from typing import List

import numpy as np


def chung_lu_weights(n: int, m: int, gamma: float, i0: float = 1.0) -> np.ndarray:
    """Expected-degree weights of a Chung-Lu graph with power-law exponent gamma."""
    i = np.arange(n, dtype=np.float64)
    w = (i + i0) ** (-1.0 / (gamma - 1.0))
    w *= (2.0 * m) / w.sum()
    cap = np.sqrt(w.sum())
    return np.minimum(w, cap)


def csr_from_edges(n: int, src: np.ndarray, dst: np.ndarray):
    """CSR (indptr int32[n+1], indices int32[nnz]) of the given directed entries,
    rows sorted by column."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    order = np.argsort(src * max(n, 1) + dst, kind="stable")   # by (src, dst), as a lexicographic sort
    src, dst = src[order], dst[order]
    counts = np.bincount(src, minlength=n)
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=indptr[1:])
    return indptr.astype(np.int32), dst.astype(np.int32)


def _sorted_unique(key: np.ndarray) -> np.ndarray:
    """The distinct values of key in increasing order (np.unique's result, by one sort)."""
    key = np.sort(key)
    if key.shape[0] == 0:
        return key
    keep = np.empty(key.shape[0], dtype=bool)
    keep[0] = True
    np.not_equal(key[1:], key[:-1], out=keep[1:])
    return key[keep]


def chung_lu_graph(n: int, avg_deg: float, gamma: float, seed: int, directed: bool = False):
    """Seeded Chung-Lu graph.  Returns (indptr, indices, weights_by_node_id).

    avg_deg is the mean number of CSR entries per row (undirected: each edge counts
    in both rows, so m_undirected = n * avg_deg / 2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = int(round(n * avg_deg / (1 if directed else 2)))
    w = chung_lu_weights(n, m, gamma)
    perm = rng.permutation(n)          # node id of the i-th weight
    w_by_id = np.empty(n, dtype=np.float64)
    w_by_id[perm] = w
    p = w_by_id / w_by_id.sum()
    u = rng.choice(n, size=m, p=p)
    v = rng.choice(n, size=m, p=p)
    keep = u != v
    u, v = u[keep], v[keep]
    if not directed:
        a, b = np.minimum(u, v), np.maximum(u, v)
        key = _sorted_unique(a.astype(np.int64) * n + b)
        a, b = key // n, key % n
        src = np.concatenate([a, b])
        dst = np.concatenate([b, a])
    else:
        key = _sorted_unique(u.astype(np.int64) * n + v)
        src, dst = key // n, key % n
    indptr, indices = csr_from_edges(n, src, dst)
    return indptr, indices, w_by_id


@dataclasses.dataclass
class Batch:
    """One call's worth of edge events.

    src/dst/op: int32/int32/int8 arrays of length k (op +1 insert, -1 delete).
    new_nodes: nodes appended (ids n_before .. n_before+new_nodes-1) before the edges.
    """
    src: np.ndarray
    dst: np.ndarray
    op: np.ndarray
    new_nodes: int

    @property
    def k(self) -> int:
        return int(self.src.shape[0])


@dataclasses.dataclass
class EdgeStream:
    n0: int
    batches: List[Batch]

    @property
    def n_final(self) -> int:
        return self.n0 + sum(b.new_nodes for b in self.batches)

    @property
    def total_edges(self) -> int:
        return sum(b.k for b in self.batches)


def edge_stream(indptr: np.ndarray, indices: np.ndarray, weights: np.ndarray, n_batches: int,
                k_lo: int, k_hi: int, p_node: float, p_del: float, seed: int,
                max_new_degree: int = 32, directed: bool = False, nodes_per_batch: int = 0,
                log_sizes: bool = False) -> EdgeStream:
    """Seeded stream of edge batches over a graph given in CSR (see module docstring).
    log_sizes: k drawn log-uniformly from [k_lo, k_hi] (round(exp(U[ln k_lo, ln(k_hi + 1)])),
    clipped) instead of uniformly."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n0 = int(indptr.shape[0] - 1)
    # initial edges (canonical for undirected) in a random order, consumed by deletions
    rows = np.repeat(np.arange(n0, dtype=np.int64), np.diff(indptr.astype(np.int64)))
    cols = indices.astype(np.int64)
    if not directed:
        sel = rows < cols
        rows, cols = rows[sel], cols[sel]
    del_order = rng.permutation(rows.shape[0])
    del_pos = 0
    w_arr = np.asarray(weights, dtype=np.float64)
    w_mean = float(w_arr.mean())
    cap = n0 + 1024
    cdf_buf = np.empty(cap, dtype=np.float64)  # prefix sums of the weights; grows with new nodes
    cdf_buf[:n0] = np.cumsum(w_arr)
    n_cur = n0
    batches = []
    for _ in range(n_batches):
        if log_sizes:
            k_other = int(min(k_hi, max(k_lo, np.floor(np.exp(rng.uniform(np.log(k_lo), np.log(k_hi + 1)))))))
        else:
            k_other = int(rng.integers(k_lo, k_hi + 1))
        src, dst, op = [], [], []
        new_nodes = 0

        cdf = cdf_buf[:n_cur]

        def draw_node():
            t = int(np.searchsorted(cdf, rng.random() * cdf[-1], side="right"))
            return min(t, n_cur - 1)

        def arrival(room):
            nonlocal new_nodes
            node = n_cur + new_nodes
            new_nodes += 1
            deg = int(round(w_arr[rng.integers(0, n0)]))
            deg = max(1, min(deg, room, max_new_degree))
            nb = set()                       # distinct existing endpoints, proportional to w
            tries = 0
            while len(nb) < deg and tries < 8 * deg:
                nb.add(draw_node())
                tries += 1
            for t in sorted(nb):
                src.append(node), dst.append(t), op.append(1)

        for _ in range(nodes_per_batch):
            arrival(max_new_degree)
        target = len(src) + k_other
        while len(src) < target:
            x = rng.random()
            if x < p_node:
                arrival(target - len(src))
            elif x < p_node + p_del and del_pos < del_order.shape[0]:
                e = del_order[del_pos]
                del_pos += 1
                src.append(int(rows[e])), dst.append(int(cols[e])), op.append(-1)
            else:
                a, b = draw_node(), draw_node()
                if a == b:
                    continue
                src.append(a), dst.append(b), op.append(1)
        batches.append(Batch(np.asarray(src, dtype=np.int32), np.asarray(dst, dtype=np.int32),
                             np.asarray(op, dtype=np.int8), new_nodes))
        # new nodes get the mean weight so later insertions can reach them
        if new_nodes:
            if n_cur + new_nodes > cap:
                cap = 2 * (n_cur + new_nodes)
                grown = np.empty(cap, dtype=np.float64)
                grown[:n_cur] = cdf_buf[:n_cur]
                cdf_buf = grown
            cdf_buf[n_cur:n_cur + new_nodes] = cdf_buf[n_cur - 1] + w_mean * np.arange(1, new_nodes + 1)
        n_cur += new_nodes
    return EdgeStream(n0=n0, batches=batches)


def gaussian_test_matrix(n_rows: int, l: int, seed: int) -> np.ndarray:
    """Standard normal n_rows x l matrix (float32, row-major): the random test matrix
    of the randomized t-SVD (Halko et al.), passed as an input to both sides."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((n_rows, l), dtype=np.float32)


def node_arrival_stream(indptr: np.ndarray, indices: np.ndarray, n0: int, directed: bool = False):
    """The paper's node-arrival protocol (Sec. 5.1, "Setting of Dynamicity"): the graph
    induced on nodes 0 .. n0-1 is the initial graph; nodes n0, n0+1, ... then arrive one at a
    time, each with its edges to the nodes already present (an undirected edge {u, v} arrives
    with the later of u and v; a directed one with the later endpoint, in its direction).
    Node ids are already a random permutation of the Chung-Lu weights, so arrival in id order
    is arrival in random order.  Returns (indptr0, indices0, EdgeStream) with one Batch per
    node, new_nodes = 1."""
    indptr = np.asarray(indptr, dtype=np.int64)
    indices = np.asarray(indices, dtype=np.int64)
    n = len(indptr) - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(indptr))
    cols = indices
    keep0 = (rows < n0) & (cols < n0)
    ip0, ix0 = csr_from_edges(n0, rows[keep0], cols[keep0])
    later = np.maximum(rows, cols)
    if directed:
        sel = later >= n0
    else:
        sel = (later >= n0) & (rows < cols)      # each undirected edge once
    r, c, lt = rows[sel], cols[sel], later[sel]
    order = np.lexsort((c, r, lt))
    r, c, lt = r[order], c[order], lt[order]
    bounds = np.searchsorted(lt, np.arange(n0, n + 1))
    batches = []
    for i, v in enumerate(range(n0, n)):
        a, b = bounds[i], bounds[i + 1]
        batches.append(Batch(src=r[a:b].astype(np.int32), dst=c[a:b].astype(np.int32),
                             op=np.ones(b - a, dtype=np.int8), new_nodes=1))
    return ip0, ix0, EdgeStream(n0=n0, batches=batches)
