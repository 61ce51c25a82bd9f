"""Oracle: dynamic graph with set semantics, and the per-update sparse change dA = B C^T.

Test infrastructure only.  Follows Sec. 2 (graph, out-degree) and Sec. 4.3 (an edge
change is the rank-one update dA = e_u e_v^T, Eq. "edge_B"); a batch is the sum of its
net entries.  Node arrival is handled as in the paper's Sec. 4.2 reduced to edges:
appending a node appends a zero row and column (the t-SVD is unchanged, V gets a zero
row), after which its edges are ordinary edge changes.
"""

from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Dict, List, Tuple

import numpy as np

from .build import build

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        vp, i32, i64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        lib.og_create.restype = vp
        lib.og_create.argtypes = [i32, i32]
        lib.og_destroy.argtypes = [vp]
        lib.og_num_nodes.restype = i32
        lib.og_num_nodes.argtypes = [vp]
        lib.og_add_nodes.restype = i32
        lib.og_add_nodes.argtypes = [vp, i32]
        lib.og_degree.restype = i32
        lib.og_degree.argtypes = [vp, i32]
        lib.og_has.restype = i32
        lib.og_has.argtypes = [vp, i32, i32]
        lib.og_insert.restype = i32
        lib.og_insert.argtypes = [vp, i32, i32]
        lib.og_erase.restype = i32
        lib.og_erase.argtypes = [vp, i32, i32]
        lib.og_neighbors.restype = i32
        lib.og_neighbors.argtypes = [vp, i32, vp]
        lib.og_load_csr.argtypes = [vp, vp, vp]
        lib.og_num_entries.restype = i64
        lib.og_num_entries.argtypes = [vp]
        lib.og_export_csr.argtypes = [vp, vp, vp]
        lib.og_push.restype = i64
        lib.og_push.argtypes = [vp, vp, i32, vp, vp, dbl, dbl, i64, i32]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Adjacency:
    """One direction of adjacency (rows = nodes), backed by the plain-C structure."""

    def __init__(self, n: int, n_cap: int):
        self.lib = _load()
        self.h = self.lib.og_create(n, n_cap)

    def __del__(self):
        if getattr(self, "h", None):
            self.lib.og_destroy(self.h)
            self.h = None

    @property
    def n(self) -> int:
        return self.lib.og_num_nodes(self.h)

    def add_nodes(self, k: int):
        if self.lib.og_add_nodes(self.h, k) < 0:
            raise ValueError("node capacity exceeded")

    def has(self, u: int, v: int) -> bool:
        return bool(self.lib.og_has(self.h, u, v))

    def insert(self, u: int, v: int) -> bool:
        return bool(self.lib.og_insert(self.h, u, v))

    def erase(self, u: int, v: int) -> bool:
        return bool(self.lib.og_erase(self.h, u, v))

    def degree(self, u: int) -> int:
        return self.lib.og_degree(self.h, u)

    def row(self, u: int) -> np.ndarray:
        out = np.empty(max(self.degree(u), 1), dtype=np.int32)
        k = self.lib.og_neighbors(self.h, u, _ptr(out))
        return out[:k].copy()

    def load_csr(self, indptr: np.ndarray, indices: np.ndarray):
        indptr = np.ascontiguousarray(indptr, dtype=np.int32)
        indices = np.ascontiguousarray(indices, dtype=np.int32)
        self.lib.og_load_csr(self.h, _ptr(indptr), _ptr(indices))

    def csr(self) -> Tuple[np.ndarray, np.ndarray]:
        nnz = self.lib.og_num_entries(self.h)
        indptr = np.empty(self.n + 1, dtype=np.int64)
        indices = np.empty(max(nnz, 1), dtype=np.int32)
        self.lib.og_export_csr(self.h, _ptr(indptr), _ptr(indices))
        return indptr, indices[:nnz]

    def degrees(self) -> np.ndarray:
        return np.array([self.degree(u) for u in range(self.n)], dtype=np.int64)


@dataclass
class SparseChange:
    """dA = I_S N I_T^T for one update: S (sources) and T (targets) sorted unique,
    N[a, b] = dA[S[a], T[b]] in {-1, 0, +1}.  `entries` lists the (u, v, delta) with
    delta != 0 in sorted (u, v) order."""
    S: np.ndarray
    T: np.ndarray
    N: np.ndarray
    entries: List[Tuple[int, int, int]]

    @property
    def empty(self) -> bool:
        return len(self.entries) == 0

    def dense(self, n: int) -> np.ndarray:
        A = np.zeros((n, n))
        for u, v, dl in self.entries:
            A[u, v] += dl
        return A


class DynGraph:
    """The dynamic graph G of Sec. 2 with set semantics for edge events."""

    def __init__(self, indptr, indices, n_cap: int, directed: bool = False):
        n = int(len(indptr) - 1)
        self.directed = directed
        self.out = Adjacency(n, n_cap)
        self.out.load_csr(indptr, indices)
        if directed:
            self.inn = Adjacency(n, n_cap)
            rows = np.repeat(np.arange(n, dtype=np.int32), np.diff(np.asarray(indptr, dtype=np.int64)))
            for u, v in zip(rows.tolist(), np.asarray(indices).tolist()):
                self.inn.insert(v, u)
        else:
            self.inn = self.out

    @property
    def n(self) -> int:
        return self.out.n

    def add_nodes(self, k: int):
        self.out.add_nodes(k)
        if self.directed:
            self.inn.add_nodes(k)

    def validate(self, src, dst, op, new_nodes: int):
        n_after = self.n + new_nodes
        for u, v, o in zip(src.tolist(), dst.tolist(), op.tolist()):
            if not (0 <= u < n_after and 0 <= v < n_after) or u == v or o not in (1, -1):
                raise ValueError("invalid edge event (%d, %d, %d)" % (u, v, o))

    def apply(self, src, dst, op) -> SparseChange:
        """Applies one update's events with set semantics and returns the net change.

        For every ordered pair (u, v) touched by the events, the final membership is
        the one set by the pair's last event (insert -> present, delete -> absent) and
        delta = final - initial.  Undirected events touch (u, v) and (v, u)."""
        last: Dict[Tuple[int, int], int] = {}
        for u, v, o in zip(np.asarray(src).tolist(), np.asarray(dst).tolist(), np.asarray(op).tolist()):
            last[(u, v)] = o
            if not self.directed:
                last[(v, u)] = o
        entries = []
        for (u, v), o in sorted(last.items()):
            initial = 1 if self.out.has(u, v) else 0
            final = 1 if o == 1 else 0
            if final != initial:
                entries.append((u, v, final - initial))
        for u, v, dl in entries:
            if dl > 0:
                self.out.insert(u, v)
                if self.directed:
                    self.inn.insert(v, u)
            else:
                self.out.erase(u, v)
                if self.directed:
                    self.inn.erase(v, u)
        S = np.array(sorted({e[0] for e in entries}), dtype=np.int64)
        T = np.array(sorted({e[1] for e in entries}), dtype=np.int64)
        N = np.zeros((len(S), len(T)))
        si = {int(u): a for a, u in enumerate(S)}
        ti = {int(v): b for b, v in enumerate(T)}
        for u, v, dl in entries:
            N[si[u], ti[v]] = dl
        return SparseChange(S, T, N, entries)


def split_updates(k: int, per_update: int) -> List[Tuple[int, int]]:
    """Edge ranges [lo, hi) of the consecutive updates one call of k events is applied as,
    at most per_update events each."""
    if per_update < 1:
        raise ValueError("per_update must be >= 1")
    return [(lo, min(lo + per_update, k)) for lo in range(0, k, per_update)]
