"""Python binding of the C ABI (argument marshalling only; every step runs in libdamf.so).

PyTorch provides device memory and streams.  Tensors passed in must be CUDA tensors of
the stated dtype; numpy arrays are copied to the device first.
"""

from __future__ import annotations

import ctypes
import functools
import inspect

import numpy as np
import torch

from . import _lib
from ._lib import Config, Stats, STATUS_NAMES


class DamfError(RuntimeError):
    def __init__(self, code: int, msg: str = ""):
        super().__init__("%s (%d)%s" % (STATUS_NAMES.get(code, "?"), code, (": " + msg) if msg else ""))
        self.code = code


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _on_stream(fn):
    """Runs fn with its `stream` argument (when one is given) as torch's current stream, so that
    the inputs it copies to the device, the outputs it allocates and the library's work are all
    ordered on that one stream; the caching allocator then hands those blocks to a later
    allocation only after that stream's work that used them."""
    pos = list(inspect.signature(fn).parameters).index("stream")

    @functools.wraps(fn)
    def run(*args, **kwargs):
        s = kwargs["stream"] if "stream" in kwargs else (args[pos] if len(args) > pos else None)
        if s is None:
            return fn(*args, **kwargs)
        with torch.cuda.stream(s):
            return fn(*args, **kwargs)
    return run


def _dev(x, dtype):
    if isinstance(x, torch.Tensor):
        if not x.is_cuda or x.dtype != dtype or not x.is_contiguous():
            x = x.to(device="cuda", dtype=dtype).contiguous()
        return x
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def make_config(n, d, alpha, eps, n_capacity=None, m_capacity=None, nnz=0, directed=False, refold_every=0,
                rsvd_oversample=10, rsvd_power_iters=4, max_push_rounds=100000, precision="mixed",
                threshold="absolute") -> Config:
    """precision: "fp32" (SIMT everywhere) or "mixed" (tensor-core GEMMs for the fold, init, query).
    threshold: "absolute" (push until max|r[u]| <= eps) or "degree" (until max|r[u]| <= eps max(deg(u), 1))."""
    n_capacity = n if n_capacity is None else n_capacity
    if m_capacity is None:
        # initial rows with 25% slack plus room for relocations and growth
        m_capacity = int(2.0 * nnz) + 64 * n_capacity + 4096
    return Config(n=n, n_capacity=n_capacity, m_capacity=m_capacity, d=d, directed=int(directed), alpha=alpha,
                  eps=eps, refold_every=refold_every, rsvd_oversample=rsvd_oversample,
                  rsvd_power_iters=rsvd_power_iters, max_push_rounds=max_push_rounds,
                  precision={"fp32": 0, "mixed": 1}[precision],
                  threshold={"absolute": 0, "degree": 1}[threshold])


def rsvd_width(cfg: Config) -> int:
    return int(_lib.load().damf_rsvd_width(ctypes.byref(cfg)))


def bytes_required(cfg: Config) -> int:
    return int(_lib.load().damf_bytes_required(ctypes.byref(cfg)))


@_on_stream
def core_svd(sigma, L, R, status=None, stream=None):
    """Top-d SVD of diag(sigma, 0) + L R^T through damf_core_svd (Step 2 of an update).
    Returns (E, H, theta) CUDA tensors; `status` (a CUDA int32 tensor of one element, optional)
    receives the device status of the computation once the stream's work is done."""
    lib = _lib.load()
    sigma, L, R = _dev(sigma, torch.float32), _dev(L, torch.float32), _dev(R, torch.float32)
    d, r = int(sigma.numel()), int(L.shape[1])
    m = d + r
    E = torch.empty((m, d), dtype=torch.float32, device="cuda")
    H = torch.empty((m, d), dtype=torch.float32, device="cuda")
    th = torch.empty(d, dtype=torch.float32, device="cuda")
    nbytes = int(lib.damf_core_svd_workspace_size(d, r))
    if nbytes == 0:
        raise DamfError(1, "core_svd sizes")
    ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    stp = ctypes.c_void_p(status.data_ptr()) if status is not None else None
    st = lib.damf_core_svd(p(sigma), p(L), p(R), d, r, p(E), p(H), p(th), p(ws), nbytes, stp, _stream_ptr(stream))
    if st != 0:
        raise DamfError(st, "core_svd")
    return E, H, th


@_on_stream
def batch_array(batches, stream=None):
    """damf_batch[] for a list of (DamfGraph, src, dst, op[, new_nodes[, k_dev]]); with a k_dev
    (device int32 tensor of one element) the arrays hold k_max events of which *k_dev are live.
    Host arrays are copied to the device on `stream` (default: the current stream), the one
    the batches are then stepped on."""
    arr = (_lib.Batch * max(len(batches), 1))()
    for i, b in enumerate(batches):
        g, src, dst, op = b[:4]
        nn = int(b[4]) if len(b) > 4 else 0
        kd = b[5] if len(b) > 5 else None
        s, t, o = _dev(src, torch.int32), _dev(dst, torch.int32), _dev(op, torch.int8)
        if kd is not None and (not isinstance(kd, torch.Tensor) or not kd.is_cuda or kd.dtype != torch.int32):
            raise ValueError("k_dev must be a CUDA int32 tensor")
        g._keep = (s, t, o, kd)   # alive until the stream has consumed them
        arr[i] = _lib.Batch(g.h.value if hasattr(g.h, "value") else g.h, s.data_ptr(), t.data_ptr(), o.data_ptr(),
                            int(s.numel()), nn, None if kd is None else kd.data_ptr())
    return arr


@_on_stream
def apply_edges_multi(batches, stream=None):
    """One batch per graph through damf_apply_edges_multi, in order on one stream: batches is a
    list of (DamfGraph, src, dst, op[, new_nodes[, k_dev]])."""
    st = _lib.load().damf_apply_edges_multi(batch_array(batches, stream), len(batches), _stream_ptr(stream))
    if st != 0:
        raise DamfError(st, "apply_edges_multi")


@_on_stream
def step_multi(batches, stream=None):
    """One step of many graphs through damf_step_multi: each graph's update and push on its own
    streams, joined back to `stream`. batches as for apply_edges_multi."""
    st = _lib.load().damf_step_multi(batch_array(batches, stream), len(batches), _stream_ptr(stream))
    if st != 0:
        raise DamfError(st, "step_multi")


def plan_slots(weights, max_blocks: int):
    """The grouped push's CTA plan for work weights (damf_plan_slots, host only): returns
    (slot of each graph, CTAs of each slot)."""
    w = np.ascontiguousarray(weights, dtype=np.float64)
    slot_of = np.zeros(w.size, dtype=np.int32)
    ctas = np.zeros(max(w.size, 1), dtype=np.int32)
    n = int(_lib.load().damf_plan_slots(w.ctypes.data_as(ctypes.c_void_p), int(w.size), int(max_blocks),
                                        slot_of.ctypes.data_as(ctypes.c_void_p), ctas.ctypes.data_as(ctypes.c_void_p)))
    if n < 0:
        raise DamfError(1, "plan_slots")
    return slot_of, ctas[:n]


class DamfFleet:
    """Many graphs stepped together, their pushes in one grouped launch (damf_fleet_*).
    The DamfGraphs stay owned by the caller and must outlive the fleet."""

    def __init__(self, graphs):
        self.lib = _lib.load()
        self.graphs = list(graphs)
        arr = (ctypes.c_void_p * len(self.graphs))(*[g.h.value for g in self.graphs])
        h = ctypes.c_void_p()
        st = self.lib.damf_fleet_create(arr, len(self.graphs), ctypes.byref(h))
        if st != 0:
            raise DamfError(st, "fleet_create")
        self.h = h

    def _check(self, st):
        if st != 0:
            raise DamfError(st, self.lib.damf_fleet_last_error(self.h).decode())

    @_on_stream
    def step(self, batches, stream=None):
        """batches: one (src, dst, op[, new_nodes[, k_dev]]) per graph, fleet order."""
        arr = batch_array([(g, *b) for g, b in zip(self.graphs, batches)], stream)
        self._keep = arr
        self._check(self.lib.damf_fleet_step(self.h, arr, _stream_ptr(stream)))

    def step_array(self, arr, stream=None):
        """A prepared damf_batch array (api.batch_array), e.g. for a captured step."""
        self._check(self.lib.damf_fleet_step(self.h, arr, _stream_ptr(stream)))

    def set_shares(self, blocks=None, exponent: float = 1.0):
        """Push CTAs per graph (list of ints), or shares proportional to (d (n + m))^exponent."""
        if blocks is None:
            self._check(self.lib.damf_fleet_set_shares(self.h, None, float(exponent)))
        else:
            a = np.ascontiguousarray(blocks, dtype=np.int32)
            if a.size != len(self.graphs):
                raise ValueError("one share per graph")
            self._check(self.lib.damf_fleet_set_shares(self.h, a.ctypes.data_as(ctypes.c_void_p), 0.0))

    def set_weights(self, weights):
        """Shares in proportion to per-graph work estimates (e.g. measured push time x CTAs)."""
        a = np.ascontiguousarray(weights, dtype=np.float64)
        if a.size != len(self.graphs):
            raise ValueError("one weight per graph")
        self._check(self.lib.damf_fleet_set_weights(self.h, a.ctypes.data_as(ctypes.c_void_p)))

    def shares(self):
        """(CTAs per graph as a list, grouped launches per step)."""
        a = np.zeros(len(self.graphs), dtype=np.int32)
        nl = ctypes.c_int32()
        self._check(self.lib.damf_fleet_get_shares(self.h, a.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nl)))
        return a.tolist(), int(nl.value)

    @property
    def launches(self) -> int:
        return int(self.lib.damf_fleet_launches(self.h))

    def set_timing(self, enable: bool = True):
        self._check(self.lib.damf_fleet_set_timing(self.h, int(enable)))

    def timing(self) -> dict:
        """{"update_ms", "push_ms", "steps"} of the steps timed since the last call."""
        a, b, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
        self._check(self.lib.damf_fleet_get_timing(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(n)))
        return {"update_ms": a.value, "push_ms": b.value, "steps": n.value}

    def close(self):
        if getattr(self, "h", None):
            self.lib.damf_fleet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class DamfGraph:
    """One graph's DAMF state on the current CUDA device (a damf_ctx)."""

    @_on_stream
    def __init__(self, indptr, indices, cfg: Config, omega, stream=None):
        self.lib = _lib.load()
        self.cfg = cfg
        self.d = cfg.d
        self.directed = bool(cfg.directed)
        ip = _dev(indptr, torch.int32)
        ix = _dev(indices, torch.int32) if len(indices) else torch.zeros(1, dtype=torch.int32, device="cuda")
        om = _dev(omega, torch.float32)
        l = rsvd_width(cfg)
        if om.shape != (cfg.n, l) and om.numel() < cfg.n * l:
            raise ValueError("omega must be n x %d" % l)
        h = ctypes.c_void_p()
        st = self.lib.damf_init_factorize(ctypes.byref(cfg), ctypes.c_void_p(ip.data_ptr()),
                                          ctypes.c_void_p(ix.data_ptr()), int(len(indices)),
                                          ctypes.c_void_p(om.data_ptr()), _stream_ptr(stream), ctypes.byref(h))
        if st != 0:
            raise DamfError(st, "init")
        self.h = h

    def _check(self, st):
        if st != 0:
            raise DamfError(st, self.lib.damf_last_error(self.h).decode())

    @_on_stream
    def save(self, stream=None) -> dict:
        """A checkpoint: the full state (CUDA tensors), the out-adjacency (host CSR) and the
        config; DamfGraph.restore(checkpoint) continues from it."""
        n, d = self.n, self.d
        t = {k: torch.empty((n, d), dtype=torch.float32, device="cuda") for k in ("Ub", "Vb", "Zb", "r")}
        t.update({k: torch.empty((d, d), dtype=torch.float32, device="cuda") for k in ("PU", "PV", "PUi", "PVi")})
        t.update({k: torch.empty(d, dtype=torch.float32, device="cuda") for k in ("sigma", "s0")})
        st = _lib.State(**{k: v.data_ptr() for k, v in t.items()})
        self._check(self.lib.damf_save_state(self.h, ctypes.byref(st), _stream_ptr(stream)))
        rp, col = self.adjacency(outgoing=True)
        cfg = Config()
        ctypes.memmove(ctypes.byref(cfg), ctypes.byref(self.cfg), ctypes.sizeof(Config))
        cfg.n = n
        return {"state": t, "updates_since_fold": int(st.updates_since_fold), "indptr": rp.astype(np.int32),
                "indices": col.copy(), "cfg": cfg}

    @classmethod
    @_on_stream
    def restore(cls, ckpt: dict, stream=None) -> "DamfGraph":
        """A new context continuing a checkpoint from DamfGraph.save (damf_restore)."""
        self = cls.__new__(cls)
        self.lib = _lib.load()
        cfg = ckpt["cfg"]
        self.cfg = cfg
        self.d = cfg.d
        self.directed = bool(cfg.directed)
        ip = _dev(ckpt["indptr"], torch.int32)
        ix = _dev(ckpt["indices"], torch.int32) if len(ckpt["indices"]) else torch.zeros(1, dtype=torch.int32,
                                                                                         device="cuda")
        t = {k: _dev(v, torch.float32) for k, v in ckpt["state"].items()}   # host tensors are copied over
        st = _lib.State(**{k: v.data_ptr() for k, v in t.items()},
                        updates_since_fold=int(ckpt["updates_since_fold"]))
        h = ctypes.c_void_p()
        code = self.lib.damf_restore(ctypes.byref(cfg), ctypes.c_void_p(ip.data_ptr()), ctypes.c_void_p(ix.data_ptr()),
                                     int(len(ckpt["indices"])), ctypes.byref(st), _stream_ptr(stream),
                                     ctypes.byref(h))
        if code != 0:
            raise DamfError(code, "restore")
        self.h = h
        return self

    @_on_stream
    def save_file(self, path: str, stream=None) -> int:
        """Writes a checkpoint (save()) to a file (paper_2306_08967_gb300.checkpoint); returns
        its size in bytes."""
        from .checkpoint import write_checkpoint
        return write_checkpoint(path, self.save(stream))

    @classmethod
    @_on_stream
    def load_file(cls, path: str, stream=None) -> "DamfGraph":
        """A new context continuing the checkpoint file at `path` (checked before any device work)."""
        from .checkpoint import read_checkpoint
        return cls.restore(read_checkpoint(path), stream)

    @property
    def n(self) -> int:
        return int(self.lib.damf_num_nodes(self.h))

    @_on_stream
    def apply_edges(self, src, dst, op, new_nodes: int = 0, stream=None):
        """Device-resident events (int32 src/dst, int8 op)."""
        s, t, o = _dev(src, torch.int32), _dev(dst, torch.int32), _dev(op, torch.int8)
        self._keep = (s, t, o)  # alive until the stream has consumed them
        self._check(self.lib.damf_apply_edges(self.h, ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                              ctypes.c_void_p(o.data_ptr()), int(s.numel()), int(new_nodes),
                                              _stream_ptr(stream)))

    @_on_stream
    def apply_edges_counted(self, src, dst, op, k_dev, new_nodes: int = 0, stream=None):
        """Device events of which the first k_dev[0] (a CUDA int32 tensor, read when the work
        runs) are live; src/dst/op hold k_max events."""
        s, t, o = _dev(src, torch.int32), _dev(dst, torch.int32), _dev(op, torch.int8)
        if not isinstance(k_dev, torch.Tensor) or not k_dev.is_cuda or k_dev.dtype != torch.int32:
            raise ValueError("k_dev must be a CUDA int32 tensor")
        self._keep = (s, t, o, k_dev)
        self._check(self.lib.damf_apply_edges_counted(self.h, ctypes.c_void_p(s.data_ptr()),
                                                      ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(o.data_ptr()),
                                                      int(s.numel()), ctypes.c_void_p(k_dev.data_ptr()),
                                                      int(new_nodes), _stream_ptr(stream)))

    def set_tuning(self, push_blocks: int = 0, push_direct_chunks: int = -1):
        """Launch shape of the following pushes (0 / -1: the defaults)."""
        t = _lib.Tuning(push_blocks=int(push_blocks), push_direct_chunks=int(push_direct_chunks))
        self._check(self.lib.damf_set_tuning(self.h, ctypes.byref(t)))

    def tuning(self) -> dict:
        """The push launch shape the next push uses."""
        t = _lib.Tuning()
        self._check(self.lib.damf_get_tuning(self.h, ctypes.byref(t)))
        return {"push_blocks": int(t.push_blocks), "push_direct_chunks": int(t.push_direct_chunks)}

    def delete_nodes(self, nodes, stream=None):
        """Removes every edge of the given nodes (host ids); the ids stay as isolated nodes."""
        a = np.ascontiguousarray(nodes, dtype=np.int32)
        self._check(self.lib.damf_delete_nodes(self.h, a.ctypes.data_as(ctypes.c_void_p), int(a.size),
                                               _stream_ptr(stream)))

    def apply_edges_host(self, src: np.ndarray, dst: np.ndarray, op: np.ndarray, new_nodes: int = 0, stream=None):
        """Host events: the library copies them to the device on the stream."""
        s = np.ascontiguousarray(src, dtype=np.int32)
        t = np.ascontiguousarray(dst, dtype=np.int32)
        o = np.ascontiguousarray(op, dtype=np.int8)
        self._check(self.lib.damf_apply_edges_host(self.h, s.ctypes.data_as(ctypes.c_void_p),
                                                   t.ctypes.data_as(ctypes.c_void_p),
                                                   o.ctypes.data_as(ctypes.c_void_p), int(s.shape[0]),
                                                   int(new_nodes), _stream_ptr(stream)))

    def ppr_refresh(self, stream=None):
        self._check(self.lib.damf_ppr_refresh(self.h, _stream_ptr(stream)))

    def join(self, stream=None):
        """Makes the stream wait for the most recent PPR push."""
        self._check(self.lib.damf_join(self.h, _stream_ptr(stream)))

    def record_event(self, event):
        """Records a torch.cuda.Event on the push stream after the most recent push."""
        self._check(self.lib.damf_record_event(self.h, ctypes.c_void_p(event.cuda_event)))

    @_on_stream
    def embeddings(self, rows=None, want=("X", "Y", "Z", "sigma"), stream=None):
        """Returns a dict of CUDA tensors: X, Y, Z (count x d) and sigma (d)."""
        if rows is None:
            count, rp = self.n, None
        else:
            rows = _dev(rows, torch.int32)
            count, rp = int(rows.numel()), ctypes.c_void_p(rows.data_ptr())
        out = {}
        ptrs = []
        for name in ("X", "Y", "Z"):
            if name in want:
                out[name] = torch.empty((count, self.d), dtype=torch.float32, device="cuda")
                ptrs.append(ctypes.c_void_p(out[name].data_ptr()))
            else:
                ptrs.append(None)
        if "sigma" in want:
            out["sigma"] = torch.empty(self.d, dtype=torch.float32, device="cuda")
            sp = ctypes.c_void_p(out["sigma"].data_ptr())
        else:
            sp = None
        self._check(self.lib.damf_get_embeddings(self.h, rp, count, ptrs[0], ptrs[1], ptrs[2], sp,
                                                 _stream_ptr(stream)))
        return out

    @_on_stream
    def score_pairs(self, src, dst, context="Z", symmetric=None, stream=None):
        """Link-prediction scores context(src[i]) . Y[dst[i]] (context "Z" enhanced or "X");
        symmetric (default: the graph is undirected) takes the larger of both directions."""
        src = _dev(src, torch.int32)
        dst = _dev(dst, torch.int32)
        count = int(src.numel())
        if int(dst.numel()) != count:
            raise ValueError("src and dst differ in length")
        sym = (not self.directed) if symmetric is None else bool(symmetric)
        out = torch.empty(count, dtype=torch.float32, device="cuda")
        self._check(self.lib.damf_score_pairs(self.h, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()),
                                              count, {"Z": 0, "X": 1}[context], int(sym),
                                              ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    @_on_stream
    def topk(self, rows, k, context="Z", symmetric=None, stream=None):
        """The k best-scoring nodes v != u for each query u in rows: (ids int32, scores float32),
        each count x k, decreasing score, equal scores by increasing id (-1 / -inf padding)."""
        rows = _dev(rows, torch.int32)
        count = int(rows.numel())
        sym = (not self.directed) if symmetric is None else bool(symmetric)
        idx = torch.empty((count, k), dtype=torch.int32, device="cuda")
        sc = torch.empty((count, k), dtype=torch.float32, device="cuda")
        self._check(self.lib.damf_topk(self.h, ctypes.c_void_p(rows.data_ptr()), count, int(k), {"Z": 0, "X": 1}[context],
                                       int(sym), ctypes.c_void_p(idx.data_ptr()), ctypes.c_void_p(sc.data_ptr()),
                                       _stream_ptr(stream)))
        return idx, sc

    @_on_stream
    def state(self, stream=None) -> dict:
        """Base state: Ub, Vb, Zb, r (n x d), PU, PV (d x d), sigma, s0 (d) as CUDA tensors."""
        n, d = self.n, self.d
        out = {k: torch.empty((n, d), dtype=torch.float32, device="cuda") for k in ("Ub", "Vb", "Zb", "r")}
        out.update({k: torch.empty((d, d), dtype=torch.float32, device="cuda") for k in ("PU", "PV")})
        out.update({k: torch.empty(d, dtype=torch.float32, device="cuda") for k in ("sigma", "s0")})
        ptr = lambda k: ctypes.c_void_p(out[k].data_ptr())
        self._check(self.lib.damf_get_state(self.h, ptr("Ub"), ptr("Vb"), ptr("Zb"), ptr("r"), ptr("PU"), ptr("PV"),
                                            ptr("sigma"), ptr("s0"), _stream_ptr(stream)))
        return out

    def adjacency(self, outgoing: bool = True, capacity: int = None):
        """Current adjacency as host CSR (row_ptr int64[n+1], col int32[nnz]; rows unsorted)."""
        capacity = int(self.cfg.m_capacity) if capacity is None else capacity
        rp = np.zeros(self.n + 1, dtype=np.int64)
        col = np.zeros(max(capacity, 1), dtype=np.int32)
        self._check(self.lib.damf_export_adjacency(self.h, int(outgoing), rp.ctypes.data_as(ctypes.c_void_p),
                                                   col.ctypes.data_as(ctypes.c_void_p), capacity))
        return rp, col[: rp[-1]]

    def last_touched(self):
        S = np.zeros(128, dtype=np.int32)   # an update touches at most 128 rows
        T = np.zeros(128, dtype=np.int32)
        ns = ctypes.c_int32()
        nt = ctypes.c_int32()
        self._check(self.lib.damf_get_last_touched(self.h, S.ctypes.data_as(ctypes.c_void_p), ctypes.byref(ns),
                                                   T.ctypes.data_as(ctypes.c_void_p), ctypes.byref(nt)))
        return S[: ns.value].copy(), T[: nt.value].copy()

    def set_timing(self, enable: bool = True):
        self._check(self.lib.damf_set_timing(self.h, int(enable)))

    def timing(self) -> dict:
        """{stage: (device ms, launches)} accumulated since the last call."""
        ms = np.zeros(len(_lib.STAGES), dtype=np.float64)
        nl = np.zeros(len(_lib.STAGES), dtype=np.int64)
        self._check(self.lib.damf_get_timing(self.h, ms.ctypes.data_as(ctypes.c_void_p),
                                             nl.ctypes.data_as(ctypes.c_void_p)))
        return {k: (float(ms[i]), int(nl[i])) for i, k in enumerate(_lib.STAGES)}

    def stats(self) -> dict:
        st = Stats()
        self._check(self.lib.damf_get_stats(self.h, ctypes.byref(st)))
        out = {k: getattr(st, k) for k, _ in Stats._fields_}
        out["push_ns"] = list(out["push_ns"])
        return out

    def sync_status(self) -> int:
        return int(self.lib.damf_sync_status(self.h))

    def check(self):
        self._check(self.sync_status())

    def close(self):
        if getattr(self, "h", None):
            self.lib.damf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
