#!/usr/bin/env python
"""Edge-update throughput and latency of the DAMF hot path on one GB300 (or N replicas).

A step is one batch of the workload through the whole hot path: damf_apply_edges
(adjacency edit, projection, residual CholQR, core SVD, transform update, row rewrite,
PPR residual fix-up) followed by damf_ppr_refresh (push until every residual <= eps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config C3] [--impl ours|reference]

The default workload is C3 (the 2M-node graph, calls of 1-256 events, the fold every 256
updates); the line adds both precisions over a longer window (precision_compare), the FP64
oracle timed on the host cores (cpu_baseline) and its error on the same batches
(err_vs_oracle). Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the same workload (bounded sample per step) and prints the same metric with "impl":
"reference".

Other workloads (not the default line):
  --config C1, C2                 the smaller single-graph workloads
  --config C4 [--graphs G]        many graphs per step: a fleet (every graph's update on its own
                                  stream, one grouped push), each step one CUDA graph replay
                                  after the push shares are autotuned; beside it the same step
                                  graph by graph, by damf_step_multi and by direct fleet calls
  --config C5 [--rates a,b,c]     serving: sessions admitted by device memory, Poisson requests
                                  in phases of rising rate, continuous batching of fleet steps
  --mode node-stream              the paper's node-arrival protocol, ms per node event
  --mode init-scale               the randomized t-SVD initialisation at the serving workload's
                                  stated size (n = 50M, m = 1B, directed), then update requests
"""

import argparse
import dataclasses
import json
import os
import sys



def _oracle_threads(argv):
    # --oracle-threads N: BLAS threads of the oracle (default: every host core), read before
    # numpy loads
    for i, a in enumerate(argv):
        if a == "--oracle-threads" and i + 1 < len(argv):
            return max(1, int(argv[i + 1]))
        if a.startswith("--oracle-threads="):
            return max(1, int(a.split("=", 1)[1]))
    return max(1, os.cpu_count() or 1)


ORACLE_THREADS = _oracle_threads(sys.argv)

if "--impl" in sys.argv and "reference" in sys.argv or "--oracle-worker" in sys.argv:
    # pin the oracle's BLAS pools before numpy loads (every host core unless --oracle-threads)
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = str(ORACLE_THREADS)

import subprocess
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edge-updates/sec and p50/p99 update latency at d=128, mixed vs plain FP32, same err"
UNIT = "edge-updates/s"


def workload_desc(c):
    return ("%s: %s Chung-Lu gamma=%.1f n=%d avg_deg=%g; d=%d alpha=%g eps=%g; batches of U[%d,%d] edges, "
            "%.0f%% node arrivals, %.0f%% deletions" % (c.name, "directed" if c.directed else "undirected", c.gamma,
                                                       c.n, c.avg_deg, c.d, c.alpha, c.eps, c.k_lo, c.k_hi,
                                                       100 * c.p_node, 100 * c.p_del))


_INPUTS = {}


def make_inputs(c, n_batches):
    """The workload's graph and its first n_batches batches (generated once per process and
    workload; the stream's first batches do not depend on how many follow them)."""
    import dataclasses as dc
    from synth import chung_lu_graph, edge_stream
    key = (c.name, c.seed, c.n)
    if key not in _INPUTS or len(_INPUTS[key][2].batches) < n_batches:
        if key in _INPUTS:
            ip, ix, w = _INPUTS[key][0], _INPUTS[key][1], _INPUTS[key][3]
        else:
            ip, ix, w = chung_lu_graph(c.n, c.avg_deg, c.gamma, seed=c.seed, directed=c.directed)
        st = edge_stream(ip, ix, w, n_batches, c.k_lo, c.k_hi, c.p_node, c.p_del, c.seed + 1,
                         max_new_degree=c.max_new_degree, directed=c.directed, nodes_per_batch=c.nodes_per_batch)
        _INPUTS[key] = (ip, ix, st, w)
    ip, ix, st, _ = _INPUTS[key]
    if len(st.batches) > n_batches:
        st = dc.replace(st, batches=st.batches[:n_batches])
    return ip, ix, st


# ---------------------------------------------------------------- oracle (CPU) leg
# The oracle's initialisation on graphs of a million nodes or more is cut to what fits in
# minutes: no randomized t-SVD power passes (two sparse products and two QR factorisations in
# place of ten and ten; the error comparison starts the device from the same randomized t-SVD)
# and no initial PPR propagation (its FIFO push from r = X_b over 2M nodes would take hours on a
# core): Z_b = 0 and r = 0, as if that propagation had converged, so the timed batches run the
# oracle's whole per-batch path (factor update, fix-up, push of the batch's residual) with a
# fix-up that reads Z_b = 0, a little less work than with the propagated Z_b.
def oracle_big(c):
    return c.n >= 1_000_000


def oracle_power_iters(c):
    return 0 if oracle_big(c) else 4


ERR_SAMPLE_ROWS = 20000   # rows of X, Y, Z the error comparison reads (all of them below this)
ORACLE_ALT_THREADS = 8    # the second thread count the oracle leg is timed at (when the host has more)


def _blas_thread_setter():
    """The OpenBLAS thread-count setter of the BLAS numpy loaded (found through the process's
    mapped libraries, as threadpoolctl does), or None."""
    import ctypes
    try:
        paths = sorted({ln.split()[-1] for ln in open("/proc/self/maps") if "openblas" in ln.lower()
                        and ln.split()[-1].startswith("/")})
    except OSError:
        return None
    for path in paths:
        try:
            h = ctypes.CDLL(path)
        except OSError:
            continue
        for name in ("scipy_openblas_set_num_threads64_", "scipy_openblas_set_num_threads",
                     "openblas_set_num_threads64_", "openblas_set_num_threads"):
            fn = getattr(h, name, None)
            if fn is not None:
                fn.argtypes, fn.restype = [ctypes.c_int], None
                return fn
    return None


def oracle_run(c, steps, warmup, time_budget_s, save_path=None, alt_threads=0):
    """Times the FP64 oracle (as it stands) on the first warmup+steps batches, stopping
    early once time_budget_s of timed work is spent.  Returns a dict; with save_path, also
    writes the oracle's final sigma and the rows of X, Y, Z of a seeded row sample there
    (npz) for the error comparison."""
    from oracle.damf import DamfOracle
    from synth import gaussian_test_matrix
    ip, ix, st = make_inputs(c, warmup + steps)
    om = gaussian_test_matrix(c.n, 160 if c.d == 128 else ((c.d + 10 + 31) // 32) * 32, seed=c.seed + 2)
    t0 = time.perf_counter()
    orc = DamfOracle(ip, ix, c.d, c.alpha, c.eps, n_cap=st.n_final, directed=c.directed, Omega=om,
                     power_iters=oracle_power_iters(c), propagate=not oracle_big(c))
    if oracle_big(c):
        orc.r[:] = 0.0
    init_s = time.perf_counter() - t0
    pushes0 = orc.pushes
    for b in st.batches[:warmup]:
        orc.apply_edges(b.src, b.dst, b.op, b.new_nodes)
        orc.ppr_refresh()
    # with alternate threads, odd batches run with ORACLE_ALT_THREADS BLAS threads: both thread
    # counts are timed on interleaved batches of the same stream within one budget
    setter = _blas_thread_setter() if alt_threads and alt_threads < ORACLE_THREADS else None
    lat, edges, alt_lat, alt_edges = [], 0, [], 0
    t_start = time.perf_counter()
    for i, b in enumerate(st.batches[warmup:warmup + steps]):
        alt = setter is not None and i % 2 == 1
        if setter is not None:
            setter(alt_threads if alt else ORACLE_THREADS)
        t = time.perf_counter()
        orc.apply_edges(b.src, b.dst, b.op, b.new_nodes)
        orc.ppr_refresh()
        if alt:
            alt_lat.append(time.perf_counter() - t)
            alt_edges += b.k
        else:
            lat.append(time.perf_counter() - t)
            edges += b.k
        if time.perf_counter() - t_start > time_budget_s:
            break
    if setter is not None:
        setter(ORACLE_THREADS)
    total = float(np.sum(lat))
    if save_path:
        n = orc.n
        rows = np.arange(n) if n <= ERR_SAMPLE_ROWS else np.sort(
            np.random.default_rng(c.seed + 5).choice(n, ERR_SAMPLE_ROWS, replace=False))
        np.savez(save_path, X=orc.X()[rows], Y=orc.Y()[rows], Z=orc.Z()[rows], sigma=orc.sigma, rows=rows, n=n,
                 batches=warmup + len(lat) + len(alt_lat), power_iters=oracle_power_iters(c), propagated=not oracle_big(c),
                 pushes=orc.pushes - pushes0)
    threads = ("1 thread" if ORACLE_THREADS == 1 else
               "%d BLAS threads (its push, in C, on one)" % ORACLE_THREADS)
    out = {"value": edges / total, "unit": UNIT, "cores": ORACLE_THREADS, "kind": "oracle", "batches": len(lat),
           "edges": edges, "seconds": total, "init_s": init_s, "pushes": int(orc.pushes - pushes0),
           "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
           "sample": "%s%d batches of the %s stream after %d warm-up batches (%d edges), FP64 oracle, "
                     "%s; initialisation untimed (%.0f s): %d randomized t-SVD power passes, %s"
                     % ("the even ones of the first " if alt_lat else "first ", len(lat) + len(alt_lat), c.name,
                        warmup, edges, threads, init_s, oracle_power_iters(c),
                        "initial PPR propagation skipped (Z_b = r = 0)" if oracle_big(c) else "initial push")}
    if alt_lat:
        out["alt_threads"] = {"cores": alt_threads, "value": alt_edges / float(np.sum(alt_lat)),
                              "batches": len(alt_lat), "edges": alt_edges,
                              "p50_ms": 1e3 * float(np.percentile(alt_lat, 50)),
                              "p99_ms": 1e3 * float(np.percentile(alt_lat, 99)),
                              "sample": "the odd batches of the same window, %d BLAS threads" % alt_threads}
    elif alt_threads and alt_threads < ORACLE_THREADS:
        out["alt_threads"] = {"cores": alt_threads, "value": None,
                              "sample": "not timed: no OpenBLAS thread setter found in the process"}
    return out


def oracle_subprocess(c, steps, budget, save_path=None, wait=True):
    """Runs the oracle leg in a child process (no GPU, its own BLAS threads). With wait=False
    returns the running process; oracle_result() collects it."""
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-worker", "--config", c.name, "--steps", str(steps),
           "--budget", str(budget), "--oracle-threads", str(ORACLE_THREADS)] + (
        ["--save-state", save_path] if save_path else [])
    nt = str(ORACLE_THREADS)
    env = dict(os.environ, OMP_NUM_THREADS=nt, OPENBLAS_NUM_THREADS=nt, MKL_NUM_THREADS=nt, CUDA_VISIBLE_DEVICES="")
    p = subprocess.Popen(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
    return oracle_result(p) if wait else p


def oracle_result(p, timeout=1800):
    try:
        out, err = p.communicate(timeout=timeout)
    except subprocess.TimeoutExpired:
        p.kill()
        out, err = p.communicate()
    for line in (out or "").splitlines()[::-1]:
        if line.startswith("{"):
            return json.loads(line)
    return {"error": (err or out or "")[-400:]}


def err_vs_oracle(c, path, precisions):
    """Replays the oracle's batches on the device (fresh context per precision, the same
    randomized t-SVD passes as the oracle) and compares sigma and, on the oracle's row sample
    (all rows up to ERR_SAMPLE_ROWS), the products X Y^T and Z Y^T: relative errors, the
    Frobenius ones through d x d Grams (|A B^T|_F^2 = tr((A^T A)(B^T B)))."""
    import torch
    from paper_2306_08967_gb300 import DamfGraph, make_config, rsvd_width
    from synth import gaussian_test_matrix
    ref = np.load(path)
    nb = int(ref["batches"])
    dev = torch.device("cuda")
    Xo, Yo, Zo = (torch.from_numpy(ref[k]).to(dev) for k in ("X", "Y", "Z"))
    rows = torch.from_numpy(ref["rows"].astype(np.int32)).to(dev)
    so = ref["sigma"]
    ip, ix, st = make_inputs(c, nb)

    def rel_fro(A, B, Ao, Bo):   # |A B^T - Ao Bo^T|_F / |Ao Bo^T|_F
        gg = torch.trace((A.T @ A) @ (B.T @ B))
        oo = torch.trace((Ao.T @ Ao) @ (Bo.T @ Bo))
        go = torch.trace((A.T @ Ao) @ (Bo.T @ B))
        return float(torch.sqrt(torch.clamp(gg - 2 * go + oo, min=0)) / torch.sqrt(oo))

    out = {"batches": nb, "rows_compared": int(rows.numel()), "rows": int(ref["n"]), "oracle_pushes": int(ref["pushes"]),
           "oracle": "FP64 incremental oracle (the paper's X-form) on the same batches; X Y^T and Z Y^T over the "
                     "rows compared (a seeded sample when the graph has more)"}
    for prec in precisions:
        cfg = make_config(c.n, c.d, c.alpha, c.eps, n_capacity=st.n_final + 16, nnz=len(ix), directed=c.directed,
                          refold_every=256, precision=prec, rsvd_power_iters=int(ref["power_iters"]))
        om = gaussian_test_matrix(c.n, rsvd_width(cfg), seed=c.seed + 2)
        g = DamfGraph(ip, ix, cfg, om)
        p0 = g.stats()["pushes"]
        for b in st.batches[:nb]:
            g.apply_edges_host(b.src, b.dst, b.op, b.new_nodes)
            g.ppr_refresh()
        g.check()
        dev_pushes = g.stats()["pushes"] - p0
        e = g.embeddings(rows=rows)
        X, Y, Z = (e[k].double() for k in ("X", "Y", "Z"))
        sg = e["sigma"].double().cpu().numpy()
        out[prec] = {"sigma_max_rel": float(np.max(np.abs(sg - so) / np.abs(so))),
                     "xyt_rel_fro": rel_fro(X, Y, Xo, Yo)}
        if bool(ref["propagated"]):
            # work against the sequential FIFO push of the oracle on the same batches: a ratio
            # well above 1 would mean redundant pushes inflating the push's algorithmic bytes
            out[prec]["pushes"] = int(dev_pushes)
            out[prec]["pushes_over_oracle_fifo"] = float(dev_pushes) / max(float(ref["pushes"]), 1.0)
        if bool(ref["propagated"]):   # else the oracle skipped its initial propagation: Z is not comparable
            out[prec]["zyt_rel_fro"] = rel_fro(Z, Y, Zo, Yo)
        if bool(ref["propagated"]) and "zyt_eps_bound" not in out:
            # each side's Z is within eps per element of Pi X (in the base space, mapped by P_X):
            # |Z Y^T - Z* Y^T|_F <= |Z - Z*|_F |Y|_2, bounded per side by |r|_F <= eps sqrt(n d)
            # times the largest scale of the base-to-embedding map; reported relative to |Zo Yo^T|_F
            zy = float(torch.sqrt(torch.trace((Zo.T @ Zo) @ (Yo.T @ Yo))))
            yn = float(torch.linalg.matrix_norm(Yo, ord=2))
            out["zyt_fro"] = zy
            out["zyt_eps_bound"] = 2 * c.eps * float(np.sqrt(X.shape[0] * c.d)) * yn * float(
                np.sqrt(np.max(so) / np.min(so[so > 0]))) / zy
        g.close()
        del X, Y, Z, e
    return out


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                out, _ = self.p.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# DRAM bytes (read + write) per k_push launch by workload, from the ncu capture summarised in
# profiles/k_push_<workload>.md; a workload is left out once k_push changes until it is
# captured again
PUSH_DRAM_BYTES = {"C3": 4.226e9}   # mean of the 20 timed launches of a 20-call C3 run (0.71-6.38 ms each)

# ---------------------------------------------------------------- ranks
def reduce_over_ranks(elapsed_ms, edges, world):
    """Replicas (one graph per rank, no collective on the data path): the job's time is the
    slowest rank's, its work the sum of the ranks' edges. Returns (max elapsed, total edges).
    Works on NCCL (CUDA tensors) and gloo (CPU tensors) process groups."""
    if world <= 1:
        return float(elapsed_ms), int(edges)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=dev)
    e = torch.tensor([float(edges)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(e, op=dist.ReduceOp.SUM)
    return float(t.item()), int(round(e.item()))


# ---------------------------------------------------------------- GPU leg
def measure_scoring(g, c, torch):
    """Link-prediction queries on the final state (Sec. 5): damf_score_pairs over 2^20 random
    pairs and damf_topk for 256 queries with k = 64, both with the enhanced context Z and
    symmetric scores on an undirected graph; inputs on the device, CUDA events."""
    n, d = g.n, c.d
    sym = not c.directed
    rng = np.random.default_rng(c.seed + 5)
    src = torch.from_numpy(rng.integers(0, n, 1 << 20).astype(np.int32)).cuda()
    dst = torch.from_numpy(rng.integers(0, n, 1 << 20).astype(np.int32)).cuda()
    rows = torch.from_numpy(rng.integers(0, n, 256).astype(np.int32)).cuda()

    def timed(fn, reps=5):
        for _ in range(2):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    ms_p = timed(lambda: g.score_pairs(src, dst, symmetric=sym))
    ms_t = timed(lambda: g.topk(rows, 64, symmetric=sym))
    g.check()
    npairs = int(src.numel())
    dirs = 2 if sym else 1
    passes = (int(rows.numel()) + 31) // 32
    return {
        "score_pairs": {"pairs": npairs, "ms": ms_p, "pairs_per_s": npairs / (ms_p / 1e3),
                        "fp32_tflops": npairs * dirs * 2 * (d * d + d) / (ms_p / 1e3) / 1e12},
        "topk": {"queries": int(rows.numel()), "k": 64, "ms": ms_t, "queries_per_s": rows.numel() / (ms_t / 1e3),
                 "scan_gb_per_s": passes * dirs * n * d * 4 / (ms_t / 1e3) / 1e9,
                 "fp32_tflops": rows.numel() * n * dirs * 2 * d / (ms_t / 1e3) / 1e12},
    }


def run_node_stream(args, c):
    """The paper's node-arrival protocol (Sec. 5.1): the graph induced on the first n0 nodes,
    then nodes arriving one at a time with their edges (one damf_apply_edges with
    new_nodes = 1, then damf_ppr_refresh, per node event). Timed on the last `steps` arrivals,
    i.e. at nearly full graph size, after `warmup` untimed arrivals."""
    import torch
    from paper_2306_08967_gb300 import DamfGraph, make_config, rsvd_width
    from synth import chung_lu_graph, gaussian_test_matrix, node_arrival_stream
    K, W = args.steps, args.warmup
    ip, ix, _ = chung_lu_graph(c.n, c.avg_deg, c.gamma, seed=c.seed, directed=c.directed)
    n0 = c.n - K - W
    ip0, ix0, st = node_arrival_stream(ip, ix, n0, directed=c.directed)
    cfg = make_config(n0, c.d, c.alpha, c.eps, n_capacity=c.n + 16, nnz=len(ix), directed=c.directed,
                      refold_every=args.refold_every, precision=args.precision)
    om = gaussian_test_matrix(n0, rsvd_width(cfg), seed=c.seed + 2)
    g = DamfGraph(ip0, ix0, cfg, om)
    dev = torch.device("cuda")
    bs = st.batches
    ks = np.array([b.k for b in bs], np.int64)
    off = np.concatenate([[0], np.cumsum(ks)])
    src = torch.from_numpy(np.concatenate([b.src for b in bs])).to(dev)
    dst = torch.from_numpy(np.concatenate([b.dst for b in bs])).to(dev)
    opv = torch.from_numpy(np.concatenate([b.op for b in bs])).to(dev)
    lib, h = g.lib, g.h
    sp = __import__("ctypes").c_void_p
    stream = torch.cuda.current_stream()
    sptr = sp(stream.cuda_stream)

    def step(i):
        o = int(off[i])
        if lib.damf_apply_edges(h, sp(src.data_ptr() + 4 * o), sp(dst.data_ptr() + 4 * o), sp(opv.data_ptr() + o),
                                int(ks[i]), 1, sptr) != 0 or lib.damf_ppr_refresh(h, sptr) != 0:
            raise RuntimeError(g.lib.damf_last_error(h))

    for i in range(W):
        step(i)
    g.check()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    for e in ev1:
        e.record(stream)
    torch.cuda.synchronize()
    with ClockSampler(dev.index or 0) as clk:
        for j in range(K):
            ev0[j].record(stream)
            step(W + j)
            g.record_event(ev1[j])
        torch.cuda.synchronize()
    g.check()
    lat = np.array([ev0[j].elapsed_time(ev1[j]) for j in range(K)])
    total_ms = float(ev0[0].elapsed_time(ev1[K - 1]))
    edges = int(ks[W:W + K].sum())
    out = {"metric": "ms per node event (the paper's node-arrival protocol)", "value": total_ms / K,
           "unit": "ms/event", "higher_is_better": False, "n_gpus": 1, "steps": K, "warmup": W,
           "events_per_s": K / (total_ms / 1e3), "edge_updates_per_s": edges / (total_ms / 1e3),
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
           "dtype": "f32", "data": "synthetic (seeded Chung-Lu graph, node ids in random order)",
           "config": {"workload": workload_desc(c) + "; node arrivals from n0 = %d, one call + one push per "
                                                     "node, the last %d arrivals timed" % (n0, K),
                      "precision": args.precision, "mean_degree_of_arrivals": edges / K},
           "clocks": clk.summary(),
           "paper_context": "the paper reports about 10 ms per update on Twitter (41.7M nodes) with 8 CPU threads"}
    g.close()
    return out


def run_ours(args, c, rank, world):
    import torch
    from paper_2306_08967_gb300 import DamfGraph, make_config, rsvd_width
    from synth import gaussian_test_matrix

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    K, W, E = args.steps, args.warmup, args.e2e_steps
    if rank > 0:   # replicas: every rank its own graph and stream of the same shape
        c = dataclasses.replace(c, seed=c.seed + 1000 * rank)
    ip, ix, st = make_inputs(c, W + K + E)
    cfg = make_config(c.n, c.d, c.alpha, c.eps, n_capacity=st.n_final + 16, nnz=len(ix), directed=c.directed,
                      refold_every=args.refold_every, precision=args.precision)
    om = gaussian_test_matrix(c.n, rsvd_width(cfg), seed=c.seed + 2)
    t0 = time.perf_counter()
    g = DamfGraph(ip, ix, cfg, om)
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t0
    if args.push_blocks or args.push_chunks >= 0:
        g.set_tuning(args.push_blocks, args.push_chunks)
    # device-resident inputs for every step
    batches = st.batches
    ks = np.array([b.k for b in batches], np.int64)
    off = np.concatenate([[0], np.cumsum(ks)])
    src = torch.from_numpy(np.concatenate([b.src for b in batches])).to(dev)
    dst = torch.from_numpy(np.concatenate([b.dst for b in batches])).to(dev)
    opv = torch.from_numpy(np.concatenate([b.op for b in batches])).to(dev)
    lib, h = g.lib, g.h
    sp = __import__("ctypes").c_void_p
    stream = torch.cuda.current_stream()
    sptr = sp(stream.cuda_stream)

    def step(i):
        o = int(off[i])
        st_ = lib.damf_apply_edges(h, sp(src.data_ptr() + 4 * o), sp(dst.data_ptr() + 4 * o), sp(opv.data_ptr() + o),
                                   int(ks[i]), int(batches[i].new_nodes), sptr)
        if st_ != 0:
            raise RuntimeError("apply_edges status %d" % st_)
        st_ = lib.damf_ppr_refresh(h, sptr)
        if st_ != 0:
            raise RuntimeError("ppr_refresh status %d" % st_)

    for i in range(W):
        step(i)
    g.check()
    s0 = g.stats()
    g.set_timing(True)
    g.timing()
    # per step: an event on the caller stream before the step's apply and an event on the
    # library's push stream after the step's push; latency = push completion - start
    ev_start = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev_done = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    for e in ev_done:
        e.record(stream)            # creates the event; re-recorded on the push stream below
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        for j in range(K):
            ev_start[j].record(stream)
            step(W + j)
            g.record_event(ev_done[j])
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    g.check()
    lat_ms = np.array([ev_start[j].elapsed_time(ev_done[j]) for j in range(K)])
    elapsed_ms = float(ev_start[0].elapsed_time(ev_done[K - 1]))
    step_ms = np.diff(np.array([0.0] + [ev_start[0].elapsed_time(ev_done[j]) for j in range(K)]))
    if args.log_jsonl and rank == 0:
        # one line per timed batch, from the events recorded in the timed region (nothing is
        # read from the device per step)
        with open(args.log_jsonl, "w") as f:
            for j in range(K):
                b = batches[W + j]
                f.write(json.dumps({"step": j, "edges": b.k, "new_nodes": b.new_nodes,
                                    "deletions": int((b.op < 0).sum()), "latency_ms": float(lat_ms[j]),
                                    "interval_ms": float(step_ms[j])}) + "\n")
    stage = g.timing()
    g.set_timing(False)
    s1 = g.stats()
    edges = int(ks[W:W + K].sum())
    elapsed_ms, total_edges = reduce_over_ranks(elapsed_ms, edges, world)
    value = total_edges / (elapsed_ms / 1e3)

    # e2e: host buffers through damf_apply_edges_host, a D2H read of sigma every step
    sig = torch.empty(c.d, dtype=torch.float32).pin_memory()
    torch.cuda.synchronize()
    t_e = time.perf_counter()
    e2e_edges, h2d = 0, 0
    for j in range(E):
        b = batches[W + K + j]
        g.apply_edges_host(b.src, b.dst, b.op, b.new_nodes)
        g.ppr_refresh()
        sig.copy_(g.embeddings(want=("sigma",))["sigma"], non_blocking=True)
        torch.cuda.current_stream().synchronize()
        e2e_edges += b.k
        h2d += b.k * 9
    e2e_s = max(time.perf_counter() - t_e, 1e-9)
    g.check()

    # error of the run: drift of the effective bases from orthonormality (U = Ub PU)
    stt = g.state()
    U = stt["Ub"].double() @ stt["PU"].double()
    V = stt["Vb"].double() @ stt["PV"].double()
    eye = torch.eye(c.d, dtype=torch.float64, device=dev)
    err = {"U_orth_max": float((U.T @ U - eye).abs().max()), "V_orth_max": float((V.T @ V - eye).abs().max())}
    sigma_final = stt["sigma"].double().cpu().numpy()
    del U, V, stt

    # roofline of the dominant kernel, from live events and device counters
    d = c.d
    B = 4 * d
    pushes = s1["pushes"] - s0["pushes"]
    push_edges = s1["push_edges"] - s0["push_edges"]
    push_bytes = pushes * 3 * B + push_edges * (8 + 2 * B)
    stage_ms = {k: v[0] for k, v in stage.items()}
    dominant = max(stage_ms, key=stage_ms.get)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    push_launches = stage["push"][1]
    push_ms_per = stage_ms["push"] / max(push_launches, 1)
    achieved = (push_bytes / max(push_launches, 1)) / (push_ms_per * 1e-3) / 1e9 if push_launches else 0.0
    roof = {"bound": "hbm", "kernel": "k_push", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
            "frac": round(achieved / hbm_peak, 4), "traffic": PUSH_DRAM_BYTES.get(c.name),
            "traffic_note": "dram read + write per launch of the current k_push from an ncu capture "
                            "(profiles/k_push_%s.md), null when none was taken of it" % c.name,
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "bytes_per_launch": push_bytes / max(push_launches, 1), "ms_per_launch": push_ms_per}
    launches = s1["launches"] - s0["launches"]
    scoring = measure_scoring(g, c, torch) if args.scoring else None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": elapsed_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded Chung-Lu graph and edge stream)",
        "config": {"workload": workload_desc(c), "precision": args.precision, "edges_timed": edges,
                   "push_shape": g.tuning(),
                   "l2": "state %.2f GB (Ub, Vb, Zb, r) > 129 MB L2; no flush" % (4 * st.n_final * d * 4 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single GPU", "refold_every": args.refold_every},
        "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99)),
                       "mean": float(lat_ms.mean()),
                       "definition": "per batch: caller-stream event before its apply to push-stream event after "
                                     "its push (batches back to back, so queueing behind the previous batch counts)"},
        "step_interval_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "e2e": {"value": e2e_edges / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d / max(E, 1),
                "d2h_bytes_per_step": 4 * d, "steps": E},
        "gpu_launches": int(launches),
        "roofline": roof,
        "stage_ms": {k: round(v, 3) for k, v in stage_ms.items()},
        "dominant_stage": dominant,
        "scoring": scoring,
        "counters": {"pushes": pushes, "push_edges": push_edges, "updates": s1["updates"] - s0["updates"],
                     "folds": s1["folds"] - s0["folds"],
                     "push_rounds": s1["push_rounds"] - s0["push_rounds"],
                     "touched_rows": s1["touched_rows"] - s0["touched_rows"], "last_sweeps": s1["last_sweeps"],
                     "jacobi_sweeps": s1["jacobi_sweeps"] - s0["jacobi_sweeps"],
                     "jacobi_full": s1["jacobi_full"] - s0["jacobi_full"],
                     "jacobi_gersh": s1["jacobi_gersh"] - s0["jacobi_gersh"],
                     "push_tasks": s1["push_tasks"] - s0["push_tasks"],
                     "push_items": s1["push_items"] - s0["push_items"],
                     "push_phase_ms": {k: (s1["push_ns"][i] - s0["push_ns"][i]) / 1e6 for i, k in
                                       enumerate(["seeding", "task_loop", "barriers", "idle_per_warp"])}},
        "init_s": init_s,
        "clocks": clk.summary(),
        "err": err,
        "_sigma": sigma_final.tolist(),
    }
    g.close()
    return out


def run_fleet(args, fw, rank, world):
    """Many graphs per step (one batch each) through a fleet (damf_fleet_step: every graph's
    update on its own stream, then one grouped push of all graphs), each step one CUDA graph
    replay after the push shares are autotuned; beside it the same step issued graph by graph
    on one stream, by direct damf_step_multi calls (one cooperative push per graph) and by
    direct (uncaptured) fleet steps."""
    import ctypes
    import torch
    from paper_2306_08967_gb300 import DamfFleet, DamfGraph, _lib, make_config, rsvd_width
    from paper_2306_08967_gb300.api import batch_array
    from paper_2306_08967_gb300.autotune import DEFAULT_DIRECT_CHUNKS, DEFAULT_EXPONENTS, tune_shares
    from synth import fleet_inputs, gaussian_test_matrix

    members = fw.members()
    if args.graphs:
        members = members[: args.graphs]
    if rank > 0:   # replicas: every rank its own fleet of the same shape
        members = [dataclasses.replace(c, seed=c.seed + 1000 * rank) for c in members]
    K, W, E, S, T = args.steps, args.warmup, args.e2e_steps, args.compare_steps, args.tune_steps
    rebalance_rounds = 3
    n_cand = len(DEFAULT_EXPONENTS) + len(DEFAULT_DIRECT_CHUNKS) + 1 + rebalance_rounds
    # warm-up, tuning (T per candidate), the three comparison forms, one untimed replay, timed, e2e,
    # phase-timed direct steps
    n_steps = W + T * n_cand + 3 * S + 1 + K + E + S
    t0 = time.perf_counter()
    data = fleet_inputs(members, n_steps, 1 if world > 1 else 0)
    gen_s = time.perf_counter() - t0
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    t0 = time.perf_counter()
    graphs = []
    for c, ip, ix, st in data:
        cfg = make_config(c.n, c.d, c.alpha, c.eps, n_capacity=c.n, nnz=len(ix), refold_every=0,
                          precision=args.precision)
        graphs.append(DamfGraph(ip, ix, cfg, gaussian_test_matrix(c.n, rsvd_width(cfg), seed=c.seed + 2)))
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t0
    G, KMAX = len(graphs), fw.k_hi
    # every step's events on the device, padded to KMAX per graph: [step][graph][KMAX]
    src = np.zeros((n_steps, G, KMAX), np.int32)
    dst = np.zeros((n_steps, G, KMAX), np.int32)
    opv = np.zeros((n_steps, G, KMAX), np.int8)
    cnt = np.zeros((n_steps, G), np.int32)
    for gi, (c, ip, ix, st) in enumerate(data):
        for t, b in enumerate(st.batches):
            src[t, gi, :b.k], dst[t, gi, :b.k], opv[t, gi, :b.k] = b.src, b.dst, b.op
            cnt[t, gi] = b.k
    d_src, d_dst = torch.from_numpy(src).to(dev), torch.from_numpy(dst).to(dev)
    d_op, d_cnt = torch.from_numpy(opv).to(dev), torch.from_numpy(cnt).to(dev)
    # the fixed buffers a captured step reads
    b_src, b_dst = torch.zeros((G, KMAX), dtype=torch.int32, device=dev), torch.zeros((G, KMAX), dtype=torch.int32,
                                                                                      device=dev)
    b_op, b_cnt = torch.zeros((G, KMAX), dtype=torch.int8, device=dev), torch.zeros(G, dtype=torch.int32, device=dev)
    sig = torch.zeros((G, 128), dtype=torch.float32, device=dev)
    batches = [(g, b_src[i], b_dst[i], b_op[i], 0, b_cnt[i:i + 1]) for i, g in enumerate(graphs)]
    arr = batch_array(batches)
    lib = _lib.load()
    fs = torch.cuda.Stream(device=dev)
    fptr = ctypes.c_void_p(fs.cuda_stream)
    pos = [0]

    def load(t):   # step t's events into the fixed buffers (device to device)
        b_src.copy_(d_src[t], non_blocking=True)
        b_dst.copy_(d_dst[t], non_blocking=True)
        b_op.copy_(d_op[t], non_blocking=True)
        b_cnt.copy_(d_cnt[t], non_blocking=True)

    def next_step():
        t = pos[0]
        pos[0] += 1
        return t

    fleet = DamfFleet(graphs)

    def capture():
        with torch.cuda.stream(fs):
            for g in graphs:
                g.join(fs)
        fs.synchronize()
        cg = torch.cuda.CUDAGraph()
        l0 = sum(g.stats()["launches"] for g in graphs) + fleet.launches
        with torch.cuda.graph(cg, stream=fs, capture_error_mode="relaxed"):
            fleet.step_array(arr, fs)
        cg.kernels = sum(g.stats()["launches"] for g in graphs) + fleet.launches - l0
        return cg

    def run_captured(cg, steps, record=None):
        with torch.cuda.stream(fs):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(fs)
            for j in range(steps):
                t = next_step()
                if record is not None:
                    record[0][j].record(fs)
                load(t)
                cg.replay()
                if record is not None:
                    record[1][j].record(fs)
            ev1.record(fs)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / max(steps, 1)

    # warm-up: direct fleet steps under the default shares
    with torch.cuda.stream(fs):
        for _ in range(W):
            load(next_step())
            fleet.step_array(arr, fs)
    fs.synchronize()
    for g in graphs:
        g.check()

    # the same step issued graph by graph on one stream (each graph's push joined before the
    # next graph's update), then by direct damf_step_multi calls, both with the default shape
    def run_sequential(steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(fs):
            ev0.record(fs)
            for _ in range(steps):
                t = next_step()
                load(t)
                for i, g in enumerate(graphs):
                    k = int(cnt[t, i])
                    g.apply_edges(b_src[i, :k], b_dst[i, :k], b_op[i, :k], stream=fs)
                    g.ppr_refresh(stream=fs)
                    g.join(fs)
            ev1.record(fs)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / max(steps, 1)

    def run_direct(steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(fs):
            ev0.record(fs)
            for _ in range(steps):
                load(next_step())
                if lib.damf_step_multi(arr, G, fptr) != 0:
                    raise RuntimeError("step_multi")
            ev1.record(fs)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / max(steps, 1)

    def run_fleet_direct(steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(fs):
            ev0.record(fs)
            for _ in range(steps):
                load(next_step())
                fleet.step_array(arr, fs)
            ev1.record(fs)
        ev1.synchronize()
        return ev0.elapsed_time(ev1) / max(steps, 1)

    seq_ms = run_sequential(S)
    direct_ms = run_direct(S)
    fleet_direct_ms = run_fleet_direct(S)

    # autotune the push shares on real steps (each candidate recaptured, one untimed replay)
    def measure():
        cg = capture()
        run_captured(cg, 1)
        return run_captured(cg, T - 1)

    last = {"ns": None, "pos": 0}

    def push_times():   # each graph's push time per step (ns, its own global timer) since the last call
        cur = np.array([float(sum(g.stats()["push_ns"][:3])) for g in graphs])
        prev, p0 = last["ns"], last["pos"]
        last["ns"], last["pos"] = cur, pos[0]
        if prev is None:
            return [1.0] * G
        return list((cur - prev) / max(pos[0] - p0, 1))

    t0 = time.perf_counter()
    tune = tune_shares(fleet, graphs, measure, push_times=push_times, rebalance_rounds=rebalance_rounds,
                       cache=args.tune_cache) if T >= 2 else None
    tune_s = time.perf_counter() - t0
    cg = capture()
    run_captured(cg, 1)
    for g in graphs:
        g.check()

    # timed: K captured steps
    ev_a = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev_b = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    t_first = pos[0]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clk:
        run_captured(cg, K, (ev_a, ev_b))
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    for g in graphs:
        g.check()
    launches = cg.kernels * K
    lat_ms = np.array([ev_a[j].elapsed_time(ev_b[j]) for j in range(K)])
    elapsed_ms = float(ev_a[0].elapsed_time(ev_b[K - 1]))
    edges = int(cnt[t_first:t_first + K].sum())
    elapsed_all, total_edges = reduce_over_ranks(elapsed_ms, edges, world)
    value = total_edges / (elapsed_all / 1e3)

    # e2e: each step's events from pinned host memory, the captured step, every graph's
    # sigma read back to the host
    h_src = torch.empty((G, KMAX), dtype=torch.int32).pin_memory()
    h_dst = torch.empty((G, KMAX), dtype=torch.int32).pin_memory()
    h_op = torch.empty((G, KMAX), dtype=torch.int8).pin_memory()
    h_cnt = torch.empty(G, dtype=torch.int32).pin_memory()
    h_sig = torch.empty((G, 128), dtype=torch.float32).pin_memory()
    with torch.cuda.stream(fs):
        for g in graphs:
            g.join(fs)
    fs.synchronize()
    rg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(rg, stream=fs, capture_error_mode="relaxed"):
        for i, g in enumerate(graphs):
            if lib.damf_get_embeddings(g.h, None, 0, None, None, None, ctypes.c_void_p(sig[i].data_ptr()), fptr):
                raise RuntimeError("readout capture")
    e2e_edges = 0
    torch.cuda.synchronize()
    t_e = time.perf_counter()
    for _ in range(E):
        t = next_step()
        h_src.numpy()[:] = src[t]
        h_dst.numpy()[:] = dst[t]
        h_op.numpy()[:] = opv[t]
        h_cnt.numpy()[:] = cnt[t]
        with torch.cuda.stream(fs):
            b_src.copy_(h_src, non_blocking=True)
            b_dst.copy_(h_dst, non_blocking=True)
            b_op.copy_(h_op, non_blocking=True)
            b_cnt.copy_(h_cnt, non_blocking=True)
            cg.replay()
            rg.replay()
            h_sig.copy_(sig, non_blocking=True)
        fs.synchronize()
        e2e_edges += int(cnt[t].sum())
    e2e_s = max(time.perf_counter() - t_e, 1e-9)
    for g in graphs:
        g.check()

    # phase split and push roofline from S more steps issued directly with the fleet's phase
    # timing (events at the fork, after every update, after the grouped push); the push's
    # algorithmic bytes come from the graphs' push counters over the same steps
    fleet.set_timing(True)
    s2 = [g.stats() for g in graphs]
    run_fleet_direct(S)
    tm = fleet.timing()
    fleet.set_timing(False)
    s3 = [g.stats() for g in graphs]
    for g in graphs:
        g.check()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    push_bytes, pushes, push_edges = 0.0, 0, 0
    for g, a, b in zip(graphs, s2, s3):
        B = 4 * g.d
        dp, de = b["pushes"] - a["pushes"], b["push_edges"] - a["push_edges"]
        pushes, push_edges = pushes + dp, push_edges + de
        push_bytes += dp * 3 * B + de * (8 + 2 * B)
    shares, n_launch = fleet.shares()
    push_ms_per = tm["push_ms"] / max(tm["steps"], 1)
    achieved = (push_bytes / max(tm["steps"], 1)) / max(push_ms_per * 1e-3, 1e-12) / 1e9
    d_mix = {dd: sum(1 for g in graphs if g.d == dd) for dd in (32, 64, 128)}
    n_all = np.array([g.n for g in graphs])
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": elapsed_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded Chung-Lu graphs and edge streams)",
        "config": {"workload": "%s: %d undirected Chung-Lu graphs, gamma %.1f, n log-uniform in [%d, %d] (total %d), "
                               "mean degree U[%g, %g], d %s; one batch of U[%d, %d] edge events per graph per step, "
                               "%.0f%% deletions; alpha %g eps %g"
                               % (fw.name, G, fw.gamma, fw.n_lo, fw.n_hi, int(n_all.sum()), fw.deg_lo, fw.deg_hi,
                                  d_mix, fw.k_lo, fw.k_hi, 100 * fw.p_del, fw.alpha, fw.eps),
                   "precision": args.precision, "edges_timed": edges, "launch": "one CUDA graph replay per step (damf_fleet_step "
                   "captured: every graph's update on its own stream, then one grouped cooperative push of all "
                   "graphs)",
                   "l2": "state of all graphs > 129 MB L2; no flush",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "latency_ms": {"p50": float(np.percentile(lat_ms, 50)), "p99": float(np.percentile(lat_ms, 99)),
                       "definition": "per step (all graphs' batches): event before the step's event copy to event "
                                     "after its replay (every graph's update and push done)"},
        "compare_ms_per_step": {"graph_by_graph_one_stream": seq_ms,
                                "step_multi_direct (one cooperative push per graph)": direct_ms,
                                "fleet_direct_default_shares": fleet_direct_ms,
                                "fleet_captured_tuned": elapsed_ms / K, "steps_each": S},
        "autotune": dict(tune or {}, seconds=tune_s, steps_per_candidate=T),
        "e2e": {"value": e2e_edges / e2e_s, "unit": UNIT,
                "h2d_bytes_per_step": G * KMAX * 9 + 4 * G, "d2h_bytes_per_step": G * 128 * 4, "steps": E},
        "gpu_launches": int(launches),
        "kernel_nodes_per_captured_step": int(cg.kernels),
        "gpu_launches_note": "kernels per captured step (counted while capturing) x timed steps",
        "roofline": {"bound": "hbm", "kernel": "k_push_group", "achieved": round(achieved, 1), "peak": hbm_peak,
                     "unit": "GB/s", "frac": round(achieved / hbm_peak, 4), "traffic": None,
                     "note": "achieved = algorithmic push bytes of all graphs per step / the grouped push's "
                             "device time per step (events around the push phase of %d direct fleet steps)"
                             % tm["steps"],
                     "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                     "grouped_launches_per_step": n_launch, "pushes": pushes, "push_edges": push_edges,
                     "bytes_per_step": push_bytes / max(tm["steps"], 1), "ms_per_step": push_ms_per},
        "phase_ms_per_step": {"updates": tm["update_ms"] / max(tm["steps"], 1), "push": push_ms_per,
                              "note": "direct fleet steps: fork to the last graph's update done; then the "
                                      "grouped push"},
        "shares": {"owners": int(sum(1 for b in shares if b > 0)), "sharing_a_cta": int(sum(1 for b in shares
                                                                                          if b == 0)),
                   "max_ctas": int(max(shares))},
        "init_s": init_s, "generate_s": gen_s,
        "clocks": clk.summary(),
    }
    fleet.close()
    for g in graphs:
        g.close()
    return out


def gpu_chung_lu_directed(n, m, gamma, seed):
    """A directed Chung-Lu graph generated on the device (torch), for sizes whose host
    generation would take tens of minutes: node i has expected out- and in-degree proportional
    to (i + 1)^(-1 / (gamma - 1)) (in-weights on a seeded random permutation of the nodes),
    m distinct edges without self-loops (endpoint pairs drawn by inverse-CDF sampling, then
    deduplicated and, if more than m remain, a seeded uniform subset of m kept). Returns the
    CSR (row_ptr int32[n + 1], col int32[m]) on the device, rows sorted."""
    import torch
    dev = torch.device("cuda")
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    w = torch.arange(1, n + 1, device=dev, dtype=torch.float64).pow_(-1.0 / (gamma - 1.0))
    cdf = torch.cumsum(w, 0)
    cdf /= cdf[-1].clone()
    del w
    perm = torch.randperm(n, device=dev, generator=gen)
    keys = []
    drawn = int(m * 1.10)
    chunk = 1 << 27
    for lo in range(0, drawn, chunk):
        k = min(chunk, drawn - lo)
        u = torch.searchsorted(cdf, torch.rand(k, device=dev, dtype=torch.float64, generator=gen))
        iv = torch.searchsorted(cdf, torch.rand(k, device=dev, dtype=torch.float64, generator=gen))
        v = perm[iv.clamp_(max=n - 1)]
        del iv
        u.clamp_(max=n - 1)
        keep = u != v
        keys.append(u[keep] * n + v[keep])
        del u, v, keep
    del cdf, perm
    keys = torch.cat(keys)
    keys, _ = torch.sort(keys)
    keys = torch.unique_consecutive(keys)
    if keys.numel() > m:
        pick = torch.randperm(keys.numel(), device=dev, generator=gen)[:m]
        pick, _ = torch.sort(pick)
        keys = keys[pick]
        del pick
    rows = keys // n
    col = (keys - rows * n).to(torch.int32)
    del keys
    counts = torch.bincount(rows, minlength=n)
    del rows
    row_ptr = torch.zeros(n + 1, device=dev, dtype=torch.int64)
    row_ptr[1:] = torch.cumsum(counts, 0)
    del counts
    torch.cuda.empty_cache()
    return row_ptr.to(torch.int32), col


def run_init_scale(args):
    """The randomized t-SVD initialisation (Algorithm 3) at the serving workload's stated size
    (one directed Chung-Lu graph of --nodes nodes and --edges edges, d = 128), then a short
    stream of update requests of 1-1024 events (10% deletions of present edges) on that graph,
    each followed by its push. The graph and the Gaussian test matrix are drawn on the device
    (seeded). Too large for the FP64 oracle (its initialisation's parity is pinned at small n
    by the GPU tests), so the factors are checked by properties that hold at any size: the
    orthonormality of U and V and the relative residuals |A v_i - sigma_i u_i| / sigma_i of
    the leading singular triplets (A the out-adjacency, FP32 sparse products)."""
    import torch
    from paper_2306_08967_gb300 import DamfGraph, bytes_required, make_config, rsvd_width
    dev = torch.device("cuda")
    n, m, d = int(args.nodes), int(args.edges), 128
    t0 = time.perf_counter()
    row_ptr, col = gpu_chung_lu_directed(n, m, args.gamma, args.seed)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    m_real = int(col.numel())
    extra = 64
    cfg = make_config(n, d, 0.15, 1e-5, n_capacity=n + extra, nnz=m_real,
                      m_capacity=int(1.15 * m_real) + 8 * (n + extra), directed=True, refold_every=256,
                      precision=args.precision)
    need = bytes_required(cfg)
    gen = torch.Generator(device=dev)
    gen.manual_seed(args.seed + 2)
    om = torch.randn((n, rsvd_width(cfg)), device=dev, dtype=torch.float32, generator=gen)
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    free0, total = torch.cuda.mem_get_info()
    t1 = time.perf_counter()
    g = DamfGraph(row_ptr, col, cfg, om)
    g.check()
    init_s = time.perf_counter() - t1
    del om
    torch.cuda.empty_cache()
    free1, _ = torch.cuda.mem_get_info()
    st0 = g.stats()
    # properties of the initial factors
    e = g.embeddings(want=("X", "Y", "sigma"))
    sig = e["sigma"].double()
    rs = torch.rsqrt(e["sigma"].clamp_min(1e-30))
    GU = torch.zeros((d, d), dtype=torch.float64, device=dev)
    GV = torch.zeros((d, d), dtype=torch.float64, device=dev)
    step = 1 << 22
    for lo in range(0, n, step):
        Uc = (e["X"][lo:lo + step] * rs).double()
        Vc = (e["Y"][lo:lo + step] * rs).double()
        GU += Uc.T @ Uc
        GV += Vc.T @ Vc
        del Uc, Vc
    eye = torch.eye(d, dtype=torch.float64, device=dev)
    orth = (float((GU - eye).abs().max()), float((GV - eye).abs().max()))
    k = 8
    A = torch.sparse_csr_tensor(row_ptr, col, torch.ones(m_real, device=dev, dtype=torch.float32), size=(n, n))
    Vk = (e["Y"][:, :k] * rs[:k]).contiguous()
    AV = A @ Vk
    Uk = e["X"][:, :k] * rs[:k]
    res = [float(torch.linalg.vector_norm((AV[:, i] - e["sigma"][i] * Uk[:, i]).double()) / sig[i]) for i in range(k)]
    av_norm = [float(torch.linalg.vector_norm(AV[:, i].double())) for i in range(k)]
    del A, Vk, AV, Uk, e
    torch.cuda.empty_cache()
    # a stream of update requests on the big graph: U[1, 1024] events, 10% deletions of present
    # edges, insertions with endpoints drawn by the generator's weight law (host, seeded)
    rng = np.random.default_rng(args.seed + 3)
    w = np.arange(1, n + 1, dtype=np.float64) ** (-1.0 / (args.gamma - 1.0))
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    del w
    K, W = int(args.steps), int(args.warmup)
    reqs = []
    rp64 = row_ptr.long()
    for _ in range(K + W):
        kk = int(rng.integers(1, 1025))
        nd = int(rng.binomial(kk, 0.10))
        ni = kk - nd
        su = np.minimum(np.searchsorted(cdf, rng.random(ni)), n - 1)
        sv = np.minimum(np.searchsorted(cdf, rng.random(ni)), n - 1)
        sv = np.where(sv == su, (sv + 1) % n, sv)
        pos = torch.from_numpy(rng.integers(0, m_real, nd)).to(dev)
        du = (torch.searchsorted(rp64, pos, right=True) - 1).cpu().numpy()
        dv = col[pos].long().cpu().numpy()
        src = np.concatenate([su, du]).astype(np.int32)
        dst = np.concatenate([sv, dv]).astype(np.int32)
        op = np.concatenate([np.ones(ni, np.int8), -np.ones(nd, np.int8)])
        reqs.append((src, dst, op))
    del cdf, rp64
    stream = torch.cuda.current_stream()
    for i in range(W):
        g.apply_edges(*reqs[i])
        g.ppr_refresh()
    g.check()
    s1 = g.stats()
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    for e1 in ev1:
        e1.record(stream)   # creates the events the library records into
    torch.cuda.synchronize()
    with ClockSampler(dev.index or 0) as clk:
        for j in range(K):
            ev0[j].record(stream)
            g.apply_edges(*reqs[W + j])
            g.ppr_refresh()
            g.record_event(ev1[j])
        torch.cuda.synchronize()
    g.check()
    s2 = g.stats()
    lat = np.array([ev0[j].elapsed_time(ev1[j]) for j in range(K)])
    total_ms = float(ev0[0].elapsed_time(ev1[K - 1]))
    edges = int(sum(len(r[0]) for r in reqs[W:]))
    out = {"metric": "randomized t-SVD initialisation time at the serving workload's size, then update latency",
           "value": init_s, "unit": "s", "higher_is_better": False, "n_gpus": 1, "dtype": "f32",
           "data": "synthetic (directed Chung-Lu graph and Gaussian test matrix drawn on the device, seeded)",
           "config": {"workload": "directed Chung-Lu gamma=%.1f n=%d m=%d (requested %d); d=128 alpha=0.15 "
                                  "eps=1e-5; %d randomized t-SVD power passes" % (args.gamma, n, m_real, m,
                                                                                  cfg.rsvd_power_iters),
                      "precision": args.precision},
           "generate_s": gen_s, "init_s": init_s,
           "init_pushes": int(st0["pushes"]), "init_push_edges": int(st0["push_edges"]),
           "device_bytes_required": int(need), "device_bytes_used_by_context": int(free0 - free1),
           "device_total_bytes": int(total),
           "checks": {"U_orth_max": orth[0], "V_orth_max": orth[1],
                      "sigma_top": [float(x) for x in sig[:k].tolist()],
                      "residual_rel_top": res, "norm_Av_top": av_norm,
                      "note": "|A v_i - sigma_i u_i| / sigma_i for the leading singular triplets (A the "
                              "out-adjacency, FP32 sparse product) and max |U^T U - I|, |V^T V - I| (FP64 "
                              "sums); the initialisation's parity with the FP64 oracle is pinned at small n "
                              "by tests/test_gpu_parity.py::test_init_matches_oracle"},
           "updates": {"requests": K, "warmup": W, "edges": edges, "edge_updates_per_s": edges / (total_ms / 1e3),
                       "ms_per_request": total_ms / K,
                       "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
                       "updates": int(s2["updates"] - s1["updates"]), "pushes": int(s2["pushes"] - s1["pushes"]),
                       "definition": "requests of U[1, 1024] events back to back on one stream; latency from an "
                                     "event before the apply to an event after the push"},
           "clocks": clk.summary()}
    g.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--config", default="C3")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--refold-every", type=int, default=256)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp32"])
    ap.add_argument("--no-compare-precision", dest="compare_precision", action="store_false",
                    help="skip timing both precisions over a longer window of the same workload")
    ap.add_argument("--precision-steps", type=int, default=300,
                    help="steps of each precision's window in the comparison (C3: ~800 updates, three folds)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-scoring", dest="scoring", action="store_false",
                    help="skip the link-prediction query timing (score_pairs, topk) after the run")
    ap.add_argument("--cpu-budget", type=float, default=30.0,
                    help="seconds of timed oracle work in the cpu_baseline leg (both thread counts)")
    ap.add_argument("--oracle-worker", action="store_true")
    ap.add_argument("--oracle-threads", type=int, default=max(1, os.cpu_count() or 1),
                    help="BLAS threads of the timed oracle (cpu_baseline and --impl reference); default: every "
                         "host core (its push, in C, runs on one)")
    ap.add_argument("--budget", type=float, default=20.0)
    ap.add_argument("--save-state", default=None)
    ap.add_argument("--log-jsonl", default=None, help="write one JSON line per timed batch (edges, latency) here; "
                    "C5: one per server step (issue and completion time, requests, edges, graphs)")
    ap.add_argument("--push-blocks", type=int, default=0, help="push CTAs (0: the library's default, 2.5 per SM)")
    ap.add_argument("--push-chunks", type=int, default=-1,
                    help="in-edge chunks a row task scatters itself before its row becomes hub items (-1: 8)")
    ap.add_argument("--graphs", type=int, default=0, help="C4: the first this many graphs of the fleet (0: all)")
    ap.add_argument("--compare-steps", type=int, default=5, help="C4: steps of each comparison launch form")
    ap.add_argument("--tune-steps", type=int, default=3, help="C4: steps per autotuner candidate (< 2: no tuning)")
    ap.add_argument("--tune-cache", default=None, help="C4: JSON file of tuned push shapes, reused for the same fleet")
    ap.add_argument("--rates", default="25,100,400", help="C5: request rates (req/s) of the phases")
    ap.add_argument("--phase-seconds", type=float, default=10.0, help="C5: seconds per rate phase")
    ap.add_argument("--budget-gb", type=float, default=0.0, help="C5: HBM budget (0: the big graph and 3/4 of "
                    "the small sessions)")
    ap.add_argument("--pool", type=int, default=48, help="C5: distinct small graphs generated")
    ap.add_argument("--drain-seconds", type=float, default=60.0, help="C5: wall time allowed after the last phase")
    ap.add_argument("--share-exponent", type=float, default=0.5, help="C5: push CTAs ~ (d (n + m))^exponent")
    ap.add_argument("--min-idle", type=float, default=3.0, help="C5: seconds without a request before a graph "
                    "may be evicted")
    ap.add_argument("--no-evict", dest="evict", action="store_false",
                    help="C5: sessions wait for memory instead of evicting idle graphs to host memory")
    ap.add_argument("--nodes", type=int, default=50_000_000, help="init-scale: nodes of the generated graph")
    ap.add_argument("--edges", type=int, default=1_000_000_000, help="init-scale: edges of the generated graph")
    ap.add_argument("--gamma", type=float, default=2.2, help="init-scale: power-law exponent")
    ap.add_argument("--seed", type=int, default=0xDA3F0500, help="init-scale: generator seed")
    ap.add_argument("--mode", default="batches", choices=["batches", "node-stream", "init-scale"],
                    help="node-stream: ms per node event under the paper's node-arrival protocol")
    args = ap.parse_args()
    from synth import CONFIGS, FLEETS, SERVING
    if args.mode == "init-scale":
        print(json.dumps(run_init_scale(args)))
        return
    if args.config in SERVING:
        os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
        print(json.dumps(run_serving(args, SERVING[args.config])))
        return
    if "." in args.config:     # one member graph of a fleet, e.g. C4.17 (the oracle's sample)
        base, idx = args.config.split(".", 1)
        c = FLEETS[base].members()[int(idx)]
    elif args.config in FLEETS:
        main_fleet(args, FLEETS[args.config])
        return
    else:
        c = CONFIGS[args.config]
    if args.oracle_worker:
        print(json.dumps(oracle_run(c, args.steps, 2, args.budget, args.save_state, alt_threads=ORACLE_ALT_THREADS)))
        return
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    if args.impl == "reference":
        if rank != 0:
            return
        # each step a bounded sample: the whole run stays within a few minutes
        budget = min(120.0, 0.5 * args.steps + 10.0)
        r = oracle_run(c, args.steps, args.warmup, budget)
        line = {"impl": "reference", "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 0,
                "steps": r["batches"], "warmup": args.warmup, "ms_per_step": 1e3 * r["seconds"] / max(r["batches"], 1),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded Chung-Lu graph and edge stream)",
                "config": {"workload": workload_desc(c), "precision": "fp64"},
                "latency_ms": {"p50": r["p50_ms"], "p99": r["p99_ms"]},
                "cpu_baseline": {"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                                 "sample": r["sample"]},
                "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    if args.mode == "node-stream":
        if rank == 0:
            print(json.dumps(run_node_stream(args, c)))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    proc, state = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle leg runs in its own process beside the GPU leg (no GPU, host cores only)
        import tempfile
        state = os.path.join(tempfile.mkdtemp(prefix="damf_oracle_"), "state.npz")
        proc = oracle_subprocess(c, 400, args.cpu_budget, state, wait=False)
    out = run_ours(args, c, rank, world)
    out.pop("_sigma")
    if args.compare_precision:
        import copy
        # both precisions over the same longer window (fresh contexts, the same batches), long
        # enough to hold folds (every refold_every updates), so that the fold's tensor-core
        # GEMMs are timed too
        cmp = {}
        for prec in [args.precision, "fp32" if args.precision == "mixed" else "mixed"]:
            a2 = copy.copy(args)
            a2.precision, a2.steps, a2.e2e_steps, a2.log_jsonl, a2.scoring = prec, args.precision_steps, 0, None, False
            o2 = run_ours(a2, c, rank, world)
            o2.pop("_sigma")
            cmp[prec] = {"value": o2["value"], "ms_per_step": o2["ms_per_step"], "steps": a2.steps,
                         "updates": o2["counters"]["updates"], "folds": o2["counters"]["folds"],
                         "fold_ms": o2["stage_ms"].get("fold"), "latency_ms": {k: o2["latency_ms"][k] for k in
                                                                               ("p50", "p99")},
                         "stage_ms_per_update": {k: round(v / max(o2["counters"]["updates"], 1), 4)
                                                 for k, v in o2["stage_ms"].items()},
                         "err": o2["err"]}
        pa = cmp[args.precision]
        cmp["speedup_mixed_over_fp32"] = (cmp["mixed"]["value"] / cmp["fp32"]["value"]) if cmp["fp32"]["value"] else None
        cmp["note"] = ("same workload and batches, fresh contexts; err = max |U^T U - I|, |V^T V - I| of the effective "
                       "bases after the window; mixed runs the fold's n x d by d x d GEMMs, the initialisation and "
                       "full-table queries on tcgen05 (TF32, three-term split), plain FP32 runs them on the SIMT "
                       "units; the per-update chain is FP32 SIMT in both (on tcgen05 its products coupled columns "
                       "of U at up to 3e-4 between folds); errors against the FP64 oracle for both are under "
                       "err_vs_oracle")
        out["precision_compare"] = cmp
        # the fold's cost per step, amortised over refold_every updates, from the longer window
        if pa["folds"]:
            per_fold = pa["fold_ms"] / pa["folds"]
            ups = out["counters"]["updates"] / max(out["steps"], 1)
            amort = per_fold * ups / max(args.refold_every, 1)
            out["fold"] = {"ms_per_fold": per_fold, "updates_per_fold": args.refold_every,
                           "folds_in_timed_steps": out["counters"]["folds"],
                           "amortized_ms_per_step": amort,
                           "value_with_amortized_fold": out["value"] * out["ms_per_step"] / (
                               out["ms_per_step"] + (amort if out["counters"]["folds"] == 0 else 0.0))}
    if rank == 0:
        if proc is not None:
            r = oracle_result(proc)
            if os.path.exists(state):
                try:
                    precs = [args.precision] + (["fp32" if args.precision == "mixed" else "mixed"]
                                                if args.compare_precision else [])
                    out["err_vs_oracle"] = err_vs_oracle(c, state, precs)
                except Exception as ex:   # reported, never fatal to the timing line
                    out["err_vs_oracle"] = {"error": repr(ex)[:300]}
                os.remove(state)
            if "value" in r:
                out["cpu_baseline"] = {"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                                       "sample": r["sample"], "p50_ms": r["p50_ms"], "p99_ms": r["p99_ms"],
                                       "init_s": r["init_s"]}
                if "alt_threads" in r:
                    out["cpu_baseline"]["alt_threads"] = r["alt_threads"]
            else:
                out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": ORACLE_THREADS, "kind": "oracle",
                                       "sample": "failed: " + r.get("error", "")}
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


def serving_inputs(sw, n_pool, big_batches, small_batches):
    """The big graph and a pool of small graphs, each with its request stream (log-uniform sizes),
    generated in spawned processes before the first GPU call."""
    from synth import fleet_inputs
    small = fleet_inputs([sw.small(i) for i in range(n_pool)], small_batches, log_sizes=True)
    big = fleet_inputs([sw.big()], big_batches, workers=1, log_sizes=True)[0]
    return big, small


def serving_timeline(reqs):
    """The serving loop's timeline, one record per server step, from the requests it served
    ((Request, phase) pairs): issue and completion time (s on the arrival clock), requests, edge
    events, the graphs that had a request in it and the earliest arrival among them."""
    steps = {}
    for r, ph in reqs:
        if r.step is None or r.t_done is None:
            continue
        e = steps.setdefault(r.step, {"step": int(r.step), "t_issue_s": r.t_issue, "t_done_s": r.t_done,
                                      "requests": 0, "edges": 0, "graphs": [], "first_arrival_s": r.t_arrive,
                                      "phase": ph})
        e["requests"] += 1
        e["edges"] += r.k
        e["graphs"].append(int(r.sid))
        e["first_arrival_s"] = min(e["first_arrival_s"], r.t_arrive)
    for e in steps.values():
        e["graphs"].sort()
    return [steps[k] for k in sorted(steps)]


def run_serving(args, sw):
    """Continuous batching of update requests over a changing set of resident graphs: a Poisson
    request stream in phases of rising rate, sessions admitted by device memory, one fleet step
    per server turn with at most one request per graph. Latency per request: arrival (host
    clock) to the host seeing its step complete."""
    import torch
    from paper_2306_08967_gb300 import bytes_required, make_config, rsvd_width
    from paper_2306_08967_gb300.serving import Server
    from synth import gaussian_test_matrix

    rates = [float(x) for x in args.rates.split(",")]
    dur = float(args.phase_seconds)
    R = sw.requests_per_session
    total_req = int(sum(rates) * dur * 1.3) + 64
    n_pool = sw.open_small + int(total_req / R) + 8
    n_pool = min(n_pool, args.pool)
    t0 = time.perf_counter()
    big, pool = serving_inputs(sw, n_pool, max(64, total_req // (sw.open_small + 1) * 3), R)
    gen_s = time.perf_counter() - t0
    print("[serving] inputs generated in %.1f s" % gen_s, file=sys.stderr, flush=True)
    torch.cuda.set_device(0)

    def spec(c, ip, ix):
        cfg = make_config(c.n, c.d, c.alpha, c.eps, nnz=len(ix), directed=True)
        return ip, ix, cfg, gaussian_test_matrix(c.n, rsvd_width(cfg), seed=c.seed + 2)

    need_big = bytes_required(spec(big[0], big[1], big[2])[2])
    need_small = [bytes_required(make_config(c.n, c.d, c.alpha, c.eps, nnz=len(ix), directed=True))
                  for c, ip, ix, _ in pool]
    free, total = torch.cuda.mem_get_info()
    budget = int(args.budget_gb * 1e9) if args.budget_gb else int(need_big + 0.75 * sum(need_small[:sw.open_small]))
    budget = min(budget, int(free * 0.9))
    srv = Server(budget, max_events=sw.k_hi, run_ahead=2, share_exponent=args.share_exponent, evict=args.evict,
                 min_idle_s=args.min_idle)
    # sessions: the big graph for the whole run, small ones each for R requests, then replaced
    srv.open(0, *spec(big[0], big[1], big[2]))
    nxt_pool = 0
    open_small = {}          # sid -> (pool index, requests submitted)
    sid_next = 1

    def open_one():
        nonlocal nxt_pool, sid_next
        c, ip, ix, _ = pool[nxt_pool % len(pool)]
        srv.open(sid_next, *spec(c, ip, ix))
        open_small[sid_next] = [nxt_pool % len(pool), 0]
        nxt_pool += 1
        sid_next += 1

    for _ in range(sw.open_small):
        open_one()
    t_init = time.perf_counter()
    srv.poll()                              # the first admissions (graph initialisations)
    srv.wait_admissions()
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t_init
    print("[serving] %d graphs initialised in %.1f s" % (len(srv.graphs), init_s), file=sys.stderr, flush=True)
    big_pos = 0
    rng = np.random.default_rng(sw.seed + 99)
    arrivals = []
    t_off = 0.0
    for ph, lam in enumerate(rates):
        a = sw.arrivals(lam, dur, sw.seed + 1000 + ph) + t_off
        arrivals += [(t, ph) for t in a]
        t_off += dur
    def progress(tag):
        print("[serving] %s t=%.1fs submitted=%d done=%d steps=%d inflight=%d resident=%d waiting=%d "
              "backlog=%d used=%.1fGB" % (tag, srv.now(), i, len(srv.completed), srv.steps_issued, len(srv.inflight),
                                         len(srv.sched.resident()), len(srv.sched.waiting), srv.sched.backlog(),
                                         srv.sched.used / 1e9), file=sys.stderr, flush=True)

    srv.t0 = time.perf_counter()           # the arrival clock starts now
    reqs = []
    i = 0
    used_max = 0
    t_report = 0.0
    wall_limit = len(rates) * dur + args.drain_seconds
    with ClockSampler(0) as clk:
        while i < len(arrivals) and srv.now() < wall_limit:
            now = srv.now()
            if now - t_report > 5.0:
                progress("run")
                t_report = now
            while i < len(arrivals) and arrivals[i][0] <= now:
                t_arr, ph = arrivals[i]
                choice = int(rng.integers(0, len(open_small) + 1))
                if choice == 0:
                    src, dst, op = (big[3].batches[big_pos % len(big[3].batches)].src,
                                    big[3].batches[big_pos % len(big[3].batches)].dst,
                                    big[3].batches[big_pos % len(big[3].batches)].op)
                    big_pos += 1
                    sid = 0
                else:
                    sid = sorted(open_small)[choice - 1]
                    pi, cnt = open_small[sid]
                    b = pool[pi][3].batches[cnt]
                    src, dst, op = b.src, b.dst, b.op
                    open_small[sid][1] += 1
                r = srv.submit(i, sid, src, dst, op, t_arrive=t_arr)
                reqs.append((r, ph))
                if sid != 0 and open_small[sid][1] == R:   # its last request: close, open the next
                    srv.close(sid)
                    del open_small[sid]
                    open_one()
                i += 1
            srv.poll()
            used_max = max(used_max, srv.sched.used)
            if i < len(arrivals) and not srv.inflight:
                time.sleep(max(0.0, min(arrivals[i][0] - srv.now(), 0.002)))
        progress("arrivals over")
        for sid in list(open_small) + [0]:   # every session ends with the trace
            srv.close(sid)
        drained = srv.drain(max(10.0, wall_limit - srv.now()))
        progress("drained" if drained else "drain cut short")
    t_end = srv.now()
    reqs = [(r, p) for r, p in reqs if r.t_done is not None]
    if args.log_jsonl:   # the loop's timeline: one line per server step
        with open(args.log_jsonl, "w") as f:
            for rec in serving_timeline(reqs):
                f.write(json.dumps(rec) + "\n")
    for g in list(srv.graphs.values()):
        g.check()
    def pct(rs):
        lat = np.array([r.t_done - r.t_arrive for r in rs]) * 1e3
        return {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                "mean": float(lat.mean()), "n": len(rs)} if len(rs) else None

    phases = []
    for ph, lam in enumerate(rates):
        rs = [r for r, p in reqs if p == ph]
        edges = sum(r.k for r in rs)
        last = max(r.t_done for r in rs) if rs else ph * dur
        phases.append({"rate_req_s": lam, "requests": len(rs), "edges": int(edges),
                       "edge_updates_s": edges / max(last - ph * dur, 1e-9),
                       "latency_ms": pct(rs),
                       "latency_ms_resident_at_arrival": pct([r for r in rs if r.resident_at_arrival]),
                       "latency_ms_waiting_for_admission": pct([r for r in rs if not r.resident_at_arrival])})
    sess = srv.sched.sessions.values()
    waits = np.array([(s.t_admit - s.t_open) for s in sess if s.t_admit is not None and s.sid != 0])
    steps = srv.steps_issued
    served = sum(r.k for r, _ in reqs)
    out = {
        "metric": METRIC, "value": served / max(t_end, 1e-9), "unit": UNIT, "n_gpus": 1,
        "steps": steps, "warmup": 0, "ms_per_step": 1e3 * t_end / max(steps, 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded directed Chung-Lu graphs, Poisson request arrivals)",
        "config": {"workload": "%s at a tenth of the stated node counts: a directed graph of n = %d (m = %d) for "
                               "the whole run and %d open sessions of directed graphs of n log-U[%d, %d] "
                               "(each closes after %d requests and a new one opens); d = %d, alpha %g, eps %g; "
                               "requests of log-U[%d, %d] edge events, Poisson arrivals in phases of %s req/s, "
                               "%g s each" % (sw.name, sw.big_n, len(big[2]), sw.open_small, sw.small_lo,
                                              sw.small_hi, R, sw.d, sw.alpha, sw.eps, sw.k_lo, sw.k_hi,
                                              args.rates, dur),
                   "budget_gb": budget / 1e9, "used_max_gb": used_max / 1e9,
                   "big_graph_gb": need_big / 1e9, "launch": "one fleet step per server turn (every resident "
                   "graph, at most one request each; graphs' updates overlapped, one grouped push)",
                   "parallelism": "single GPU"},
        "value_definition": "all served edge events / (last completion - first arrival), over every phase",
        "phases": phases,
        "e2e": {"value": served / max(t_end, 1e-9), "unit": UNIT,
                "h2d_bytes_per_step": 9 * served / max(steps, 1), "d2h_bytes_per_step": 0,
                "note": "every request goes host -> device (pinned staging, one copy per step); completion is "
                        "observed on the host through an event"},
        "sessions": {"opened": len(srv.sched.sessions), "evict": args.evict, "min_idle_s": args.min_idle,
                     "evictions": int(sum(x.evictions for x in srv.sched.sessions.values())),
                     "admission_wait_s": {
            "p50": float(np.percentile(waits, 50)) if len(waits) else None,
            "p99": float(np.percentile(waits, 99)) if len(waits) else None}},
        "gpu_launches": int(srv.kernel_count()),
        "gpu_launches_note": "kernels of every graph (initialisations included) and fleet of the run",
        "init_s": init_s, "generate_s": gen_s, "clocks": clk.summary(),
    }
    srv.shutdown()
    return out


def main_fleet(args, fw):
    # more hardware work queues for the graphs' streams (read when the CUDA context starts)
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    members = fw.members()[: args.graphs] if args.graphs else fw.members()
    # the oracle's sample: the fleet member closest to the median size
    order = np.argsort([c.n for c in members])
    sample = members[int(order[len(order) // 2])]
    if args.impl == "reference":
        if rank != 0:
            return
        budget = min(120.0, 0.5 * args.steps + 10.0)
        r = oracle_run(sample, args.steps, args.warmup, budget)
        line = {"impl": "reference", "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": 0,
                "steps": r["batches"], "warmup": args.warmup, "ms_per_step": 1e3 * r["seconds"] / max(r["batches"], 1),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic (seeded Chung-Lu graphs and edge streams)",
                "config": {"workload": "%s: the oracle on one member graph (%s, n = %d, d = %d)"
                                       % (fw.name, sample.name, sample.n, sample.d), "precision": "fp64"},
                "cpu_baseline": {"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                                 "sample": r["sample"]},
                "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return
    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    out = run_fleet(args, fw, rank, world)
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            r = oracle_subprocess(sample, 400, args.cpu_budget)
            if "value" in r:
                out["cpu_baseline"] = {"value": r["value"], "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                                       "sample": r["sample"] + "; graph %s (n = %d, d = %d, the median size of the "
                                       "fleet); edge-updates/s of one graph at a time" % (sample.name, sample.n,
                                                                                          sample.d)}
            else:
                out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                       "sample": "failed: " + r.get("error", "")}
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
