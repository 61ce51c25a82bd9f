#!/usr/bin/env python
"""Edge-update throughput and latency of the DAMF hot path on one GB300 (or N replicas).

A step is one batch of the workload through the whole hot path: damf_apply_edges
(adjacency edit, projection, residual CholQR, core SVD, transform update, row rewrite,
PPR residual fix-up) followed by damf_ppr_refresh (push until every residual <= eps).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config C2] [--impl ours|reference]

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on the same
workload (bounded sample per step) and prints the same metric with "impl": "reference".
"""

import argparse
import dataclasses
import json
import os
import sys

if "--impl" in sys.argv and "reference" in sys.argv or "--oracle-worker" in sys.argv:
    # the oracle runs single-threaded: pin BLAS pools before numpy loads
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"

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


def make_inputs(c, n_batches):
    from synth import chung_lu_graph, edge_stream
    ip, ix, w = chung_lu_graph(c.n, c.avg_deg, c.gamma, seed=c.seed, directed=c.directed)
    st = edge_stream(ip, ix, w, n_batches, c.k_lo, c.k_hi, c.p_node, c.p_del, c.seed + 1,
                     max_new_degree=c.max_new_degree, directed=c.directed, nodes_per_batch=c.nodes_per_batch)
    return ip, ix, st


# ---------------------------------------------------------------- oracle (CPU) leg
def oracle_run(c, steps, warmup, time_budget_s, save_path=None):
    """Times the FP64 oracle (as it stands) on the first warmup+steps batches, stopping
    early once time_budget_s of timed work is spent.  Returns a dict; with save_path, also
    writes the oracle's final X, Y, Z and sigma there (npz) for the error comparison."""
    from oracle.damf import DamfOracle
    from synth import gaussian_test_matrix
    ip, ix, st = make_inputs(c, warmup + steps)
    om = gaussian_test_matrix(c.n, 160 if c.d == 128 else ((c.d + 10 + 31) // 32) * 32, seed=c.seed + 2)
    t0 = time.perf_counter()
    orc = DamfOracle(ip, ix, c.d, c.alpha, c.eps, n_cap=st.n_final, directed=c.directed, Omega=om)
    init_s = time.perf_counter() - t0
    for b in st.batches[:warmup]:
        orc.apply_edges(b.src, b.dst, b.op, b.new_nodes)
        orc.ppr_refresh()
    lat, edges = [], 0
    t_start = time.perf_counter()
    for b in st.batches[warmup:warmup + steps]:
        t = time.perf_counter()
        orc.apply_edges(b.src, b.dst, b.op, b.new_nodes)
        orc.ppr_refresh()
        lat.append(time.perf_counter() - t)
        edges += b.k
        if time.perf_counter() - t_start > time_budget_s:
            break
    total = time.perf_counter() - t_start
    if save_path:
        n = orc.n
        np.savez(save_path, X=orc.X()[:n], Y=orc.Y()[:n], Z=orc.Z()[:n], sigma=orc.sigma,
                 batches=warmup + len(lat))
    return {"value": edges / total, "unit": UNIT, "cores": 1, "kind": "oracle", "batches": len(lat),
            "edges": edges, "seconds": total, "init_s": init_s,
            "p50_ms": 1e3 * float(np.percentile(lat, 50)), "p99_ms": 1e3 * float(np.percentile(lat, 99)),
            "sample": "first %d batches of the %s stream after %d warm-up batches (%d edges), FP64 oracle, "
                      "1 thread" % (len(lat), c.name, warmup, edges)}


def oracle_subprocess(c, steps, budget, save_path=None):
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-worker", "--config", c.name, "--steps", str(steps),
           "--budget", str(budget)] + (["--save-state", save_path] if save_path else [])
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    out = subprocess.run(cmd, env=env, capture_output=True, text=True, timeout=1800)
    for line in out.stdout.splitlines()[::-1]:
        if line.startswith("{"):
            return json.loads(line)
    return {"error": (out.stderr or out.stdout)[-400:]}


def err_vs_oracle(c, path, precisions):
    """Replays the oracle's batches on the device (fresh context per precision) and compares
    sigma, X Y^T and Z Y^T with the oracle's FP64 result: relative errors, the Frobenius
    ones through d x d Grams (|A B^T|_F^2 = tr((A^T A)(B^T B)))."""
    import torch
    from paper_2306_08967_gb300 import DamfGraph, make_config, rsvd_width
    from synth import gaussian_test_matrix
    ref = np.load(path)
    nb = int(ref["batches"])
    dev = torch.device("cuda")
    Xo, Yo, Zo = (torch.from_numpy(ref[k]).to(dev) for k in ("X", "Y", "Z"))
    so = ref["sigma"]
    ip, ix, st = make_inputs(c, nb)

    def rel_fro(A, B, Ao, Bo):   # |A B^T - Ao Bo^T|_F / |Ao Bo^T|_F
        gg = torch.trace((A.T @ A) @ (B.T @ B))
        oo = torch.trace((Ao.T @ Ao) @ (Bo.T @ Bo))
        go = torch.trace((A.T @ Ao) @ (Bo.T @ B))
        return float(torch.sqrt(torch.clamp(gg - 2 * go + oo, min=0)) / torch.sqrt(oo))

    out = {"batches": nb, "oracle": "FP64 incremental oracle (the paper's X-form) on the same batches"}
    for prec in precisions:
        cfg = make_config(c.n, c.d, c.alpha, c.eps, n_capacity=st.n_final + 16, nnz=len(ix), directed=c.directed,
                          refold_every=256, precision=prec)
        om = gaussian_test_matrix(c.n, rsvd_width(cfg), seed=c.seed + 2)
        g = DamfGraph(ip, ix, cfg, om)
        for b in st.batches[:nb]:
            g.apply_edges_host(b.src, b.dst, b.op, b.new_nodes)
            g.ppr_refresh()
        g.check()
        e = g.embeddings()
        X, Y, Z = (e[k].double() for k in ("X", "Y", "Z"))
        sg = e["sigma"].double().cpu().numpy()
        out[prec] = {"sigma_max_rel": float(np.max(np.abs(sg - so) / np.abs(so))),
                     "xyt_rel_fro": rel_fro(X, Y, Xo, Yo), "zyt_rel_fro": rel_fro(Z, Y, Zo, Yo)}
        if "zyt_eps_bound" not in out:
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


# DRAM bytes (read + write) of one k_push launch of the C2 workload, from the ncu capture
# summarised in profiles/k_push_C2.md; None once k_push changes until it is captured again
PUSH_DRAM_BYTES = 478.21e6

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
            "frac": round(achieved / hbm_peak, 4), "traffic": PUSH_DRAM_BYTES if c.name == "C2" else None,
            "traffic_note": "dram read + write of one captured launch of the current k_push (ncu, "
                            "profiles/k_push_C2.md); most of the algorithmic bytes are L2 atomics",
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "bytes_per_launch": push_bytes / max(push_launches, 1), "ms_per_launch": push_ms_per}
    launches = s1["launches"] - s0["launches"]
    scoring = measure_scoring(g, c, torch) if args.scoring else None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": elapsed_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded Chung-Lu graph and edge stream)",
        "config": {"workload": workload_desc(c), "precision": args.precision, "edges_timed": edges,
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--config", default="C2")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--refold-every", type=int, default=256)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp32"])
    ap.add_argument("--no-compare-precision", dest="compare_precision", action="store_false",
                    help="skip timing the other precision build of the path on the same workload")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-scoring", dest="scoring", action="store_false",
                    help="skip the link-prediction query timing (score_pairs, topk) after the run")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    ap.add_argument("--oracle-worker", action="store_true")
    ap.add_argument("--budget", type=float, default=20.0)
    ap.add_argument("--save-state", default=None)
    ap.add_argument("--mode", default="batches", choices=["batches", "node-stream"],
                    help="node-stream: ms per node event under the paper's node-arrival protocol")
    args = ap.parse_args()
    from synth import CONFIGS
    c = CONFIGS[args.config]
    if args.oracle_worker:
        print(json.dumps(oracle_run(c, args.steps, 2, args.budget, args.save_state)))
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
    out = run_ours(args, c, rank, world)
    sig_a = np.array(out.pop("_sigma"))
    if args.compare_precision:
        import copy
        a2 = copy.copy(args)
        a2.precision = "fp32" if args.precision == "mixed" else "mixed"
        a2.e2e_steps = 0
        o2 = run_ours(a2, c, rank, world)
        sig_b = np.array(o2.pop("_sigma"))
        out["precision_compare"] = {
            args.precision: {"value": out["value"], "ms_per_step": out["ms_per_step"], "err": out["err"],
                             "fold_ms": out["stage_ms"].get("fold")},
            a2.precision: {"value": o2["value"], "ms_per_step": o2["ms_per_step"], "err": o2["err"],
                           "fold_ms": o2["stage_ms"].get("fold")},
            "sigma_max_rel_diff": float(np.max(np.abs(sig_a - sig_b) / np.abs(sig_b))),
            "note": "same workload and stream; err = max |U^T U - I|, |V^T V - I| of the effective bases "
                    "after the run; mixed runs the fold's n x d by d x d GEMMs on tcgen05 (TF32, 3-term split)"}
    if rank == 0:
        if not args.no_cpu_baseline and world == 1:
            import tempfile
            state = os.path.join(tempfile.mkdtemp(prefix="damf_oracle_"), "state.npz")
            r = oracle_subprocess(c, 400, args.cpu_budget, state)
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
            else:
                out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle",
                                       "sample": "failed: " + r.get("error", "")}
        print(json.dumps(out))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
