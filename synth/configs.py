"""Named workloads (sizes and distributions of the paper-shaped synthetic inputs).

C1  small FP64-checkable case: undirected Chung-Lu, gamma 2.5, n = 2,000, ~10k edges,
    d = 16, alpha = 0.15, eps = 1e-4; 100 batches of 10 insertions plus 1 node arrival.
C2  single-GPU workload: undirected Chung-Lu, gamma 2.2, n = 200,000, mean degree 10,
    d = 128, alpha = 0.15, eps = 1e-5; 10,000 batches of U[1, 64] edges with 5% node
    arrivals and 10% deletions.
C3  large graph: undirected Chung-Lu, gamma 2.1, n = 2,000,000, m = 40M edges (mean degree
    40), d = 128; 50,000 batches of U[1, 256] edges (up to four updates per call), node
    arrivals and deletions as in C2 (the workload states neither; C2's rates are used), alpha
    and eps as in C2, the fold every 256 updates.
C5  serving (the workload's graph of n = 50M, m = 1B and 32 graphs of 1M-5M nodes need about
    300 GB at d = 128, more than one GPU holds; run here at a tenth of the node counts): one
    directed Chung-Lu graph, gamma 2.2, n = 5M, m = 100M, and sessions of directed graphs with
    n log-uniform in [100k, 500k] (32 open at a time; each closes after 50 requests and a new
    one opens), d = 128, alpha and eps as in C2; Poisson arrivals of requests
    of log-uniform size in [1, 1024] edge events (10% deletions), each to a uniformly chosen
    open session; admission by the bytes each graph needs against an HBM budget.
C4  many graphs: 256 undirected Chung-Lu graphs, n log-uniform in [1,000, 500,000], mean
    degree uniform in [4, 32], d drawn from {32, 64, 128}; one batch of U[1, 128] edge events
    per graph per step. The workload names no node arrivals, deletion rate, gamma, alpha or
    eps: 10% deletions, no arrivals (so the step replays as one captured launch), and C2's
    gamma, alpha and eps are used.
"""

import dataclasses
import math

import numpy as np

SEED_BASE = 0xDA3F0000


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n: int
    avg_deg: float
    gamma: float
    d: int
    alpha: float
    eps: float
    n_batches: int
    k_lo: int
    k_hi: int
    p_node: float
    p_del: float
    nodes_per_batch: int
    seed: int
    directed: bool = False
    max_new_degree: int = 32

    @property
    def n_cap(self) -> int:
        # room for every node arrival the stream can make
        per_batch = self.nodes_per_batch + self.k_hi
        return self.n + self.n_batches * per_batch if self.p_node > 0 else self.n + self.n_batches * self.nodes_per_batch


CONFIGS = {
    "C1": Workload("C1", n=2000, avg_deg=10.0, gamma=2.5, d=16, alpha=0.15, eps=1e-4, n_batches=100,
                   k_lo=10, k_hi=10, p_node=0.0, p_del=0.0, nodes_per_batch=1, seed=SEED_BASE + 0),
    "C2": Workload("C2", n=200_000, avg_deg=10.0, gamma=2.2, d=128, alpha=0.15, eps=1e-5, n_batches=10_000,
                   k_lo=1, k_hi=64, p_node=0.05, p_del=0.10, nodes_per_batch=0, seed=SEED_BASE + 1),
    "C3": Workload("C3", n=2_000_000, avg_deg=40.0, gamma=2.1, d=128, alpha=0.15, eps=1e-5, n_batches=50_000,
                   k_lo=1, k_hi=256, p_node=0.05, p_del=0.10, nodes_per_batch=0, seed=SEED_BASE + 2),
}


def small_config(name: str = "C1", **over) -> Workload:
    return dataclasses.replace(CONFIGS[name], **over)


@dataclasses.dataclass(frozen=True)
class FleetWorkload:
    """Many independent graphs stepped together (one batch per graph per step)."""
    name: str
    graphs: int
    n_lo: int
    n_hi: int
    deg_lo: float
    deg_hi: float
    ds: tuple
    gamma: float
    alpha: float
    eps: float
    k_lo: int
    k_hi: int
    p_del: float
    seed: int

    def members(self) -> list:
        """The graphs as Workloads: n log-uniform in [n_lo, n_hi], mean degree uniform in
        [deg_lo, deg_hi], d uniform over ds; each graph's own seed."""
        rng = np.random.Generator(np.random.PCG64(self.seed))
        out = []
        for i in range(self.graphs):
            n = int(round(math.exp(rng.uniform(math.log(self.n_lo), math.log(self.n_hi)))))
            deg = float(rng.uniform(self.deg_lo, self.deg_hi))
            d = int(self.ds[int(rng.integers(0, len(self.ds)))])
            out.append(Workload("%s.%d" % (self.name, i), n=n, avg_deg=deg, gamma=self.gamma, d=d, alpha=self.alpha,
                                eps=self.eps, n_batches=0, k_lo=self.k_lo, k_hi=self.k_hi, p_node=0.0,
                                p_del=self.p_del, nodes_per_batch=0, seed=self.seed + 7919 * (i + 1)))
        return out


FLEETS = {
    "C4": FleetWorkload("C4", graphs=256, n_lo=1000, n_hi=500_000, deg_lo=4.0, deg_hi=32.0, ds=(32, 64, 128),
                        gamma=2.2, alpha=0.15, eps=1e-5, k_lo=1, k_hi=128, p_del=0.10, seed=SEED_BASE + 3),
}


def member_inputs(c: Workload, n_batches: int, log_sizes: bool = False):
    """One graph's inputs: (indptr, indices, EdgeStream of n_batches batches)."""
    from .chung_lu import chung_lu_graph, edge_stream
    ip, ix, w = chung_lu_graph(c.n, c.avg_deg, c.gamma, seed=c.seed, directed=c.directed)
    st = edge_stream(ip, ix, w, n_batches, c.k_lo, c.k_hi, c.p_node, c.p_del, c.seed + 1,
                     max_new_degree=c.max_new_degree, directed=c.directed, nodes_per_batch=c.nodes_per_batch,
                     log_sizes=log_sizes)
    return ip, ix, st


def fleet_inputs(members, n_batches: int, workers: int = 0, log_sizes: bool = False):
    """member_inputs for every graph, in a pool of `workers` spawned processes (0: the host's
    cores, at most 16; 1: in this process). Spawned, so that it is safe in a process that
    already uses a GPU. Returns [(workload, indptr, indices, stream)] in member order."""
    import os
    members = list(members)
    if workers <= 0:
        workers = min(16, os.cpu_count() or 1, len(members))
    if workers <= 1:
        return [(c, *member_inputs(c, n_batches, log_sizes)) for c in members]
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(member_inputs, members, [n_batches] * len(members), [log_sizes] * len(members),
                          chunksize=1))
    return [(c, *r) for c, r in zip(members, res)]


@dataclasses.dataclass(frozen=True)
class ServingWorkload:
    """Sessions of graphs served together; requests arrive as a Poisson process."""
    name: str
    big_n: int
    big_deg: float
    small_lo: int
    small_hi: int
    small_deg: float
    open_small: int          # small sessions open at a time
    requests_per_session: int
    d: int
    gamma: float
    alpha: float
    eps: float
    k_lo: int
    k_hi: int
    p_del: float
    seed: int

    def big(self) -> Workload:
        return Workload(self.name + ".big", n=self.big_n, avg_deg=self.big_deg, gamma=self.gamma, d=self.d,
                        alpha=self.alpha, eps=self.eps, n_batches=0, k_lo=self.k_lo, k_hi=self.k_hi, p_node=0.0,
                        p_del=self.p_del, nodes_per_batch=0, seed=self.seed, directed=True)

    def small(self, i: int) -> Workload:
        rng = np.random.Generator(np.random.PCG64(self.seed + 104729 * (i + 1)))
        n = int(round(math.exp(rng.uniform(math.log(self.small_lo), math.log(self.small_hi)))))
        return Workload("%s.s%d" % (self.name, i), n=n, avg_deg=self.small_deg, gamma=self.gamma, d=self.d,
                        alpha=self.alpha, eps=self.eps, n_batches=0, k_lo=self.k_lo, k_hi=self.k_hi, p_node=0.0,
                        p_del=self.p_del, nodes_per_batch=0, seed=self.seed + 7919 * (i + 1), directed=True)

    def arrivals(self, rate: float, duration: float, seed: int) -> np.ndarray:
        """Poisson arrival times (s) in [0, duration) at `rate` requests per second."""
        rng = np.random.Generator(np.random.PCG64(seed))
        t = np.cumsum(rng.exponential(1.0 / rate, size=int(rate * duration * 1.5) + 16))
        return t[t < duration]


SERVING = {
    "C5": ServingWorkload("C5", big_n=5_000_000, big_deg=20.0, small_lo=100_000, small_hi=500_000, small_deg=12.0,
                          open_small=32, requests_per_session=50, d=128, gamma=2.2, alpha=0.15, eps=1e-5, k_lo=1,
                          k_hi=1024, p_del=0.10, seed=SEED_BASE + 4),
}
