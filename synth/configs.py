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
"""

import dataclasses

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
