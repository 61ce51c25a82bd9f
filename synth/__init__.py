"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module generates inputs only: Chung-Lu power-law graphs standing in for the
paper's datasets (Table "Statistics of Datasets", Sec. 5.1), edge-event streams in
the paper's dynamic setting (Sec. 5.1 "Setting of Dynamicity": node arrivals plus
edge changes), and the Gaussian test matrix of the randomized t-SVD used at
initialisation (Appendix A, Algorithm 3).  It contains none of the method's
arithmetic and imports neither the oracle nor the CUDA package.
"""

from .chung_lu import (  # noqa: F401
    Batch,
    EdgeStream,
    chung_lu_graph,
    chung_lu_weights,
    edge_stream,
    gaussian_test_matrix,
    csr_from_edges,
    node_arrival_stream,
)
from .configs import (CONFIGS, FLEETS, SERVING, FleetWorkload, ServingWorkload, fleet_inputs,  # noqa: F401
                      member_inputs, small_config)
