"""Plain FP64 CPU oracle for DAMF (arXiv 2306.08967).  TEST INFRASTRUCTURE ONLY.

Only the tests, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import or run anything in this package.  It shares no code with the CUDA
library (`paper_2306_08967_gb300`) and the library never imports it.

Contents, each following the cited passage of the paper:
  tsvd.py   t-SVD (Sec. 4.1, Eq. "ne"); the brute-force update that Theorem 2
            (Sec. 4.3) says the incremental update must equal; the randomized
            t-SVD of the initialisation (Appendix A, Algorithm 3).
  graph.py  the dynamic graph with set semantics and the net change dA = B C^T
            of an update (Sec. 4.3, Eq. "edge_B"); the plain-C adjacency.
  damf.py   the incremental update in the paper's X-form (Algorithms 1-2,
            Eqs. "update", "f_edge", "g_edge", "x_edge", "y_edge").
  ppr.py    PPR (Sec. 4.4, Eq. "ppr"): dense closed form, the literal series,
            power iteration, the graph-change residual fix-up, and the
            sequential FIFO push (plain C, oracle/c/oracle_graph.c), with the
            absolute or the degree-scaled threshold.
  scoring.py  link-prediction scores and the per-query top-k ranking (Sec. 5,
            "Link Prediction", "Graph Reconstruction").

Pins (tests/test_oracle_*.py, `-m "not gpu"`): closed-form spectra of cliques,
stars and cycles; Theorem 2 against the brute-force t-SVD on random tiny graphs;
Proposition 1; the PPR closed form against the literal series; alpha = 1 giving
Z = X (the paper's ablation); a constant signal as a fixed point; the push's
epsilon bound; the residual invariant after graph changes; set semantics of the
graph against an independent dense replay.
"""
