/*
 * damf.h -- C ABI of the DAMF per-update hot path on one GPU (sm_103a).
 *
 * DAMF (Dynamic Adjacency Matrix Factorization, arXiv 2306.08967) keeps a rank-d
 * truncated SVD  A ~ U Sigma V^T  of a graph's adjacency matrix while edges and
 * nodes change, and a Personalized-PageRank-enhanced context embedding
 * Z = PPR(U Sigma^{1/2}) (Sec. 4.4, Eq. "ppr").  The library stores U and V as
 * node-row bases times d x d transforms (U = U_b P_U, V = V_b P_V; the lazy base
 * space of Sec. 4.1, Eq. "update"), so an update rewrites only the rows the
 * change touches (Lemma 1) plus four d x d matrices.
 *
 * Conventions shared by every entry point
 *   - Pointers marked (device) are CUDA device pointers owned by the caller; the
 *     library reads them during the call's stream work and keeps no reference.
 *     Pointers marked (host) are ordinary host memory, read before the call returns.
 *   - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *     stream.  All work is enqueued asynchronously on it.
 *   - A returned status covers argument checks made on the host.  Errors found on
 *     the device (invalid edge ids, capacity exhaustion, a bounded wait that ran
 *     out, non-finite values) are recorded in a device status word and returned by
 *     damf_sync_status(); after such an error the context is poisoned and every
 *     later call returns that status until damf_destroy().
 *   - Dense arrays are row-major float32 with rows of d entries (16-byte aligned
 *     when the pointer is 16-byte aligned).  Node ids are int32 in [0, n).
 *   - One context must be used from one stream at a time.
 */
#ifndef DAMF_H_
#define DAMF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct damf_ctx damf_ctx; /* opaque; owns all device state */

typedef enum {
  DAMF_OK = 0,
  DAMF_ERR_INVALID = 1,        /* bad argument or edge event (id out of range, self-loop, op not +-1) */
  DAMF_ERR_CAPACITY = 2,       /* node or edge capacity exhausted; the update was not applied */
  DAMF_ERR_CUDA = 3,           /* a CUDA runtime call failed; damf_last_error() has the text */
  DAMF_ERR_NUMERIC = 4,        /* non-finite value in Sigma, a transform or a residual factor */
  DAMF_ERR_TIMEOUT = 5,        /* a bounded device-side wait ran out */
  DAMF_ERR_NOT_CONVERGED = 6,  /* the PPR push hit max_push_rounds phases before every residual was <= eps */
  DAMF_ERR_BOUNDS = 7          /* a device bounds check failed (only in a library built with DAMF_CHECK: row ids
                                  below the node capacity, adjacency offsets inside m_capacity, queue items
                                  inside their arrays); the access was skipped */
} damf_status;

typedef struct {
  int32_t n;                /* nodes of the initial graph */
  int32_t n_capacity;       /* maximum node count (node arrivals append ids n, n+1, ...) */
  int64_t m_capacity;       /* stored adjacency entries, slack and relocations included
                               (undirected edges are stored twice; directed graphs keep
                               an out- and an in-adjacency, each within m_capacity) */
  int32_t d;                /* rank of the factorisation: 16, 32, 64 or 128 */
  int32_t directed;         /* 0: undirected (each event touches (u,v) and (v,u)); 1: directed */
  double alpha;             /* PPR damping factor, 0 < alpha <= 1 (Eq. "ppr") */
  double eps;               /* PPR tolerance: the push stops when max_j |r[u][j]| <= eps for all u */
  int32_t refold_every;     /* fold the transforms into the bases every this many updates; 0 = never */
  int32_t rsvd_oversample;  /* randomized t-SVD: l = round_up(d + rsvd_oversample, 32) test vectors */
  int32_t rsvd_power_iters; /* randomized t-SVD power iterations q */
  int32_t max_push_rounds;  /* cap on push phases per damf_ppr_refresh (a phase runs the work queue
                               until it drains; another follows only when the queue overflowed) */
  int32_t precision;        /* 0: plain FP32 (SIMT for every kernel); 1: mixed, the n x d by d x d
                               GEMMs of the fold, the initialisation and the full query run on
                               the tensor cores (tcgen05, TF32 with a three-term split that keeps
                               FP32 accuracy); the small dense factor update is FP32 in both */
  int32_t threshold;        /* push threshold: 0 absolute, the push stops when max_j |r[u][j]| <= eps
                               for all u (then |Z_b - Pi X_b| <= eps elementwise); 1 degree-scaled,
                               max_j |r[u][j]| <= eps * max(deg(u), 1) with deg the out-degree (the
                               c of the push cost in Sec. 4.5; |Z_b - Pi X_b| <= eps Pi deg) */
} damf_config;

/* Workspace the library allocates on the device for `cfg` (bytes).  Lets a caller
 * admit a graph only when it fits in free device memory.  0 for an invalid cfg. */
size_t damf_bytes_required(const damf_config* cfg);

/* Randomized-t-SVD sample width l for `cfg` (columns of the Omega argument below). */
int32_t damf_rsvd_width(const damf_config* cfg);

/*
 * Creates a context and computes the initial state (Appendix A, Algorithm 3):
 * a rank-d randomized t-SVD A ~ U Sigma V^T (Halko et al., cited at Algorithm 3),
 * U_b = U, V_b = V, P_U = P_V = I, then the PPR residual r = U_b Sigma^{1/2},
 * Z_b = 0 and a push to tolerance eps (Algorithm 3, lines 4-5).
 *   row_ptr (device) int32[n+1], col_idx (device) int32[m]: the initial adjacency in
 *     CSR; an undirected graph must list both (u,v) and (v,u); no self-loops.
 *   omega (device) float32[n x l], l = damf_rsvd_width(cfg): standard normal test
 *     matrix (the caller draws it so that results are reproducible across devices).
 *   out: receives the context; *out is NULL on failure.
 * Returns DAMF_ERR_INVALID for a bad cfg, DAMF_ERR_CAPACITY when a device allocation
 * fails for want of memory (everything allocated so far is freed), DAMF_ERR_CUDA when
 * another CUDA call fails.  Synchronises `stream` before returning (setup path, not the
 * per-update path).
 */
damf_status damf_init_factorize(const damf_config* cfg, const int32_t* row_ptr, const int32_t* col_idx,
                                int64_t m, const float* omega, void* stream, damf_ctx** out);

/*
 * Applies one call's edge events (Algorithm 2; Algorithm 1 "UpdateEmbeddingE" with
 * B C^T = dA, Sec. 4.3, Eqs. "edge_B", "f_edge", "g_edge", "x_edge", "y_edge").
 *   new_nodes: nodes appended before the edges (ids n .. n+new_nodes-1); a node
 *     arrival is a zero row and column followed by ordinary edge changes (Sec. 4.2).
 *   src, dst (device) int32[k], op (device) int8[k]: event i inserts (op = +1) or
 *     deletes (op = -1) edge (src[i], dst[i]); an undirected event covers both
 *     directions.  Set semantics: per ordered pair the last event decides whether
 *     the edge is present; inserting a present edge or deleting an absent one is a
 *     no-op.
 * The events are applied as ceil(k/64) consecutive updates of at most 64 events
 * each (rank r <= 128).  Each update: edits the adjacency; projects dA onto the
 * bases (W_B = U^T B, W_C = V^T C); re-orthogonalises the residual blocks by
 * Cholesky of their Gram matrices (Prop. 1 for a block); takes the SVD of the
 * (d+r) x (d+r) core; folds the rotation into P_U, P_V and their inverses; rewrites
 * the touched base rows; and updates the PPR residual for the changed signal rows
 * and the changed out-rows.  The PPR push itself is damf_ppr_refresh().
 * Device-side validation: ids < n + new_nodes, no self-loop, op = +-1; on failure
 * nothing is written and the status becomes DAMF_ERR_INVALID.
 */
damf_status damf_apply_edges(damf_ctx* ctx, const int32_t* src, const int32_t* dst, const int8_t* op,
                             int32_t k, int32_t new_nodes, void* stream);

/*
 * damf_apply_edges (Algorithm 2; Algorithm 1 "UpdateEmbeddingE", Sec. 4.3) with the event
 * count on the device: the live events are the first
 * *k_dev of src/dst/op (k_dev: device int32, read when the work runs, clamped to
 * [0, k_max]); the arrays hold k_max entries.  The call enqueues ceil(k_max / 64) updates;
 * an update whose events all lie beyond the live count finds no net change and leaves the
 * state as it is.  So one captured call (CUDA graph) replays batches of any size up to
 * k_max, written into the same buffers between replays; the result of each replay equals
 * damf_apply_edges on the live events.  DAMF_ERR_INVALID for a NULL k_dev.
 */
damf_status damf_apply_edges_counted(damf_ctx* ctx, const int32_t* src, const int32_t* dst, const int8_t* op,
                                     int32_t k_max, const int32_t* k_dev, int32_t new_nodes, void* stream);

/* One batch of events for one graph (damf_apply_edges_multi). */
typedef struct {
  damf_ctx* ctx;          /* the graph's context */
  const int32_t* src;     /* (device) int32[k] */
  const int32_t* dst;     /* (device) int32[k] */
  const int8_t* op;       /* (device) int8[k], +1 insert, -1 delete */
  int32_t k;              /* events (with k_dev: the capacity of the arrays, k_max) */
  int32_t new_nodes;      /* node arrivals appended before the events */
  const int32_t* k_dev;   /* NULL, or (device) int32: the live event count, as for
                             damf_apply_edges_counted */
} damf_batch;

/*
 * Applies one batch to each of num_graphs independent graphs (the batching pattern: many
 * graphs of uneven size per call), in order, on `stream`: each entry is exactly
 * damf_apply_edges(batches[i].ctx, ...), so every graph's result is the same as when its
 * batch is applied alone. Each graph's push still runs on its own context's stream
 * (damf_ppr_refresh). Every batch's host-side checks (arguments, node capacity) are taken
 * before any work is enqueued: a batch they reject poisons its own context and no graph of
 * the call gets new work. Otherwise returns the first non-OK status (the remaining batches
 * are not applied); DAMF_ERR_INVALID for num_graphs < 0 or a NULL batches array / context.
 */
damf_status damf_apply_edges_multi(const damf_batch* batches, int32_t num_graphs, void* stream);

/*
 * One step of many independent graphs (the batching pattern: graphs of uneven size and
 * rank, one batch each; per graph Algorithm 2 followed by the push of Sec. 4.4): for every
 * entry, the batch's update (as damf_apply_edges, or
 * damf_apply_edges_counted when k_dev is set) and then its push (damf_ppr_refresh), run on
 * streams the graph's context owns, forked from `stream` after the work enqueued on it
 * before the call; `stream` then waits for every graph's update and push.  The graphs'
 * kernels overlap on the device, and each graph's result equals its result when its batch
 * is applied and pushed alone.  Capturable in one CUDA graph (join each context, damf_join,
 * before the capture starts); a replay then runs the whole step as one launch.  A context
 * may appear once per call (DAMF_ERR_INVALID otherwise, nothing enqueued).  A batch that the
 * host-side checks (arguments, node capacity) reject poisons its own context and nothing is
 * enqueued for any graph; after a later failure (a CUDA call) the graphs before it have been
 * enqueued.  Returns the first non-OK status.
 */
damf_status damf_step_multi(const damf_batch* batches, int32_t num_graphs, void* stream);

/*
 * Fleets: many independent graphs stepped together with their pushes in one launch.
 *
 * damf_step_multi runs one cooperative push per graph, and cooperative launches do not run
 * side by side, so a fleet of small graphs spends its time in one push after another.  A
 * fleet instead pushes all its graphs in one grouped cooperative launch (one per threshold
 * mode): graph i owns a share of the CTAs and runs its own push (Sec. 4.4) over them, with
 * its own work queue and its own barrier among its CTAs, so each graph's result is the same
 * as when it is pushed alone.  Graphs too small for a CTA of their own share one, which
 * pushes them one after another.
 */
typedef struct damf_fleet damf_fleet;

/* Creates a fleet over count distinct contexts (ctxs: host array; the fleet order; the
 * contexts stay owned by the caller and must outlive the fleet; out receives the fleet, freed
 * by damf_fleet_destroy).  Shares start proportional to d (n + m) (m the
 * initial adjacency entries).  Synchronous (uploads its tables).  DAMF_ERR_INVALID for
 * count < 1, a NULL, repeated or poisoned context. */
damf_status damf_fleet_create(damf_ctx* const* ctxs, int32_t count, damf_fleet** out);

/*
 * One step (per graph Algorithm 2, then the push of Sec. 4.4 for all graphs in one grouped
 * launch): batches[i] (host array in fleet order; its ctx NULL or the fleet's i-th context;
 * its event arrays on the device, read when the step runs) is applied to
 * graph i as by damf_apply_edges (damf_apply_edges_counted when k_dev is set), each graph's
 * update on its context's own stream, forked from `stream`; then the grouped push of every
 * graph; `stream` waits for all of it.  Capturable in one CUDA graph (join every context,
 * damf_join, before the capture starts; new_nodes = 0 and refold_every = 0 keep the host
 * bookkeeping of a captured step the same at every replay).  Afterwards each context reads
 * and joins like after damf_ppr_refresh.  A batch that the host-side checks (arguments, node
 * capacity) reject poisons its own context, and nothing is enqueued for any graph.
 */
damf_status damf_fleet_step(damf_fleet* fleet, const damf_batch* batches, void* stream);

/* Sets the CTAs of each graph's push: blocks (host int32[count], each >= 1, the graphs of one
 * threshold mode summing to at most the resident push CTAs), or with blocks = NULL shares in
 * proportion to (d (n + m))^exponent, exponent in [0, 4]: a graph whose share is below one CTA
 * shares a CTA with other such graphs (first fit, largest first).  Also takes each
 * context's push_direct_chunks (damf_set_tuning) as it is now.  Synchronous: once the fleet
 * has taken a step it waits for all device work (pushes already enqueued or replayed read the
 * old tables); not while a capture is in progress.  A CUDA graph that captured a step of this fleet must be captured again:
 * its grouped push no longer matches the tables, and a replay only sets DAMF_ERR_INVALID on
 * the fleet's contexts.  DAMF_ERR_INVALID (shares unchanged) for bad values. */
damf_status damf_fleet_set_shares(damf_fleet* fleet, const int32_t* blocks, double exponent);

/* Sets the shares from per-graph work estimates (host double[count], each > 0, e.g. a
 * graph's measured push time times its CTAs): CTAs in proportion to the weights, graphs below
 * one CTA's worth packed as with damf_fleet_set_shares (and, like it, synchronous, not while
 * capturing, and requiring captured steps to be captured again).
 * DAMF_ERR_INVALID (shares unchanged) for a weight that is not > 0. */
damf_status damf_fleet_set_weights(damf_fleet* fleet, const double* weights);

/* Phase timing of the following (uncaptured) fleet steps: when enabled, each step records
 * events at its fork, after every graph's update and after the pushes. */
damf_status damf_fleet_set_timing(damf_fleet* fleet, int32_t enable);

/* Waits for the timed steps and returns their summed update-phase and push-phase device time
 * (ms) and their number, then starts counting afresh; any pointer may be NULL. */
damf_status damf_fleet_get_timing(damf_fleet* fleet, double* update_ms, double* push_ms, int32_t* steps);

/* The CTAs each graph's push owns alone (host int32[count], fleet order; 0 for a small graph
 * that shares one CTA with other small graphs, which it pushes after or before them) and the
 * number of grouped launches per step; either pointer may be NULL. */
damf_status damf_fleet_get_shares(const damf_fleet* fleet, int32_t* blocks, int32_t* launches);

/* Kernels the fleet itself has launched (two per grouped push: queue reset and push); the
 * updates' kernels count in each context's damf_stats.launches. */
int64_t damf_fleet_launches(const damf_fleet* fleet);

/*
 * Fault injection on the host (a test hook): the device allocation number `after` from now
 * on (0 = the next) made by damf_init_factorize / damf_restore fails as cudaMalloc out of
 * memory does; the call then returns DAMF_ERR_CAPACITY having freed what it had allocated.
 * One failure per arming; after < 0 disarms.  Not thread-safe (process-wide).
 */
void damf_debug_fail_allocations(int32_t after);

/*
 * Failure detection without a GPU fault: runs one of the push's bounded waits against a
 * condition that never comes true, with an iteration limit of `limit` (1 .. the library's own
 * limit; each iteration sleeps up to about a microsecond), and writes the device status the
 * wait left in *status_out: DAMF_ERR_TIMEOUT (5) when it gave up as it must.  which = 0: the
 * grid barrier, counting one CTA more than are launched; which = 1: the wait for a queue
 * position that nobody fills while a task is still counted.  Uses its own small device
 * allocation (no context) and synchronises `stream`; the device stays usable.
 * DAMF_ERR_INVALID for bad arguments, DAMF_ERR_CUDA when a CUDA call fails.
 */
damf_status damf_selftest_wait(int32_t which, int64_t limit, int32_t* status_out, void* stream);

/* The CTA plan of one grouped push, on the host (what damf_fleet_set_shares and
 * damf_fleet_set_weights compute; exposed for capacity planning and tests).  weights (host
 * double[count], each > 0): the graphs' work; max_blocks: the resident push CTAs.  Graph i's
 * fair share is x_i = max_blocks w_i / sum(w); a graph with x_i >= 1 owns floor(x_i) CTAs,
 * the others are packed largest-first into one-CTA slots of total share <= 1, CTAs left over
 * go to the owners by largest remainder (if the slots do not fit, the packing limit grows by
 * 1.25x until they do).  Writes slot_of[i] (host int32[count]) and ctas[s] (host int32[count];
 * a slot holding several graphs has one CTA).  Returns the number of slots; -1 for bad
 * arguments. */
int32_t damf_plan_slots(const double* weights, int32_t count, int32_t max_blocks, int32_t* slot_of, int32_t* ctas);

/* Text of the fleet's most recent error. */
const char* damf_fleet_last_error(const damf_fleet* fleet);

/* Waits for the fleet's pushes and frees the fleet (not the contexts).  A CUDA graph that
 * captured damf_fleet_step of this fleet must not be replayed afterwards (it reads the
 * fleet's tables). */
void damf_fleet_destroy(damf_fleet* fleet);

/* Launch shape of a context's PPR push (damf_set_tuning, damf_get_tuning). */
typedef struct {
  int32_t push_blocks;        /* CTAs of the persistent push, 256 threads each; 0 = the most that
                                 leave room for the factor chain (2.5 per SM).  Larger
                                 values (up to the push's own occupancy, four per SM) give the
                                 push more warps, but then the next update's factor chain no
                                 longer runs beside it; values above the occupancy are clamped
                                 to it.  Graphs that share the GPU (damf_step_multi) take fewer,
                                 so that their pushes overlap. */
  int32_t push_direct_chunks; /* a row with more in-edges than this many chunks (a chunk is 8,
                                 16, 32, 32 in-edges for d = 128, 64, 32, 16) is pushed as hub
                                 items of 8 in-edges spread over warps; -1 = 8 chunks */
} damf_tuning;

/* Sets the push launch shape for the following pushes (the results stay within the push
 * bound; the order of the floating-point adds changes).  DAMF_ERR_INVALID for
 * push_blocks < 0 or push_direct_chunks outside [-1, 1024] (context unchanged). */
damf_status damf_set_tuning(damf_ctx* ctx, const damf_tuning* tuning);

/* The launch shape the next push uses (defaults and clamping resolved). */
damf_status damf_get_tuning(const damf_ctx* ctx, damf_tuning* tuning);

/*
 * Node deletion (not treated by the paper, whose events add nodes): removes every edge of
 * each node in nodes (host int32[count], ids < n), i.e. zeroes row u and column u of A, as
 * ordinary updates: the node's current adjacency rows (out, and in for a directed graph) are
 * expanded on the device into deletion events, applied like damf_apply_edges (so the result
 * is the rank-d t-SVD of the previous product plus that change, Theorem 2), in chunks of at
 * most 4096 events. The id stays valid as an isolated node; no id is renumbered. Reads each
 * node's degree from the device (synchronises `stream` once per node and direction). The
 * push (damf_ppr_refresh) follows as for any update. DAMF_ERR_INVALID (context usable) for
 * a bad id or argument.
 */
damf_status damf_delete_nodes(damf_ctx* ctx, const int32_t* nodes, int32_t count, void* stream);

/* Same as damf_apply_edges with src, dst, op in (host) memory: the library copies
 * them to the device on `stream` (k <= 4096). */
damf_status damf_apply_edges_host(damf_ctx* ctx, const int32_t* src, const int32_t* dst, const int8_t* op,
                                  int32_t k, int32_t new_nodes, void* stream);

/*
 * Dynamic embedding enhancement (Sec. 4.4; Algorithm 2, last step): pushes on the current
 * graph until max_j |r[u][j]| <= eps for every u (eps * max(deg(u), 1) with the
 * degree-scaled threshold), keeping the invariant  Pi X_b = Z_b + Pi r  with
 * Pi = alpha (I - (1-alpha) D^{-1} A)^{-1}, so that |Z_b - Pi X_b| <= eps elementwise.
 * One persistent launch over a device work queue seeded with the rows whose residual
 * changed since the last push.  DAMF_ERR_NOT_CONVERGED (via damf_sync_status) when
 * max_push_rounds phases did not finish; DAMF_ERR_TIMEOUT when a bounded wait runs out.
 */
damf_status damf_ppr_refresh(damf_ctx* ctx, void* stream);

/*
 * Ordering of the push.  damf_ppr_refresh runs the push on a stream the context owns,
 * after all work enqueued on `stream` before the call; the next damf_apply_edges on
 * `stream` overlaps its read-only part (net change, projection, residual factors, core
 * SVD, transform update) with that push and waits for it before editing the adjacency
 * and the PPR state.  damf_get_embeddings waits for it when Z is requested (X, Y and sigma
 * are final when the update's work on `stream` is), damf_get_state always.
 * damf_join makes `stream` wait for the most recent push (e.g. before the caller reads
 * results produced by it through other means); damf_record_event records a caller's
 * cudaEvent_t (passed as void*) on the push stream after the most recent push.
 *
 * CUDA graph capture: damf_apply_edges (device events), damf_ppr_refresh and damf_join can
 * be captured on `stream`. Call damf_join on `stream` before the capture begins and end the
 * captured work with damf_join (which brings the push stream back into the capture). A
 * replay repeats the captured calls with their k, new_nodes and event pointers (the caller
 * rewrites the event buffers between replays); the host-side fold schedule and node count
 * do not advance on replay, so capture with refold_every = 0 and new_nodes = 0.
 */
damf_status damf_join(damf_ctx* ctx, void* stream);
damf_status damf_record_event(damf_ctx* ctx, void* event);

/*
 * Query (Sec. 4.6, "Query Node's Embedding"): X = U_b P_U Sigma^{1/2},
 * Y = V_b P_V Sigma^{1/2}, Z = Z_b S0^{-1/2} P_U Sigma^{1/2} (S0 = Sigma at the last
 * fold; PPR is linear, so the enhanced embedding maps like X).
 *   rows (device) int32[count] node ids, or NULL for rows 0..count-1.
 *   X, Y, Z (device) float32[count x d] outputs, sigma (device) float32[d]; any
 *   output may be NULL.
 * Only Z depends on the push: with Z = NULL the call follows the work enqueued on `stream`
 * and does not wait for the most recent damf_ppr_refresh, so reading Σ (or X, Y) after each
 * update leaves that push running beside the next update's factor chain.
 */
damf_status damf_get_embeddings(damf_ctx* ctx, const int32_t* rows, int32_t count, float* X, float* Y,
                                float* Z, float* sigma, void* stream);

/*
 * Link-prediction scores (Sec. 5, "Link Prediction", and the appendix "Additional Details of
 * Link Prediction"): the score of the pair (u, v) is the inner product of u's context vector
 * with v's content vector, Z[u] . Y[v] (context = 0, the PPR-enhanced context) or X[u] . Y[v]
 * (context = 1), with X, Y, Z as in damf_get_embeddings. symmetric = 1 scores an undirected
 * pair as the larger of score(u, v) and score(v, u); 0 scores the directed pair (u, v).
 * Computed from the base state through G = P_U Sigma P_V^T (no n x d buffers).
 *   src, dst (device) int32[count] node ids; scores (device) float32[count] output.
 * An id outside [0, n) gives score 0 and DAMF_ERR_INVALID through damf_sync_status.
 * Waits for the most recent push (see damf_join). DAMF_ERR_INVALID for a bad argument
 * (count < 0, context or symmetric not 0/1, a NULL array); such a rejection leaves the
 * context usable.
 */
damf_status damf_score_pairs(damf_ctx* ctx, const int32_t* src, const int32_t* dst, int32_t count,
                             int32_t context, int32_t symmetric, float* scores, void* stream);

/*
 * Top-k link candidates (the ranking behind precision@K of Sec. 5, "Graph Reconstruction"):
 * for each query node u = rows[i], the k nodes v != u with the largest score(u, v) (same
 * score, context and symmetric as damf_score_pairs), in decreasing score; equal scores in
 * increasing node id.
 *   rows (device) int32[count]; out_idx (device) int32[count x k] (row-major, -1 where fewer
 *   than k candidates exist); out_score (device) float32[count x k] (-inf there).
 *   1 <= k <= 64. Queries run in passes of 32; each pass reads V_b (and the context base for
 *   symmetric scores) once. An invalid query id gives a row of -1 and DAMF_ERR_INVALID
 *   through damf_sync_status. A bad argument (k, context, symmetric, NULL arrays) is
 *   rejected with DAMF_ERR_INVALID and leaves the context usable.
 */
damf_status damf_topk(damf_ctx* ctx, const int32_t* rows, int32_t count, int32_t k, int32_t context,
                      int32_t symmetric, int32_t* out_idx, float* out_score, void* stream);

/*
 * Copies the base state to caller buffers (device), rows 0..n-1: Ub, Vb, Zb, r are
 * float32[n x d]; PU, PV float32[d x d] (U = Ub PU, V = Vb PV); sigma, s0 float32[d]
 * (the PPR signal is X_b = Ub diag(s0)).  Any pointer may be NULL.  For tests,
 * inspection and checkpointing.
 */
damf_status damf_get_state(damf_ctx* ctx, float* Ub, float* Vb, float* Zb, float* r, float* PU, float* PV,
                           float* sigma, float* s0, void* stream);

/*
 * Checkpoint and resume (no counterpart in the paper; the state is that of Sec. 4: the bases
 * and transforms of the U-form, Sigma, and the PPR base signal's Z_b and r of Sec. 4.4).  A
 * context's full state, in buffers the caller owns: U_b, V_b, Z_b,
 * r (device) float32[n x d]; P_U, P_V and their inverses (device) float32[d x d] (the
 * library updates the inverses incrementally, so they are saved rather than recomputed);
 * Sigma and s0 (device) float32[d]; and the host count of updates since the last fold.
 */
typedef struct {
  float* Ub;
  float* Vb;
  float* Zb;
  float* r;
  float* PU;
  float* PV;
  float* PUi;
  float* PVi;
  float* sigma;
  float* s0;
  int32_t updates_since_fold;
} damf_state;

/* Copies the state into st's buffers on `stream` after the most recent push (n = the
 * context's current node count, damf_num_nodes) and sets st->updates_since_fold.  With the
 * adjacency from damf_export_adjacency (outgoing) it is everything damf_restore needs. */
damf_status damf_save_state(damf_ctx* ctx, damf_state* st, void* stream);

/*
 * Creates a context from a saved state instead of a factorisation: cfg as for the original
 * (cfg->n = the saved node count; capacities may differ), the adjacency in CSR (device,
 * int32 row_ptr[n+1] and col_idx[m], rows in the exported order), the saved buffers (device;
 * read, not kept).  The result continues the original: the same further calls give
 * bit-identical factors and adjacency (the push, whose add order depends on timing, keeps its
 * eps bound); the next push starts from every row.  A directed graph's in-adjacency is rebuilt
 * from the out-adjacency.  Synchronises `stream`.  DAMF_ERR_INVALID for a bad cfg or a NULL
 * buffer; DAMF_ERR_CAPACITY when a device allocation fails for want of memory (nothing is
 * left allocated), DAMF_ERR_CUDA when another CUDA call fails.
 */
damf_status damf_restore(const damf_config* cfg, const int32_t* row_ptr, const int32_t* col_idx, int64_t m,
                         const damf_state* saved, void* stream, damf_ctx** out);

/*
 * Copies the current adjacency into (host) CSR buffers: row_ptr int64[n+1] and
 * col int32[col_capacity] (row order as stored, not sorted).  outgoing = 1 gives the
 * out-adjacency A[u][.], 0 the in-adjacency (same as outgoing for undirected graphs).
 * Blocks on the device.  DAMF_ERR_CAPACITY when col_capacity is too small.
 */
damf_status damf_export_adjacency(damf_ctx* ctx, int32_t outgoing, int64_t* row_ptr, int32_t* col,
                                  int64_t col_capacity);

/*
 * Touched sets of the most recent update (Lemma 1: the rows of U_b, V_b it rewrote):
 * S (host) int32[128] sorted source rows, T (host) int32[128] sorted target rows.
 * Blocks on the device.
 */
damf_status damf_get_last_touched(damf_ctx* ctx, int32_t* S, int32_t* nS, int32_t* T, int32_t* nT);

/*
 * Step 2 of an update on its own (Sec. 4.5 "Rediagonalization", Eq. "svd_small_edge"):
 * the top-d SVD  E Theta H^T  of the (d + r) x (d + r) core
 *     M = [[diag(sigma), 0], [0, 0]] + L R^T,
 * computed by the kernels of the update path (one-sided block Jacobi on an 8-CTA thread-block
 * cluster, then H = M^T E Theta^{-1}).  No context.
 *   sigma (device) float32[d]; L, R (device) float32[(d+r) x r] row-major (L = [W_B; R_B],
 *   R = [W_C; R_C] in the paper's notation); d in {16, 32, 64, 128}, 1 <= r <= 128.
 *   E, H (device) float32[(d+r) x d] row-major: column k is the k-th left / right
 *   singular vector (non-increasing singular values); theta (device) float32[d].
 *   workspace (device): at least damf_core_svd_workspace_size(d, r) bytes, 256-byte
 *   aligned, owned by the caller; it holds a status word and a copy of M.
 *   status (device) int32, optional (NULL: not written): when the call's stream work is
 *   done it holds the device status of the computation: DAMF_OK, DAMF_ERR_NUMERIC (a
 *   non-finite singular value or vector) or DAMF_ERR_NOT_CONVERGED (the Jacobi sweeps ran
 *   out; the results are then only approximate).  Read it after synchronising the stream.
 * Returns DAMF_ERR_INVALID for bad sizes or NULL pointers, DAMF_ERR_CAPACITY for a short
 * workspace, DAMF_ERR_CUDA when a launch fails; DAMF_OK covers the enqueue only (device
 * errors arrive through `status`).  Asynchronous on `stream`.
 */
size_t damf_core_svd_workspace_size(int32_t d, int32_t r);
damf_status damf_core_svd(const float* sigma, const float* L, const float* R, int32_t d, int32_t r, float* E,
                          float* H, float* theta, void* workspace, size_t workspace_bytes, int32_t* status,
                          void* stream);

/*
 * damf_core_svd without a workspace, for callers that cannot allocate device memory:
 * for example an engine plugin that receives only input and output pointers from a host
 * framework whose allocator owns all device memory, or code on a latency-critical path
 * that must not call cudaMalloc (it can synchronise the device).  The paper has no
 * counterpart; this is a deployment variant of Step 2.
 *   Arguments and results are those of damf_core_svd, `status` included (the status word
 *   itself lives in the library's array, which the caller cannot read, so pass `status` to
 *   learn of a device error).  The caller still provides and owns every input and output.
 *   Nothing is allocated: the scratch (a status word and the assembled core) is one static
 *   device array of 263,168 bytes compiled into the library, which every GPU that loads the
 *   library holds until the process exits.
 *   Limit: d + r <= 256 (d in {16, 32, 64, 128}, 1 <= r <= 128); a larger r returns
 *   DAMF_ERR_CAPACITY, bad d or NULL pointers DAMF_ERR_INVALID.
 *   Every call looks the array's device address up with the caller's device current (so the
 *   address stays right after a device reset); the first call on a device also loads the
 *   library's device code there: make that first call before any stream capture.
 *   All calls on a device share the one array and each call overwrites it (the status
 *   word is cleared at the start of every call): calls that overlap on the GPU (other
 *   streams or threads) race and give undefined results; serialise them.
 */
damf_status damf_core_svd_noalloc(const float* sigma, const float* L, const float* R, int32_t d, int32_t r,
                                  float* E, float* H, float* theta, int32_t* status, void* stream);

/* Current node count as known to the host (initial n plus all node arrivals). */
int32_t damf_num_nodes(const damf_ctx* ctx);

typedef struct {
  int64_t updates;          /* rank-r updates applied (non-empty) */
  int64_t edges_applied;    /* events passed to damf_apply_edges* */
  int64_t entries_changed;  /* net adjacency entries changed (set semantics) */
  int64_t pushes;           /* node pushes (rows moved from r to Z_b) */
  int64_t push_edges;       /* in-edges traversed by pushes */
  int64_t push_rounds;      /* push phases (1 per push unless the work queue overflowed) */
  int64_t fixup_edges;      /* adjacency entries gathered by the graph-change fix-up */
  int64_t touched_rows;     /* sum over updates of |S| + |T| */
  int64_t folds;            /* refolds of the transforms into the bases */
  int32_t last_rank;        /* r of the most recent update */
  int32_t last_status;      /* device status word */
  int64_t launches;         /* kernels launched by this context so far */
  int32_t last_sweeps;      /* Jacobi sweeps of the most recent update's core SVD */
  int32_t reserved;
  int64_t jacobi_sweeps;    /* Jacobi sweeps over all updates */
  int64_t jacobi_full;      /* updates whose core needed sweeps over every pair */
  int64_t jacobi_gersh;     /* updates that needed the exact Gershgorin gap check */
  int64_t push_tasks;       /* push row tasks (a row taken from the queue, pushed or found below eps) */
  int64_t push_items;       /* push hub-item tasks (one chunk of a hub's in-edges) */
  int64_t push_ns[4];       /* push time seen by one CTA (ns): seeding, task loop, grid barriers; [3] the time a warp
                               waited for work, averaged over the push's warps */
} damf_stats;

/* Stages timed by damf_set_timing (indices into damf_get_timing's arrays). */
enum {
  DAMF_STAGE_PREPARE = 0,    /* adjacency edit, set semantics, S, T, N (one CTA) */
  DAMF_STAGE_FIXUP = 1,      /* PPR residual change of changed out-rows */
  DAMF_STAGE_GATHER = 2,     /* U[S] = Ub[S] PU, V[T] = Vb[T] PV */
  DAMF_STAGE_CHOL = 3,       /* residual Grams and Cholesky factors */
  DAMF_STAGE_CORE = 4,       /* core assembly and block Jacobi SVD (8-CTA cluster) */
  DAMF_STAGE_TRANSFORMS = 5, /* H, re-orthonormalised E and H, Theta, R^{-1} E[d:], K, K^{-1}, transform products */
  DAMF_STAGE_SCATTER = 6,    /* base-row rewrite and PPR signal change */
  DAMF_STAGE_PUSH = 7,       /* persistent PPR push */
  DAMF_STAGE_FOLD = 8,       /* periodic fold of the transforms into the bases */
  DAMF_NUM_STAGES = 9
};

/* Enables (1) or disables (0) per-stage timing: CUDA events recorded on the call's
 * stream around each stage's launches.  Costs a few microseconds of host time per stage. */
damf_status damf_set_timing(damf_ctx* ctx, int32_t enable);

/* Accumulated device milliseconds and launch counts per stage since the last call
 * (arrays of DAMF_NUM_STAGES; either may be NULL), then resets them.  Blocks. */
damf_status damf_get_timing(damf_ctx* ctx, double* ms, int64_t* launches);

/* Copies the device counters (blocking on the context's work). */
damf_status damf_get_stats(damf_ctx* ctx, damf_stats* out);

/* Reads the device status word (blocking) and returns it. */
damf_status damf_sync_status(damf_ctx* ctx);

/* Text of the most recent error on this context ("" if none). */
const char* damf_last_error(const damf_ctx* ctx);

/* Frees all device state.  NULL is ignored. */
void damf_destroy(damf_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* DAMF_H_ */
