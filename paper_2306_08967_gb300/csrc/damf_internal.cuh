// Internal declarations shared by the library's translation units.
//
// Device data layout (one context, all in HBM):
//   Ub, Vb      float [n_cap x d]   node-row bases; U = Ub PU, V = Vb PV
//   Zb, r       float [n_cap x d]   PPR state in base space (signal Xb = Ub diag(s0))
//   PU, PV, PUi, PVi  float [d x d] accumulated transforms and their inverses
//   sigma, s0   float [d]           singular values; s0 = sqrt(sigma) at the last fold
//   out / in    slack adjacency: start/len/cap int32 [n_cap], col int32 [m_cap]
//   workspace   the small per-update matrices (rank r <= kMaxR), push lists, rho
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "damf.h"

namespace damf {

constexpr int kMaxR = 128;                // maximum rank of one update
constexpr int kEdgesPerUpdate = 64;       // events per update (undirected: 2 entries each)
constexpr int kMaxEntries = 2 * kEdgesPerUpdate;
constexpr int kMaxD = 128;
constexpr int kMaxM = kMaxD + kMaxR;      // 256: largest core
constexpr int kChainThreads = 512;        // one-CTA chain kernels: leave room beside a push
constexpr long long kSpinLimit = 1ll << 26;  // iterations of a bounded wait (with nanosleep)
constexpr int kTopQ = 32;                 // queries per top-k pass (score.cu)
constexpr int kMaxTopK = 64;              // largest k of damf_topk
constexpr int kTopMaxCtas = 256;          // top-k scan CTAs at most
constexpr int kFixSplit = 16;             // CTAs that share one changed row of the PPR fix-up

// Grid barrier state for persistent cooperative kernels.
struct GridBar {
  unsigned int count;
  unsigned int gen;
};

// Device header: status word, counters, per-update sizes.
struct DevHeader {
  int status;            // first device error (damf_status), 0 = ok
  int nS, nT;            // touched sets of the current update
  int nedit;             // net entries changed by the current update
  int nrowS;             // distinct source rows edited (== nS)
  int rankB, rankC;      // pivots kept by the residual Cholesky factors
  int pending;           // rows queued for the next push (signal or graph changed)
  int check_all;         // next push starts from every node (set by the fold)
  int n_nodes;           // node count after the most recent update (the push's row range)
  unsigned int epoch;    // stamp generation for push dedupe
  long long tail_out, tail_in;   // adjacency bump allocators
  // counters (damf_stats)
  long long updates, edges_applied, entries_changed, pushes, push_edges, push_rounds, fixup_edges,
      touched_rows, folds;
  int last_rank;
  int last_sweeps;       // Jacobi sweeps of the most recent update
  long long jacobi_sweeps, jacobi_full, jacobi_gersh;
  long long push_tasks, push_items;
  unsigned long long push_ns[4];   // block 0 of the push: seeding, task loop, barriers; [3] mean idle (ns)
  // push work queue (ppr.cu), zeroed before each launch: qstate = (tasks not finished << 32) |
  // queue tail; q_head = next queue position to claim; bump counters of rho slots and items
  // Each word every warp of the push hits (qstate at each publication, q_head at each claim)
  // sits on its own 128-byte line, so that their atomics queue at different L2 slices.
  alignas(128) unsigned long long qstate;
  alignas(128) int q_head;
  alignas(128) int overflow;
  int rho_tail;
  int item_tail;
  int ovf_count;    // hub items that found the queue full (processed at the end of the phase)
  // grouped push: warps of other graphs may join this graph's task loop while help_open is set
  // (between the seeding barrier and the end of the loop); helpers counts those inside
  int help_open;
  int helpers;
  alignas(128) GridBar bar;
};

struct Adj {
  int32_t* start;
  int32_t* len;
  int32_t* cap;
  int32_t* col;
  long long m_cap;
};

// The long rows of an adjacency cut into chunks for the initialisation's SpMM (dense.cu).
struct SpmmPlan {
  int nlong = 0, nchunks = 0;
  int* rows = nullptr;      // [nlong] long rows, increasing
  int* first = nullptr;     // [nlong + 1] chunks of row i: first[i] .. first[i + 1] - 1
  int2* chunks = nullptr;   // [nchunks] (first entry, entry count)
  float* P = nullptr;       // [nchunks x l] partial sums
};
cudaError_t spmm_plan(const Adj& a, int n, int l, SpmmPlan* p, cudaStream_t s);
void spmm_plan_free(SpmmPlan* p);
cudaError_t spmm(const Adj& a, int n, const float* X, int l, float* Y, const SpmmPlan* plan, cudaStream_t s);

struct Workspace {
  int32_t* S;        // [kMaxR]
  int32_t* T;        // [kMaxR]
  float* N;          // [kMaxR x kMaxR] net change, rows S, cols T
  int4* edits;       // [kMaxEntries] (u, v, delta, s_index), (u, v) order
  int4* editsT;      // [kMaxEntries] (v, u, delta, -), (v, u) order (directed in-adjacency)
  int32_t* Sfirst;   // [kMaxR + 1] edits of row S[q]: edits[Sfirst[q] .. Sfirst[q+1])
  int32_t* Tfirst;   // [kMaxR + 1] editsT of row T[q]
  long long* relocS; // [kMaxR] new start of a relocated out-row (-1: fits)
  long long* relocT; // [kMaxR]
  int32_t* rcapS;    // [kMaxR] its new capacity
  int32_t* rcapT;
  int32_t* deg_old;  // [kMaxR] out-degree of S rows before/after
  int32_t* deg_new;
  float* UST;        // [kMaxR x d] rows U[S] = Ub[S] PU
  float* VT;         // [kMaxR x d] rows V[T] = Vb[T] PV
  float* WCt;        // [kMaxR x d] N V[T]  (= W_C^T)
  float* RB;         // [kMaxR x kMaxR] upper Cholesky factor (dropped rows zero)
  float* RC;
  float* M;          // [kMaxM x kMaxM] core, column-major with leading dimension m
  float* E;          // [kMaxM x d] left singular vectors (column k = k-th largest)
  float* H;          // [kMaxM x d]
  float* theta;      // [d]
  // refinement of the core SVD (update.cu): P = E^T L, Q = H^T R, T = E^T M H
  float* foP;        // [d x kMaxR]
  float* foQ;        // [d x kMaxR]
  float* foT;        // [d x d]
  // PPR fix-up: partial sums of the CTAs that share a row, and per-row arrival counters
  float* fixpart;    // [kMaxR x kFixSplit x d]
  int32_t* fixcnt;   // [kMaxR], zero between launches
  float* YB;         // [kMaxR x d]  R_B^{-1} E[d:]
  float* YC;         // [kMaxR x d]  R_C^{-1} H[d:]
  float* KU;         // [d x d]
  float* KV;
  float* KUi;
  float* KVi;
  float* tmp;        // [4 x d x d] scratch for products
  // push
  int32_t* queue;    // [qcap] push tasks: row id >= 0, item i as -(i + 2), -1 empty
  long long qcap;
  int4* work;        // [work_cap] hub items (rho slot, first in-edge, in-edge count, -)
  long long work_cap;
  float* rho;        // [rho_cap x d] residuals of the hub pushes
  long long rho_cap;
  int32_t* ovf;      // [work_cap] ids of hub items that found the queue full
  uint32_t* stamp;   // [n_cap] 1 while the row is in the push queue
  int32_t* pend;     // [n_cap] rows queued for the next push
  uint32_t* pstamp;  // [n_cap]
  // link-prediction scores (score.cu), one region
  float* sG;         // [d x d] PU diag(sigma) PV^T
  float* sIs0;       // [d] 1/s0
  float* sLq;        // [kTopQ x d] query rows times G
  float* sRq;        // [kTopQ x d] query content rows times G^T
  int32_t* sQid;     // [kTopQ] query node ids (-1: invalid)
  unsigned long long* sPart;  // [kTopMaxCtas x kTopQ x kMaxTopK] per-CTA sorted keys
  // fold
  float* gram;       // [2 x d x d] reduced Grams
  float* gram_part;  // [gram_parts x d x d]
  int gram_parts;
};

struct Ctx {
  damf_config cfg;
  int d;
  int n;           // host-tracked node count
  int l;           // randomized t-SVD width
  DevHeader* hdr;
  float *Ub, *Vb, *Zb, *r;
  float *PU, *PV, *PUi, *PVi, *sigma, *s0;
  Adj out, in;
  Workspace ws;
  long long m_init;      // adjacency entries of the initial graph (a size hint for shares)
  int push_blocks;       // requested persistent push grid size (0: push_max)
  int push_max;          // default push CTAs on the device, 2.5 per SM (0: not yet known)
  int push_occ;          // co-resident push CTAs when the push takes the whole occupancy
  int push_direct_chunks;  // in-edge chunks a row task scatters itself (-1: default)
  // damf_step_multi runs this graph's update on its own stream, forked from the caller's
  cudaStream_t own_stream;
  cudaEvent_t ev_fork;    // caller-stream point the graph's work follows
  cudaEvent_t ev_done;    // the graph's update and push, joined on own_stream
  int updates_since_fold;
  int32_t* host_stage;   // pinned staging for damf_apply_edges_host
  int32_t* dev_stage;    // device copy of staged events
  char errbuf[256];
  int sticky;            // host-side poisoned status
  int check_all_next;    // next push starts from every row (after a fold)
  // the PPR push runs on its own stream so the next update's factor chain overlaps it
  cudaStream_t push_stream;
  cudaEvent_t ev_caller;  // caller-stream work a push must follow
  cudaEvent_t ev_push;    // the most recent push
  cudaEvent_t ev_push_cap;  // the most recent push recorded inside a stream capture
  unsigned long long push_capture_id;  // capture that recorded ev_push_cap (0: none)
  long long launches;    // kernels this context has launched (host count)
  // per-stage timing (api.cu)
  int timing;
  cudaEvent_t* ev;       // 2 * kTimerPairs events
  int* ev_stage;         // stage of each pair
  int ev_used;
  double stage_ms[DAMF_NUM_STAGES];
  long long stage_launches[DAMF_NUM_STAGES];
  void* allocs[96];
  int nallocs;
};

// ---- small device helpers ----
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void set_status(DevHeader* h, int code) {
  atomicCAS(&h->status, 0, code);
}

// Device bounds checks of a DAMF_CHECK build: true when cond holds; otherwise the status
// becomes DAMF_ERR_BOUNDS and the caller skips the access. Compiled out (always true) in the
// default build.
#ifdef DAMF_CHECK
#define DAMF_DCHECK(h, cond) ((cond) ? true : (set_status((h), DAMF_ERR_BOUNDS), false))
#else
#define DAMF_DCHECK(h, cond) true
#endif

// Bounded sense-free grid barrier: every block must call it the same number of times.
// Returns false (and records DAMF_ERR_TIMEOUT) when a wait runs out.
__device__ __forceinline__ bool grid_barrier(GridBar* bar, DevHeader* h, unsigned int nblocks,
                                             long long limit = kSpinLimit) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    volatile unsigned int* vgen = &bar->gen;
    unsigned int gen = *vgen;
    __threadfence();
    unsigned int arrived = atomicAdd(&bar->count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      long long it = 0;
      while (*vgen == gen) {
        if (++it > limit) {
          ok = 0;
          set_status(h, DAMF_ERR_TIMEOUT);
          break;
        }
        if (it > 4096) __nanosleep(64);   // short phases finish within the first spins
      }
    }
    __threadfence();
    ok_s = ok;
  }
  __syncthreads();
  return ok_s != 0;
}

// ---- launchers implemented in the .cu files ----
cudaError_t launch_edit(Ctx* c, cudaStream_t s);
// k events, or (kdev != NULL) the first *kdev of them clamped to [0, k]; the update starting
// at event lo takes events lo .. lo + k - 1 of the arrays, of which *kdev - lo are live
cudaError_t launch_validate(Ctx* c, const int32_t* src, const int32_t* dst, const int8_t* op, int k,
                            const int32_t* kdev, int n_after, cudaStream_t s);
cudaError_t launch_prepare(Ctx* c, const int32_t* src, const int32_t* dst, const int8_t* op, int k,
                           const int32_t* kdev, int lo, cudaStream_t s);
cudaError_t launch_fixup(Ctx* c, cudaStream_t s);
cudaError_t launch_gather(Ctx* c, cudaStream_t s);
cudaError_t launch_chol(Ctx* c, cudaStream_t s);
cudaError_t launch_core(Ctx* c, cudaStream_t s);
cudaError_t launch_transforms(Ctx* c, cudaStream_t s);
cudaError_t launch_scatter(Ctx* c, cudaStream_t s);
int push_default_direct_chunks();
cudaError_t launch_wait_selftest(DevHeader* h, int32_t* queue, int which, long long limit, cudaStream_t s);
// One graph's push operands (the grouped push reads them from device memory).
struct PushArgs {
  DevHeader* h;
  Adj in;                  // in-adjacency (the out-adjacency of an undirected graph)
  const int32_t* outdeg;
  Workspace ws;
  float* Zb;
  float* r;
  float alpha, eps;
  int max_phases;
  int direct_max;          // in-edges a row task scatters itself
  int d;
  int ncap;                // node capacity: every row id is below it (checked in DAMF_CHECK builds)
};
PushArgs push_args(const Ctx* c, int direct_chunks);
int push_group_max_blocks(int scaled);
// Grouped push of descs[0 .. ngraphs): table holds (nslots, blocks, plan), then sfirst[nslots + 1]
// (CTA prefix sums, ending at `blocks`), then gfirst[nslots + 1] (graph prefix sums, ending at
// ngraphs); a slot of several graphs has one CTA. A launch whose (nslots, blocks, plan) differ
// from the table's does nothing but set DAMF_ERR_INVALID on its graphs.
cudaError_t launch_push_group(const PushArgs* descs, int ngraphs, const int* table, int nslots, int blocks,
                              int plan, int scaled, cudaStream_t s);
cudaError_t launch_push(Ctx* c, int check_all, cudaStream_t s);
cudaError_t launch_expand_row(Ctx* c, int u, int cnt, int incoming, int32_t* src, int32_t* dst, int8_t* op,
                              cudaStream_t s);
cudaError_t launch_score_pairs(Ctx* c, const int32_t* src, const int32_t* dst, int count, int context, int symmetric,
                               float* scores, cudaStream_t s);
cudaError_t launch_topk(Ctx* c, const int32_t* rows, int count, int k, int context, int symmetric, int32_t* out_idx,
                        float* out_score, cudaStream_t s);
cudaError_t launch_fold(Ctx* c, cudaStream_t s);
cudaError_t launch_query(Ctx* c, const int32_t* rows, int count, float* X, float* Y, float* Z, float* sigma,
                         cudaStream_t s);
cudaError_t build_adjacency(Ctx* c, Adj* a, const int32_t* row_ptr, const int32_t* col_idx, int64_t m, int n,
                            long long* tail_dev, int transpose, cudaStream_t s);
cudaError_t init_factorize(Ctx* c, const int32_t* row_ptr, const int32_t* col_idx, int64_t m, const float* omega,
                           cudaStream_t s);

// dense helpers (dense.cu)
// C[rows x N] (+)= A[rows x K] * B[K x N]; A row i taken from A + idx[i]*lda when idx != nullptr.
cudaError_t gemm_rowgather(const float* A, int lda, const int32_t* idx, const int* rows_dev, int rows_max,
                           const float* B, int K, int N, float* C, int ldc, int accumulate, cudaStream_t s);
// n x K by K x N product for a context (tensor cores in mixed precision where covered)
cudaError_t gemm_ctx(Ctx* c, const float* A, int lda, long long n, const float* B, int K, int N, float* C, int ldc,
                     const float* ascale, const float* cscale, cudaStream_t s);
// tall-skinny C[n x N] = A[n x K] B[K x N] (K, N <= 160, multiples of 16)
cudaError_t gemm_tall(const float* A, int lda, long long n, const float* B, int K, int N, float* C, int ldc,
                      cudaStream_t s);
// partial Grams of A[n x K]: out[K x K] = A^T A (uses ws.gram_part)
cudaError_t gram_tall(Ctx* c, const float* A, int lda, long long n, int K, float* out, cudaStream_t s);
// one-CTA Cholesky (lower, G = L L^T) and inverse of L^T; out Linvt[K x K] with A * Linvt orthonormal
cudaError_t chol_inv_upper(const float* G, int K, float* Rinv, DevHeader* h, cudaStream_t s);
// dense one-sided block Jacobi SVD (8-CTA cluster) of an m x m column-major matrix: top-d
// (E, theta, H); report_nc = 1 records DAMF_ERR_NOT_CONVERGED in h when the sweeps run out
cudaError_t jacobi_svd_dense(const float* Min, int m, int d, float* E, float* H, float* theta, int report_nc,
                             DevHeader* h, cudaStream_t s);

}  // namespace damf
