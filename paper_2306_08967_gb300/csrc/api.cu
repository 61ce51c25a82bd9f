// C ABI entry points (include/damf.h): context lifetime, per-call orchestration on the
// caller's stream, and the initial factorisation (Appendix A, Algorithm 3).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "damf_internal.cuh"

namespace damf {
cudaError_t chol_inv_upper2(const float* G, int K, float* R, float* Rinv, DevHeader* h, cudaStream_t s);
cudaError_t small_mm(const float* A, const float* B, float* C, int K, cudaStream_t s);
cudaError_t gemm_tall_scaled(const float* A, int lda, long long n, const float* B, int K, int N, float* C, int ldc,
                             const float* ascale, const float* cscale, cudaStream_t s);
}  // namespace damf

using namespace damf;

struct damf_ctx {
  Ctx c;
};

namespace {

constexpr int kHostStageMax = 4096;
constexpr int kTimerPairs = 16384;

void harvest_timing(Ctx* c) {
  if (!c->ev || c->ev_used == 0) return;
  cudaDeviceSynchronize();
  for (int i = 0; i < c->ev_used; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[2 * i], c->ev[2 * i + 1]) == cudaSuccess) c->stage_ms[c->ev_stage[i]] += ms;
  }
  c->ev_used = 0;
}

// Records a start event for `stage` when timing is on; returns the pair index or -1.
int timer_begin(Ctx* c, int stage, cudaStream_t s) {
  if (!c->timing || !c->ev) return -1;
  if (c->ev_used == kTimerPairs) harvest_timing(c);
  const int i = c->ev_used++;
  c->ev_stage[i] = stage;
  cudaEventRecord(c->ev[2 * i], s);
  return i;
}

void timer_end(Ctx* c, int i, int stage, int launches, cudaStream_t s) {
  c->stage_launches[stage] += launches;
  if (i >= 0) cudaEventRecord(c->ev[2 * i + 1], s);
}

#define DAMF_STAGE(stage, nl, call, what)          \
  do {                                            \
    const int ti_ = timer_begin(c, stage, s);      \
    DAMF_CUDA(call, what);                        \
    timer_end(c, ti_, stage, nl, s);              \
  } while (0)
// kernels per update: prepare, gather, wct, chol, assemble, jacobi, hmat, ns_gram, ns_apply,
// fo_pq, fo_t, fo_apply, fo_norm_theta, trans, inverse, products, commit, edit, fixup, scatter
constexpr int kLaunchesPerUpdate = 20;
// fold: 2 x (gram part + reduce), 2 x (congruence + chol), core, jacobi, hmat, 4 small_mm,
// finish, 4 tall GEMMs
constexpr int kLaunchesPerFold = 4 + 4 + 1 + 2 + 4 + 1 + 4;

bool cfg_ok(const damf_config* cfg) {
  if (!cfg) return false;
  if (!(cfg->d == 16 || cfg->d == 32 || cfg->d == 64 || cfg->d == 128)) return false;
  if (cfg->n < 1 || cfg->n_capacity < cfg->n) return false;
  if (cfg->m_capacity < 1 || cfg->m_capacity > 0x7fffffffll) return false;
  if (!(cfg->alpha > 0.0 && cfg->alpha <= 1.0) || !(cfg->eps > 0.0)) return false;
  if (cfg->rsvd_oversample < 0 || cfg->rsvd_power_iters < 0 || cfg->max_push_rounds < 1) return false;
  if (cfg->refold_every < 0) return false;
  if (cfg->precision != 0 && cfg->precision != 1) return false;
  if (cfg->threshold != 0 && cfg->threshold != 1) return false;
  return true;
}

int width_of(const damf_config* cfg) {
  int l = cfg->d + cfg->rsvd_oversample;
  l = (l + 31) / 32 * 32;
  if (l > 160) l = 160;
  if (l < cfg->d) l = cfg->d;
  return l;
}

// hub items of one push phase, and the rho slots holding the vectors of pushed hub rows; a
// hub row that finds either full is scattered by its own warp instead, so the caps bound
// memory on very large graphs (2^28 items, 2^23 slots: 5.4 + 4.3 GB at d = 128) without
// changing any result
long long work_cap_of(const damf_config* cfg) {
  const long long w = 2 * ((long long)cfg->n_capacity + cfg->m_capacity / 4 + 64);
  return w > (1ll << 28) ? (1ll << 28) : w;
}

long long rho_slots_of(const damf_config* cfg) {
  const long long s = 2ll * cfg->n_capacity;
  return s > (1ll << 23) ? (1ll << 23) : s;
}

// push queue positions of one phase (a phase that needs more rescans every row); the
// environment variable DAMF_PUSH_QUEUE_CAP overrides it (testing the overflow path)
long long qcap_of(const damf_config* cfg) {
  long long q = 4ll * cfg->n_capacity + (1ll << 20);
  if (const char* ev = getenv("DAMF_PUSH_QUEUE_CAP")) {
    const long long v = atoll(ev);
    if (v >= 64) q = v;
  }
  return q > 0x7fffff00ll ? 0x7fffff00ll : q;
}

// CTAs (and FP32 partial Grams) of a tall Gram: about 2,048 rows each, at most 8,192 (a part's
// FP32 sum then spans <= 6,200 rows at n = 50M; the parts are added in FP64)
int gram_parts_of(const damf_config* cfg) {
  long long p = (cfg->n_capacity + 2047) / 2048;
  if (p > 8192) p = 8192;
  if (p < 1) p = 1;
  return (int)p;
}

// Sizes of every device allocation, in order (shared by damf_bytes_required and create).
// scoring scratch: G, 1/s0, Lq, Rq, query ids, per-CTA top-k keys (256-byte aligned parts)
size_t score_part(size_t bytes) { return (bytes + 255) & ~(size_t)255; }
size_t score_bytes(size_t d) {
  return score_part(d * d * 4) + score_part(d * 4) + 2 * score_part((size_t)kTopQ * d * 4) + score_part(kTopQ * 4) +
         score_part((size_t)kTopMaxCtas * kTopQ * kMaxTopK * 8);
}

struct Plan {
  size_t sz[96];
  int count;
};

Plan plan_of(const damf_config* cfg) {
  Plan p{};
  const size_t n = (size_t)cfg->n_capacity, d = (size_t)cfg->d, m = (size_t)cfg->m_capacity;
  const size_t nd = n * d * sizeof(float);
  const size_t dd = d * d * sizeof(float);
  size_t* s = p.sz;
  int k = 0;
  s[k++] = sizeof(DevHeader);
  s[k++] = nd; s[k++] = nd; s[k++] = nd; s[k++] = nd;      // Ub Vb Zb r
  s[k++] = dd; s[k++] = dd; s[k++] = dd; s[k++] = dd;      // PU PV PUi PVi
  s[k++] = d * sizeof(float); s[k++] = d * sizeof(float);  // sigma s0
  for (int a = 0; a < (cfg->directed ? 2 : 1); ++a) {
    s[k++] = n * 4; s[k++] = n * 4; s[k++] = n * 4; s[k++] = m * 4;  // start len cap col
  }
  s[k++] = kMaxR * 4; s[k++] = kMaxR * 4;                   // S T
  s[k++] = (size_t)kMaxR * kMaxR * 4;                        // N
  s[k++] = (size_t)kMaxEntries * sizeof(int4);               // edits
  s[k++] = (size_t)kMaxEntries * sizeof(int4);               // editsT
  s[k++] = (kMaxR + 1) * 4; s[k++] = (kMaxR + 1) * 4;        // Sfirst Tfirst
  s[k++] = kMaxR * 8; s[k++] = kMaxR * 8;                    // relocS relocT
  s[k++] = kMaxR * 4; s[k++] = kMaxR * 4;                    // rcapS rcapT
  s[k++] = kMaxR * 4; s[k++] = kMaxR * 4;                    // deg_old deg_new
  s[k++] = (size_t)kMaxR * d * 4; s[k++] = (size_t)kMaxR * d * 4; s[k++] = (size_t)kMaxR * d * 4;  // UST VT WCt
  s[k++] = (size_t)kMaxR * kMaxR * 4; s[k++] = (size_t)kMaxR * kMaxR * 4;                              // RB RC
  s[k++] = (size_t)kMaxM * kMaxM * 4;                        // M
  s[k++] = (size_t)kMaxM * d * 4; s[k++] = (size_t)kMaxM * d * 4;  // E H
  s[k++] = d * 4;                                            // theta
  s[k++] = (2 * (size_t)kMaxR * d + d * d) * sizeof(float);   // foP foQ foT
  s[k++] = ((size_t)kMaxR * kFixSplit * d + kMaxR) * sizeof(float);   // fixpart fixcnt
  s[k++] = (size_t)kMaxR * d * 4; s[k++] = (size_t)kMaxR * d * 4;  // YB YC
  s[k++] = dd; s[k++] = dd; s[k++] = dd; s[k++] = dd;        // KU KV KUi KVi
  s[k++] = 4 * dd;                                           // tmp
  s[k++] = (size_t)qcap_of(cfg) * 4;                         // push queue
  s[k++] = (size_t)work_cap_of(cfg) * sizeof(int4);          // hub items
  s[k++] = (size_t)rho_slots_of(cfg) * d * sizeof(float);   // rho
  s[k++] = (size_t)work_cap_of(cfg) * 4;                     // overflowed hub items
  s[k++] = n * 4; s[k++] = n * 4; s[k++] = n * 4;            // stamp pend pstamp
  s[k++] = 2 * (size_t)160 * 160 * 4;                        // gram (room for the init width)
  s[k++] = (size_t)gram_parts_of(cfg) * 160 * 160 * 4;       // gram_part
  s[k++] = score_bytes(d);                                   // link-prediction scratch
  p.count = k;
  return p;
}

damf_status fail(Ctx* c, damf_status st, const char* what, cudaError_t e) {
  if (c) {
    snprintf(c->errbuf, sizeof(c->errbuf), "%s: %s", what, e == cudaSuccess ? "" : cudaGetErrorString(e));
    if (st != DAMF_OK && c->sticky == DAMF_OK) c->sticky = st;
  }
  return st;
}

// A rejected argument of a query: the message is kept, the context stays usable.
damf_status reject(Ctx* c, const char* what) {
  snprintf(c->errbuf, sizeof(c->errbuf), "%s", what);
  return DAMF_ERR_INVALID;
}

// Device allocations of a context go through here: the test hook damf_debug_fail_allocations
// can make the n-th one fail as cudaMalloc out of memory does (fault injection on the host).
int g_fail_alloc_after = -1;

cudaError_t dev_alloc(void** p, size_t bytes) {
  if (g_fail_alloc_after == 0) {
    g_fail_alloc_after = -1;
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  if (g_fail_alloc_after > 0) --g_fail_alloc_after;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) cudaGetLastError();   // not sticky: clear it
  return e;
}

// Makes `s` wait for the most recent push. Under stream capture: a push captured in the same
// capture is waited for through its own event; a push from before the capture is the caller's
// to join before capturing (so nothing is added). Outside a capture: the last push recorded
// outside any capture (work after a graph replay is ordered by the graph's final join).
cudaError_t wait_push(Ctx* c, cudaStream_t s) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  unsigned long long id = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cap, &id);
  if (e != cudaSuccess) return e;
  if (cap == cudaStreamCaptureStatusNone) return cudaStreamWaitEvent(s, c->ev_push, 0);
  return c->push_capture_id == id ? cudaStreamWaitEvent(s, c->ev_push_cap, 0) : cudaSuccess;
}

// Records that the most recent push of `c` ends at the current tail of `s` (the stream the
// push ran on): its own event inside a stream capture (keyed by the capture), ev_push outside.
cudaError_t note_push(Ctx* c, cudaStream_t s) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  unsigned long long id = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cap, &id);
  if (e != cudaSuccess) return e;
  const bool captured = cap != cudaStreamCaptureStatusNone;
  c->push_capture_id = captured ? id : 0;
  return cudaEventRecord(captured ? c->ev_push_cap : c->ev_push, s);
}

#define DAMF_CUDA(call, what)                                  \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return fail(c, DAMF_ERR_CUDA, what, e_); \
  } while (0)

void free_all(Ctx* c) {
  if (c->push_stream) cudaStreamDestroy(c->push_stream);
  if (c->ev_caller) cudaEventDestroy(c->ev_caller);
  if (c->ev_push) cudaEventDestroy(c->ev_push);
  if (c->ev_push_cap) cudaEventDestroy(c->ev_push_cap);
  if (c->own_stream) cudaStreamDestroy(c->own_stream);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_done) cudaEventDestroy(c->ev_done);
  c->own_stream = nullptr;
  c->ev_fork = c->ev_done = c->ev_push_cap = nullptr;
  c->push_stream = nullptr;
  c->ev_caller = c->ev_push = nullptr;
  if (c->ev) {
    for (int i = 0; i < 2 * kTimerPairs; ++i)
      if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    free(c->ev);
    free(c->ev_stage);
    c->ev = nullptr;
  }
  for (int i = 0; i < c->nallocs; ++i) cudaFree(c->allocs[i]);
  c->nallocs = 0;
  if (c->host_stage) cudaFreeHost(c->host_stage);
  c->host_stage = nullptr;
}

__global__ void k_init_state(float* Ub, float* r, const float* sigma, float* s0, float* PU, float* PV, float* PUi,
                             float* PVi, int n, int d) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < (long long)n * d) {
    const int k = (int)(i % d);
    r[i] = Ub[i] * sqrtf(fmaxf(sigma[k], 0.0f));
  }
  if (i < (long long)d * d) {
    const float v = (i / d == i % d) ? 1.0f : 0.0f;
    PU[i] = PV[i] = PUi[i] = PVi[i] = v;
  }
  if (i < d) s0[i] = sqrtf(fmaxf(sigma[i], 0.0f));
}

}  // namespace

namespace damf {

// Randomized t-SVD (Halko et al. 2011, randomized subspace iteration; Algorithm 3 line 1):
// Q = orth(A Omega); q times: Q' = orth(A^T Q), Q = orth(A Q'); Bt = A^T Q = Q2 R2;
// R2^T = E Theta H^T (Jacobi);  U = Q E, V = Q2 H.  orth() is CholQR applied twice.
cudaError_t init_factorize(Ctx* c, const int32_t*, const int32_t*, int64_t, const float* omega, cudaStream_t s) {
  const int n = c->n, l = c->l, d = c->d;
  const size_t nl = (size_t)n * l * sizeof(float);
  float *Y = nullptr, *Q = nullptr, *Q2 = nullptr, *G = nullptr, *R = nullptr, *Ri = nullptr, *R2 = nullptr,
        *Rt = nullptr;
  cudaError_t e;
  const Adj& out = c->out;
  const Adj& in = c->cfg.directed ? c->in : c->out;
  SpmmPlan pout, pin_;   // long rows of the out- and (directed) in-adjacency
  const SpmmPlan* pin = c->cfg.directed ? &pin_ : &pout;
  const size_t ll = (size_t)l * l * sizeof(float);
  if ((e = cudaMalloc(&Y, nl)) != cudaSuccess) goto done;
  if ((e = cudaMalloc(&Q, nl)) != cudaSuccess) goto done;
  if ((e = cudaMalloc(&Q2, nl)) != cudaSuccess) goto done;
  if ((e = cudaMalloc(&G, ll)) != cudaSuccess) goto done;
  if ((e = cudaMalloc(&R, ll)) != cudaSuccess) goto done;
  if ((e = cudaMalloc(&Ri, ll)) != cudaSuccess) goto done;
  if ((e = cudaMalloc(&R2, ll)) != cudaSuccess) goto done;
  if ((e = cudaMalloc(&Rt, ll)) != cudaSuccess) goto done;
  if ((e = spmm_plan(out, n, l, &pout, s)) != cudaSuccess) goto done;
  if (c->cfg.directed && (e = spmm_plan(in, n, l, &pin_, s)) != cudaSuccess) goto done;
  {
    // orth(X) in place into dst with its triangular factor accumulated in Racc (optional)
    auto orth = [&](const float* X, float* dst, float* Racc) -> cudaError_t {
      cudaError_t ee;
      if ((ee = gram_tall(c, X, l, n, l, G, s)) != cudaSuccess) return ee;
      if ((ee = chol_inv_upper2(G, l, Racc ? R : nullptr, Ri, c->hdr, s)) != cudaSuccess) return ee;
      if ((ee = gemm_ctx(c, X, l, n, Ri, l, l, dst, l, nullptr, nullptr, s)) != cudaSuccess) return ee;
      if ((ee = gram_tall(c, dst, l, n, l, G, s)) != cudaSuccess) return ee;
      if ((ee = chol_inv_upper2(G, l, Racc ? Rt : nullptr, Ri, c->hdr, s)) != cudaSuccess) return ee;
      if ((ee = gemm_ctx(c, dst, l, n, Ri, l, l, dst, l, nullptr, nullptr, s)) != cudaSuccess) return ee;
      if (Racc) {  // X = dst (Rt R): R_total = Rt R
        if ((ee = small_mm(Rt, R, Racc, l, s)) != cudaSuccess) return ee;
      }
      return cudaSuccess;
    };
    if ((e = spmm(out, n, omega, l, Y, &pout, s)) != cudaSuccess) goto done;
    if ((e = orth(Y, Q, nullptr)) != cudaSuccess) goto done;
    for (int it = 0; it < c->cfg.rsvd_power_iters; ++it) {
      if ((e = spmm(in, n, Q, l, Y, pin, s)) != cudaSuccess) goto done;
      if ((e = orth(Y, Q2, nullptr)) != cudaSuccess) goto done;
      if ((e = spmm(out, n, Q2, l, Y, &pout, s)) != cudaSuccess) goto done;
      if ((e = orth(Y, Q, nullptr)) != cudaSuccess) goto done;
    }
    if ((e = spmm(in, n, Q, l, Y, pin, s)) != cudaSuccess) goto done;  // Bt = A^T Q
    if ((e = orth(Y, Q2, R2)) != cudaSuccess) goto done;         // Bt = Q2 R2
    // R2 row-major == (R2^T) column-major: the Jacobi input is R2^T
    if ((e = jacobi_svd_dense(R2, l, d, c->ws.E, c->ws.H, c->ws.theta, 0, c->hdr, s)) != cudaSuccess) goto done;
    if ((e = gemm_ctx(c, Q, l, n, c->ws.E, l, d, c->Ub, d, nullptr, nullptr, s)) != cudaSuccess) goto done;
    if ((e = gemm_ctx(c, Q2, l, n, c->ws.H, l, d, c->Vb, d, nullptr, nullptr, s)) != cudaSuccess) goto done;
    if ((e = cudaMemcpyAsync(c->sigma, c->ws.theta, sizeof(float) * d, cudaMemcpyDeviceToDevice, s)) != cudaSuccess)
      goto done;
    const long long tot = (long long)n * d;
    k_init_state<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(c->Ub, c->r, c->sigma, c->s0, c->PU, c->PV, c->PUi,
                                                                c->PVi, n, d);
    if ((e = cudaGetLastError()) != cudaSuccess) goto done;
    e = cudaStreamSynchronize(s);
  }
done:
  cudaStreamSynchronize(s);
  spmm_plan_free(&pout);
  spmm_plan_free(&pin_);
  cudaFree(Y);
  cudaFree(Q);
  cudaFree(Q2);
  cudaFree(G);
  cudaFree(R);
  cudaFree(Ri);
  cudaFree(R2);
  cudaFree(Rt);
  return e;
}

}  // namespace damf

// ---- fleets: many graphs stepped together, their pushes in one grouped launch ----
struct FleetLaunch {
  int scaled;        // threshold mode of its graphs
  int first_graph;   // its graphs: descriptor positions first_graph .. first_graph + count
  int count;
  int nslots;
  int blocks;
  int table_off;     // its sfirst / gfirst table in d_table
};

struct damf_fleet {
  std::vector<damf_ctx*> ctxs;   // fleet order (damf_fleet_step's batches follow it)
  std::vector<int> blocks;       // CTAs each graph owns alone (0: it shares one CTA with others)
  std::vector<FleetLaunch> launches;
  PushArgs* d_descs = nullptr;   // per launch position
  int* d_table = nullptr;
  size_t table_cap = 0;
  cudaStream_t push_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_done = nullptr;
  long long launches_total = 0;
  int plan_id = 0;               // changes with every plan; captured launches carry theirs
  int stepped = 0;               // damf_fleet_step was called (directly or while capturing)
  // phase timing (damf_fleet_set_timing): per step, events at the fork, before and after the pushes
  int timing = 0;
  std::vector<cudaEvent_t> tev;
  size_t tev_used = 0;
  char errbuf[256] = {0};
};

namespace {

damf_status fleet_fail(damf_fleet* f, damf_status st, const char* what, cudaError_t e = cudaSuccess) {
  snprintf(f->errbuf, sizeof(f->errbuf), "%s%s%s", what, e == cudaSuccess ? "" : ": ",
           e == cudaSuccess ? "" : cudaGetErrorString(e));
  return st;
}

struct Slot {
  int blocks;
  std::vector<int> graphs;   // fleet indices
};

// Slots of `w.size()` graphs with work weights w over at most maxb CTAs (Slot.graphs holds
// positions in w): graph j's fair share is x_j = maxb w_j / sum(w); a graph with x_j >= cap
// owns floor(x_j) CTAs (at least one), the rest are packed first-fit-decreasing into one-CTA
// bins of total share <= cap, and CTAs left over go to the owners by largest remainders; cap
// starts at 1 and grows until the slots fit. When no graph owns CTAs (more graphs than CTAs),
// nobody could take the CTAs the last growth step left over, so cap is then narrowed by
// bisection towards the smallest one that fits, keeping the plan with the most bins.
void pack_slots(const std::vector<double>& w, int maxb, std::vector<Slot>* out) {
  const int cnt = (int)w.size();
  std::vector<double> x(cnt);
  double wsum = 0.0;
  for (int j = 0; j < cnt; ++j) wsum += w[j];
  for (int j = 0; j < cnt; ++j) x[j] = maxb * w[j] / wsum;
  std::vector<int> by_x(cnt);
  for (int j = 0; j < cnt; ++j) by_x[j] = j;
  std::sort(by_x.begin(), by_x.end(), [&](int a, int b) { return x[a] > x[b] || (x[a] == x[b] && a < b); });
  std::vector<Slot> owners, bins;
  std::vector<double> rem;
  // the slots for one cap; returns the CTAs they take
  auto attempt = [&](double cap) -> long long {
    owners.clear();
    bins.clear();
    rem.clear();
    std::vector<double> bin_load;
    for (int j : by_x) {
      if (x[j] >= cap) {
        owners.push_back(Slot{std::max(1, (int)std::floor(x[j])), {j}});
        rem.push_back(x[j] - std::floor(x[j]));
        continue;
      }
      size_t b = 0;
      while (b < bins.size() && bin_load[b] + x[j] > cap) ++b;
      if (b == bins.size()) {
        bins.push_back(Slot{1, {}});
        bin_load.push_back(0.0);
      }
      bins[b].graphs.push_back(j);
      bin_load[b] += x[j];
    }
    long long used = (long long)bins.size();
    for (const Slot& o : owners) used += o.blocks;
    return used;
  };
  double lo = 0.0;   // the largest cap seen that did not fit
  for (double cap = 1.0;; cap *= 1.25) {
    long long used = attempt(cap);
    if (used > maxb) {   // cap >= maxb leaves one bin, so this ends
      lo = cap;
      continue;
    }
    if (owners.empty() && used < maxb && lo > 0.0) {
      std::vector<Slot> best = bins;
      long long best_used = used;
      double hi = cap;
      for (int it = 0; it < 40 && best_used < maxb; ++it) {
        const double mid = 0.5 * (lo + hi);
        const long long u = attempt(mid);
        if (u > maxb) {
          lo = mid;
        } else {
          hi = mid;
          if (u > best_used && owners.empty()) {
            best = bins;
            best_used = u;
          }
        }
      }
      *out = best;
      return;
    }
    std::vector<int> order(owners.size());
    for (size_t k = 0; k < owners.size(); ++k) order[k] = (int)k;
    std::sort(order.begin(), order.end(), [&](int a, int b) { return rem[a] > rem[b] || (rem[a] == rem[b] && a < b); });
    for (long long left = maxb - used, k = 0; left > 0 && !owners.empty(); --left, ++k)
      owners[order[k % (long long)owners.size()]].blocks += 1;
    *out = owners;
    out->insert(out->end(), bins.begin(), bins.end());
    return;
  }
}

// Slots of one threshold mode's graphs (idx, fleet positions) over at most maxb CTAs: with
// `given`, one slot per graph with those CTAs; otherwise pack_slots on the weights (given, or
// (d (n + m))^exponent).
bool plan_slots(const damf_fleet* f, const std::vector<int>& idx, int maxb, const int32_t* given, double exponent,
                const double* weights, std::vector<Slot>* out) {
  out->clear();
  if (given) {
    long long tot = 0;
    for (int i : idx) {
      out->push_back(Slot{given[i], {i}});
      tot += given[i];
    }
    return tot <= maxb;
  }
  std::vector<double> w(idx.size());
  for (size_t j = 0; j < idx.size(); ++j) {
    const Ctx& c = f->ctxs[idx[j]]->c;
    w[j] = weights ? weights[idx[j]] : std::pow((double)c.d * (double)(c.n + c.m_init + 1), exponent);
  }
  pack_slots(w, maxb, out);
  for (Slot& sl : *out)
    for (int& g : sl.graphs) g = idx[g];
  return true;
}

// Builds every launch's slots and uploads the descriptor and slot tables; the fleet's plan
// changes only when every launch could be planned.
damf_status fleet_plan(damf_fleet* f, const int32_t* given, double exponent, const double* weights = nullptr) {
  const int G = (int)f->ctxs.size();
  std::vector<int> blocks(G, 0);
  std::vector<FleetLaunch> launches;
  std::vector<PushArgs> descs;
  std::vector<int> table;
  for (int scaled = 0; scaled < 2; ++scaled) {
    std::vector<int> idx;
    for (int i = 0; i < G; ++i)
      if ((f->ctxs[i]->c.cfg.threshold != 0) == (scaled != 0)) idx.push_back(i);
    if (idx.empty()) continue;
    const int maxb = push_group_max_blocks(scaled);
    if (maxb < 1) return fleet_fail(f, DAMF_ERR_CUDA, "fleet: no resident push CTA");
    std::vector<Slot> slots;
    if (!plan_slots(f, idx, maxb, given, exponent, weights, &slots))
      return fleet_fail(f, DAMF_ERR_INVALID, "fleet: shares exceed the resident push CTAs");
    FleetLaunch L{scaled, (int)descs.size(), 0, (int)slots.size(), 0, (int)table.size()};
    std::vector<int> sfirst(1, 0), gfirst(1, 0);
    const int plan_id = f->plan_id + 1;
    for (const Slot& sl : slots) {
      for (int gi : sl.graphs) {
        descs.push_back(push_args(&f->ctxs[gi]->c, f->ctxs[gi]->c.push_direct_chunks));
        blocks[gi] = sl.graphs.size() == 1 ? sl.blocks : 0;
      }
      L.count += (int)sl.graphs.size();
      L.blocks += sl.blocks;
      sfirst.push_back(L.blocks);
      gfirst.push_back(L.count);
    }
    table.push_back((int)slots.size());
    table.push_back(L.blocks);
    table.push_back(plan_id);
    table.insert(table.end(), sfirst.begin(), sfirst.end());
    table.insert(table.end(), gfirst.begin(), gfirst.end());
    launches.push_back(L);
  }
  // pushes of earlier steps (direct or replayed from a CUDA graph) may still read the
  // tables: let them finish before the tables change (a fleet never stepped has none)
  cudaError_t e = f->stepped ? cudaDeviceSynchronize() : cudaSuccess;
  if (e == cudaSuccess && !f->d_descs) e = cudaMalloc(&f->d_descs, sizeof(PushArgs) * (size_t)G);
  if (e == cudaSuccess && table.size() > f->table_cap) {
    if (f->d_table) cudaFree(f->d_table);
    f->d_table = nullptr;
    f->table_cap = table.size() + 64;
    e = cudaMalloc(&f->d_table, sizeof(int) * f->table_cap);
  }
  if (e == cudaSuccess) e = cudaMemcpy(f->d_descs, descs.data(), sizeof(PushArgs) * descs.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(f->d_table, table.data(), sizeof(int) * table.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fleet_fail(f, DAMF_ERR_CUDA, "fleet tables", e);
  f->blocks = blocks;
  f->launches = launches;
  f->plan_id += 1;
  return DAMF_OK;
}

cudaError_t fleet_mark(damf_fleet* f, cudaStream_t s) {
  if (!f->timing) return cudaSuccess;
  if (f->tev_used == f->tev.size()) {
    if (f->tev.size() >= 3 * 4096) return cudaSuccess;   // full: the later steps go unmeasured
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return e;
    f->tev.push_back(ev);
  }
  return cudaEventRecord(f->tev[f->tev_used++], s);
}

void fleet_free(damf_fleet* f) {
  if (f->d_descs) cudaFree(f->d_descs);
  if (f->d_table) cudaFree(f->d_table);
  if (f->push_stream) cudaStreamDestroy(f->push_stream);
  if (f->ev_fork) cudaEventDestroy(f->ev_fork);
  if (f->ev_done) cudaEventDestroy(f->ev_done);
  for (cudaEvent_t ev : f->tev) cudaEventDestroy(ev);
  delete f;
}

}  // namespace

extern "C" {

size_t damf_bytes_required(const damf_config* cfg) {
  if (!cfg_ok(cfg)) return 0;
  Plan p = plan_of(cfg);
  size_t t = 0;
  for (int i = 0; i < p.count; ++i) t += (p.sz[i] + 255) & ~(size_t)255;
  return t;
}

int32_t damf_rsvd_width(const damf_config* cfg) { return cfg_ok(cfg) ? width_of(cfg) : 0; }

// A context for cfg and the adjacency (row_ptr, col_idx): with omega, its initial state by the
// randomized t-SVD and a push from every row (damf_init_factorize); with saved, the state
// copied from a damf_save_state (damf_restore).
static damf_status ctx_open(const damf_config* cfg, const int32_t* row_ptr, const int32_t* col_idx, int64_t m,
                            const float* omega, const damf_state* saved, void* stream, damf_ctx** out) {
  cudaStream_t s = (cudaStream_t)stream;
  damf_ctx* x = (damf_ctx*)calloc(1, sizeof(damf_ctx));
  if (!x) return DAMF_ERR_CUDA;
  Ctx* c = &x->c;
  c->cfg = *cfg;
  c->d = cfg->d;
  c->n = cfg->n;
  c->l = width_of(cfg);
  c->m_init = m;
  Plan p = plan_of(cfg);
  void* ptr[64];
  for (int i = 0; i < p.count; ++i) {
    cudaError_t e = dev_alloc(&ptr[i], p.sz[i]);
    if (e != cudaSuccess) {
      free_all(c);
      free(x);
      return e == cudaErrorMemoryAllocation ? DAMF_ERR_CAPACITY : DAMF_ERR_CUDA;
    }
    c->allocs[c->nallocs++] = ptr[i];
    cudaMemsetAsync(ptr[i], 0, p.sz[i], s);
  }
  int k = 0;
  c->hdr = (DevHeader*)ptr[k++];
  c->Ub = (float*)ptr[k++]; c->Vb = (float*)ptr[k++]; c->Zb = (float*)ptr[k++]; c->r = (float*)ptr[k++];
  c->PU = (float*)ptr[k++]; c->PV = (float*)ptr[k++]; c->PUi = (float*)ptr[k++]; c->PVi = (float*)ptr[k++];
  c->sigma = (float*)ptr[k++]; c->s0 = (float*)ptr[k++];
  Adj* adjs[2] = {&c->out, &c->in};
  for (int a = 0; a < (cfg->directed ? 2 : 1); ++a) {
    adjs[a]->start = (int32_t*)ptr[k++]; adjs[a]->len = (int32_t*)ptr[k++];
    adjs[a]->cap = (int32_t*)ptr[k++]; adjs[a]->col = (int32_t*)ptr[k++];
    adjs[a]->m_cap = cfg->m_capacity;
  }
  if (!cfg->directed) c->in = c->out;
  Workspace& w = c->ws;
  w.S = (int32_t*)ptr[k++]; w.T = (int32_t*)ptr[k++]; w.N = (float*)ptr[k++]; w.edits = (int4*)ptr[k++];
  w.editsT = (int4*)ptr[k++]; w.Sfirst = (int32_t*)ptr[k++]; w.Tfirst = (int32_t*)ptr[k++];
  w.relocS = (long long*)ptr[k++]; w.relocT = (long long*)ptr[k++];
  w.rcapS = (int32_t*)ptr[k++]; w.rcapT = (int32_t*)ptr[k++];
  w.deg_old = (int32_t*)ptr[k++]; w.deg_new = (int32_t*)ptr[k++];
  w.UST = (float*)ptr[k++]; w.VT = (float*)ptr[k++]; w.WCt = (float*)ptr[k++];
  w.RB = (float*)ptr[k++]; w.RC = (float*)ptr[k++]; w.M = (float*)ptr[k++];
  w.E = (float*)ptr[k++]; w.H = (float*)ptr[k++]; w.theta = (float*)ptr[k++];
  w.foP = (float*)ptr[k++];
  w.foQ = w.foP + (size_t)kMaxR * cfg->d;
  w.foT = w.foQ + (size_t)kMaxR * cfg->d;
  w.fixpart = (float*)ptr[k++];
  w.fixcnt = (int32_t*)(w.fixpart + (size_t)kMaxR * kFixSplit * cfg->d);
  w.YB = (float*)ptr[k++]; w.YC = (float*)ptr[k++];
  w.KU = (float*)ptr[k++]; w.KV = (float*)ptr[k++]; w.KUi = (float*)ptr[k++]; w.KVi = (float*)ptr[k++];
  w.tmp = (float*)ptr[k++];
  w.queue = (int32_t*)ptr[k++]; w.qcap = qcap_of(cfg);
  w.work = (int4*)ptr[k++]; w.work_cap = work_cap_of(cfg);
  w.rho = (float*)ptr[k++]; w.rho_cap = rho_slots_of(cfg);
  w.ovf = (int32_t*)ptr[k++];
  w.stamp = (uint32_t*)ptr[k++]; w.pend = (int32_t*)ptr[k++]; w.pstamp = (uint32_t*)ptr[k++];
  w.gram = (float*)ptr[k++]; w.gram_part = (float*)ptr[k++]; w.gram_parts = gram_parts_of(cfg);
  {
    char* sp = (char*)ptr[k++];
    const size_t d = (size_t)cfg->d;
    w.sG = (float*)sp; sp += score_part(d * d * 4);
    w.sIs0 = (float*)sp; sp += score_part(d * 4);
    w.sLq = (float*)sp; sp += score_part((size_t)kTopQ * d * 4);
    w.sRq = (float*)sp; sp += score_part((size_t)kTopQ * d * 4);
    w.sQid = (int32_t*)sp; sp += score_part(kTopQ * 4);
    w.sPart = (unsigned long long*)sp;
  }
  cudaError_t e;
  unsigned int one = 1;
  const int n0 = cfg->n;
  if ((e = cudaMemcpyAsync(&c->hdr->epoch, &one, sizeof(one), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemcpyAsync(&c->hdr->n_nodes, &n0, sizeof(n0), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
      (e = cudaMemsetAsync(w.queue, 0xff, (size_t)w.qcap * 4, s)) != cudaSuccess ||   // empty slots: -1
      (e = cudaStreamSynchronize(s)) != cudaSuccess) {
    free_all(c);
    free(x);
    return DAMF_ERR_CUDA;
  }
  long long tail = 0;
  e = build_adjacency(c, &c->out, row_ptr, col_idx, m, cfg->n, &tail, 0, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&c->hdr->tail_out, &tail, sizeof(tail), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && cfg->directed) {
    e = build_adjacency(c, &c->in, row_ptr, col_idx, m, cfg->n, &tail, 1, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&c->hdr->tail_in, &tail, sizeof(tail), cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->push_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_caller, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_push, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_push_cap, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_done, cudaEventDisableTiming);
  c->push_direct_chunks = -1;
  if (!saved) {
    if (e == cudaSuccess) e = init_factorize(c, row_ptr, col_idx, m, omega, s);
    if (e == cudaSuccess) e = launch_push(c, 1, s);
  } else {
    const size_t nd = (size_t)cfg->n * cfg->d * sizeof(float), dd = (size_t)cfg->d * cfg->d * sizeof(float);
    const size_t dv = (size_t)cfg->d * sizeof(float);
    const cudaMemcpyKind kd = cudaMemcpyDeviceToDevice;
    float* dst[10] = {c->Ub, c->Vb, c->Zb, c->r, c->PU, c->PV, c->PUi, c->PVi, c->sigma, c->s0};
    const float* src[10] = {saved->Ub, saved->Vb, saved->Zb, saved->r, saved->PU, saved->PV, saved->PUi, saved->PVi,
                            saved->sigma, saved->s0};
    const size_t sz[10] = {nd, nd, nd, nd, dd, dd, dd, dd, dv, dv};
    for (int i = 0; i < 10 && e == cudaSuccess; ++i) e = cudaMemcpyAsync(dst[i], src[i], sz[i], kd, s);
    c->updates_since_fold = saved->updates_since_fold;
    c->check_all_next = 1;   // the next push looks at every row (whatever was pending at the save)
  }
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_push, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free_all(c);
    free(x);
    return e == cudaErrorMemoryAllocation ? DAMF_ERR_CAPACITY : DAMF_ERR_CUDA;
  }
  int st = 0;
  cudaMemcpy(&st, &c->hdr->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (st != 0) {
    free_all(c);
    free(x);
    return (damf_status)st;
  }
  if (cudaMallocHost(&c->host_stage, sizeof(int32_t) * 3 * kHostStageMax) == cudaSuccess) {
    if (cudaMalloc(&c->dev_stage, sizeof(int32_t) * 3 * kHostStageMax) == cudaSuccess)
      c->allocs[c->nallocs++] = c->dev_stage;
  }
  *out = x;
  return DAMF_OK;
}

damf_status damf_init_factorize(const damf_config* cfg, const int32_t* row_ptr, const int32_t* col_idx, int64_t m,
                                const float* omega, void* stream, damf_ctx** out) {
  if (!out) return DAMF_ERR_INVALID;
  *out = nullptr;
  if (!cfg_ok(cfg) || !row_ptr || !omega || m < 0 || (m > 0 && !col_idx)) return DAMF_ERR_INVALID;
  if (width_of(cfg) < cfg->d + 1 && cfg->rsvd_oversample > 0) return DAMF_ERR_INVALID;
  return ctx_open(cfg, row_ptr, col_idx, m, omega, nullptr, stream, out);
}

damf_status damf_restore(const damf_config* cfg, const int32_t* row_ptr, const int32_t* col_idx, int64_t m,
                         const damf_state* saved, void* stream, damf_ctx** out) {
  if (!out) return DAMF_ERR_INVALID;
  *out = nullptr;
  if (!cfg_ok(cfg) || !row_ptr || !saved || m < 0 || (m > 0 && !col_idx)) return DAMF_ERR_INVALID;
  if (!saved->Ub || !saved->Vb || !saved->Zb || !saved->r || !saved->PU || !saved->PV || !saved->PUi ||
      !saved->PVi || !saved->sigma || !saved->s0 || saved->updates_since_fold < 0)
    return DAMF_ERR_INVALID;
  return ctx_open(cfg, row_ptr, col_idx, m, nullptr, saved, stream, out);
}

damf_status damf_save_state(damf_ctx* x, damf_state* st, void* stream) {
  if (!x || !st) return DAMF_ERR_INVALID;
  Ctx* c = &x->c;
  if (c->sticky) return (damf_status)c->sticky;
  if (!st->Ub || !st->Vb || !st->Zb || !st->r || !st->PU || !st->PV || !st->PUi || !st->PVi || !st->sigma ||
      !st->s0)
    return reject(c, "save_state: a NULL buffer");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nd = (size_t)c->n * c->d * sizeof(float), dd = (size_t)c->d * c->d * sizeof(float);
  const size_t dv = (size_t)c->d * sizeof(float);
  const cudaMemcpyKind kd = cudaMemcpyDeviceToDevice;
  DAMF_CUDA(wait_push(c, s), "join push");
  float* dst[10] = {st->Ub, st->Vb, st->Zb, st->r, st->PU, st->PV, st->PUi, st->PVi, st->sigma, st->s0};
  const float* src[10] = {c->Ub, c->Vb, c->Zb, c->r, c->PU, c->PV, c->PUi, c->PVi, c->sigma, c->s0};
  const size_t sz[10] = {nd, nd, nd, nd, dd, dd, dd, dd, dv, dv};
  for (int i = 0; i < 10; ++i) DAMF_CUDA(cudaMemcpyAsync(dst[i], src[i], sz[i], kd, s), "save");
  st->updates_since_fold = c->updates_since_fold;
  return DAMF_OK;
}

// Events src/dst/op[0 .. k), or the first *kdev of them (clamped to [0, k]) when kdev is
// given: ceil(k / 64) updates are enqueued either way, and an update whose events are all
// beyond the live count finds no net change and leaves every state untouched.
// The host-side checks of one batch (arguments, node capacity), taken before any of its work
// is enqueued; a failed one poisons that context only.
static damf_status batch_args_ok(damf_ctx* x, const int32_t* src, const int32_t* dst, const int8_t* op, int32_t k,
                                 int32_t new_nodes) {
  if (!x) return DAMF_ERR_INVALID;
  Ctx* c = &x->c;
  if (c->sticky) return (damf_status)c->sticky;
  if (k < 0 || new_nodes < 0 || (k > 0 && (!src || !dst || !op))) return fail(c, DAMF_ERR_INVALID, "arguments", cudaSuccess);
  if ((long long)c->n + new_nodes > c->cfg.n_capacity) return fail(c, DAMF_ERR_CAPACITY, "node capacity", cudaSuccess);
  return DAMF_OK;
}

// The same checks for every batch of a multi-graph call (ctxs[i], or batches[i].ctx when ctxs
// is null), so that a rejected batch leaves every graph of the call without new work.
static damf_status batches_args_ok(const damf_batch* batches, int32_t count, damf_ctx* const* ctxs) {
  for (int32_t i = 0; i < count; ++i) {
    const damf_batch& b = batches[i];
    const damf_status st = batch_args_ok(ctxs ? ctxs[i] : b.ctx, b.src, b.dst, b.op, b.k, b.new_nodes);
    if (st != DAMF_OK) return st;
  }
  return DAMF_OK;
}

static damf_status apply_impl(damf_ctx* x, const int32_t* src, const int32_t* dst, const int8_t* op, int32_t k,
                              const int32_t* kdev, int32_t new_nodes, cudaStream_t s) {
  const damf_status ok = batch_args_ok(x, src, dst, op, k, new_nodes);
  if (ok != DAMF_OK) return ok;
  Ctx* c = &x->c;
  const int n_after = c->n + new_nodes;
  DAMF_CUDA(launch_validate(c, src, dst, op, k, kdev, n_after, s), "validate");
  c->launches += 1;
  c->n = n_after;
  for (int lo = 0; lo < k; lo += kEdgesPerUpdate) {
    const int kk = (k - lo) < kEdgesPerUpdate ? (k - lo) : kEdgesPerUpdate;
    // read-only part: net change, projection, residual factors, core SVD, transforms.
    // It runs on the caller's stream while the previous push may still run on the
    // push stream (both only read the adjacency).
    DAMF_STAGE(DAMF_STAGE_PREPARE, 1, launch_prepare(c, src, dst, op, kk, kdev, lo, s), "prepare");
    DAMF_STAGE(DAMF_STAGE_GATHER, 1, launch_gather(c, s), "gather");
    DAMF_STAGE(DAMF_STAGE_CHOL, 2, launch_chol(c, s), "chol");
    DAMF_STAGE(DAMF_STAGE_CORE, 2, launch_core(c, s), "core");
    DAMF_STAGE(DAMF_STAGE_TRANSFORMS, 11, launch_transforms(c, s), "transforms");
    // writes to the adjacency, Zb and r follow the push
    DAMF_CUDA(wait_push(c, s), "join push");
    DAMF_STAGE(DAMF_STAGE_PREPARE, 1, launch_edit(c, s), "edit");
    DAMF_STAGE(DAMF_STAGE_FIXUP, 1, launch_fixup(c, s), "fixup");
    DAMF_STAGE(DAMF_STAGE_SCATTER, 1, launch_scatter(c, s), "scatter");
    c->launches += kLaunchesPerUpdate;
    if (c->cfg.refold_every > 0 && ++c->updates_since_fold >= c->cfg.refold_every) {
      DAMF_STAGE(DAMF_STAGE_FOLD, kLaunchesPerFold, launch_fold(c, s), "fold");
      c->launches += kLaunchesPerFold;
      c->updates_since_fold = 0;
      c->check_all_next = 1;
    }
  }
  return DAMF_OK;
}

damf_status damf_apply_edges(damf_ctx* x, const int32_t* src, const int32_t* dst, const int8_t* op, int32_t k,
                             int32_t new_nodes, void* stream) {
  return apply_impl(x, src, dst, op, k, nullptr, new_nodes, (cudaStream_t)stream);
}

damf_status damf_apply_edges_counted(damf_ctx* x, const int32_t* src, const int32_t* dst, const int8_t* op,
                                     int32_t k_max, const int32_t* k_dev, int32_t new_nodes, void* stream) {
  if (x && !k_dev) return fail(&x->c, DAMF_ERR_INVALID, "arguments", cudaSuccess);
  return apply_impl(x, src, dst, op, k_max, k_dev, new_nodes, (cudaStream_t)stream);
}

damf_status damf_delete_nodes(damf_ctx* x, const int32_t* nodes, int32_t count, void* stream) {
  if (!x) return DAMF_ERR_INVALID;
  Ctx* c = &x->c;
  if (c->sticky) return (damf_status)c->sticky;
  if (count < 0 || (count > 0 && !nodes) || !c->dev_stage) return reject(c, "delete_nodes: bad argument");
  for (int32_t i = 0; i < count; ++i)
    if (nodes[i] < 0 || nodes[i] >= c->n) return reject(c, "delete_nodes: node id out of range");
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* es = c->dev_stage;
  int32_t* ed = c->dev_stage + kHostStageMax;
  int8_t* eo = (int8_t*)(c->dev_stage + 2 * kHostStageMax);
  for (int32_t i = 0; i < count; ++i) {
    const int u = nodes[i];
    // the rows' current lengths (earlier deletions of this call may have shortened them)
    int32_t dg[2] = {0, 0};
    DAMF_CUDA(cudaMemcpyAsync(&dg[0], c->out.len + u, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "degree");
    if (c->cfg.directed)
      DAMF_CUDA(cudaMemcpyAsync(&dg[1], c->in.len + u, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "degree");
    DAMF_CUDA(cudaStreamSynchronize(s), "degree sync");
    if (dg[0] + dg[1] <= kHostStageMax) {   // both rows in one call
      if (dg[0] > 0) DAMF_CUDA(launch_expand_row(c, u, dg[0], 0, es, ed, eo, s), "expand row");
      if (dg[1] > 0) DAMF_CUDA(launch_expand_row(c, u, dg[1], 1, es + dg[0], ed + dg[0], eo + dg[0], s), "expand row");
      c->launches += (dg[0] > 0) + (dg[1] > 0);
      if (dg[0] + dg[1] > 0) {
        const damf_status st = damf_apply_edges(x, es, ed, eo, dg[0] + dg[1], 0, stream);
        if (st != DAMF_OK) return st;
      }
      continue;
    }
    for (int incoming = 0; incoming < (c->cfg.directed ? 2 : 1); ++incoming) {
      int32_t deg = dg[incoming];
      while (deg > 0) {
        const int cnt = deg < kHostStageMax ? deg : kHostStageMax;
        DAMF_CUDA(launch_expand_row(c, u, cnt, incoming, es, ed, eo, s), "expand row");
        c->launches += 1;
        const damf_status st = damf_apply_edges(x, es, ed, eo, cnt, 0, stream);
        if (st != DAMF_OK) return st;
        deg -= cnt;
      }
    }
  }
  return DAMF_OK;
}

damf_status damf_apply_edges_multi(const damf_batch* batches, int32_t num_graphs, void* stream) {
  if (num_graphs < 0 || (num_graphs > 0 && !batches)) return DAMF_ERR_INVALID;
  for (int32_t i = 0; i < num_graphs; ++i)
    if (!batches[i].ctx) return DAMF_ERR_INVALID;
  const damf_status ok = batches_args_ok(batches, num_graphs, nullptr);
  if (ok != DAMF_OK) return ok;
  for (int32_t i = 0; i < num_graphs; ++i) {
    const damf_batch& b = batches[i];
    const damf_status st = apply_impl(b.ctx, b.src, b.dst, b.op, b.k, b.k_dev, b.new_nodes, (cudaStream_t)stream);
    if (st != DAMF_OK) return st;
  }
  return DAMF_OK;
}

damf_status damf_step_multi(const damf_batch* batches, int32_t num_graphs, void* stream) {
  if (num_graphs < 0 || (num_graphs > 0 && !batches)) return DAMF_ERR_INVALID;
  for (int32_t i = 0; i < num_graphs; ++i) {
    if (!batches[i].ctx) return DAMF_ERR_INVALID;
    if (batches[i].ctx->c.sticky) return (damf_status)batches[i].ctx->c.sticky;
    for (int32_t j = 0; j < i; ++j)
      if (batches[j].ctx == batches[i].ctx) return reject(&batches[i].ctx->c, "step_multi: a graph appears twice");
  }
  const damf_status ok = batches_args_ok(batches, num_graphs, nullptr);
  if (ok != DAMF_OK) return ok;
  cudaStream_t caller = (cudaStream_t)stream;
  for (int32_t i = 0; i < num_graphs; ++i) {
    const damf_batch& b = batches[i];
    Ctx* c = &b.ctx->c;
    // fork: the graph's update and push on its own streams, after the caller's earlier work
    DAMF_CUDA(cudaEventRecord(c->ev_fork, caller), "fork");
    DAMF_CUDA(cudaStreamWaitEvent(c->own_stream, c->ev_fork, 0), "fork");
    damf_status st = apply_impl(b.ctx, b.src, b.dst, b.op, b.k, b.k_dev, b.new_nodes, c->own_stream);
    if (st == DAMF_OK) st = damf_ppr_refresh(b.ctx, c->own_stream);
    if (st != DAMF_OK) return st;
    // join: the caller's stream waits for the push
    DAMF_CUDA(wait_push(c, c->own_stream), "join push");
    DAMF_CUDA(cudaEventRecord(c->ev_done, c->own_stream), "join");
    DAMF_CUDA(cudaStreamWaitEvent(caller, c->ev_done, 0), "join");
  }
  return DAMF_OK;
}

damf_status damf_set_tuning(damf_ctx* x, const damf_tuning* t) {
  if (!x || !t) return DAMF_ERR_INVALID;
  Ctx* c = &x->c;
  if (t->push_blocks < 0 || t->push_direct_chunks < -1 || t->push_direct_chunks > 1024)
    return reject(c, "set_tuning: value out of range");
  c->push_blocks = t->push_blocks;
  c->push_direct_chunks = t->push_direct_chunks;
  return DAMF_OK;
}

damf_status damf_get_tuning(const damf_ctx* x, damf_tuning* t) {
  if (!x || !t) return DAMF_ERR_INVALID;
  const Ctx* c = &x->c;
  t->push_blocks = c->push_blocks > 0 ? (c->push_occ > 0 && c->push_blocks > c->push_occ ? c->push_occ : c->push_blocks)
                                      : c->push_max;
  t->push_direct_chunks = c->push_direct_chunks >= 0 ? c->push_direct_chunks : push_default_direct_chunks();
  return DAMF_OK;
}

damf_status damf_apply_edges_host(damf_ctx* x, const int32_t* src, const int32_t* dst, const int8_t* op, int32_t k,
                                  int32_t new_nodes, void* stream) {
  if (!x) return DAMF_ERR_INVALID;
  Ctx* c = &x->c;
  if (c->sticky) return (damf_status)c->sticky;
  if (k < 0 || k > kHostStageMax || (k > 0 && (!src || !dst || !op)) || !c->host_stage || !c->dev_stage)
    return fail(c, DAMF_ERR_INVALID, "arguments", cudaSuccess);
  cudaStream_t s = (cudaStream_t)stream;
  // the previous call's copy out of the staging buffer must be complete before reuse
  DAMF_CUDA(cudaStreamSynchronize(s), "stage sync");
  memcpy(c->host_stage, src, sizeof(int32_t) * k);
  memcpy(c->host_stage + kHostStageMax, dst, sizeof(int32_t) * k);
  memcpy((int8_t*)(c->host_stage + 2 * kHostStageMax), op, (size_t)k);
  if (k > 0) {
    DAMF_CUDA(cudaMemcpyAsync(c->dev_stage, c->host_stage, sizeof(int32_t) * k, cudaMemcpyHostToDevice, s), "h2d");
    DAMF_CUDA(cudaMemcpyAsync(c->dev_stage + kHostStageMax, c->host_stage + kHostStageMax, sizeof(int32_t) * k,
                              cudaMemcpyHostToDevice, s),
              "h2d");
    DAMF_CUDA(cudaMemcpyAsync(c->dev_stage + 2 * kHostStageMax, c->host_stage + 2 * kHostStageMax, (size_t)k,
                              cudaMemcpyHostToDevice, s),
              "h2d");
  }
  return damf_apply_edges(x, c->dev_stage, c->dev_stage + kHostStageMax, (const int8_t*)(c->dev_stage + 2 * kHostStageMax),
                          k, new_nodes, stream);
}

damf_status damf_ppr_refresh(damf_ctx* x, void* stream) {
  if (!x) return DAMF_ERR_INVALID;
  Ctx* c = &x->c;
  if (c->sticky) return (damf_status)c->sticky;
  DAMF_CUDA(cudaEventRecord(c->ev_caller, (cudaStream_t)stream), "record");
  cudaStream_t s = c->push_stream;
  DAMF_CUDA(cudaStreamWaitEvent(s, c->ev_caller, 0), "push wait");
  DAMF_STAGE(DAMF_STAGE_PUSH, 1, launch_push(c, c->check_all_next, s), "push");
  DAMF_CUDA(note_push(c, s), "record");
  c->launches += 1;
  c->check_all_next = 0;
  return DAMF_OK;
}

damf_status damf_join(damf_ctx* x, void* stream) {
  if (!x) return DAMF_ERR_INVALID;
  Ctx* c = &x->c;
  DAMF_CUDA(wait_push(c, (cudaStream_t)stream), "join");
  return DAMF_OK;
}

damf_status damf_record_event(damf_ctx* x, void* event) {
  if (!x || !event) return DAMF_ERR_INVALID;
  Ctx* c = &x->c;
  DAMF_CUDA(cudaEventRecord((cudaEvent_t)event, c->push_stream), "record");
  return DAMF_OK;
}

damf_status damf_get_embeddings(damf_ctx* x, const int32_t* rows, int32_t count, float* X, float* Y, float* Z,
                                float* sigma, void* stream) {
  if (!x) return DAMF_ERR_INVALID;
  Ctx* c = &x->c;
  if (c->sticky) return (damf_status)c->sticky;
  if (count < 0 || (!rows && count > c->n)) return fail(c, DAMF_ERR_INVALID, "count", cudaSuccess);
  // only Z reads the push's output; X, Y and sigma follow the update's work on `stream`
  if (Z) DAMF_CUDA(wait_push(c, (cudaStream_t)stream), "join push");
  DAMF_CUDA(launch_query(c, rows, count, X, Y, Z, sigma, (cudaStream_t)stream), "query");
  return DAMF_OK;
}

damf_status damf_score_pairs(damf_ctx* x, const int32_t* src, const int32_t* dst, int32_t count, int32_t context,
                             int32_t symmetric, float* scores, void* stream) {
  if (!x) return DAMF_ERR_INVALID;
  Ctx* c = &x->c;
  if (c->sticky) return (damf_status)c->sticky;
  if (count < 0 || (context != 0 && context != 1) || (symmetric != 0 && symmetric != 1) ||
      (count > 0 && (!src || !dst || !scores)))
    return reject(c, "score_pairs: bad argument");
  DAMF_CUDA(wait_push(c, (cudaStream_t)stream), "join push");
  DAMF_CUDA(launch_score_pairs(c, src, dst, count, context, symmetric, scores, (cudaStream_t)stream), "score_pairs");
  return DAMF_OK;
}

damf_status damf_topk(damf_ctx* x, const int32_t* rows, int32_t count, int32_t k, int32_t context, int32_t symmetric,
                      int32_t* out_idx, float* out_score, void* stream) {
  if (!x) return DAMF_ERR_INVALID;
  Ctx* c = &x->c;
  if (c->sticky) return (damf_status)c->sticky;
  if (count < 0 || k < 1 || k > kMaxTopK || (context != 0 && context != 1) || (symmetric != 0 && symmetric != 1) ||
      (count > 0 && (!rows || !out_idx || !out_score)))
    return reject(c, "topk: bad argument (1 <= k <= 64, context and symmetric 0 or 1)");
  DAMF_CUDA(wait_push(c, (cudaStream_t)stream), "join push");
  DAMF_CUDA(launch_topk(c, rows, count, k, context, symmetric, out_idx, out_score, (cudaStream_t)stream), "topk");
  return DAMF_OK;
}

int32_t damf_num_nodes(const damf_ctx* x) { return x ? x->c.n : 0; }

damf_status damf_set_timing(damf_ctx* x, int32_t enable) {
  if (!x) return DAMF_ERR_INVALID;
  Ctx* c = &x->c;
  if (enable && !c->ev) {
    c->ev = (cudaEvent_t*)calloc(2 * kTimerPairs, sizeof(cudaEvent_t));
    c->ev_stage = (int*)calloc(kTimerPairs, sizeof(int));
    if (!c->ev || !c->ev_stage) return fail(c, DAMF_ERR_CAPACITY, "timing", cudaSuccess);
    for (int i = 0; i < 2 * kTimerPairs; ++i) DAMF_CUDA(cudaEventCreate(&c->ev[i]), "timing");
  }
  if (!enable) harvest_timing(c);
  c->timing = enable ? 1 : 0;
  return DAMF_OK;
}

damf_status damf_get_timing(damf_ctx* x, double* ms, int64_t* launches) {
  if (!x) return DAMF_ERR_INVALID;
  Ctx* c = &x->c;
  harvest_timing(c);
  for (int k = 0; k < DAMF_NUM_STAGES; ++k) {
    if (ms) ms[k] = c->stage_ms[k];
    if (launches) launches[k] = c->stage_launches[k];
    c->stage_ms[k] = 0.0;
    c->stage_launches[k] = 0;
  }
  return DAMF_OK;
}

damf_status damf_get_state(damf_ctx* x, float* Ub, float* Vb, float* Zb, float* r, float* PU, float* PV,
                           float* sigma, float* s0, void* stream) {
  if (!x) return DAMF_ERR_INVALID;
  Ctx* c = &x->c;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nd = (size_t)c->n * c->d * sizeof(float), dd = (size_t)c->d * c->d * sizeof(float);
  const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
  DAMF_CUDA(wait_push(c, s), "join push");
  if (Ub) DAMF_CUDA(cudaMemcpyAsync(Ub, c->Ub, nd, k, s), "state");
  if (Vb) DAMF_CUDA(cudaMemcpyAsync(Vb, c->Vb, nd, k, s), "state");
  if (Zb) DAMF_CUDA(cudaMemcpyAsync(Zb, c->Zb, nd, k, s), "state");
  if (r) DAMF_CUDA(cudaMemcpyAsync(r, c->r, nd, k, s), "state");
  if (PU) DAMF_CUDA(cudaMemcpyAsync(PU, c->PU, dd, k, s), "state");
  if (PV) DAMF_CUDA(cudaMemcpyAsync(PV, c->PV, dd, k, s), "state");
  if (sigma) DAMF_CUDA(cudaMemcpyAsync(sigma, c->sigma, c->d * sizeof(float), k, s), "state");
  if (s0) DAMF_CUDA(cudaMemcpyAsync(s0, c->s0, c->d * sizeof(float), k, s), "state");
  return DAMF_OK;
}

damf_status damf_export_adjacency(damf_ctx* x, int32_t outgoing, int64_t* row_ptr, int32_t* col,
                                  int64_t col_capacity) {
  if (!x || !row_ptr || (!col && col_capacity > 0)) return DAMF_ERR_INVALID;
  Ctx* c = &x->c;
  const Adj& a = (outgoing || !c->cfg.directed) ? c->out : c->in;
  DAMF_CUDA(cudaDeviceSynchronize(), "export");
  long long tails[2];
  DAMF_CUDA(cudaMemcpy(tails, &c->hdr->tail_out, sizeof(tails), cudaMemcpyDeviceToHost), "export");
  const long long tail = (outgoing || !c->cfg.directed) ? tails[0] : tails[1];
  const int n = c->n;
  int32_t* st = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* ln = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
  int32_t* cl = (int32_t*)malloc(sizeof(int32_t) * (size_t)(tail > 0 ? tail : 1));
  damf_status ret = DAMF_OK;
  if (!st || !ln || !cl) {
    ret = DAMF_ERR_CAPACITY;
  } else if (cudaMemcpy(st, a.start, sizeof(int32_t) * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
             cudaMemcpy(ln, a.len, sizeof(int32_t) * n, cudaMemcpyDeviceToHost) != cudaSuccess ||
             (tail > 0 && cudaMemcpy(cl, a.col, sizeof(int32_t) * (size_t)tail, cudaMemcpyDeviceToHost) != cudaSuccess)) {
    ret = DAMF_ERR_CUDA;
  } else {
    long long pos = 0;
    for (int u = 0; u < n && ret == DAMF_OK; ++u) {
      row_ptr[u] = pos;
      if (pos + ln[u] > col_capacity) {
        ret = DAMF_ERR_CAPACITY;
        break;
      }
      memcpy(col + pos, cl + st[u], sizeof(int32_t) * (size_t)ln[u]);
      pos += ln[u];
    }
    if (ret == DAMF_OK) row_ptr[n] = pos;
  }
  free(st);
  free(ln);
  free(cl);
  return ret;
}

damf_status damf_get_last_touched(damf_ctx* x, int32_t* S, int32_t* nS, int32_t* T, int32_t* nT) {
  if (!x || !S || !nS || !T || !nT) return DAMF_ERR_INVALID;
  Ctx* c = &x->c;
  DAMF_CUDA(cudaDeviceSynchronize(), "touched");
  int sz[2];
  DAMF_CUDA(cudaMemcpy(sz, &c->hdr->nS, sizeof(sz), cudaMemcpyDeviceToHost), "touched");
  *nS = sz[0];
  *nT = sz[1];
  if (sz[0] > 0) DAMF_CUDA(cudaMemcpy(S, c->ws.S, sizeof(int32_t) * sz[0], cudaMemcpyDeviceToHost), "touched");
  if (sz[1] > 0) DAMF_CUDA(cudaMemcpy(T, c->ws.T, sizeof(int32_t) * sz[1], cudaMemcpyDeviceToHost), "touched");
  return DAMF_OK;
}

damf_status damf_get_stats(damf_ctx* x, damf_stats* o) {
  if (!x || !o) return DAMF_ERR_INVALID;
  Ctx* c = &x->c;
  DevHeader h;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&h, c->hdr, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(c, DAMF_ERR_CUDA, "stats", e);
  o->updates = h.updates;
  o->edges_applied = h.edges_applied;
  o->entries_changed = h.entries_changed;
  o->pushes = h.pushes;
  o->push_edges = h.push_edges;
  o->push_rounds = h.push_rounds;
  o->fixup_edges = h.fixup_edges;
  o->touched_rows = h.touched_rows;
  o->folds = h.folds;
  o->last_rank = h.last_rank;
  o->last_status = h.status;
  o->launches = c->launches;
  o->last_sweeps = h.last_sweeps;
  o->jacobi_sweeps = h.jacobi_sweeps;
  o->jacobi_full = h.jacobi_full;
  o->jacobi_gersh = h.jacobi_gersh;
  o->push_tasks = h.push_tasks;
  o->push_items = h.push_items;
  for (int i = 0; i < 4; ++i) o->push_ns[i] = (int64_t)h.push_ns[i];
  return DAMF_OK;
}

damf_status damf_sync_status(damf_ctx* x) {
  if (!x) return DAMF_ERR_INVALID;
  Ctx* c = &x->c;
  int st = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&st, &c->hdr->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(c, DAMF_ERR_CUDA, "sync", e);
  if (st != 0 && c->sticky == 0) {
    c->sticky = st;
    snprintf(c->errbuf, sizeof(c->errbuf), "device status %d", st);
  }
  return (damf_status)(c->sticky ? c->sticky : st);
}

const char* damf_last_error(const damf_ctx* x) { return x ? x->c.errbuf : "null context"; }

void damf_destroy(damf_ctx* x) {
  if (!x) return;
  cudaDeviceSynchronize();
  free_all(&x->c);
  free(x);
}

void damf_debug_fail_allocations(int32_t after) { g_fail_alloc_after = after < 0 ? -1 : after; }

damf_status damf_selftest_wait(int32_t which, int64_t limit, int32_t* status_out, void* stream) {
  if (!status_out || (which != 0 && which != 1) || limit < 1 || limit > (int64_t)kSpinLimit) return DAMF_ERR_INVALID;
  cudaStream_t s = (cudaStream_t)stream;
  DevHeader* h = nullptr;
  int32_t* q = nullptr;
  cudaError_t e = cudaMalloc(&h, sizeof(DevHeader));
  if (e == cudaSuccess) e = cudaMalloc(&q, sizeof(int32_t));
  if (e == cudaSuccess) e = cudaMemsetAsync(h, 0, sizeof(DevHeader), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(q, 0xff, sizeof(int32_t), s);   // the position stays empty (-1)
  const unsigned long long one_task = 1ull << 32;                          // one unfinished task, tail 0
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h->qstate, &one_task, sizeof(one_task), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_wait_selftest(h, q, which, (long long)limit, s);
  int32_t st = -1;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, &h->status, sizeof(st), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (h) cudaFree(h);
  if (q) cudaFree(q);
  if (e != cudaSuccess) return DAMF_ERR_CUDA;
  *status_out = st;
  return DAMF_OK;
}

int32_t damf_plan_slots(const double* weights, int32_t count, int32_t max_blocks, int32_t* slot_of, int32_t* ctas) {
  if (!weights || !slot_of || !ctas || count < 1 || max_blocks < 1) return -1;
  std::vector<double> w(weights, weights + count);
  for (double x : w)
    if (!(x > 0.0 && x < 1e300)) return -1;
  std::vector<Slot> slots;
  pack_slots(w, max_blocks, &slots);
  for (size_t s = 0; s < slots.size(); ++s) {
    ctas[s] = slots[s].blocks;
    for (int g : slots[s].graphs) slot_of[g] = (int32_t)s;
  }
  return (int32_t)slots.size();
}

damf_status damf_fleet_create(damf_ctx* const* ctxs, int32_t count, damf_fleet** out) {
  if (!out) return DAMF_ERR_INVALID;
  *out = nullptr;
  if (count < 1 || !ctxs) return DAMF_ERR_INVALID;
  for (int32_t i = 0; i < count; ++i) {
    if (!ctxs[i] || ctxs[i]->c.sticky) return DAMF_ERR_INVALID;
    for (int32_t j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return DAMF_ERR_INVALID;
  }
  damf_fleet* f = new (std::nothrow) damf_fleet();
  if (!f) return DAMF_ERR_CUDA;
  f->ctxs.assign(ctxs, ctxs + count);
  cudaError_t e = cudaStreamCreateWithFlags(&f->push_stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&f->ev_done, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    fleet_free(f);
    return DAMF_ERR_CUDA;
  }
  const damf_status st = fleet_plan(f, nullptr, 1.0);
  if (st != DAMF_OK) {
    fleet_free(f);
    return st;
  }
  *out = f;
  return DAMF_OK;
}

damf_status damf_fleet_set_shares(damf_fleet* f, const int32_t* blocks, double exponent) {
  if (!f) return DAMF_ERR_INVALID;
  if (blocks) {
    for (size_t i = 0; i < f->ctxs.size(); ++i)
      if (blocks[i] < 1) return fleet_fail(f, DAMF_ERR_INVALID, "fleet: a share below one CTA");
  } else if (!(exponent >= 0.0 && exponent <= 4.0)) {
    return fleet_fail(f, DAMF_ERR_INVALID, "fleet: exponent outside [0, 4]");
  }
  return fleet_plan(f, blocks, exponent);   // a rejected plan leaves the previous one in place
}

damf_status damf_fleet_set_weights(damf_fleet* f, const double* weights) {
  if (!f || !weights) return DAMF_ERR_INVALID;
  for (size_t i = 0; i < f->ctxs.size(); ++i)
    if (!(weights[i] > 0.0 && weights[i] < 1e300)) return fleet_fail(f, DAMF_ERR_INVALID, "fleet: a weight not > 0");
  return fleet_plan(f, nullptr, 1.0, weights);
}

damf_status damf_fleet_get_shares(const damf_fleet* f, int32_t* blocks, int32_t* launches) {
  if (!f) return DAMF_ERR_INVALID;
  if (blocks)
    for (size_t i = 0; i < f->blocks.size(); ++i) blocks[i] = f->blocks[i];
  if (launches) *launches = (int32_t)f->launches.size();
  return DAMF_OK;
}

damf_status damf_fleet_step(damf_fleet* f, const damf_batch* batches, void* stream) {
  if (!f || !batches) return DAMF_ERR_INVALID;
  const int G = (int)f->ctxs.size();
  for (int i = 0; i < G; ++i) {
    if (batches[i].ctx && batches[i].ctx != f->ctxs[i]) return fleet_fail(f, DAMF_ERR_INVALID, "fleet: batch order");
    if (f->ctxs[i]->c.sticky) return (damf_status)f->ctxs[i]->c.sticky;
  }
  const damf_status ok = batches_args_ok(batches, G, f->ctxs.data());
  if (ok != DAMF_OK) return ok;
  cudaStream_t caller = (cudaStream_t)stream;
  f->stepped = 1;
  cudaError_t e = fleet_mark(f, caller);
  if (e == cudaSuccess) e = cudaEventRecord(f->ev_fork, caller);
  if (e != cudaSuccess) return fleet_fail(f, DAMF_ERR_CUDA, "fleet fork", e);
  // every graph's update on its own stream; the fleet's push stream then waits for all of them
  for (int i = 0; i < G; ++i) {
    damf_ctx* x = f->ctxs[i];
    Ctx* c = &x->c;
    const damf_batch& b = batches[i];
    DAMF_CUDA(cudaStreamWaitEvent(c->own_stream, f->ev_fork, 0), "fleet fork");
    const damf_status st = apply_impl(x, b.src, b.dst, b.op, b.k, b.k_dev, b.new_nodes, c->own_stream);
    if (st != DAMF_OK) return st;
    DAMF_CUDA(cudaEventRecord(c->ev_done, c->own_stream), "fleet join");
    DAMF_CUDA(cudaStreamWaitEvent(f->push_stream, c->ev_done, 0), "fleet join");
  }
  // the pushes: one grouped cooperative launch per threshold mode
  e = fleet_mark(f, f->push_stream);
  if (e != cudaSuccess) return fleet_fail(f, DAMF_ERR_CUDA, "fleet timing", e);
  for (size_t l = 0; l < f->launches.size(); ++l) {
    const FleetLaunch& L = f->launches[l];
    e = launch_push_group(f->d_descs + L.first_graph, L.count, f->d_table + L.table_off, L.nslots, L.blocks,
                          f->plan_id, L.scaled, f->push_stream);
    if (e != cudaSuccess) {
      for (int i = 0; i < G; ++i) fail(&f->ctxs[i]->c, DAMF_ERR_CUDA, "fleet push", e);
      return fleet_fail(f, DAMF_ERR_CUDA, "fleet push", e);
    }
    f->launches_total += 2;
  }
  for (int i = 0; i < G; ++i) {
    Ctx* c = &f->ctxs[i]->c;
    DAMF_CUDA(note_push(c, f->push_stream), "fleet record");
    c->check_all_next = 0;
  }
  e = fleet_mark(f, f->push_stream);
  if (e == cudaSuccess) e = cudaEventRecord(f->ev_done, f->push_stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, f->ev_done, 0);
  if (e != cudaSuccess) return fleet_fail(f, DAMF_ERR_CUDA, "fleet join", e);
  return DAMF_OK;
}

damf_status damf_fleet_set_timing(damf_fleet* f, int32_t enable) {
  if (!f) return DAMF_ERR_INVALID;
  f->timing = enable ? 1 : 0;
  f->tev_used = 0;
  return DAMF_OK;
}

damf_status damf_fleet_get_timing(damf_fleet* f, double* update_ms, double* push_ms, int32_t* steps) {
  if (!f) return DAMF_ERR_INVALID;
  double a = 0.0, b = 0.0;
  int n = 0;
  for (size_t i = 0; i + 3 <= f->tev_used; i += 3) {
    cudaError_t e = cudaEventSynchronize(f->tev[i + 2]);
    float t01 = 0.f, t12 = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t01, f->tev[i], f->tev[i + 1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t12, f->tev[i + 1], f->tev[i + 2]);
    if (e != cudaSuccess) return fleet_fail(f, DAMF_ERR_CUDA, "fleet timing", e);
    a += t01;
    b += t12;
    ++n;
  }
  f->tev_used = 0;
  if (update_ms) *update_ms = a;
  if (push_ms) *push_ms = b;
  if (steps) *steps = n;
  return DAMF_OK;
}

int64_t damf_fleet_launches(const damf_fleet* f) { return f ? f->launches_total : 0; }

const char* damf_fleet_last_error(const damf_fleet* f) { return f ? f->errbuf : "no fleet"; }

void damf_fleet_destroy(damf_fleet* f) {
  if (!f) return;
  cudaStreamSynchronize(f->push_stream);
  fleet_free(f);
}

}  // extern "C"
