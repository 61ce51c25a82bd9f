// Dynamic embedding enhancement (Sec. 4.4; Step 4 of Sec. 4.5): the PPR push.
//
// State (Zb, r) keeps  Pi X_b = Zb + Pi r  with P = D^{-1} A, Pi = alpha (I - (1-alpha) P)^{-1}.
// Because Pi = alpha I + (1-alpha) Pi P, pushing any vector x out of r[u] (r[u] -= x,
// Zb[u] += alpha x, r[w] += (1-alpha) A[w][u] / deg(w) x for every in-neighbour w of u) keeps
// the invariant, whatever the order and whatever x. The push stops when no row has
// max_j |r[u][j]| > eps; then |Zb - Pi X_b| <= eps elementwise since Pi is row-substochastic.
// With the degree-scaled threshold (damf_config.threshold = 1) the eps of row u reads
// eps * max(deg(u), 1), deg the out-degree, and |Zb - Pi X_b|[i] <= (Pi t)[i] for those t.
//
// One persistent cooperative launch, no rounds: a FIFO work queue of tasks in HBM.
//   * task "row u": clear u's in-queue flag, read v = r[u]; if max|v| > eps, remove exactly v
//     (float4 atomic add of -v), add alpha v to Zb[u] (atomic), and scatter coef * v to the
//     in-neighbours of u; a row with many in-edges (a hub) instead stores v in a rho slot and
//     queues one "item" task per kItemEdges of its in-edges, which spreads it over every warp.
//   * task "item": scatter a hub's stored v to up to kItemEdges of its in-edges.
// Every add returns the old value, so the thread whose add (or removal) is the last on an
// element sees what it leaves there; a row left above eps is queued unless its flag says it
// already is. The flag is cleared before the row is read, so an add that lands after that read
// queues the row again. A row can thus be pushed by two warps at once; all changes to r and
// Zb are atomic adds, so both pushes count.
// Termination: qstate holds (unfinished tasks << 32) | tail in one 64-bit word. A task is
// counted before it is published and uncounted in the same atomic that counts the tasks it
// queued (or later), so the count reaches 0 only when no task is queued or running. A warp
// claims kClaim positions at a time (q_head), keeps the tasks it queues in a shared-memory
// buffer, and publishes them (one atomic, release stores) once 16 are buffered and before it
// waits for an empty slot; it leaves when the count is 0. The queue words sit on their own
// cache lines (every warp hits them); a claim's hub items read their in-edges in one pass and
// share the hub's row through a per-warp shared-memory slot.
// The queue does not wrap within a phase. When it is full, rows stay flagged and unqueued and
// the overflow flag is set; after the phase every row is cleared and checked again.
// Every wait is bounded (kSpinLimit with __nanosleep; DAMF_ERR_TIMEOUT).
#include <string.h>

#include "damf_internal.cuh"

namespace damf {

// CTAs of the push per SM, in halves: five halves = 2.5 per SM on average (every other SM
// holds three), which leaves registers, threads and shared memory on at least half the SMs
// for the next update's factor chain (an 8-CTA cluster of 512 threads at 64 registers fits
// beside two push CTAs). Measured on C3: 304 CTAs 3.21 ms per push and 5.21 ms per call, 380
// CTAs 2.89 and 4.91, 456 CTAs 2.70 and 5.61 (the chain waits for SMs). A context's grid is
// this many unless damf_set_tuning asks otherwise.
constexpr int kPushHalfBlocksPerSM = 5;
// A row with more than this many chunks of in-edges is a hub: its chunks become item tasks
// (per context: damf_set_tuning).
constexpr int kPushDirectChunks = 8;
// in-edges per hub item: small items spread a hub over many warps (measured: 8 beats 32)
constexpr int kItemEdges = 8;

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kTask = 1ull << 32;   // one unfinished task in qstate

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// adds the time since the last mark to slot i and sets a new mark
__device__ __forceinline__ void time_mark(unsigned long long* s_t, int i) {
  const unsigned long long t = gtimer();
  s_t[i] += t - s_t[4];
  s_t[4] = t;
}

__device__ __forceinline__ float4 f4_ldcg(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }

__device__ __forceinline__ float max_abs4(float4 v) {
  return fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w)));
}

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_volatile64(const unsigned long long* p) {
  return *reinterpret_cast<const volatile unsigned long long*>(p);
}

// A warp runs one task at a time. A row of D floats is held by a row group of LPR lanes (a
// float4 each); each of the RPW groups holds the same row and takes its own in-edges, CHL at
// a time, so a chunk is EPC = RPW * CHL in-edges (one owner lane per in-edge).
template <int D>
struct PushShape {
  static constexpr int LPR = D / 4;
  static constexpr int RPW = 32 / LPR;
  // atomics in flight per lane: four (returns in 16 registers) measured as fast as eight,
  // which pushed the task loop past 64 registers into local-memory spills
  static constexpr int CHL = 4;
  static constexpr int EPC = RPW * CHL;   // 4, 8, 16, 32 for D = 128, 64, 32, 16
};

// maximum over the LPR lanes of a row group (every lane of the warp takes part)
template <int LPR>
__device__ __forceinline__ float group_max(float m) {
#pragma unroll
  for (int o = 1; o < LPR; o <<= 1) m = fmaxf(m, __shfl_xor_sync(kFull, m, o));
  return m;
}

template <bool SCALED>
__device__ __forceinline__ float threshold(float eps, int deg) {
  return SCALED ? eps * (float)max(deg, 1) : eps;
}

__device__ __forceinline__ unsigned exch_acq_rel(uint32_t* p, unsigned v) {
  unsigned old;
  asm volatile("atom.exch.acq_rel.gpu.global.b32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void st_release(int32_t* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr int kQBuf = 256;    // per-warp buffer of tasks to publish (shared memory)
constexpr int kClaim = 4;     // queue positions a warp claims at a time

// A warp's counters, kept by its lane 0 in shared memory (registers are the push's scarce
// resource: what does not fit in 64 per thread spills to local memory, whose reloads miss L1).
struct WarpStats {
  long long pushes, edges;   // rows pushed, in-edges scattered
  unsigned long long wait;   // ns spent waiting for a queue slot
  int rows, items;           // row and item tasks taken
};

// A warp's tasks to publish and the count of its finished tasks not yet uncounted.
struct WarpQ {
  int32_t* buf;   // [kQBuf] in shared memory
  float* rho;     // [128] in shared memory: the hub row of the claim's items
  int n;          // buffered entries (warp-uniform)
  int done;       // finished tasks (warp-uniform)
  int32_t* ovf;   // list of hub items that found the queue full
  uint32_t* inq;  // in-queue flags of the rows
};

// Claims the buffered rows (in-queue flags), then publishes the kept entries and uncounts the
// finished tasks in one atomic on qstate
// (count += n - done, tail += n), then stores the entries with release semantics, so that a
// consumer that sees an entry also sees the count that includes it and everything the warp
// wrote before (rho, items). Entries past the queue's end are uncounted again and set the
// overflow flag. Warp-level: every lane calls it.
__device__ __forceinline__ void flush(WarpQ& wq, DevHeader* h, int32_t* queue, long long qcap, int lane,
                                      int32_t* ovf) {
  if (wq.n == 0 && wq.done == 0) return;
  __syncwarp();
  // claim the buffered rows: a row whose in-queue flag was set already is queued (or being
  // queued) by someone else and is dropped; all exchanges are in flight at once
  constexpr int kRounds = kQBuf / 32;
  unsigned keep = 0;   // bit j: entry lane + 32 j stays
#pragma unroll
  for (int j = 0; j < kRounds; ++j) {
    const int i = lane + 32 * j;
    if (i < wq.n) {
      const int e = wq.buf[i];
      keep |= (unsigned)(e < -1 || exch_acq_rel(wq.inq + e, 1u) == 0u) << j;
    }
  }
  int kept = 0;
#pragma unroll
  for (int j = 0; j < kRounds; ++j) {
    if (32 * j >= wq.n) break;   // warp-uniform
    const int i = lane + 32 * j;
    const int e = i < wq.n ? wq.buf[i] : 0;
    const bool k = i < wq.n && ((keep >> j) & 1u);
    const unsigned m = __ballot_sync(kFull, k);
    __syncwarp();                // this round's entries are read before any is overwritten
    if (k) wq.buf[kept + __popc(m & ((1u << lane) - 1u))] = e;
    kept += __popc(m);
  }
  __syncwarp();
  wq.n = kept;
  unsigned long long base = 0;
  if (lane == 0)
    base = atomicAdd(&h->qstate, (unsigned long long)(long long)(wq.n - wq.done) * kTask + (unsigned)wq.n);
  base = __shfl_sync(kFull, base, 0) & 0xffffffffull;
  int lost = 0;
  for (int i = lane; i < wq.n; i += 32) {
    const long long pos = (long long)base + i;
    if (pos < qcap) {
      st_release(queue + pos, wq.buf[i]);
    } else {
      ++lost;
      // a row stays flagged and is found again by the rescan; a hub item holds mass already
      // taken out of r, so it is kept for the end of the phase
      if (wq.buf[i] < -1) ovf[atomicAdd(&h->ovf_count, 1)] = -wq.buf[i] - 2;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lost += __shfl_xor_sync(kFull, lost, o);
  if (lost && lane == 0) {
    atomicAdd(&h->qstate, (unsigned long long)(-(long long)lost * (long long)kTask));
    atomicExch(&h->overflow, 1);
  }
  __syncwarp();
  wq.n = 0;
  wq.done = 0;
}

// Adds the entries of the lanes with `want` to the warp's buffer (flushing it first when full).
__device__ __forceinline__ void stage(bool want, int entry, WarpQ& wq, DevHeader* h, int32_t* queue, long long qcap,
                                      int lane) {
  const unsigned m = __ballot_sync(kFull, want);
  if (!m) return;
  if (wq.n + __popc(m) > kQBuf) flush(wq, h, queue, qcap, lane, wq.ovf);
  if (want) wq.buf[wq.n + __popc(m & ((1u << lane) - 1u))] = entry;
  wq.n += __popc(m);
  __syncwarp();
}

// Queues row w for the lanes with `want`: buffered now, claimed at the flush unless it is
// queued already (in-queue flag; the exchange is a release, so the add that made w cross
// comes before it).
__device__ __forceinline__ void enqueue_rows(bool want, int w, WarpQ& wq, DevHeader* h, uint32_t* inq,
                                             int32_t* queue, long long qcap, int lane) {
  stage(want, w, wq, h, queue, qcap, lane);
}

// Scatter (warp-level): adds coef(w) * v to r[w] for the in-edges col[st .. st+ne) of a row,
// coef(w) = (1-alpha)/deg(w). The in-edges and their out-degrees are loaded 32 at a time, one
// per lane; then chunks of EPC in-edges follow, group g taking in-edges g, g + RPW, ... of
// the chunk with all CHL atomics in flight before any result is looked at. Each w an add left
// above its threshold is queued (unless enq is false: the adds only). Every lane calls it.
template <int D, bool SCALED>
__device__ __forceinline__ void scatter_edges(const float4 v, int st, int ne, const int32_t* __restrict__ col,
                                              const int32_t* __restrict__ outdeg, float* r, float beta, float eps,
                                              WarpQ& wq, DevHeader* h, uint32_t* inq, int32_t* queue, long long qcap,
                                              int lane, int sub, int q, bool enq = true, bool pre0 = false,
                                              int w_pre = 0, int d_pre = 1, int ncap = 0x7fffffff) {
  constexpr int LPR = PushShape<D>::LPR;
  constexpr int RPW = PushShape<D>::RPW;
  constexpr int CHL = PushShape<D>::CHL;
  constexpr int EPC = PushShape<D>::EPC;
  const unsigned gmask = (LPR == 32) ? kFull : ((1u << LPR) - 1u);
  for (int b0 = 0; b0 < ne; b0 += 32) {   // warp-uniform
    const int nb = min(32, ne - b0);
    int w_own = 0, d_own = 1;
    float c_own = 0.f;
    if (b0 == 0 && pre0) {   // the caller loaded the first 32 in-edges and their degrees
      w_own = w_pre;
      d_own = d_pre;
      if (lane < nb) c_own = beta / (float)d_own;
    } else if (lane < nb) {
      w_own = __ldg(col + st + b0 + lane);
      if (DAMF_DCHECK(h, (unsigned)w_own < (unsigned)ncap)) {
        d_own = __ldg(outdeg + w_own);
        c_own = beta / (float)d_own;
      } else {
        w_own = 0;   // an add of zero to row 0 in place of the bad neighbour
      }
    }
    for (int c0 = 0; c0 < nb; c0 += EPC) {   // warp-uniform; the chunk's in-edges are lanes c0 ..
      const int ncur = min(EPC, nb - c0);
      float4 nv[CHL];
#pragma unroll
      for (int c = 0; c < CHL; ++c) {
        const int e = c * RPW + sub;
        const int src = min(c0 + e, 31);
        const int w = __shfl_sync(kFull, w_own, src);
        const float coef = __shfl_sync(kFull, c_own, src);
        nv[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (e < ncur) {
          const float4 add = make_float4(coef * v.x, coef * v.y, coef * v.z, coef * v.w);
          const float4 old = atomicAdd(reinterpret_cast<float4*>(r + (size_t)w * D) + q, add);
          nv[c] = make_float4(old.x + add.x, old.y + add.y, old.z + add.z, old.w + add.w);
        }
      }
      if (!enq) continue;   // warp-uniform: the adds only (a rescan follows)
      // lane l = c0 + c * RPW + g owns the chunk's in-edge c * RPW + g: its bit is group g's
      // part of step c's ballot
      const int le = lane - c0;
      bool crossed = false;
#pragma unroll
      for (int c = 0; c < CHL; ++c) {
        const float thr = SCALED ? __shfl_sync(kFull, threshold<true>(eps, d_own), min(c0 + c * RPW + sub, 31)) : eps;
        const unsigned b = __ballot_sync(kFull, max_abs4(nv[c]) > thr);
        if (le >= 0 && le / RPW == c) crossed = ((b >> ((le % RPW) * LPR)) & gmask) != 0u;
      }
      enqueue_rows(le >= 0 && le < ncur && crossed, w_own, wq, h, inq, queue, qcap, lane);
    }
  }
}

// Waits (lane 0) for queue position p: returns its entry, or -1 when no task is left (the
// unfinished count is 0), the device status is set, or the wait runs out (DAMF_ERR_TIMEOUT).
__device__ __forceinline__ int wait_slot(DevHeader* h, int32_t* queue, long long p, long long qcap,
                                         long long limit = kSpinLimit) {
  for (long long it = 0;; ++it) {
    if (p < qcap) {
      const int e = ld_acquire(queue + p);
      if (e != -1) {
        queue[p] = -1;                 // read once per phase; empty again for the next launch
        return e;
      }
    }
    if ((ld_volatile64(&h->qstate) >> 32) == 0ull) return -1;
    if (*reinterpret_cast<volatile int*>(&h->status) != 0) return -1;
    if (it > limit) {
      set_status(h, DAMF_ERR_TIMEOUT);
      return -1;
    }
    if (it > 32) __nanosleep(it > 2048 ? 1024 : 128);
  }
}

// The task loop of one graph's push for one warp: claims queue positions kClaim at a time and
// runs the row and item tasks it finds, until no task is left (the unfinished count is zero),
// the device status is set, or a wait runs out. The warp's counters accumulate in my_*.
// Owners call it between the grid barriers of a phase; in a grouped push, warps whose own
// graphs are done call it on another graph's queue while that graph's loop is open.
template <int D, bool SCALED>
__device__ __forceinline__ void task_loop(const PushArgs& a, WarpQ& wq, WarpStats& st_w) {
  DevHeader* const h = a.h;
  const Adj in = a.in;
  const int32_t* __restrict__ outdeg = a.outdeg;
  const Workspace& ws = a.ws;
  float* const Zb = a.Zb;
  float* const r = a.r;
  const float alpha = a.alpha, eps = a.eps;
  const int direct_max = a.direct_max;
  constexpr int LPR = PushShape<D>::LPR;
  constexpr int RPW = PushShape<D>::RPW;
  const int lane = threadIdx.x & 31;
  const int sub = lane / LPR, q = lane % LPR;
  const float beta = 1.0f - alpha;
  const long long qcap = ws.qcap;
  int32_t* queue = ws.queue;
  uint32_t* inq = ws.stamp;
  // ---- task loop: claim kClaim positions at a time, lanes 0 .. kClaim-1 read their slots ----
  bool quit = false;
  while (!quit) {
    long long p0 = 0;
    if (lane == 0) p0 = atomicAdd(&h->q_head, kClaim);
    p0 = __shfl_sync(kFull, p0, 0);
    int eb = -1;
    if (lane < kClaim && p0 + lane < qcap) {
      eb = ld_acquire(queue + p0 + lane);
      if (eb != -1) queue[p0 + lane] = -1;   // read once per phase; empty again for the next launch
    }
    // and the entries' read-only data in the same pass: a row's in-edge range (and out-degree),
    // an item's (rho slot, first in-edge, count)
    int m0 = 0, m1 = 0, m2 = 1;
    if (lane < kClaim && eb != -1) {
      if (eb >= 0) {
        m0 = __ldg(in.start + eb);
        m1 = __ldg(in.len + eb);
        if (SCALED) m2 = __ldg(outdeg + eb);
      } else {
        const int4 wi = __ldcg(ws.work + (-eb - 2));
        m0 = wi.y;
        m1 = wi.z;
        m2 = wi.x;
      }
    }
    // the in-edges of every claimed hub item and their out-degrees, two loads for the whole
    // claim instead of two per item: lane kItemEdges b + j holds in-edge j of entry b
    int iw = 0, idg = 1;
    if constexpr (kClaim * kItemEdges == 32) {
      const int bb = lane / kItemEdges, j = lane % kItemEdges;
      const int e_b = __shfl_sync(kFull, eb, bb);
      const int st_b = __shfl_sync(kFull, m0, bb), n_b = __shfl_sync(kFull, m1, bb);
      const bool want = e_b < -1 && j < n_b &&
                        DAMF_DCHECK(h, st_b >= 0 && n_b <= kItemEdges && (long long)st_b + n_b <= in.m_cap);
      if (want) iw = __ldg(in.col + st_b + j);
      if (want && DAMF_DCHECK(h, (unsigned)iw < (unsigned)a.ncap)) idg = __ldg(outdeg + iw);
      else iw = 0;
    }
    // consecutive items of one hub share its rho row: read once per claim
    int rho_slot = -1;
    for (int b = 0; b < kClaim; ++b) {
    const long long p = p0 + b;
    int e = __shfl_sync(kFull, eb, b);
    const bool pre = e != -1;    // the batch pass read this entry's data
    int st = __shfl_sync(kFull, m0, b), deg = __shfl_sync(kFull, m1, b), aux = __shfl_sync(kFull, m2, b);
    if (e == -1) {
      flush(wq, h, queue, qcap, lane, ws.ovf);   // publish and uncount before waiting
      if (lane == 0) {
        const unsigned long long t0 = gtimer();
        e = wait_slot(h, queue, p, qcap);
        st_w.wait += gtimer() - t0;
      }
      e = __shfl_sync(kFull, e, 0);
      if (e == -1) {
        quit = true;                     // positions after p are not filled either
        break;
      }
    }
    // a dequeued id outside its array (DAMF_CHECK builds): the task is dropped (counted done)
    if (!(e >= 0 ? DAMF_DCHECK(h, e < a.ncap) : DAMF_DCHECK(h, (long long)(-e - 2) < ws.work_cap))) {
      wq.done += 1;
      continue;
    }
    if (e >= 0) {
      if (lane == 0) ++st_w.rows;
      // row task. The flag is cleared first; the removal of v below is ordered after the
      // clear (fence), so an add that lands after the removal finds the flag clear and queues
      // u again, while an add between the read of v and the removal shows in `left`.
      const int u = e;
      if (lane == 0) atomicExch(inq + u, 0u);
      __syncwarp();
      // group 0 reads r[u] once and hands it to the other groups, so that every group
      // scatters exactly the v that group 0 removes
      if (!pre) {
        st = __ldg(in.start + u);
        deg = __ldg(in.len + u);
        aux = SCALED ? __ldg(outdeg + u) : 1;
      }
      if (!DAMF_DCHECK(h, st >= 0 && deg >= 0 && (long long)st + deg <= in.m_cap)) deg = 0;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (sub == 0) v = f4_ldcg(r + (size_t)u * D + 4 * q);
      // the first 32 in-edges and their out-degrees are requested beside the row, so that they
      // arrive while the removal below is still in flight
      const bool pre0 = deg <= direct_max;
      int w0 = 0, d0 = 1;
      if (pre0 && lane < min(deg, 32)) w0 = __ldg(in.col + st + lane);
      if (RPW > 1) {
        v.x = __shfl_sync(kFull, v.x, q);
        v.y = __shfl_sync(kFull, v.y, q);
        v.z = __shfl_sync(kFull, v.z, q);
        v.w = __shfl_sync(kFull, v.w, q);
      }
      if (pre0 && lane < min(deg, 32) && DAMF_DCHECK(h, (unsigned)w0 < (unsigned)a.ncap)) d0 = __ldg(outdeg + w0);
      const int dout = aux;
      const float thr_u = threshold<SCALED>(eps, dout);
      bool go = group_max<LPR>(max_abs4(v)) > thr_u;   // the same in every group: warp-uniform
      if (!go) {
        // about to let u go: the read above may have passed the flag's clear, so an add whose
        // adder still found the flag set (its claim is a release) could be missing from v.
        // After a fence that orders the clear first, a second read must see every such add.
        __syncwarp();
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        if (sub == 0) v = f4_ldcg(r + (size_t)u * D + 4 * q);
        if (RPW > 1) {
          v.x = __shfl_sync(kFull, v.x, q);
          v.y = __shfl_sync(kFull, v.y, q);
          v.z = __shfl_sync(kFull, v.z, q);
          v.w = __shfl_sync(kFull, v.w, q);
        }
        go = group_max<LPR>(max_abs4(v)) > thr_u;
      }
      if (go) {
        float lm = 0.f;                           // max |r[u]| right after the removal of v
        __syncwarp();
        asm volatile("fence.acq_rel.gpu;" ::: "memory");   // the flag's clear comes first
        if (sub == 0) {
          const float4 old =
              atomicAdd(reinterpret_cast<float4*>(r + (size_t)u * D) + q, make_float4(-v.x, -v.y, -v.z, -v.w));
          lm = max_abs4(make_float4(old.x - v.x, old.y - v.y, old.z - v.z, old.w - v.w));
          atomicAdd(reinterpret_cast<float4*>(Zb + (size_t)u * D) + q,
                    make_float4(alpha * v.x, alpha * v.y, alpha * v.z, alpha * v.w));
        }
        if (lane == 0) {
          st_w.pushes += 1;
          st_w.edges += deg;
        }
        bool direct = true;
        if (deg > direct_max) {
          // hub: a rho slot and one item task per kItemEdges in-edges
          const int nch = (deg + kItemEdges - 1) / kItemEdges;
          int slot = 0, ib = 0;
          if (lane == 0) {
            slot = atomicAdd(&h->rho_tail, 1);
            ib = atomicAdd(&h->item_tail, nch);
          }
          slot = __shfl_sync(kFull, slot, 0);
          ib = __shfl_sync(kFull, ib, 0);
          if ((long long)slot < ws.rho_cap && (long long)ib + nch <= ws.work_cap) {
            direct = false;
            if (sub == 0) __stcg(reinterpret_cast<float4*>(ws.rho + (size_t)slot * D) + q, v);
            for (int c0 = 0; c0 < nch; c0 += 32) {   // warp-uniform
              const int c2 = c0 + lane;
              if (c2 < nch)
                __stcg(ws.work + ib + c2,
                       make_int4(slot, st + c2 * kItemEdges, min(kItemEdges, deg - c2 * kItemEdges), 0));
              stage(c2 < nch, -(ib + c2 + 2), wq, h, queue, qcap, lane);
            }
          }
        }
        if (direct)
          scatter_edges<D, SCALED>(v, st, deg, in.col, outdeg, r, beta, eps, wq, h, inq, queue, qcap, lane, sub, q,
                                   true, pre0, w0, d0, a.ncap);
        // u itself: adds that reached r[u] between the read of v and its removal are still there
        lm = __shfl_sync(kFull, group_max<LPR>(lm), 0);
        enqueue_rows(lane == 0 && lm > thr_u, u, wq, h, inq, queue, qcap, lane);
      }
    } else {
      // item task: one chunk of a hub's in-edges
      if (lane == 0) ++st_w.items;
      if (!pre) {
        const int4 wi = __ldcg(ws.work + (-e - 2));
        st = wi.y;
        deg = wi.z;
        aux = wi.x;
      }
      if (!DAMF_DCHECK(h, aux >= 0 && (long long)aux < ws.rho_cap && st >= 0 && deg >= 0 && deg <= kItemEdges &&
                              (long long)st + deg <= in.m_cap)) {
        deg = 0;
        aux = 0;
      }
      float4 rv;
      if (aux != rho_slot) {   // warp-uniform; the row is kept in the warp's shared slot, not in registers
        rv = f4_ldcg(ws.rho + (size_t)aux * D + 4 * q);
        if (sub == 0) reinterpret_cast<float4*>(wq.rho)[q] = rv;
        __syncwarp();
        rho_slot = aux;
      } else {
        rv = reinterpret_cast<const float4*>(wq.rho)[q];
      }
      int w0 = 0, d0 = 1;
      if (pre && kClaim * kItemEdges == 32) {   // the claim's pass loaded them: in-edge `lane` of this entry sits in lane kItemEdges b + lane
        const int src = min(b * kItemEdges + lane, 31);
        w0 = __shfl_sync(kFull, iw, src);
        d0 = __shfl_sync(kFull, idg, src);
      } else {
        if (lane < deg) w0 = __ldg(in.col + st + lane);
        if (lane < deg && DAMF_DCHECK(h, (unsigned)w0 < (unsigned)a.ncap)) d0 = __ldg(outdeg + w0);
      }
      scatter_edges<D, SCALED>(rv, st, deg, in.col, outdeg, r, beta, eps, wq, h, inq, queue, qcap, lane, sub,
                               q, true, true, w0, d0, a.ncap);
    }
    wq.done += 1;
    }
    // publish once enough is buffered (and always before waiting, above): fewer atomics on
    // the queue word, which every warp of the push shares
    if (wq.n >= 16) flush(wq, h, queue, qcap, lane, ws.ovf);
  }
  flush(wq, h, queue, qcap, lane, ws.ovf);
}

// The push of one graph by `nblocks` CTAs of 256 threads (this one is CTA `blk` of them): the
// whole launch for one graph (k_push), or one graph's share of a launch over many (k_push_group).
// s_t (5 words) and s_buf (8 warps x kQBuf) are the CTA's shared timers and warp queue buffers.
template <int D, bool SCALED>
__device__ __forceinline__ void push_body(const PushArgs& a, int n, int check_all, unsigned blk, unsigned nblocks,
                                          unsigned long long* s_t, int32_t (*s_buf)[kQBuf], float (*s_rho)[kMaxD],
                                          WarpStats* s_ws) {
  DevHeader* const h = a.h;
  const Adj in = a.in;
  const int32_t* __restrict__ outdeg = a.outdeg;
  const Workspace& ws = a.ws;
  float* const r = a.r;
  const float alpha = a.alpha, eps = a.eps;
  const int max_phases = a.max_phases;
  constexpr int LPR = PushShape<D>::LPR;
  constexpr int RPW = PushShape<D>::RPW;
  const int lane = threadIdx.x & 31;
  const int sub = lane / LPR, q = lane % LPR;
  const long long gwarp = ((long long)blk * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)nblocks * blockDim.x) >> 5;
  const unsigned epoch0 = h->epoch;
  const float beta = 1.0f - alpha;
  const long long qcap = ws.qcap;
  int32_t* queue = ws.queue;
  uint32_t* inq = ws.stamp;
  WarpStats& st_w = s_ws[threadIdx.x >> 5];   // this warp's counters (lane 0 keeps them)
  if (lane == 0) st_w = WarpStats{0, 0, 0ull, 0, 0};
  const int npend = h->pending;
  // block 0's view of where the time goes (ns): seeding, task loop, barriers; [4] is the last
  // mark. Kept in shared memory, where it costs no registers.
  const bool timer = blk == 0 && threadIdx.x == 0;
  if (timer) {
    s_t[0] = s_t[1] = s_t[2] = s_t[3] = 0ull;
    s_t[4] = gtimer();
  }
  WarpQ wq{s_buf[threadIdx.x >> 5], s_rho[threadIdx.x >> 5], 0, 0, ws.ovf, ws.stamp};
  int phase = 0;
  for (;; ++phase) {
    if (phase >= max_phases) {
      if (blk == 0 && threadIdx.x == 0) set_status(h, DAMF_ERR_NOT_CONVERGED);
      break;
    }
    // ---- seeding: the rows whose residual changed (or every row), when above eps ----
    const bool all = check_all || phase > 0;
    const int ncand = all ? n : npend;
    for (long long base = gwarp * RPW; base < ncand; base += nwarps * RPW) {
      const long long ci = base + sub;
      const bool valid = ci < ncand;
      const int u = valid ? (all ? (int)ci : __ldcg(ws.pend + ci)) : 0;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      int dout = 1;
      if (valid) {
        v = f4_ldcg(r + (size_t)u * D + 4 * q);
        if (SCALED) dout = __ldg(outdeg + u);
      }
      const bool above = group_max<LPR>(max_abs4(v)) > threshold<SCALED>(eps, dout);
      enqueue_rows(valid && above && q == 0, u, wq, h, inq, queue, qcap, lane);
    }
    flush(wq, h, queue, qcap, lane, ws.ovf);
    if (timer) time_mark(s_t, 0);
    if (!grid_barrier(&h->bar, h, nblocks)) return;
    if (timer) time_mark(s_t, 2);
    if (blk == 0 && threadIdx.x == 0) atomicExch(&h->help_open, 1);   // the queue is seeded

    // ---- task loop ----
    task_loop<D, SCALED>(a, wq, st_w);
    if (timer) time_mark(s_t, 1);
    if (!grid_barrier(&h->bar, h, nblocks)) return;   // every warp has left the task loop
    if (blk == 0 && threadIdx.x == 0) atomicExch(&h->help_open, 0);   // no task is left to help with
    const bool again = *reinterpret_cast<volatile int*>(&h->overflow) != 0 &&
                       *reinterpret_cast<volatile int*>(&h->status) == 0;
    if (!again) {
      if (timer) time_mark(s_t, 2);
      ++phase;
      break;
    }
    // overflow: scatter the hub items that found the queue full (their mass is out of r
    // already), unflag every row and start a phase that checks them all
    {
      const int novf = *reinterpret_cast<volatile int*>(&h->ovf_count);
      for (long long i = gwarp; i < novf; i += nwarps) {
        const int4 wi = __ldcg(ws.work + __ldcg(ws.ovf + i));
        const bool ok = DAMF_DCHECK(h, wi.x >= 0 && (long long)wi.x < ws.rho_cap && wi.y >= 0 && wi.z >= 0 &&
                                           (long long)wi.y + wi.z <= in.m_cap);
        const float4 rv = f4_ldcg(ws.rho + (size_t)(ok ? wi.x : 0) * D + 4 * q);
        scatter_edges<D, SCALED>(rv, wi.y, ok ? wi.z : 0, in.col, outdeg, r, beta, eps, wq, h, inq, queue, qcap, lane,
                                 sub, q, false, false, 0, 1, a.ncap);
      }
    }
    for (long long u = (long long)blk * blockDim.x + threadIdx.x; u < n; u += (long long)nblocks * blockDim.x)
      inq[u] = 0u;
    // helpers that joined before the gate closed leave before the queue words are reset
    if (blk == 0 && threadIdx.x == 0) {
      __threadfence();   // the gate's close (above) is ordered before this read of helpers
      long long it = 0;
      while (*reinterpret_cast<volatile int*>(&h->helpers) != 0) {
        if (++it > kSpinLimit) {
          set_status(h, DAMF_ERR_TIMEOUT);
          break;
        }
        __nanosleep(64);
      }
    }
    if (!grid_barrier(&h->bar, h, nblocks)) return;   // everyone has read the overflow flag
    if (blk == 0 && threadIdx.x == 0) {
      h->qstate = 0ull;
      h->q_head = 0;
      h->overflow = 0;
      h->rho_tail = 0;
      h->item_tail = 0;
      h->ovf_count = 0;
    }
    if (!grid_barrier(&h->bar, h, nblocks)) return;
    if (timer) time_mark(s_t, 2);
  }
  if (timer)
    for (int i = 0; i < 3; ++i) h->push_ns[i] += s_t[i];
  // counters and bookkeeping (block 0 after the last barrier; everyone has left the loop)
  if (lane == 0) {
    const WarpStats w = st_w;
    if (w.pushes || w.edges) {
      atomicAdd((unsigned long long*)&h->pushes, (unsigned long long)w.pushes);
      atomicAdd((unsigned long long*)&h->push_edges, (unsigned long long)w.edges);
    }
    if (w.wait) atomicAdd(&h->push_ns[3], w.wait / (unsigned long long)nwarps);
    if (w.rows || w.items) {
      atomicAdd((unsigned long long*)&h->push_tasks, (unsigned long long)w.rows);
      atomicAdd((unsigned long long*)&h->push_items, (unsigned long long)w.items);
    }
  }
  if (blk == 0 && threadIdx.x == 0) {
    h->push_rounds += phase;
    h->pending = 0;
    h->check_all = 0;
    h->epoch = epoch0 + 2u;
  }
}

// 64 registers at most (min. 4 CTAs' worth per SM): two push CTAs (32k registers) then leave room
// on every SM for the 768-thread core SVD CTA of the next update, which runs beside the push
template <int D, bool SCALED>
__global__ void __launch_bounds__(256, 4) k_push(PushArgs a, int n, int check_all) {
  __shared__ unsigned long long s_t[5];
  __shared__ int32_t s_buf[8][kQBuf];   // 256 threads: 8 warps
  __shared__ __align__(16) float s_rho[8][kMaxD];
  __shared__ WarpStats s_ws[8];
  push_body<D, SCALED>(a, n, check_all, blockIdx.x, gridDim.x, s_t, s_buf, s_rho, s_ws);
}

// Zeroes the work-queue words of every graph of a grouped push (one thread per graph).
__global__ void k_push_reset(const PushArgs* __restrict__ descs, int count) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= count) return;
  DevHeader* h = descs[g].h;
  h->qstate = 0ull;
  h->q_head = 0;
  h->overflow = 0;
  h->rho_tail = 0;
  h->item_tail = 0;
  h->ovf_count = 0;
  h->help_open = 0;
  h->helpers = 0;
}

constexpr int kHelpMinTasks = 64;   // a graph with fewer unfinished tasks is left to its own warps
constexpr int kHelpRounds = 256;    // graphs one warp may help in turn

// A warp whose own graphs are pushed joins the task loop of the open graph with the most
// unfinished tasks, until none is left with at least kHelpMinTasks. It registers (helpers) and
// then checks the gate, so that a graph that closes its gate and then finds helpers == 0 has no
// warp of another graph left in its loop; its tasks' counters go to that graph's header.
template <bool SCALED>
__device__ __forceinline__ void help_others(const PushArgs* __restrict__ descs, int ngraphs, int32_t* buf,
                                            float* rho, WarpStats& st_w) {
  const int lane = threadIdx.x & 31;
  for (int round = 0; round < kHelpRounds; ++round) {
    unsigned best = 0;
    int bg = -1;
    for (int g = lane; g < ngraphs; g += 32) {
      DevHeader* hg = descs[g].h;
      if (*reinterpret_cast<volatile int*>(&hg->help_open) != 0) {
        const unsigned u = (unsigned)(ld_volatile64(&hg->qstate) >> 32);
        if (u > best) {
          best = u;
          bg = g;
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned ob = __shfl_xor_sync(kFull, best, o);
      const int og = __shfl_xor_sync(kFull, bg, o);
      if (ob > best || (ob == best && og > bg)) {
        best = ob;
        bg = og;
      }
    }
    if (bg < 0 || best < (unsigned)kHelpMinTasks) return;
    const PushArgs& a = descs[bg];
    int ok = 0;
    if (lane == 0) {
      atomicAdd(&a.h->helpers, 1);
      __threadfence();
      ok = *reinterpret_cast<volatile int*>(&a.h->help_open);
      if (!ok) atomicSub(&a.h->helpers, 1);
    }
    if (!__shfl_sync(kFull, ok, 0)) continue;
    WarpQ wq{buf, rho, 0, 0, a.ws.ovf, a.ws.stamp};
    if (lane == 0) st_w = WarpStats{0, 0, 0ull, 0, 0};
    switch (a.d) {
      case 16: task_loop<16, SCALED>(a, wq, st_w); break;
      case 32: task_loop<32, SCALED>(a, wq, st_w); break;
      case 64: task_loop<64, SCALED>(a, wq, st_w); break;
      default: task_loop<128, SCALED>(a, wq, st_w); break;
    }
    if (lane == 0) {
      const WarpStats w = st_w;
      if (w.pushes || w.edges) {
        atomicAdd((unsigned long long*)&a.h->pushes, (unsigned long long)w.pushes);
        atomicAdd((unsigned long long*)&a.h->push_edges, (unsigned long long)w.edges);
      }
      if (w.rows || w.items) {
        atomicAdd((unsigned long long*)&a.h->push_tasks, (unsigned long long)w.rows);
        atomicAdd((unsigned long long*)&a.h->push_items, (unsigned long long)w.items);
      }
      __threadfence();
      atomicSub(&a.h->helpers, 1);
    }
    __syncwarp();
  }
}

// The pushes of many graphs in one cooperative launch, in slots: slot s owns CTAs
// sfirst[s] .. sfirst[s+1]-1 and graphs gfirst[s] .. gfirst[s+1]-1 of descs. A slot of one graph
// runs that graph's push over its CTAs (its own queue, header and grid barrier among them); a
// slot of several graphs has one CTA, which pushes them one after another. The rank d of each
// graph selects the row shape; node count and full seeding come from the graph's device header,
// so one captured launch serves every step. Three CTAs per SM (80 registers): the kernel holds
// the task loop for every d, and at four (64 registers) it spilled 1.9 KB per thread; on the
// 256-graph fleet three ran the push phase in 283 ms per step against 333 ms for four.
template <bool SCALED>
__global__ void __launch_bounds__(256, 3) k_push_group(const PushArgs* __restrict__ descs, const int* __restrict__ table,
                                                       int nslots, int plan, int ngraphs) {
  __shared__ PushArgs sa;
  __shared__ int s_s, s_n, s_all;
  __shared__ unsigned long long s_t[5];
  __shared__ int32_t s_buf[8][kQBuf];   // 256 threads: 8 warps
  __shared__ __align__(16) float s_rho[8][kMaxD];
  __shared__ WarpStats s_ws[8];
  // a launch captured under an earlier plan of the fleet must not run on this plan's tables:
  // every CTA returns before any barrier and the graphs' status reports it
  if (table[0] != nslots || table[1] != (int)gridDim.x || table[2] != plan) {
    if (blockIdx.x == 0)
      for (int g = threadIdx.x; g < ngraphs; g += blockDim.x) set_status(descs[g].h, DAMF_ERR_INVALID);
    return;
  }
  const int* __restrict__ sfirst = table + 3;
  const int* __restrict__ gfirst = sfirst + nslots + 1;
  if (threadIdx.x == 0) {
    int lo = 0, hi = nslots - 1;   // the last slot with sfirst[s] <= blockIdx.x
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sfirst[mid] <= (int)blockIdx.x) lo = mid;
      else hi = mid - 1;
    }
    s_s = lo;
  }
  __syncthreads();
  const int slot = s_s;
  const unsigned blk = blockIdx.x - (unsigned)sfirst[slot];
  const unsigned nb = (unsigned)(sfirst[slot + 1] - sfirst[slot]);
  const int g1 = gfirst[slot + 1];
  for (int g = gfirst[slot]; g < g1; ++g) {
    __syncthreads();   // the previous graph's push no longer reads sa
    {
      const int* src = reinterpret_cast<const int*>(descs + g);
      int* dst = reinterpret_cast<int*>(&sa);
      for (int i = threadIdx.x; i < (int)(sizeof(PushArgs) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_n = *reinterpret_cast<volatile int*>(&sa.h->n_nodes);
      s_all = *reinterpret_cast<volatile int*>(&sa.h->check_all);
    }
    __syncthreads();
    switch (sa.d) {
      case 16: push_body<16, SCALED>(sa, s_n, s_all, blk, nb, s_t, s_buf, s_rho, s_ws); break;
      case 32: push_body<32, SCALED>(sa, s_n, s_all, blk, nb, s_t, s_buf, s_rho, s_ws); break;
      case 64: push_body<64, SCALED>(sa, s_n, s_all, blk, nb, s_t, s_buf, s_rho, s_ws); break;
      default: push_body<128, SCALED>(sa, s_n, s_all, blk, nb, s_t, s_buf, s_rho, s_ws); break;
    }
  }
  // this CTA's graphs are pushed: its warps help the graphs still running
  help_others<SCALED>(descs, gfirst[nslots], s_buf[threadIdx.x >> 5], s_rho[threadIdx.x >> 5], s_ws[threadIdx.x >> 5]);
}

PushArgs push_args(const Ctx* c, int direct_chunks) {
  PushArgs a;
  memset(&a, 0, sizeof(a));
  a.h = c->hdr;
  a.in = c->cfg.directed ? c->in : c->out;
  a.outdeg = c->out.len;
  a.ws = c->ws;
  a.Zb = c->Zb;
  a.r = c->r;
  a.alpha = (float)c->cfg.alpha;
  a.eps = (float)c->cfg.eps;
  a.max_phases = c->cfg.max_push_rounds;
  a.d = c->d;
  a.ncap = c->cfg.n_capacity;
  const int epc = c->d == 128 ? PushShape<128>::EPC : c->d == 64 ? PushShape<64>::EPC
                : c->d == 32 ? PushShape<32>::EPC : PushShape<16>::EPC;
  a.direct_max = (direct_chunks >= 0 ? direct_chunks : kPushDirectChunks) * epc;
  return a;
}

// co-resident CTAs of the grouped push on the current device: a fleet's push runs after every
// update of its step, so it may take the whole occupancy (not only two CTAs per SM)
template <bool SCALED>
static int group_max_blocks() {
  static int cached = 0;
  if (cached == 0) {
    cudaFuncSetAttribute(k_push_group<SCALED>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push_group<SCALED>, 256, 0);
    cached = sms * (per_sm < 1 ? 1 : per_sm);
  }
  return cached;
}

int push_group_max_blocks(int scaled) { return scaled ? group_max_blocks<true>() : group_max_blocks<false>(); }

cudaError_t launch_push_group(const PushArgs* descs, int ngraphs, const int* table, int nslots, int blocks,
                              int plan, int scaled, cudaStream_t s) {
  if (ngraphs <= 0 || nslots <= 0) return cudaSuccess;
  k_push_reset<<<(ngraphs + 255) / 256, 256, 0, s>>>(descs, ngraphs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&descs, (void*)&table, &nslots, &plan, &ngraphs};
  return scaled ? cudaLaunchCooperativeKernel((void*)k_push_group<true>, dim3(blocks), dim3(256), args, 0, s)
                : cudaLaunchCooperativeKernel((void*)k_push_group<false>, dim3(blocks), dim3(256), args, 0, s);
}

template <int D, bool SCALED>
static cudaError_t push_impl(Ctx* c, int check_all, cudaStream_t s) {
  if (c->push_max == 0) {
    cudaFuncSetAttribute(k_push<D, SCALED>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    int per_sm = 0, dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push<D, SCALED>, 256, 0);
    if (per_sm < 1) per_sm = 1;
    c->push_occ = sms * per_sm;
    c->push_max = 2 * per_sm > kPushHalfBlocksPerSM ? sms * kPushHalfBlocksPerSM / 2 : sms * per_sm;
  }
  // a cooperative grid must fit on the device at once
  const int blocks = c->push_blocks > 0 ? (c->push_blocks < c->push_occ ? c->push_blocks : c->push_occ) : c->push_max;
  const int chunks = c->push_direct_chunks;
  // qstate .. helpers (the queue words, on their own cache lines, and the padding between them)
  static_assert(offsetof(DevHeader, helpers) > offsetof(DevHeader, qstate), "queue words in header order");
  const size_t qbytes = offsetof(DevHeader, helpers) + sizeof(int) - offsetof(DevHeader, qstate);
  cudaError_t e = cudaMemsetAsync(&c->hdr->qstate, 0, qbytes, s);
  if (e != cudaSuccess) return e;
  PushArgs a = push_args(c, chunks);
  int n = c->n;
  check_all = check_all ? 1 : 0;
  void* args[] = {&a, &n, &check_all};
  return cudaLaunchCooperativeKernel((void*)k_push<D, SCALED>, dim3(blocks), dim3(256), args, 0, s);
}

template <bool SCALED>
static cudaError_t push_dispatch(Ctx* c, int check_all, cudaStream_t s) {
  switch (c->d) {
    case 16: return push_impl<16, SCALED>(c, check_all, s);
    case 32: return push_impl<32, SCALED>(c, check_all, s);
    case 64: return push_impl<64, SCALED>(c, check_all, s);
    default: return push_impl<128, SCALED>(c, check_all, s);
  }
}

int push_default_direct_chunks() { return kPushDirectChunks; }

// Failure detection without a fault: the push's own bounded waits, run against conditions that
// never come true, must give up after `limit` iterations, record DAMF_ERR_TIMEOUT and return.
// which = 0: a grid barrier that counts one CTA more than the launch has (this one CTA
// waits for a second that never arrives); which = 1: a wait for a queue position that nobody
// fills while one task is still counted as unfinished.
__global__ void k_wait_selftest(DevHeader* h, int32_t* queue, int which, long long limit) {
  if (which == 0) {
    grid_barrier(&h->bar, h, gridDim.x + 1, limit);
  } else if (threadIdx.x == 0) {
    wait_slot(h, queue, 0, 1, limit);
  }
}

cudaError_t launch_wait_selftest(DevHeader* h, int32_t* queue, int which, long long limit, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(h, queue, which, limit);
  return cudaGetLastError();
}

cudaError_t launch_push(Ctx* c, int check_all, cudaStream_t s) {
  return c->cfg.threshold ? push_dispatch<true>(c, check_all, s) : push_dispatch<false>(c, check_all, s);
}

}  // namespace damf
