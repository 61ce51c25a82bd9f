// Graph store and per-update sparse change.
//
//  * slack adjacency: each row owns [start, start+cap) of col[], holds len entries;
//    a row that overflows is relocated to the bump tail with doubled capacity.
//  * k_prepare (one CTA per update): set semantics of the events (last event per
//    ordered pair decides; delta = final - initial membership), the touched sets
//    S (rows with a changed entry) and T (columns), the net-change matrix
//    N[a][b] = dA[S_a][T_b] so that dA = I_S N I_T^T (Sec. 4.3, Eq. "edge_B" summed
//    over the update), and the adjacency edit.  Capacity is checked before any write.
//  * k_fixup: the PPR residual change for changed out-rows.  With P = D^{-1} A and
//    Pi^{-1} = (I - (1-alpha) P) / alpha, the residual r = X_b - Pi^{-1} Z_b changes by
//    ((1-alpha)/alpha) (P' - P) Z_b; only rows u in S change (Sec. 4.4, Step 4).
#include <algorithm>
#include <vector>

#include <cub/device/device_segmented_sort.cuh>

#include "damf_internal.cuh"

namespace damf {

// Events in use: k, or *kdev clamped to [0, k] when the count lives on the device.
__device__ __forceinline__ int live_events(int k, const int32_t* kdev, int lo) {
  if (!kdev) return k;
  const int kd = *kdev - lo;
  return kd < 0 ? 0 : (kd < k ? kd : k);
}

__global__ void k_validate(DevHeader* h, const int32_t* src, const int32_t* dst, const int8_t* op, int kmax,
                           const int32_t* kdev, int n_after) {
  const int k = live_events(kmax, kdev, 0);
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) h->n_nodes = n_after;
  if (i >= k) return;
  int u = src[i], v = dst[i], o = op[i];
  bool bad = u < 0 || v < 0 || u >= n_after || v >= n_after || u == v || (o != 1 && o != -1);
  if (bad) set_status(h, DAMF_ERR_INVALID);
  if (i == 0) atomicAdd((unsigned long long*)&h->edges_applied, (unsigned long long)k);
}

cudaError_t launch_validate(Ctx* c, const int32_t* src, const int32_t* dst, const int8_t* op, int k,
                            const int32_t* kdev, int n_after, cudaStream_t s) {
  // launched for every call: it also records the node count the push works over
  k_validate<<<k > 0 ? (k + 255) / 256 : 1, 256, 0, s>>>(c->hdr, src, dst, op, k, kdev, n_after);
  return cudaGetLastError();
}

// Warp searches row u for v; returns the position or -1.  Four 32-entry chunks are loaded
// per round, so a long row costs a quarter of the dependent round trips.
__device__ __forceinline__ int row_find(const Adj& a, int u, int v) {
  const int lane = threadIdx.x & 31;
  const int st = a.start[u], ln = a.len[u];
  for (int base = 0; base < ln; base += 128) {
    int x[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = base + 32 * c + lane;
      x[c] = j < ln ? a.col[st + j] : -1;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const unsigned hit = __ballot_sync(0xffffffffu, x[c] == v);
      if (hit) return base + 32 * c + __ffs(hit) - 1;
    }
  }
  return -1;
}

// Whether entry (u, v) is present: row u of the out-adjacency holds v exactly when row v of
// the in-adjacency (the out-adjacency itself for an undirected graph) holds u, so the
// shorter of the two rows is searched (a hub's row is then rarely scanned).
__device__ __forceinline__ bool has_entry(const Adj& out, const Adj& in, int u, int v) {
  return in.len[v] < out.len[u] ? row_find(in, v, u) >= 0 : row_find(out, u, v) >= 0;
}

__device__ __forceinline__ int grown_cap(int cap, int need) {
  int c = max(2 * cap, need + 4);
  return (c + 3) & ~3;
}

// Edits the rows listed in rows[0..nrows) of adjacency a; entries (row, col, delta) of
// row q are ent[first[q] .. first[q+1]).  One warp per row.  Relocation space was
// reserved by the caller at reloc_base[q] (or -1 when the row fits).
__device__ void apply_row_edits(Adj a, const int* rows, int nrows, const int* first, const int4* ent,
                                const long long* reloc_base, const int* reloc_cap, int* deg_new) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int q = warp; q < nrows; q += nw) {
    const int u = rows[q];
    if (reloc_base[q] >= 0) {  // move the row to its new home first
      const int st = a.start[u], ln = a.len[u];
      const long long nb = reloc_base[q];
      for (int j = lane; j < ln; j += 32) a.col[nb + j] = a.col[st + j];
      __syncwarp();
      if (lane == 0) {
        a.start[u] = (int)nb;
        a.cap[u] = reloc_cap[q];
      }
      __syncwarp();
    }
    // deletions first, so the row never holds more than max(len, new len) entries
    for (int e = first[q]; e < first[q + 1]; ++e) {
      const int4 x = ent[e];
      if (x.z >= 0) continue;
      const int pos = row_find(a, u, x.y);
      if (lane == 0 && pos >= 0) {
        const int st = a.start[u], ln = a.len[u];
        a.col[st + pos] = a.col[st + ln - 1];
        a.len[u] = ln - 1;
      }
      __syncwarp();
    }
    if (lane == 0) {
      for (int e = first[q]; e < first[q + 1]; ++e) {
        const int4 x = ent[e];
        if (x.z <= 0) continue;
        const int st = a.start[u], ln = a.len[u];
        a.col[st + ln] = x.y;
        a.len[u] = ln + 1;
      }
    }
    __syncwarp();
    if (lane == 0 && deg_new) deg_new[q] = a.len[u];
  }
}

template <int DIRECTED>
__global__ void __launch_bounds__(512) k_prepare(DevHeader* h, Adj out, Adj in, Workspace ws, const int32_t* src,
                                                 const int32_t* dst, const int8_t* op, int kmax,
                                                 const int32_t* kdev, int lo) {
  const int k = live_events(kmax, kdev, lo);
  __shared__ unsigned long long key[kMaxEntries];
  __shared__ int evt[kMaxEntries];
  __shared__ int eop[kMaxEntries];
  __shared__ unsigned long long skey[kMaxEntries];
  __shared__ int sop[kMaxEntries];
  __shared__ int sdelta[kMaxEntries];
  __shared__ int3 ed[kMaxEntries];     // compacted edits, key order (u, v, delta)
  __shared__ int3 edT[kMaxEntries];    // directed: (v, u, delta) in (v, u) order
  __shared__ int ne, nedit, nS, nT, nTrow, fail;
  __shared__ int Srow[kMaxR + 1], Sfirst[kMaxR + 1];
  __shared__ int Tcol[kMaxR + 1], Tfirst[kMaxR + 1];
  __shared__ long long relocS[kMaxR], relocT[kMaxR];
  __shared__ int rcapS[kMaxR], rcapT[kMaxR];
  const int tid = threadIdx.x;
  if (h->status != 0) {
    if (tid == 0) h->nS = h->nT = h->nedit = 0;
    return;
  }
  if (tid == 0) {
    ne = DIRECTED ? k : 2 * k;
    fail = 0;
  }
  __syncthreads();
  for (int i = tid; i < k; i += blockDim.x) {
    const unsigned int u = (unsigned int)src[i], v = (unsigned int)dst[i];
    key[DIRECTED ? i : 2 * i] = ((unsigned long long)u << 32) | v;
    evt[DIRECTED ? i : 2 * i] = i;
    eop[DIRECTED ? i : 2 * i] = op[i];
    if (!DIRECTED) {
      key[2 * i + 1] = ((unsigned long long)v << 32) | u;
      evt[2 * i + 1] = i;
      eop[2 * i + 1] = op[i];
    }
  }
  __syncthreads();
  // sort entries by (key, event index): rank by counting
  for (int i = tid; i < ne; i += blockDim.x) {
    int rk = 0;
    const unsigned long long ki = key[i];
    const int ti = evt[i];
    for (int j = 0; j < ne; ++j) {
      const unsigned long long kj = key[j];
      rk += (kj < ki) || (kj == ki && evt[j] < ti);
    }
    skey[rk] = ki;
    sop[rk] = eop[i];
  }
  __syncthreads();
  // last event per ordered pair decides; membership lookup (one warp per pair)
  {
    const int warp = tid >> 5, lane = tid & 31, nw = blockDim.x >> 5;
    for (int i = warp; i < ne; i += nw) {
      const bool last = (i == ne - 1) || (skey[i + 1] != skey[i]);
      int dl = 0;
      if (last) {
        const int u = (int)(skey[i] >> 32), v = (int)(skey[i] & 0xffffffffu);
        const int initial = has_entry(out, in, u, v) ? 1 : 0;
        const int fin = sop[i] > 0 ? 1 : 0;
        dl = fin - initial;
      }
      if (lane == 0) sdelta[i] = dl;
    }
  }
  __syncthreads();
  if (tid < 32) {  // compaction and S (edits are in (u, v) order), 32 entries at a time
    const int lane = tid;
    const unsigned below = (1u << lane) - 1u;
    int m = 0, s = 0, prevu = -1;   // edits and rows so far, the last edit's row
    for (int base = 0; base < ne; base += 32) {
      const int i = base + lane;
      const bool live = i < ne && sdelta[i] != 0;
      const int u = live ? (int)(skey[i] >> 32) : -1;
      const unsigned lmask = __ballot_sync(0xffffffffu, live);
      const unsigned lb = lmask & below;
      const int pu = __shfl_sync(0xffffffffu, u, lb ? 31 - __clz(lb) : 0);
      const bool head = live && (lb ? pu : prevu) != u;   // first edit of its row
      const unsigned hmask = __ballot_sync(0xffffffffu, head);
      const int pos = m + __popc(lb);
      if (live) ed[pos] = make_int3(u, (int)(skey[i] & 0xffffffffu), sdelta[i]);
      if (head) {
        const int q = s + __popc(hmask & below);
        Srow[q] = u;
        Sfirst[q] = pos;
      }
      m += __popc(lmask);
      s += __popc(hmask);
      if (lmask) prevu = __shfl_sync(0xffffffffu, u, 31 - __clz(lmask));
    }
    if (lane == 0) {
      Sfirst[s] = m;
      nedit = m;
      nS = s;
    }
  }
  __syncthreads();
  // T: sorted unique columns; edT = edits ordered by (v, u)
  for (int i = tid; i < nedit; i += blockDim.x) {
    int rk = 0;
    const int3 x = ed[i];
    for (int j = 0; j < nedit; ++j) {
      const int3 y = ed[j];
      rk += (y.y < x.y) || (y.y == x.y && y.x < x.x);
    }
    edT[rk] = make_int3(x.y, x.x, x.z);
  }
  __syncthreads();
  if (tid < 32) {  // T's heads: the first edit of each column, 32 edits at a time
    const int lane = tid;
    const unsigned below = (1u << lane) - 1u;
    int t = 0, prevv = -1;   // columns so far, the last edit's column
    for (int base = 0; base < nedit; base += 32) {
      const int i = base + lane;
      const int v = i < nedit ? edT[i].x : -1;
      const int pv = __shfl_up_sync(0xffffffffu, v, 1);
      const bool head = i < nedit && (lane == 0 ? prevv : pv) != v;
      const unsigned hmask = __ballot_sync(0xffffffffu, head);
      if (head) {
        const int q = t + __popc(hmask & below);
        Tcol[q] = v;
        Tfirst[q] = i;
      }
      t += __popc(hmask);
      prevv = __shfl_sync(0xffffffffu, v, 31);
    }
    if (lane == 0) {
      Tfirst[t] = nedit;
      nT = t;
      nTrow = t;
    }
  }
  __syncthreads();
  // capacity check (before any write): one thread per touched row, then a prefix sum
  // of the relocation sizes (thread 0, shared memory only)
  for (int q = tid; q < nS; q += blockDim.x) {
    const int u = Srow[q];
    int ins = 0, del = 0;
    for (int e = Sfirst[q]; e < Sfirst[q + 1]; ++e) (ed[e].z > 0 ? ins : del)++;
    const int nl = out.len[u] - del + ins;
    rcapS[q] = nl > out.cap[u] ? grown_cap(out.cap[u], nl) : 0;
  }
  if (DIRECTED) {
    for (int q = tid; q < nTrow; q += blockDim.x) {
      const int v = Tcol[q];
      int ins = 0, del = 0;
      for (int e = Tfirst[q]; e < Tfirst[q + 1]; ++e) (edT[e].z > 0 ? ins : del)++;
      const int nl = in.len[v] - del + ins;
      rcapT[q] = nl > in.cap[v] ? grown_cap(in.cap[v], nl) : 0;
    }
  }
  __syncthreads();
  if (tid < 32) {   // relocation offsets: exclusive prefix sums in one warp, 32 rows at a time
    const int lane = tid;
    auto plan = [&](const int* rcap, long long* reloc, int cnt, long long t0) {
      long long need = 0;
      for (int base = 0; base < cnt; base += 32) {
        const int q = base + lane;
        const long long c = q < cnt ? rcap[q] : 0;
        long long incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const long long y = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += y;
        }
        if (q < cnt) reloc[q] = c ? t0 + need + (incl - c) : -1;
        need += __shfl_sync(0xffffffffu, incl, 31);
      }
      return need;
    };
    const long long t0 = h->tail_out;
    const long long need = plan(rcapS, relocS, nS, t0);
    bool over = t0 + need > out.m_cap;
    long long needT = 0;
    if (DIRECTED) {
      const long long t1 = h->tail_in;
      needT = plan(rcapT, relocT, nTrow, t1);
      over = over || t1 + needT > in.m_cap;
    }
    if (lane == 0) {
      if (over) {
        fail = 1;
        set_status(h, DAMF_ERR_CAPACITY);
      } else {
        h->tail_out = t0 + need;
        if (DIRECTED) h->tail_in += needT;
      }
    }
  }
  __syncthreads();
  if (fail) {
    if (tid == 0) h->nS = h->nT = h->nedit = 0;
    return;
  }
  // write the sets, N, the edit lists and the relocation plan; the adjacency itself is
  // edited later by k_edit (a PPR push may still be reading it)
  for (int i = tid; i < nS; i += blockDim.x) {
    ws.S[i] = Srow[i];
    ws.deg_old[i] = out.len[Srow[i]];
    ws.relocS[i] = relocS[i];
    ws.rcapS[i] = rcapS[i];
  }
  for (int i = tid; i <= nS; i += blockDim.x) ws.Sfirst[i] = Sfirst[i];
  for (int i = tid; i < nT; i += blockDim.x) {
    ws.T[i] = Tcol[i];
    if (DIRECTED) {
      ws.relocT[i] = relocT[i];
      ws.rcapT[i] = rcapT[i];
    }
  }
  for (int i = tid; i <= nT; i += blockDim.x) ws.Tfirst[i] = Tfirst[i];
  for (int i = tid; i < nS * nT; i += blockDim.x) ws.N[i] = 0.0f;
  __syncthreads();
  for (int e = tid; e < nedit; e += blockDim.x) {
    const int3 x = ed[e];
    int a = 0, b = 0;   // positions of x's row in S and column in T (both sorted, unique)
    for (int hi = nS - 1; a < hi;) {
      const int mid = (a + hi) >> 1;
      if (Srow[mid] < x.x) a = mid + 1;
      else hi = mid;
    }
    for (int hi = nT - 1; b < hi;) {
      const int mid = (b + hi) >> 1;
      if (Tcol[mid] < x.y) b = mid + 1;
      else hi = mid;
    }
    ws.N[a * nT + b] = (float)x.z;
    ws.edits[e] = make_int4(x.x, x.y, x.z, a);
    if (DIRECTED) ws.editsT[e] = make_int4(edT[e].x, edT[e].y, edT[e].z, 0);
  }
  if (tid == 0) {
    h->nS = nS;
    h->nT = nT;
    h->nedit = nedit;
  }
}

// Applies the planned adjacency edit of the current update (after any push that reads
// the adjacency has finished), records the new out-degrees, queues the rows whose PPR
// residual changes for the next push, and counts the update.
template <int DIRECTED>
__global__ void __launch_bounds__(512) k_edit(DevHeader* h, Adj out, Adj in, Workspace ws) {
  if (h->status != 0) return;
  const int nS = h->nS, nT = h->nT, nedit = h->nedit;
  if (nedit == 0) return;
  const int tid = threadIdx.x;
  apply_row_edits(out, ws.S, nS, ws.Sfirst, ws.edits, ws.relocS, ws.rcapS, ws.deg_new);
  if (DIRECTED) {
    __syncthreads();
    apply_row_edits(in, ws.T, nT, ws.Tfirst, ws.editsT, ws.relocT, ws.rcapT, nullptr);
  }
  if (tid == 0) {
    h->updates += 1;
    h->entries_changed += nedit;
    h->touched_rows += nS + nT;
    h->last_rank = nS;
  }
  // rows whose residual changes (signal delta and fix-up) are queued for the next push
  for (int i = tid; i < nS; i += blockDim.x) {
    const int u = ws.S[i];
    if (atomicExch(&ws.pstamp[u], h->epoch) != h->epoch) {
      const int p = atomicAdd(&h->pending, 1);
      ws.pend[p] = u;
    }
  }
}

cudaError_t launch_edit(Ctx* c, cudaStream_t s) {
  if (c->cfg.directed)
    k_edit<1><<<1, 512, 0, s>>>(c->hdr, c->out, c->in, c->ws);
  else
    k_edit<0><<<1, 512, 0, s>>>(c->hdr, c->out, c->out, c->ws);
  return cudaGetLastError();
}

cudaError_t launch_prepare(Ctx* c, const int32_t* src, const int32_t* dst, const int8_t* op, int k,
                           const int32_t* kdev, int lo, cudaStream_t s) {
  if (c->cfg.directed)
    k_prepare<1><<<1, 512, 0, s>>>(c->hdr, c->out, c->in, c->ws, src + lo, dst + lo, op + lo, k, kdev, lo);
  else
    k_prepare<0><<<1, 512, 0, s>>>(c->hdr, c->out, c->out, c->ws, src + lo, dst + lo, op + lo, k, kdev, lo);
  return cudaGetLastError();
}

// ---- graph-change fix-up of the PPR residual (one CTA per changed out-row) ----
// r[u] += (a - b) sum_{v in N'(u)} Zb[v] + b (sum_{added} Zb[v] - sum_{removed} Zb[v])
// with a = c/deg'(u) (0 if deg' = 0), b = c/deg(u) (0 if deg = 0), c = (1-alpha)/alpha:
// this equals c (mean_{N'(u)} Zb - mean_{N(u)} Zb) because N(u) = N'(u) - added + removed.
// One changed row u per blockIdx.x, its adjacency row split over kFixSplit CTAs (blockIdx.y,
// interleaved groups of rows, four loads in flight per warp): a hub's thousands of
// neighbours are read by many SMs at once. Each CTA leaves its partial sum in the workspace;
// the last of the row's CTAs (counted by an atomic per row, reset by that CTA) adds the
// partials in CTA order to r[u], so the result does not depend on which CTA finishes last.
template <int D>
__global__ void __launch_bounds__(256) k_fixup(DevHeader* h, Adj out, Workspace ws, const float* __restrict__ Zb,
                                               float* r, float c_alpha) {
  constexpr int LPR = D / 4;          // lanes per row (float4 each)
  constexpr int RPW = 32 / LPR;       // rows per warp step
  constexpr int UNR = 4;              // row loads in flight per lane
  __shared__ float4 part[8][32];
  __shared__ int last;
  const int a_idx = blockIdx.x, cta = blockIdx.y;
  if (h->status != 0 || a_idx >= h->nS) return;
  const int u = ws.S[a_idx];
  const int dold = ws.deg_old[a_idx], dnew = ws.deg_new[a_idx];
  const float ca = dnew > 0 ? c_alpha / (float)dnew : 0.0f;
  const float cb = dold > 0 ? c_alpha / (float)dold : 0.0f;
  const float w = ca - cb;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sub = lane / LPR, q = lane % LPR;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const int st = out.start[u], ln = out.len[u];
  // rows of the group: j = (g * kFixSplit + cta) * 8 RPW + warp RPW + sub, g = 0, 1, ...
  const int stride = kFixSplit * 8 * RPW;
  for (int j0 = cta * 8 * RPW + warp * RPW + sub; j0 < ln; j0 += UNR * stride) {
    float4 z[UNR];
#pragma unroll
    for (int t = 0; t < UNR; ++t) {
      const int j = j0 + t * stride;
      z[t] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (j < ln) {
        const int v = __ldg(out.col + st + j);
        z[t] = __ldg(reinterpret_cast<const float4*>(Zb + (size_t)v * D) + q);
      }
    }
#pragma unroll
    for (int t = 0; t < UNR; ++t) {
      acc.x = fmaf(w, z[t].x, acc.x);
      acc.y = fmaf(w, z[t].y, acc.y);
      acc.z = fmaf(w, z[t].z, acc.z);
      acc.w = fmaf(w, z[t].w, acc.w);
    }
  }
  const int nedit = h->nedit;
  if (cta == 0) {
    for (int e = warp * RPW + sub; e < nedit; e += 8 * RPW) {
      const int4 x = ws.edits[e];
      if (x.x != u) continue;
      const float4 z = reinterpret_cast<const float4*>(Zb + (size_t)x.y * D)[q];
      const float we = x.z > 0 ? cb : -cb;
      acc.x += we * z.x, acc.y += we * z.y, acc.z += we * z.z, acc.w += we * z.w;
    }
  }
  // reduce the RPW sub-rows of the warp, then the 8 warps
#pragma unroll
  for (int o = LPR; o < 32; o <<= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
    acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
  }
  part[warp][lane] = acc;
  __syncthreads();
  float4* mine = reinterpret_cast<float4*>(ws.fixpart + ((size_t)a_idx * kFixSplit + cta) * D);
  if (warp == 0 && lane < LPR) {
    float4 s = part[0][lane];
    for (int wi = 1; wi < 8; ++wi) {
      const float4 t = part[wi][lane];
      s.x += t.x, s.y += t.y, s.z += t.z, s.w += t.w;
    }
    __stcg(mine + lane, s);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ws.fixcnt + a_idx, 1) == kFixSplit - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (warp == 0 && lane < LPR) {
    const float4* all = reinterpret_cast<const float4*>(ws.fixpart + (size_t)a_idx * kFixSplit * D);
    float4 s = __ldcg(all + lane);
    for (int c = 1; c < kFixSplit; ++c) {
      const float4 t = __ldcg(all + (size_t)c * LPR + lane);
      s.x += t.x, s.y += t.y, s.z += t.z, s.w += t.w;
    }
    float4* ru = reinterpret_cast<float4*>(r + (size_t)u * D) + lane;
    float4 cur = *ru;
    cur.x += s.x, cur.y += s.y, cur.z += s.z, cur.w += s.w;
    *ru = cur;
  }
  if (threadIdx.x == 0) {
    ws.fixcnt[a_idx] = 0;   // ready for the next update (the kernel boundary orders it)
    atomicAdd((unsigned long long*)&h->fixup_edges, (unsigned long long)(ln + nedit));
  }
}

cudaError_t launch_fixup(Ctx* c, cudaStream_t s) {
  const float ca = (float)((1.0 - c->cfg.alpha) / c->cfg.alpha);
  const dim3 grid(kMaxR, kFixSplit);
  switch (c->d) {
    case 16: k_fixup<16><<<grid, 256, 0, s>>>(c->hdr, c->out, c->ws, c->Zb, c->r, ca); break;
    case 32: k_fixup<32><<<grid, 256, 0, s>>>(c->hdr, c->out, c->ws, c->Zb, c->r, ca); break;
    case 64: k_fixup<64><<<grid, 256, 0, s>>>(c->hdr, c->out, c->ws, c->Zb, c->r, ca); break;
    default: k_fixup<128><<<grid, 256, 0, s>>>(c->hdr, c->out, c->ws, c->Zb, c->r, ca); break;
  }
  return cudaGetLastError();
}

// ---- adjacency construction from a caller CSR ----
__global__ void k_row_len(const int32_t* row_ptr, int n, int32_t* len, int32_t* cap) {
  int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  int l = row_ptr[u + 1] - row_ptr[u];
  len[u] = l;
  int c = l + max(4, l >> 2);
  cap[u] = (c + 3) & ~3;
}

__global__ void k_copy_rows(const int32_t* row_ptr, const int32_t* col_idx, int n, const int32_t* start,
                            int32_t* col) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  const int b = row_ptr[warp], e = row_ptr[warp + 1], st = start[warp];
  for (int j = b + lane; j < e; j += 32) col[st + (j - b)] = col_idx[j];
}

__global__ void k_in_count(const int32_t* col_idx, long long m, int32_t* cnt) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < m) atomicAdd(&cnt[col_idx[i]], 1);
}

__global__ void k_in_fill(const int32_t* row_ptr, const int32_t* col_idx, int n, const int32_t* start, int32_t* fillpos,
                          int32_t* col) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= n) return;
  for (int j = row_ptr[warp] + lane; j < row_ptr[warp + 1]; j += 32) {
    const int v = col_idx[j];
    const int p = atomicAdd(&fillpos[v], 1);
    col[start[v] + p] = warp;
  }
}

// Node deletion: the first cnt entries of row u as deletion events (u, w, -1), or (w, u, -1)
// for a row of the in-adjacency.
__global__ void k_expand_row(Adj a, int u, int cnt, int incoming, int32_t* src, int32_t* dst, int8_t* op) {
  const int st = a.start[u];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    const int w = a.col[st + i];
    src[i] = incoming ? w : u;
    dst[i] = incoming ? u : w;
    op[i] = -1;
  }
}

cudaError_t launch_expand_row(Ctx* c, int u, int cnt, int incoming, int32_t* src, int32_t* dst, int8_t* op,
                              cudaStream_t s) {
  const Adj a = incoming ? c->in : c->out;
  k_expand_row<<<(cnt + 255) / 256, 256, 0, s>>>(a, u, cnt, incoming, src, dst, op);
  return cudaGetLastError();
}

// Every row of the in-adjacency is sorted by source id, so the in-rows do not depend on the
// order in which k_in_fill's atomics ran: two contexts built from the same graph hold the
// same adjacency, and sums over in-rows round the same way. The rows are the segments
// [start[u], start[u] + len[u]) of col; a segmented sort (CUB's, setup path only) handles
// the hub rows of millions of entries that a per-row insertion sort took minutes on.
__global__ void k_seg_end(const int32_t* __restrict__ start, const int32_t* __restrict__ len, int n, int32_t* end) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < n) end[u] = start[u] + len[u];
}

static cudaError_t sort_rows(Adj* a, int n, long long span, cudaStream_t s) {
  if (n <= 0 || span <= 0) return cudaSuccess;
  int32_t* end = nullptr;
  int32_t* tmp = nullptr;
  void* ts = nullptr;
  size_t tb = 0;
  cudaError_t e = cudaMalloc(&end, sizeof(int32_t) * (size_t)n);
  if (e == cudaSuccess) {
    k_seg_end<<<(n + 255) / 256, 256, 0, s>>>(a->start, a->len, n, end);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cub::DeviceSegmentedSort::SortKeys(nullptr, tb, a->col, tmp, (int)span, n, a->start, end, s);
  if (e == cudaSuccess) e = cudaMalloc(&tmp, sizeof(int32_t) * (size_t)span);
  if (e == cudaSuccess) e = cudaMalloc(&ts, tb > 0 ? tb : 16);
  if (e == cudaSuccess) e = cub::DeviceSegmentedSort::SortKeys(ts, tb, a->col, tmp, (int)span, n, a->start, end, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(a->col, tmp, sizeof(int32_t) * (size_t)span, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(end);
  cudaFree(tmp);
  cudaFree(ts);
  return e;
}

__global__ void k_cap_from_len(const int32_t* len, int n, int32_t* cap) {
  int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  int l = len[u];
  int c = l + max(4, l >> 2);
  cap[u] = (c + 3) & ~3;
}

cudaError_t build_adjacency(Ctx* c, Adj* a, const int32_t* row_ptr, const int32_t* col_idx, int64_t m, int n,
                            long long* tail_host, int transpose, cudaStream_t s) {
  cudaError_t e;
  const int nb = (n + 255) / 256;
  if (!transpose) {
    k_row_len<<<nb, 256, 0, s>>>(row_ptr, n, a->len, a->cap);
  } else {
    cudaMemsetAsync(a->len, 0, sizeof(int32_t) * (size_t)n, s);
    if (m > 0) k_in_count<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(col_idx, m, a->len);
    k_cap_from_len<<<nb, 256, 0, s>>>(a->len, n, a->cap);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // exclusive scan of the capacities on the host (setup path)
  std::vector<int32_t> cap(n), start(n);
  if ((e = cudaMemcpyAsync(cap.data(), a->cap, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  long long acc = 0;
  for (int u = 0; u < n; ++u) {
    start[u] = (int32_t)acc;
    acc += cap[u];
  }
  if (acc > a->m_cap || acc > 0x7fffffffll) return cudaErrorMemoryAllocation;
  *tail_host = acc;
  if ((e = cudaMemcpyAsync(a->start, start.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s)) !=
      cudaSuccess)
    return e;
  const int wb = (int)(((long long)n * 32 + 255) / 256);
  if (!transpose) {
    k_copy_rows<<<wb, 256, 0, s>>>(row_ptr, col_idx, n, a->start, a->col);
  } else {
    int32_t* fillpos = c->ws.queue;  // >= n ints of scratch, unused until the first push
    cudaMemsetAsync(fillpos, 0, sizeof(int32_t) * (size_t)n, s);
    k_in_fill<<<wb, 256, 0, s>>>(row_ptr, col_idx, n, a->start, fillpos, a->col);
    cudaMemsetAsync(fillpos, 0xff, sizeof(int32_t) * (size_t)n, s);   // empty queue slots again
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = sort_rows(a, n, acc, s)) != cudaSuccess) return e;
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

}  // namespace damf
