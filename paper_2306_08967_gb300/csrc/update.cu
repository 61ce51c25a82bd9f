// The factor update for one batch of net changes dA = I_S N I_T^T (Sec. 4.3, Thm 2),
// in U-form: U = Ub PU, V = Vb PV, Sigma kept separately (X = U Sigma^{1/2}).
//
// Choice of factors: B = I_S (orthonormal columns, one per touched source row) and
// C = I_T N^T, so that B C^T = dA and r = |S|.  Then
//   Step 1 (orthogonalisation, Alg. 1):  W_B = U^T B = U[S]^T,  W_C = V^T C = (N V[T])^T,
//          residual Grams  G_B = B^T B - W_B^T W_B = I - U[S] U[S]^T,
//                          G_C = N N^T - (N V[T]) (N V[T])^T        (Prop. 1 for a block),
//          R_B, R_C upper Cholesky factors (pivots below a tolerance are dropped: the
//          residual column is dependent, e.g. rank(N) < |S| when events share endpoints).
//   Step 2 (rediagonalisation):  M = [[Sigma, 0], [0, 0]] + [W_B; R_B] [W_C; R_C]^T,
//          top-d SVD  M = E Theta H^T  (Eq. "svd_small_edge"; jacobi.cu).
//   Step 3 (space projection):   Y_B = R_B^{-1} E[d:],  K_U = E[:d] - W_B Y_B,
//          PU <- PU K_U, PUi <- K_U^{-1} PUi, Ub[S] += Y_B PUi   (Eqs. "f_edge", "x_edge",
//          "update" with the Sigma^{1/2} scalings moved to query time), same for V with
//          Y_C = R_C^{-1} H[d:], K_V = H[:d] - W_C Y_C, Vb[T] += (N^T Y_C) PVi;  Sigma <- Theta.
//   Step 4 input: r[S] += (Ub[S] change) diag(s0), the change of the PPR signal Ub diag(s0).
#include "damf_internal.cuh"

namespace damf {

constexpr float kPivotTol = 1e-5f;   // relative Cholesky pivot tolerance (FP32)

// Register tiles of a D x D output over up to 512 threads: TR rows x TC columns per thread.
template <int D>
struct MMShape {
  static constexpr int TR = D >= 128 ? 4 : D >= 64 ? 2 : 1;   // rows per thread
  static constexpr int TC = D >= 128 ? 8 : D >= 64 ? 4 : D >= 32 ? 2 : 1;   // columns per thread
  static constexpr int NTJ = D / TC;
  static constexpr int NT = (D / TR) * NTJ;   // threads that compute (512, or 256 for D = 16)
};


// ---- a2: gather U[S] = Ub[S] PU and V[T] = Vb[T] PV (16 rows per CTA) ----
template <int D>
__global__ void __launch_bounds__(256) k_gather(DevHeader* h, Workspace ws, const float* __restrict__ Ub,
                                                const float* __restrict__ Vb, const float* __restrict__ PU,
                                                const float* __restrict__ PV) {
  extern __shared__ float smem[];
  float* P = smem;               // D x D
  float* A = smem + D * D;       // 16 x D
  if (h->status != 0) return;
  const int side = blockIdx.y;
  const int nrows = side == 0 ? h->nS : h->nT;
  const int r0 = blockIdx.x * 16;
  if (r0 >= nrows) return;
  const int32_t* idx = side == 0 ? ws.S : ws.T;
  const float* base = side == 0 ? Ub : Vb;
  const float* Pm = side == 0 ? PU : PV;
  float* outp = side == 0 ? ws.UST : ws.VT;
  const int tid = threadIdx.x;
  for (int i = tid; i < D * D / 4; i += 256) reinterpret_cast<float4*>(P)[i] = reinterpret_cast<const float4*>(Pm)[i];
  for (int i = tid; i < 16 * D / 4; i += 256) {
    const int rr = i / (D / 4), q = i % (D / 4);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r0 + rr < nrows && DAMF_DCHECK(h, idx[r0 + rr] >= 0 && idx[r0 + rr] < h->n_nodes))
      v = reinterpret_cast<const float4*>(base + (size_t)idx[r0 + rr] * D)[q];
    reinterpret_cast<float4*>(A)[i] = v;
  }
  __syncthreads();
  for (int o = tid; o < 16 * D; o += 256) {
    const int rr = o / D, j = o % D;
    if (r0 + rr >= nrows) continue;
    float s = 0.f;
#pragma unroll 8
    for (int k = 0; k < D; ++k) s = fmaf(A[rr * D + k], P[k * D + j], s);
    outp[(r0 + rr) * D + j] = s;
  }
}

// ---- a2 (second half): W_C^T = N V[T]  (16 rows per CTA) ----
template <int D>
__global__ void __launch_bounds__(256) k_wct(DevHeader* h, Workspace ws) {
  extern __shared__ float smem[];
  float* Vs = smem;                 // nT x D
  float* Ns = smem + kMaxR * D;     // 16 x nT
  if (h->status != 0) return;
  const int nS = h->nS, nT = h->nT;
  const int r0 = blockIdx.x * 16;
  if (r0 >= nS) return;
  for (int i = threadIdx.x; i < nT * D / 4; i += blockDim.x)
    reinterpret_cast<float4*>(Vs)[i] = reinterpret_cast<const float4*>(ws.VT)[i];
  for (int i = threadIdx.x; i < 16 * nT; i += blockDim.x) {
    const int rr = i / nT, b = i % nT;
    Ns[i] = (r0 + rr < nS) ? ws.N[(r0 + rr) * nT + b] : 0.0f;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < 16 * D; o += blockDim.x) {
    const int rr = o / D, j = o % D;
    if (r0 + rr >= nS) continue;
    float s = 0.f;
    for (int b = 0; b < nT; ++b) s = fmaf(Ns[rr * nT + b], Vs[b * D + j], s);
    ws.WCt[(r0 + rr) * D + j] = s;
  }
}

// ---- a3: residual Grams and semi-definite Cholesky (one CTA per Gram) ----
// Rows a0 .. a0 + 3 of a residual Gram (read by every lane at once) against the columns
// lane + 32 c (consecutive rows of X, other banks), two column blocks per paired FMA. Only
// the upper triangle is read later, so the column pairs q < P0 (blocks 2 q, 2 q + 1, all left
// of a0) are skipped. Each entry is the same sequence of FMAs as one column at a time: the
// N N^T terms (CTA 1) in increasing t, then the X X^T terms in increasing k.
template <int D, int P0>
__device__ __forceinline__ void chol_gram_rows(float* G, const float* X, const float* Ns, bool isC, int nS, int nT,
                                               int a0, int lane) {
  constexpr int LDX = D + 1, LDN = kMaxR + 1, LG = kMaxR + 1;
  static_assert(kMaxR == 128, "four column blocks of 32");
  const int ncol = (nS + 31) / 32;   // column blocks of 32 in use
  float2 acc[4][2];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 2; ++q) acc[r][q] = make_float2(0.f, 0.f);
  if (isC) {
    for (int t = 0; t < nT; ++t) {
      float na[4];
      float2 nb[2];
#pragma unroll
      for (int r = 0; r < 4; ++r) na[r] = Ns[(a0 + r) * LDN + t];
#pragma unroll
      for (int q = P0; q < 2; ++q)
        nb[q] = make_float2(2 * q < ncol ? Ns[(lane + 64 * q) * LDN + t] : 0.0f,
                            2 * q + 1 < ncol ? Ns[(lane + 64 * q + 32) * LDN + t] : 0.0f);
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = P0; q < 2; ++q) acc[r][q] = __ffma2_rn(make_float2(na[r], na[r]), nb[q], acc[r][q]);
    }
  }
#pragma unroll 2
  for (int k = 0; k < D; ++k) {
    float xa[4];
    float2 xb[2];
#pragma unroll
    for (int r = 0; r < 4; ++r) xa[r] = X[(a0 + r) * LDX + k];
#pragma unroll
    for (int q = P0; q < 2; ++q)
      xb[q] = make_float2(2 * q < ncol ? X[(lane + 64 * q) * LDX + k] : 0.0f,
                          2 * q + 1 < ncol ? X[(lane + 64 * q + 32) * LDX + k] : 0.0f);
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = P0; q < 2; ++q) acc[r][q] = __ffma2_rn(make_float2(-xa[r], -xa[r]), xb[q], acc[r][q]);
  }
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = P0; q < 2; ++q)
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int a = a0 + r, b = lane + 64 * q + 32 * hh;
        if (a < nS && b < nS) G[a * LG + b] = (hh ? acc[r][q].y : acc[r][q].x) + ((!isC && a == b) ? 1.0f : 0.0f);
      }
}

template <int D>
__global__ void __launch_bounds__(kChainThreads, 2) k_chol(DevHeader* h, Workspace ws) {   // <= 64 registers
  // CTA 0: G_B = I - U[S] U[S]^T -> R_B; CTA 1: G_C = N N^T - (N V[T])(N V[T])^T -> R_C
  extern __shared__ float smem[];
  constexpr int LDX = D + 1;             // padded strides: a warp reads rows b, b + 1, ... of X
  constexpr int LDN = kMaxR + 1;         // and of N in different banks
  const bool isC = blockIdx.x == 1;
  constexpr int LG = kMaxR + 1;          // padded stride of G: lanes on consecutive rows hit other banks
  float* G = smem;                       // kMaxR x LG
  float* X = G + kMaxR * LG;             // nS x LDX: U[S] or W_C^T
  float* Ns = X + kMaxR * LDX;           // nS x LDN (CTA 1)
  __shared__ float scale;
  __shared__ int kept;
  if (h->status != 0) return;
  const int nS = h->nS, nT = h->nT;
  if (nS == 0) return;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5;
  const float* src = isC ? ws.WCt : ws.UST;
  // rows nS .. kMaxR - 1 are zero (the register tiles below read them)
  for (int i = tid; i < kMaxR * D; i += nt) X[(i / D) * LDX + i % D] = i < nS * D ? src[i] : 0.0f;
  if (isC)   // a warp per two rows of N, four loads per row in flight
    for (int r0 = 2 * warp; r0 < kMaxR; r0 += 2 * (nt / 32)) {
      float v[2][4];
#pragma unroll
      for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int t = lane + 32 * q;
          v[rr][q] = (r0 + rr < nS && t < nT) ? ws.N[(r0 + rr) * nT + t] : 0.0f;
        }
#pragma unroll
      for (int rr = 0; rr < 2; ++rr)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (lane + 32 * q < nT) Ns[(r0 + rr) * LDN + lane + 32 * q] = v[rr][q];
    }
  __syncthreads();
  // the Gram's upper triangle: a warp per four rows
  for (int a0 = 4 * warp; a0 < nS; a0 += 4 * (nt / 32)) {
    if (a0 < 64) chol_gram_rows<D, 0>(G, X, Ns, isC, nS, nT, a0, lane);
    else chol_gram_rows<D, 1>(G, X, Ns, isC, nS, nT, a0, lane);
  }
  __syncthreads();
  if (warp == 0) {   // the pivot scale: the largest diagonal entry (at least 1)
    float mx = 1.0f;
    for (int a = lane; a < nS; a += 32) mx = fmaxf(mx, G[a * LG + a]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) {
      scale = mx * kPivotTol;
      kept = 0;
    }
  }
  __syncthreads();
  // blocked right-looking Cholesky G = R^T R (R upper), panels of 32 rows; a pivot <= tol
  // makes its row of R zero. Per panel [k0, k1): warp 0 factors the diagonal block in
  // registers, the 16 warps solve the panel's trailing columns (forward substitution with
  // R11^T, lane l holding row k0 + l), then everyone updates the trailing block. Every entry
  // sees the same operations in the same order as in the plain column-by-column algorithm.
  constexpr int kTrailBlocks = kMaxR / 32 - 1;   // column blocks of 32 right of a panel
  for (int k0 = 0; k0 < nS; k0 += 32) {
    const int k1 = min(k0 + 32, nS);
    const int nb = k1 - k0;
    if (warp == 0) {
      // lane b holds column k0 + b of the diagonal block, rows k0 .. k0 + b; lanes past the
      // panel hold zero columns, whose pivots (0 <= tol) are dropped and change nothing
      float g[32];
#pragma unroll
      for (int a = 0; a < 32; ++a) g[a] = (a <= lane && lane < nb) ? G[(k0 + a) * LG + k0 + lane] : 0.0f;
      int kp = 0;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float p = __shfl_sync(0xffffffffu, g[j], j);
        const float pv = p > scale ? sqrtf(p) : 0.0f;
        const float ip = pv > 0.f ? 1.0f / pv : 0.0f;
        kp += pv > 0.f;
        g[j] = lane == j ? pv : (lane > j ? g[j] * ip : 0.0f);   // row j of R
#pragma unroll
        for (int a = 0; a < 32; ++a) {                           // G[a][b] -= R[j][a] R[j][b]
          if (a > j) g[a] = fmaf(-__shfl_sync(0xffffffffu, g[j], a), g[j], g[a]);
          // (fixed trip count: g stays in registers; in lanes b < a this writes the lower
          // entry G[a][b], which is set to zero at step a before any use and never stored)
        }
      }
#pragma unroll
      for (int a = 0; a < 32; ++a)
        if (a <= lane && lane < nb) G[(k0 + a) * LG + k0 + lane] = g[a];
      if (lane == 0) kept += kp;
    }
    __syncthreads();
    // trailing columns c >= k1 of the panel's rows, four per warp at once:
    // R[k][c] = (G[k][c] - sum_{i<k} R[i][k] R[i][c]) / R[k][k]
    const int ncol = nS - k1;
    const int row = k0 + lane;
    for (int c0 = 4 * warp; c0 < ncol; c0 += 4 * (nt / 32)) {
      float x[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) x[q] = (row < k1 && c0 + q < ncol) ? G[row * LG + k1 + c0 + q] : 0.0f;
      for (int k = 0; k < nb; ++k) {
        const float rkk = G[(k0 + k) * LG + k0 + k];
        const bool below = lane > k && row < k1;
        const float rk = below ? G[(k0 + k) * LG + row] : 0.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          float y = __shfl_sync(0xffffffffu, x[q], k);
          y = rkk > 0.f ? y / rkk : 0.0f;
          if (lane == k) x[q] = y;
          else if (below) x[q] = fmaf(-rk, y, x[q]);
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (row < k1 && c0 + q < ncol) G[row * LG + k1 + c0 + q] = x[q];
    }
    __syncthreads();
    // trailing update of the upper triangle, G[a][b] -= sum_k R[k][a] R[k][b] (k1 <= a <= b):
    // a warp takes rows a0 .. a0 + 3 against the columns k1 + lane + 32 c
    for (int a0 = k1 + 4 * warp; a0 < nS; a0 += 4 * (nt / 32)) {
      float acc[4][kTrailBlocks];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < kTrailBlocks; ++c) acc[r][c] = 0.f;
      for (int k = k0; k < k1; ++k) {
        float ra[4], rb[kTrailBlocks];
#pragma unroll
        for (int r = 0; r < 4; ++r) ra[r] = a0 + r < nS ? G[k * LG + a0 + r] : 0.0f;
#pragma unroll
        for (int c = 0; c < kTrailBlocks; ++c) {
          const int b = k1 + lane + 32 * c;
          rb[c] = b < nS ? G[k * LG + b] : 0.0f;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < kTrailBlocks; ++c) acc[r][c] = fmaf(ra[r], rb[c], acc[r][c]);
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < kTrailBlocks; ++c) {
          const int a = a0 + r, b = k1 + lane + 32 * c;
          if (a <= b && b < nS) G[a * LG + b] -= acc[r][c];
        }
    }
    __syncthreads();
  }
  float* R = isC ? ws.RC : ws.RB;
  for (int i = tid; i < nS * nS; i += nt) {
    const int a = i / nS, b = i % nS;
    R[a * kMaxR + b] = b >= a ? G[a * LG + b] : 0.0f;
  }
  if (tid == 0) {
    if (isC)
      h->rankC = kept;
    else
      h->rankB = kept;
  }
}

// ---- core assembly: M = diag(sigma, 0) + L R^T, column-major with ld = m ----
template <int D>
__global__ void __launch_bounds__(256) k_assemble(DevHeader* h, Workspace ws, const float* __restrict__ sigma) {
  if (h->status != 0) return;
  const int nS = h->nS;
  if (nS == 0) return;
  const int m = D + nS;
  const int j = blockIdx.x;  // column
  if (j >= m) return;
  __shared__ float Rj[kMaxR];
  for (int a = threadIdx.x; a < nS; a += blockDim.x)
    Rj[a] = j < D ? ws.WCt[a * D + j] : ws.RC[(j - D) * kMaxR + a];
  __syncthreads();
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    float s = (i == j && i < D) ? sigma[i] : 0.0f;
    if (i < D) {
#pragma unroll 8
      for (int a = 0; a < nS; ++a) s = fmaf(ws.UST[a * D + i], Rj[a], s);   // loads of 8 rows in flight
    } else {
      const float* rb = ws.RB + (i - D) * kMaxR;
#pragma unroll 8
      for (int a = 0; a < nS; ++a) s = fmaf(rb[a], Rj[a], s);
    }
    ws.M[(size_t)j * m + i] = s;
  }
}

// ---- H = M^T E Theta^{-1} (top-d right singular vectors) ----
template <int D>
__global__ void __launch_bounds__(128) k_hmat(DevHeader* h, Workspace ws) {
  if (h->status != 0) return;
  const int nS = h->nS;
  if (nS == 0) return;
  const int m = D + nS;
  const int j = blockIdx.x;
  if (j >= m) return;
  __shared__ float Mj[kMaxM];
  for (int i = threadIdx.x; i < m; i += blockDim.x) Mj[i] = ws.M[(size_t)j * m + i];
  __syncthreads();
  for (int k = threadIdx.x; k < D; k += blockDim.x) {
    float s = 0.f;
#pragma unroll 8
    for (int i = 0; i < m; ++i) s = fmaf(Mj[i], ws.E[i * D + k], s);   // eight rows' loads in flight
    const float t = ws.theta[k];
    ws.H[j * D + k] = t > 0.f ? s / t : 0.0f;
  }
}

// ---- one Newton-Schulz step on E and H: X <- X (3 I - X^T X) / 2 ----
// E's columns are orthonormal to the Jacobi tolerance; H = M^T E Theta^{-1} inherits that
// error amplified by the spread of the singular values.  One step of the iteration for the
// orthonormal polar factor squares the orthonormality error of both, so the updated bases
// stay orthonormal to FP32 level between folds.
// (a) G = X^T X over the m rows: 32 x 32 output tiles, blockIdx.z selects E or H
template <int D>
__global__ void __launch_bounds__(256) k_ns_gram(DevHeader* h, Workspace ws) {
  __shared__ float xa[32][33], xb[32][33];
  if (h->status != 0 || h->nS == 0) return;
  const int m = D + h->nS;
  const float* X = blockIdx.z == 0 ? ws.E : ws.H;
  float* G = ws.tmp + (size_t)blockIdx.z * D * D;
  const int ta = blockIdx.x * 32, tb = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int r0 = 0; r0 < m; r0 += 32) {
    __syncthreads();
    for (int i = ty; i < 32; i += 8) {
      const int row = r0 + i;
      xa[i][tx] = (row < m && ta + tx < D) ? X[row * D + ta + tx] : 0.0f;
      xb[i][tx] = (row < m && tb + tx < D) ? X[row * D + tb + tx] : 0.0f;
    }
    __syncthreads();
    for (int i = 0; i < 32; ++i) {
      const float b = xb[i][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(xa[i][ty + 8 * q], b, acc[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int a = ta + ty + 8 * q, b = tb + tx;
    if (a < D && b < D) G[a * D + b] = acc[q];
  }
}

// (b) X <- X (1.5 I - 0.5 G), 16 rows per CTA, blockIdx.y selects E or H (rows are owned by
// one CTA, so the update is in place)
template <int D>
__global__ void __launch_bounds__(256) k_ns_apply(DevHeader* h, Workspace ws) {
  extern __shared__ float smem[];
  float* Gs = smem;            // D x D: 1.5 I - 0.5 G
  float* Xs = smem + D * D;    // 16 x D
  if (h->status != 0 || h->nS == 0) return;
  const int m = D + h->nS;
  const int r0 = blockIdx.x * 16;
  if (r0 >= m) return;
  float* X = blockIdx.y == 0 ? ws.E : ws.H;
  const float* G = ws.tmp + (size_t)blockIdx.y * D * D;
  for (int i = threadIdx.x; i < D * D; i += blockDim.x) {
    const int a = i / D, b = i % D;
    Gs[i] = (a == b ? 1.5f : 0.0f) - 0.5f * G[i];
  }
  for (int i = threadIdx.x; i < 16 * D; i += blockDim.x) {
    const int rr = i / D;
    Xs[i] = (r0 + rr < m) ? X[(r0 + rr) * D + i % D] : 0.0f;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < 16 * D; o += blockDim.x) {
    const int rr = o / D, j = o % D;
    if (r0 + rr >= m) continue;
    float s = 0.f;
#pragma unroll 8
    for (int k = 0; k < D; ++k) s = fmaf(Xs[rr * D + k], Gs[k * D + j], s);
    X[(r0 + rr) * D + j] = s;
  }
}

// ---- Step 2 refinement: consistent singular pairs, exact norms, Theta from the core itself ----
// One-sided Jacobi leaves the columns orthogonal only to its tolerance; E (normalised columns)
// and H = M^T E Theta^{-1}, each made orthonormal by Newton-Schulz, then pair up with a first-
// order error of that size (~1e-6 relative in E Theta H^T per update at d = 128), and in FP32
// the normalised columns keep a norm bias of a few 1e-8 that the bases inherit update after
// update; the largest singular value drifted up by ~3e-7 per update. So after Newton-Schulz:
//   (1) T = E^T M H (d x d, nearly diagonal), with M = diag(sigma, 0) + L R^T,
//       L = [W_B; R_B], R = [W_C; R_C]:  T = E[:d]^T diag(sigma) H[:d] + P Q^T,
//       P = E^T L, Q = H^T R (d x r);
//   (2) the first-order SVD of T = (I + A) Theta' (I + B)^T with A, B skew:
//       A_jk = (t_k F_jk + t_j F_kj) / (t_k^2 - t_j^2), B_jk = (t_j F_jk + t_k F_kj) / (t_k^2 - t_j^2)
//       for the off-diagonal part F of T and t = diag(T) (pairs too close to separate, or whose
//       correction would not be small, are left as they are); E <- E (I + A), H <- H (I + B);
//   (3) every column of E and H scaled to unit norm, the norm summed in FP64 and each element
//       scaled in FP64 and rounded once;
//   (4) theta_k = e_k^T M h_k, the Rayleigh quotient with the original core, summed in FP64
//       (the products of FP32 operands are exact in FP64; FP32 sums of these dot products were
//       measured biased by ~4e-7 relative, which the update would accumulate).
// (1)-(2) are FP32; (3)-(4) take (d + r) d FP64 products per update.

// (a) P[k][a] = (L^T e_k)_a and Q[k][a] = (R^T h_k)_a: one CTA per k, one thread per column a.
template <int D, typename Acc>
__device__ __forceinline__ void fo_pq_col(const Workspace& ws, int nS, const float* ev, const float* hv, int a,
                                          Acc& p, Acc& q) {
  p = 0;
  q = 0;
  const float4* ur = reinterpret_cast<const float4*>(ws.UST + (size_t)a * D);
  const float4* wr = reinterpret_cast<const float4*>(ws.WCt + (size_t)a * D);
#pragma unroll 4
  for (int i4 = 0; i4 < D / 4; ++i4) {
    const float4 u = ur[i4], w = wr[i4];
    const int i = 4 * i4;
    p = fma((Acc)ev[i], (Acc)u.x, p);
    p = fma((Acc)ev[i + 1], (Acc)u.y, p);
    p = fma((Acc)ev[i + 2], (Acc)u.z, p);
    p = fma((Acc)ev[i + 3], (Acc)u.w, p);
    q = fma((Acc)hv[i], (Acc)w.x, q);
    q = fma((Acc)hv[i + 1], (Acc)w.y, q);
    q = fma((Acc)hv[i + 2], (Acc)w.z, q);
    q = fma((Acc)hv[i + 3], (Acc)w.w, q);
  }
  // R_B and R_C are upper triangular: column a has rows 0 .. a (eight rows' loads in flight
  // before their products, the sums in row order)
  for (int b0 = 0; b0 <= a; b0 += 8) {
    float rb[8], rc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      rb[j] = b0 + j <= a ? ws.RB[(b0 + j) * kMaxR + a] : 0.0f;
      rc[j] = b0 + j <= a ? ws.RC[(b0 + j) * kMaxR + a] : 0.0f;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (b0 + j <= a) {
        p = fma((Acc)ev[D + b0 + j], (Acc)rb[j], p);
        q = fma((Acc)hv[D + b0 + j], (Acc)rc[j], q);
      }
    }
  }
}

template <int D>
__global__ void __launch_bounds__(128) k_fo_pq(DevHeader* h, Workspace ws) {
  __shared__ float ev[kMaxM], hv[kMaxM];
  if (h->status != 0 || h->nS == 0) return;
  const int nS = h->nS, m = D + nS;
  const int k = blockIdx.x, tid = threadIdx.x;
  for (int i = tid; i < m; i += blockDim.x) {
    ev[i] = ws.E[i * D + k];
    hv[i] = ws.H[i * D + k];
  }
  __syncthreads();
  if (tid < nS) {
    float p, q;
    fo_pq_col<D, float>(ws, nS, ev, hv, tid, p, q);
    ws.foP[(size_t)k * kMaxR + tid] = p;
    ws.foQ[(size_t)k * kMaxR + tid] = q;
  }
}

// (b) T = E[:d]^T diag(sigma) H[:d] + P Q^T in TS x TS output tiles (256 threads).
template <int D>
__global__ void __launch_bounds__(256) k_fo_t(DevHeader* h, Workspace ws, const float* __restrict__ sigma) {
  constexpr int TS = D < 32 ? D : 32;
  extern __shared__ __align__(16) float fo_smem[];
  float* Ps = fo_smem;               // TS x (kMaxR + 1)
  float* Qs = Ps + TS * (kMaxR + 1);  // TS x (kMaxR + 1)
  float* Es = Qs + TS * (kMaxR + 1);  // D x TS
  float* Hs = Es + D * TS;            // D x TS
  if (h->status != 0 || h->nS == 0) return;
  const int nS = h->nS;
  const int j0 = blockIdx.x * TS, k0 = blockIdx.y * TS, tid = threadIdx.x;
  for (int o = tid; o < TS * nS; o += blockDim.x) {
    const int t = o / nS, a = o % nS;
    Ps[t * (kMaxR + 1) + a] = ws.foP[(size_t)(j0 + t) * kMaxR + a];
    Qs[t * (kMaxR + 1) + a] = ws.foQ[(size_t)(k0 + t) * kMaxR + a];
  }
  for (int o = tid; o < D * TS; o += blockDim.x) {
    const int i = o / TS, t = o % TS;
    Es[o] = ws.E[i * D + j0 + t];
    Hs[o] = ws.H[i * D + k0 + t];
  }
  __syncthreads();
  for (int o = tid; o < TS * TS; o += blockDim.x) {
    const int tj = o / TS, tk = o % TS;
    float s = 0.f;
    for (int i = 0; i < D; ++i) s = fmaf(sigma[i] * Es[i * TS + tj], Hs[i * TS + tk], s);
    float s2 = 0.f;
    for (int a = 0; a < nS; ++a) s2 = fmaf(Ps[tj * (kMaxR + 1) + a], Qs[tk * (kMaxR + 1) + a], s2);
    ws.foT[(size_t)(j0 + tj) * D + k0 + tk] = s + s2;
  }
}

// (c) X <- X (I + A) for E (blockIdx.y = 0) and X <- X (I + B) for H (blockIdx.y = 1), 16 rows per
// CTA (rows are owned by one CTA, so the update is in place); the small terms are summed first.
template <int D>
__global__ void __launch_bounds__(256) k_fo_apply(DevHeader* h, Workspace ws) {
  extern __shared__ float smem[];
  float* Gs = smem;            // D x D: A or B
  float* Xs = smem + D * D;    // 16 x D
  float* Ts = Xs + 16 * D;     // D x (D + 1): T, read once with coalesced loads
  if (h->status != 0 || h->nS == 0) return;
  const int m = D + h->nS;
  const int r0 = blockIdx.x * 16;
  if (r0 >= m) return;
  const int side = blockIdx.y;
  float* X = side == 0 ? ws.E : ws.H;
  const float* T = ws.foT;
  for (int o = threadIdx.x; o < D * D; o += blockDim.x) Ts[(o / D) * (D + 1) + o % D] = T[o];
  __syncthreads();
  for (int o = threadIdx.x; o < D * D; o += blockDim.x) {
    const int j = o / D, k = o % D;
    float g = 0.0f;
    if (j != k) {
      const float tj = Ts[j * (D + 1) + j], tk = Ts[k * (D + 1) + k];
      const float fjk = Ts[j * (D + 1) + k], fkj = Ts[k * (D + 1) + j];
      const float den = tk * tk - tj * tj;
      if (fabsf(den) >= 1e-4f * (tj * tj + tk * tk) && den != 0.0f) {
        const float id = 1.0f / den;
        const float a = (tk * fjk + tj * fkj) * id;
        const float b = (tj * fjk + tk * fkj) * id;
        if (fabsf(a) <= 1e-2f && fabsf(b) <= 1e-2f) g = side == 0 ? a : b;
      }
    }
    Gs[o] = g;
  }
  for (int i = threadIdx.x; i < 16 * D; i += blockDim.x) {
    const int rr = i / D;
    Xs[i] = (r0 + rr < m) ? X[(r0 + rr) * D + i % D] : 0.0f;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < 16 * D; o += blockDim.x) {
    const int rr = o / D, k = o % D;
    if (r0 + rr >= m) continue;
    float s = 0.f;
#pragma unroll 8
    for (int j = 0; j < D; ++j) s = fmaf(Xs[rr * D + j], Gs[j * D + k], s);
    X[(r0 + rr) * D + k] = Xs[rr * D + k] + s;
  }
}

template <typename Acc>
__device__ __forceinline__ Acc block_sum128(Acc v, Acc* part) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();   // part may still be read from an earlier sum
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  return part[0] + part[1] + part[2] + part[3];
}

// Double-float accumulation (an unevaluated pair hi + lo of floats): sums of exact products
// (TwoProduct by an FMA, TwoSum by Knuth's branch-free form) carry about 48 bits, as FP64
// sums of FP32 products do, at FP32 instruction rates (FP64 runs at ~1/64 of FP32 here).
// The __f*_rn intrinsics keep the compiler from fusing the roundings the error terms rely on.
struct DFloat {
  float hi, lo;
};

__device__ __forceinline__ DFloat df_add_prod(DFloat acc, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float pe = fmaf(a, b, -p);              // a b = p + pe exactly
  const float s = __fadd_rn(acc.hi, p);
  const float bb = __fsub_rn(s, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));   // acc.hi + p = s + err
  return {s, __fadd_rn(acc.lo, __fadd_rn(err, pe))};
}

__device__ __forceinline__ DFloat df_add(DFloat a, DFloat b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float bb = __fsub_rn(s, a.hi);
  const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
  return {s, __fadd_rn(__fadd_rn(a.lo, b.lo), err)};
}

// (d) unit columns (norms summed in FP64, each element scaled in FP64 and rounded once) and
// theta_k = e_k^T M h_k with double-float sums. One CTA of 128 threads per k.
template <int D>
__global__ void __launch_bounds__(128) k_fo_norm_theta(DevHeader* h, Workspace ws, const float* __restrict__ sigma) {
  __shared__ float ev[kMaxM], hv[kMaxM];
  __shared__ double part[4];
  __shared__ DFloat dpart[4];
  if (h->status != 0 || h->nS == 0) return;
  const int nS = h->nS, m = D + nS;
  const int k = blockIdx.x, tid = threadIdx.x;
  double se = 0, sh = 0;
  for (int i = tid; i < m; i += blockDim.x) {
    const float e = ws.E[i * D + k], f = ws.H[i * D + k];
    ev[i] = e;
    hv[i] = f;
    se = fma((double)e, (double)e, se);
    sh = fma((double)f, (double)f, sh);
  }
  se = block_sum128<double>(se, part);
  sh = block_sum128<double>(sh, part);
  const double ie = se > 0 ? 1.0 / sqrt(se) : 0.0;
  const double ih = sh > 0 ? 1.0 / sqrt(sh) : 0.0;
  for (int i = tid; i < m; i += blockDim.x) {
    const float e = (float)((double)ev[i] * ie), f = (float)((double)hv[i] * ih);
    ev[i] = e;
    hv[i] = f;
    ws.E[i * D + k] = e;
    ws.H[i * D + k] = f;
  }
  __syncthreads();
  DFloat acc = {0.f, 0.f};
  for (int i = tid; i < D; i += blockDim.x) {
    // sigma_i e_i h_i: (sigma_i e_i) split exactly, then times h_i
    const float t = __fmul_rn(sigma[i], ev[i]);
    const float te = fmaf(sigma[i], ev[i], -t);
    acc = df_add_prod(acc, t, hv[i]);
    acc.lo = __fadd_rn(acc.lo, __fmul_rn(te, hv[i]));
  }
  if (tid < nS) {
    const int a = tid;
    DFloat p = {0.f, 0.f}, q = {0.f, 0.f};
    const float4* ur = reinterpret_cast<const float4*>(ws.UST + (size_t)a * D);
    const float4* wr = reinterpret_cast<const float4*>(ws.WCt + (size_t)a * D);
    for (int i4 = 0; i4 < D / 4; ++i4) {
      const float4 u = ur[i4], w = wr[i4];
      const int i = 4 * i4;
      p = df_add_prod(p, ev[i], u.x);
      p = df_add_prod(p, ev[i + 1], u.y);
      p = df_add_prod(p, ev[i + 2], u.z);
      p = df_add_prod(p, ev[i + 3], u.w);
      q = df_add_prod(q, hv[i], w.x);
      q = df_add_prod(q, hv[i + 1], w.y);
      q = df_add_prod(q, hv[i + 2], w.z);
      q = df_add_prod(q, hv[i + 3], w.w);
    }
    // R_B and R_C are upper triangular: column a has rows 0 .. a; eight rows' loads are issued
    // before their sums, so the loop does not wait on one L2 round trip per row
    for (int b0 = 0; b0 <= a; b0 += 8) {
      float rb[8], rc[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int b = b0 + j;
        rb[j] = b <= a ? ws.RB[b * kMaxR + a] : 0.0f;
        rc[j] = b <= a ? ws.RC[b * kMaxR + a] : 0.0f;
      }
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (b0 + j <= a) {
          p = df_add_prod(p, ev[D + b0 + j], rb[j]);
          q = df_add_prod(q, hv[D + b0 + j], rc[j]);
        }
      }
    }
    // p q = p.hi q.hi + p.hi q.lo + p.lo q.hi (+ p.lo q.lo, below the precision kept)
    acc = df_add_prod(acc, p.hi, q.hi);
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(__fmul_rn(p.hi, q.lo), __fmul_rn(p.lo, q.hi)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    DFloat other;
    other.hi = __shfl_xor_sync(0xffffffffu, acc.hi, o);
    other.lo = __shfl_xor_sync(0xffffffffu, acc.lo, o);
    acc = df_add(acc, other);
  }
  if ((tid & 31) == 0) dpart[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    DFloat t = dpart[0];
    for (int w = 1; w < 4; ++w) t = df_add(t, dpart[w]);
    ws.theta[k] = __fadd_rn(t.hi, t.lo);
  }
}

// ---- Step 3 part 1: Y = R^{-1} E[d:] and K = E[:d] - W Y (block 0: U side, block 1: V side) ----
// Blocked back substitution over row blocks of 32, bottom block first: a warp solves the
// block's 32 x 32 triangle for its D/16 columns in registers (lane l holds row l, the solved
// value of row j is broadcast by a shuffle), then the rows above take the block's
// contribution as one product; two barriers per block instead of one per row.
template <int D>
__global__ void __launch_bounds__(kChainThreads) k_trans(DevHeader* h, Workspace ws) {
  constexpr int LDR = kMaxR + 1;      // padded row stride: a lane per row reads one column
  constexpr int CPW = D / 16;         // columns per warp (16 warps)
  extern __shared__ float smem[];
  float* R = smem;                    // kMaxR x LDR
  float* Y = R + kMaxR * LDR;         // nS x D
  float* Wts = Y + kMaxR * D;         // nS x D
  if (h->status != 0) return;
  const int nS = h->nS;
  if (nS == 0) return;
  const int side = blockIdx.x;
  const float* Rg = side == 0 ? ws.RB : ws.RC;
  const float* Eg = side == 0 ? ws.E : ws.H;     // (D + nS) x D row-major
  const float* Wt = side == 0 ? ws.UST : ws.WCt;  // nS x D  (W^T)
  float* Yg = side == 0 ? ws.YB : ws.YC;
  float* K = side == 0 ? ws.KU : ws.KV;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
  for (int i = tid; i < nS * nS; i += nt) {
    const int a = i / nS, b = i % nS;
    R[a * LDR + b] = Rg[a * kMaxR + b];
  }
  for (int i = tid; i < nS * D; i += nt) {
    Y[i] = Eg[D * D + i];
    Wts[i] = Wt[i];
  }
  __syncthreads();
  const int nblk = (nS + 31) / 32;
  for (int blk = nblk - 1; blk >= 0; --blk) {
    const int r0 = blk * 32;
    const int row = r0 + lane;
    const bool live = row < nS;
    if (warp < 16) {
      float x[CPW];
#pragma unroll
      for (int c = 0; c < CPW; ++c) x[c] = live ? Y[row * D + warp * CPW + c] : 0.0f;
      for (int j = min(31, nS - 1 - r0); j >= 0; --j) {
        const float p = R[(r0 + j) * LDR + r0 + j];
        const float ip = p > 0.f ? 1.0f / p : 0.0f;
        const float rl = (lane < j) ? R[row * LDR + r0 + j] : 0.0f;
#pragma unroll
        for (int c = 0; c < CPW; ++c) {
          float yj = __shfl_sync(0xffffffffu, x[c], j);
          yj *= ip;
          if (lane == j) x[c] = yj;
          else if (lane < j) x[c] = fmaf(-rl, yj, x[c]);
        }
      }
      if (live)
#pragma unroll
        for (int c = 0; c < CPW; ++c) Y[row * D + warp * CPW + c] = x[c];
    }
    __syncthreads();
    // rows above the block: Y[i] -= R[i, block] Y[block]
    const int nb = min(32, nS - r0);
    if constexpr (D == 128) {
      // warp w takes the rows w, w + 16, ... (at most six: r0 <= kMaxR - 32), lane l the
      // columns 4 l .. 4 l + 3: one 16-byte read of a block row serves all the rows
      static_assert(kMaxR - 32 <= 6 * 16, "six rows per warp");
      float4 acc[6];
#pragma unroll
      for (int q = 0; q < 6; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int j = 0; j < nb; ++j) {
        const float4 y = *reinterpret_cast<const float4*>(Y + (r0 + j) * D + 4 * lane);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
          const int i = warp + 16 * q;
          if (i < r0) {
            const float rij = R[i * LDR + r0 + j];
            acc[q].x = fmaf(rij, y.x, acc[q].x);
            acc[q].y = fmaf(rij, y.y, acc[q].y);
            acc[q].z = fmaf(rij, y.z, acc[q].z);
            acc[q].w = fmaf(rij, y.w, acc[q].w);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const int i = warp + 16 * q;
        if (i < r0) {
          float4* yi = reinterpret_cast<float4*>(Y + i * D + 4 * lane);
          float4 v = *yi;
          v.x -= acc[q].x;
          v.y -= acc[q].y;
          v.z -= acc[q].z;
          v.w -= acc[q].w;
          *yi = v;
        }
      }
    } else {
      for (int o = tid; o < r0 * D; o += nt) {
        const int i = o / D, col = o % D;
        float s = 0.f;
        for (int j = 0; j < nb; ++j) s = fmaf(R[i * LDR + r0 + j], Y[(r0 + j) * D + col], s);
        Y[o] -= s;
      }
    }
    __syncthreads();
  }
  for (int i = tid; i < nS * D; i += nt) Yg[i] = Y[i];
  // K = E[:d] - W Y with W = Wts^T: register tiles (TR x TC outputs per thread)
  using S = MMShape<D>;
  if constexpr (D == 128) {
    // rows 4 ti .. 4 ti + 3 and columns 4 tj .. + 3, 64 + 4 tj .. + 3 (as in smem_mm): one
    // 16-byte read of W^T and two of Y per a, paired FMAs; the same FMAs in increasing a
    const int i0 = (tid >> 4) * 4, j0 = (tid & 15) * 4;
    float2 acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int a = 0; a < nS; ++a) {
      const float4 w = *reinterpret_cast<const float4*>(Wts + a * D + i0);
      const float4 bl = *reinterpret_cast<const float4*>(Y + a * D + j0);
      const float4 bh = *reinterpret_cast<const float4*>(Y + a * D + 64 + j0);
      const float wr[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const float2 a2 = make_float2(wr[r], wr[r]);
        acc[r][0] = __ffma2_rn(a2, make_float2(bl.x, bl.y), acc[r][0]);
        acc[r][1] = __ffma2_rn(a2, make_float2(bl.z, bl.w), acc[r][1]);
        acc[r][2] = __ffma2_rn(a2, make_float2(bh.x, bh.y), acc[r][2]);
        acc[r][3] = __ffma2_rn(a2, make_float2(bh.z, bh.w), acc[r][3]);
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = i0 + r;
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int j = hh * 64 + j0;
        const float4 e = *reinterpret_cast<const float4*>(Eg + i * D + j);
        *reinterpret_cast<float4*>(K + i * D + j) =
            make_float4(e.x - acc[r][2 * hh].x, e.y - acc[r][2 * hh].y, e.z - acc[r][2 * hh + 1].x,
                        e.w - acc[r][2 * hh + 1].y);
      }
    }
  } else if (tid < S::NT) {
    const int i0 = (tid / S::NTJ) * S::TR, j0 = (tid % S::NTJ) * S::TC;
    float acc[S::TR][S::TC];
#pragma unroll
    for (int r = 0; r < S::TR; ++r)
#pragma unroll
      for (int c = 0; c < S::TC; ++c) acc[r][c] = 0.f;
    for (int a = 0; a < nS; ++a) {
      float av[S::TR], bv[S::TC];
#pragma unroll
      for (int r = 0; r < S::TR; ++r) av[r] = Wts[a * D + i0 + r];
#pragma unroll
      for (int c = 0; c < S::TC; ++c) bv[c] = Y[a * D + j0 + c];
#pragma unroll
      for (int r = 0; r < S::TR; ++r)
#pragma unroll
        for (int c = 0; c < S::TC; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
#pragma unroll
    for (int r = 0; r < S::TR; ++r)
#pragma unroll
      for (int c = 0; c < S::TC; ++c) {
        const int i = i0 + r, j = j0 + c;
        K[i * D + j] = Eg[i * D + j] - acc[r][c];
      }
  }
}

// ---- K^{-1}: Newton-Schulz when K is close to a scaled orthogonal matrix, else Gauss-Jordan ----
// Gauss-Jordan with partial pivoting: [K | I] in shared memory with a padded row stride
// (2D + 1: column reads are free of bank conflicts); each warp owns rows, each lane columns;
// the pivot row's live window [p, 2D) is read once per step into registers.
template <int D>
__device__ __forceinline__ void gj_inverse(DevHeader* h, const float* K, float* Ki, float* smem) {
  constexpr int LD = 2 * D + 1;
  constexpr int CPL = (2 * D + 31) / 32;   // columns per lane
  float* Aug = smem;   // D x LD
  __shared__ int piv_row;
  __shared__ float piv_val;
  __shared__ float colv[D];
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  for (int o = tid; o < D * 2 * D; o += nt) {
    const int i = o / (2 * D), j = o % (2 * D);
    Aug[i * LD + j] = j < D ? K[i * D + j] : (j - D == i ? 1.0f : 0.0f);
  }
  __syncthreads();
  for (int p = 0; p < D; ++p) {
    if (warp == 0) {  // pivot search in column p, rows p..D-1
      float best = -1.f;
      int br = p;
      for (int i = p + lane; i < D; i += 32) {
        const float a = fabsf(Aug[i * LD + p]);
        if (a > best) best = a, br = i;
      }
      for (int o = 16; o > 0; o >>= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int orr = __shfl_xor_sync(0xffffffffu, br, o);
        if (ob > best || (ob == best && orr < br)) best = ob, br = orr;
      }
      if (lane == 0) {
        piv_row = br;
        piv_val = Aug[br * LD + p];
      }
    }
    __syncthreads();
    if (!(fabsf(piv_val) > 1e-30f)) {
      if (tid == 0) set_status(h, DAMF_ERR_NUMERIC);
      return;
    }
    const int pr = piv_row;
    const float inv = 1.0f / piv_val;
    for (int j = p + tid; j < 2 * D; j += nt) {  // swap rows p, pr and scale the pivot row
      const float a = Aug[p * LD + j], b = Aug[pr * LD + j];
      Aug[pr * LD + j] = a;
      Aug[p * LD + j] = b * inv;
    }
    __syncthreads();
    for (int i = tid; i < D; i += nt) colv[i] = Aug[i * LD + p];
    float pv[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int j = p + lane + 32 * c;
      pv[c] = j < 2 * D ? Aug[p * LD + j] : 0.0f;
    }
    __syncthreads();
    for (int i = warp; i < D; i += nw) {
      if (i == p) continue;
      const float f = colv[i];
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int j = p + lane + 32 * c;
        if (j < 2 * D) Aug[i * LD + j] = fmaf(-f, pv[c], Aug[i * LD + j]);
      }
    }
    __syncthreads();
  }
  for (int o = tid; o < D * D; o += nt) {
    const int i = o / D, j = o % D;
    Ki[o] = Aug[i * LD + D + j];
  }
}

// Register-tiled product of D x D matrices in shared memory (row stride D) by up to 512 threads:
// MODE 0: C = A B;  MODE 1: C = I - A B;  MODE 2: C = A + A B (A and C must differ).
// (not inlined: the product gets the kernel's whole register budget, nothing spills in its loop)
template <int D, int MODE>
__device__ __noinline__ void smem_mm(const float* A, const float* B, float* C) {
  if constexpr (D == 128) {
    // 512 threads, 4 rows x 8 columns each: rows 4 ti .. 4 ti + 3, columns 4 tj .. 4 tj + 3 and
    // 64 + 4 tj .. 64 + 4 tj + 3 (a half-warp reads 256 contiguous bytes of a row of B, the
    // other half-warp the same: no bank conflicts); two k at a time from one 8-byte read of
    // each row of A, and column pairs through paired FMAs. Every output is the same
    // sequence of FMAs in increasing k as in the generic path below.
    const int tid = threadIdx.x;
    if (tid >= 512) return;
    const int i0 = (tid >> 4) * 4, j0 = (tid & 15) * 4;
    float2 acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);
#pragma unroll 2
    for (int k = 0; k < D; k += 2) {
      float2 a2r[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a2r[r] = *reinterpret_cast<const float2*>(A + (i0 + r) * D + k);
#pragma unroll
      for (int kk = 0; kk < 2; ++kk) {
        const float4 bl = *reinterpret_cast<const float4*>(B + (k + kk) * D + j0);
        const float4 bh = *reinterpret_cast<const float4*>(B + (k + kk) * D + 64 + j0);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float av = kk == 0 ? a2r[r].x : a2r[r].y;
          const float2 a2 = make_float2(av, av);
          acc[r][0] = __ffma2_rn(a2, make_float2(bl.x, bl.y), acc[r][0]);
          acc[r][1] = __ffma2_rn(a2, make_float2(bl.z, bl.w), acc[r][1]);
          acc[r][2] = __ffma2_rn(a2, make_float2(bh.x, bh.y), acc[r][2]);
          acc[r][3] = __ffma2_rn(a2, make_float2(bh.z, bh.w), acc[r][3]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int i = i0 + r;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = h * 64 + j0;
        float4 v = make_float4(acc[r][2 * h].x, acc[r][2 * h].y, acc[r][2 * h + 1].x, acc[r][2 * h + 1].y);
        if (MODE == 1) {
          v.x = (i == j ? 1.0f : 0.0f) - v.x;
          v.y = (i == j + 1 ? 1.0f : 0.0f) - v.y;
          v.z = (i == j + 2 ? 1.0f : 0.0f) - v.z;
          v.w = (i == j + 3 ? 1.0f : 0.0f) - v.w;
        }
        if (MODE == 2) {
          const float4 a = *reinterpret_cast<const float4*>(A + i * D + j);
          v.x += a.x;
          v.y += a.y;
          v.z += a.z;
          v.w += a.w;
        }
        *reinterpret_cast<float4*>(C + i * D + j) = v;
      }
    }
    return;
  }
  using S = MMShape<D>;
  const int tid = threadIdx.x;
  if (tid >= S::NT) return;
  const int i0 = (tid / S::NTJ) * S::TR, j0 = (tid % S::NTJ) * S::TC;
  float acc[S::TR][S::TC];
#pragma unroll
  for (int r = 0; r < S::TR; ++r)
#pragma unroll
    for (int c = 0; c < S::TC; ++c) acc[r][c] = 0.f;
#pragma unroll 4
  for (int k = 0; k < D; ++k) {
    float a[S::TR], b[S::TC];
#pragma unroll
    for (int r = 0; r < S::TR; ++r) a[r] = A[(i0 + r) * D + k];
#pragma unroll
    for (int c = 0; c < S::TC; ++c) b[c] = B[k * D + j0 + c];
#pragma unroll
    for (int r = 0; r < S::TR; ++r)
#pragma unroll
      for (int c = 0; c < S::TC; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
  }
#pragma unroll
  for (int r = 0; r < S::TR; ++r)
#pragma unroll
    for (int c = 0; c < S::TC; ++c) {
      const int i = i0 + r, j = j0 + c;
      float v = acc[r][c];
      if (MODE == 1) v = (i == j ? 1.0f : 0.0f) - v;
      if (MODE == 2) v += A[i * D + j];
      C[i * D + j] = v;
    }
}

// max over the block (kChainThreads threads) of v
__device__ __forceinline__ float block_max512(float v, float* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float m = 0.f;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmaxf(m, red[w]);
  return m;
}

// One CTA per side (block 0: K_U, block 1: K_V). K relates the old and the new bases and is
// close to orthogonal after a small change, so X0 = K^T (scaled by d / |K|_F^2) starts the
// Newton-Schulz iteration X <- X + X (I - K X), whose residual squares each step; when the
// start is too far (|I - K X0|_F >= 0.9) or the residual stops shrinking, Gauss-Jordan with
// partial pivoting takes over. Three d x d buffers; K is re-read from global memory (L2) in
// each step, its buffer having received the new X.
constexpr int kNSInvSteps = 12;
constexpr float kNSInvTol = 2e-6f;   // max |I - K X| accepted (FP32 level for d <= 128)

template <int D>
__global__ void __launch_bounds__(kChainThreads, 2) k_inverse(DevHeader* h, Workspace ws) {   // <= 64 registers
  extern __shared__ float smem[];
  __shared__ float red[kChainThreads / 32];
  if (h->status != 0 || h->nS == 0) return;
  const float* K = blockIdx.x == 0 ? ws.KU : ws.KV;
  float* Ki = blockIdx.x == 0 ? ws.KUi : ws.KVi;
  const int tid = threadIdx.x, nt = blockDim.x;
  float* b0 = smem;
  float* b1 = smem + D * D;
  float* W = smem + 2 * D * D;
  float ss = 0.f;
  for (int o = tid; o < D * D; o += nt) {
    const float v = K[o];
    b0[o] = v;
    ss = fmaf(v, v, ss);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = ss;
  __syncthreads();
  float fro = 0.f;
  for (int w = 0; w < nt / 32; ++w) fro += red[w];
  const float scale = fro > 0.f ? (float)D / fro : 0.0f;
  __syncthreads();
  for (int o = tid; o < D * D; o += nt) {
    const int i = o / D, j = o % D;
    b1[o] = b0[j * D + i] * scale;   // X0 = scaled K^T
  }
  __syncthreads();
  float* Kb = b0;
  float* Xb = b1;
  bool ok = false;
  float prev = 3.0e38f;
  for (int it = 0; it < kNSInvSteps && fro > 0.f; ++it) {
    smem_mm<D, 1>(Kb, Xb, W);   // W = I - K X
    __syncthreads();
    float mx = 0.f, f2 = 0.f;
    for (int o = tid; o < D * D; o += nt) {
      const float w = W[o];
      mx = fmaxf(mx, fabsf(w));
      f2 = fmaf(w, w, f2);
    }
    const float res = block_max512(mx, red);
    if (res <= kNSInvTol) {
      ok = true;
      break;
    }
    if (it == 0) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) f2 += __shfl_xor_sync(0xffffffffu, f2, o);
      __syncthreads();
      if ((tid & 31) == 0) red[tid >> 5] = f2;
      __syncthreads();
      float ff = 0.f;
      for (int w = 0; w < nt / 32; ++w) ff += red[w];
      if (!(ff < 0.81f)) break;     // |I - K X0|_F >= 0.9: the iteration may not converge
    } else if (!(res < 0.5f * prev)) {
      break;                        // not shrinking any more (rounding floor or divergence)
    }
    prev = res;
    smem_mm<D, 2>(Xb, W, Kb);       // K's buffer <- X + X W
    __syncthreads();
    float* t = Kb;
    Kb = Xb;
    Xb = t;
    for (int o = tid; o < D * D; o += nt) Kb[o] = K[o];   // K again, into the old X's buffer
    __syncthreads();
  }
  if (ok) {
    for (int o = tid; o < D * D; o += nt) Ki[o] = Xb[o];
    return;
  }
  __syncthreads();
  gj_inverse<D>(h, K, Ki, smem);
}

// ---- d x d products into tmp: PU K_U, K_U^{-1} PUi, PV K_V, K_V^{-1} PVi ----
template <int D>
__global__ void __launch_bounds__(256) k_products(DevHeader* h, Workspace ws, const float* __restrict__ PU,
                                                  const float* __restrict__ PUi, const float* __restrict__ PV,
                                                  const float* __restrict__ PVi) {
  constexpr int TS = D < 32 ? D : 32;
  constexpr int NT = D / TS;
  __shared__ float As[TS][D + 1];
  __shared__ float Bs[D][TS + 1];
  if (h->status != 0 || h->nS == 0) return;
  const int prod = blockIdx.x / (NT * NT), tile = blockIdx.x % (NT * NT);
  const int ti = tile / NT, tj = tile % NT;
  const float *A, *B;
  switch (prod) {
    case 0: A = PU, B = ws.KU; break;
    case 1: A = ws.KUi, B = PUi; break;
    case 2: A = PV, B = ws.KV; break;
    default: A = ws.KVi, B = PVi; break;
  }
  float* C = ws.tmp + (size_t)prod * D * D;
  for (int o = threadIdx.x; o < TS * D; o += blockDim.x) {
    const int i = o / D, k = o % D;
    As[i][k] = A[(ti * TS + i) * D + k];
  }
  for (int o = threadIdx.x; o < D * TS; o += blockDim.x) {
    const int k = o / TS, j = o % TS;
    Bs[k][j] = B[k * D + tj * TS + j];
  }
  __syncthreads();
  for (int o = threadIdx.x; o < TS * TS; o += blockDim.x) {
    const int i = o / TS, j = o % TS;
    float s = 0.f;
#pragma unroll 8
    for (int k = 0; k < D; ++k) s = fmaf(As[i][k], Bs[k][j], s);
    C[(ti * TS + i) * D + tj * TS + j] = s;
  }
}

// ---- commit the new transforms and Sigma; non-finite check ----
template <int D>
__global__ void __launch_bounds__(256) k_commit(DevHeader* h, Workspace ws, float* PU, float* PUi, float* PV,
                                                float* PVi, float* sigma) {
  __shared__ int bad;
  if (h->status != 0 || h->nS == 0) return;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  float* dst[4] = {PU, PUi, PV, PVi};
  const int part = blockIdx.x;  // one block per matrix
  for (int o = threadIdx.x; o < D * D; o += blockDim.x) {
    const float v = ws.tmp[(size_t)part * D * D + o];
    if (!isfinite(v)) bad = 1;
  }
  if (part == 0)
    for (int k = threadIdx.x; k < D; k += blockDim.x)
      if (!isfinite(ws.theta[k])) bad = 1;
  __syncthreads();
  if (bad) {
    if (threadIdx.x == 0) set_status(h, DAMF_ERR_NUMERIC);
    return;
  }
  for (int o = threadIdx.x; o < D * D; o += blockDim.x) dst[part][o] = ws.tmp[(size_t)part * D * D + o];
  if (part == 0)
    for (int k = threadIdx.x; k < D; k += blockDim.x) sigma[k] = ws.theta[k];
}

// ---- a6: Ub[S] += Y_B PUi,  Vb[T] += (N^T Y_C) PVi,  r[S] += (Ub[S] change) diag(s0) ----
template <int D>
__global__ void __launch_bounds__(256) k_scatter(DevHeader* h, Workspace ws, float* Ub, float* Vb, float* r,
                                                 const float* __restrict__ PUi, const float* __restrict__ PVi,
                                                 const float* __restrict__ s0) {
  extern __shared__ float smem[];
  float* P = smem;             // D x D
  float* A = smem + D * D;     // 16 x D
  float* Ys = A + 16 * D;      // nS x D: Y_C (side 1)
  if (h->status != 0) return;
  const int nS = h->nS, nT = h->nT;
  if (nS == 0) return;
  const int side = blockIdx.y;
  const int nrows = side == 0 ? nS : nT;
  const int r0 = blockIdx.x * 16;
  if (r0 >= nrows) return;
  const float* Pm = side == 0 ? PUi : PVi;
  const int tid = threadIdx.x;
  for (int i = tid; i < D * D / 4; i += 256) reinterpret_cast<float4*>(P)[i] = reinterpret_cast<const float4*>(Pm)[i];
  if (side == 1)
    for (int i = tid; i < nS * D / 4; i += 256)
      reinterpret_cast<float4*>(Ys)[i] = reinterpret_cast<const float4*>(ws.YC)[i];
  __syncthreads();
  for (int o = tid; o < 16 * D; o += 256) {
    const int rr = o / D, k = o % D;
    float v = 0.f;
    if (r0 + rr < nrows) {
      if (side == 0) {
        v = ws.YB[(r0 + rr) * D + k];
      } else {   // (N^T Y_C)[b]: the column b of N is the same for the whole warp (a broadcast)
        const int b = r0 + rr;
        for (int a = 0; a < nS; ++a) v = fmaf(__ldg(ws.N + a * nT + b), Ys[a * D + k], v);
      }
    }
    A[o] = v;
  }
  __syncthreads();
  for (int o = tid; o < 16 * D; o += 256) {
    const int rr = o / D, j = o % D;
    if (r0 + rr >= nrows) continue;
    float s = 0.f;
#pragma unroll 8
    for (int k = 0; k < D; ++k) s = fmaf(A[rr * D + k], P[k * D + j], s);
    const int u = side == 0 ? ws.S[r0 + rr] : ws.T[r0 + rr];
    if (!DAMF_DCHECK(h, u >= 0 && u < h->n_nodes)) continue;
    if (side == 0) {
      const size_t row = (size_t)u * D;
      Ub[row + j] += s;
      r[row + j] += s * s0[j];
    } else {
      Vb[(size_t)u * D + j] += s;
    }
  }
}

// The update's projection U[S] = Ub[S] PU, V[T] = Vb[T] PV stays on the SIMT units in both
// precisions: on the tensor cores (kind::tf32, three-term split, accumulation in TMEM) its
// error of ~1e-6 per product, amplified by residual Grams with small pivots (hub rows nearly
// inside the span of U), coupled columns of U at up to 3e-4 between folds on C3, against 5e-5
// with FP32 products, for no measurable gain in speed.
template <int D>
static cudaError_t gather_impl(Ctx* c, cudaStream_t s) {
  const size_t sm = (size_t)(D * D + 16 * D) * sizeof(float);
  cudaFuncSetAttribute(k_gather<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_gather<D><<<dim3(kMaxR / 16, 2), 256, sm, s>>>(c->hdr, c->ws, c->Ub, c->Vb, c->PU, c->PV);
  return cudaGetLastError();
}

template <int D>
static cudaError_t chol_impl(Ctx* c, cudaStream_t s) {
  const size_t smw = (size_t)(kMaxR * D + 16 * kMaxR) * sizeof(float);
  cudaFuncSetAttribute(k_wct<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smw);
  k_wct<D><<<kMaxR / 16, 256, smw, s>>>(c->hdr, c->ws);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t sm = (size_t)(kMaxR * (kMaxR + 1) + kMaxR * (D + 1) + kMaxR * (kMaxR + 1)) * sizeof(float);
  cudaFuncSetAttribute(k_chol<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_chol<D><<<2, kChainThreads, sm, s>>>(c->hdr, c->ws);
  return cudaGetLastError();
}

template <int D>
static cudaError_t refine_core(Ctx* c, cudaStream_t s) {
  cudaError_t e;
  k_fo_pq<D><<<D, 128, 0, s>>>(c->hdr, c->ws);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  constexpr int TS = D < 32 ? D : 32;
  const size_t smt = ((size_t)2 * TS * (kMaxR + 1) + (size_t)2 * D * TS) * sizeof(float);
  cudaFuncSetAttribute(k_fo_t<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smt);
  k_fo_t<D><<<dim3(D / TS, D / TS), 256, smt, s>>>(c->hdr, c->ws, c->sigma);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t sma = (size_t)(D * D + 16 * D + D * (D + 1)) * sizeof(float);
  cudaFuncSetAttribute(k_fo_apply<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sma);
  k_fo_apply<D><<<dim3(kMaxM / 16, 2), 256, sma, s>>>(c->hdr, c->ws);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_fo_norm_theta<D><<<D, 128, 0, s>>>(c->hdr, c->ws, c->sigma);
  return cudaGetLastError();
}

template <int D>
static cudaError_t trans_impl(Ctx* c, cudaStream_t s) {
  cudaError_t e;
  k_hmat<D><<<kMaxM, 128, 0, s>>>(c->hdr, c->ws);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  {
    constexpr int GT = (D + 31) / 32;
    k_ns_gram<D><<<dim3(GT, GT, 2), 256, 0, s>>>(c->hdr, c->ws);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t sma = (size_t)(D * D + 16 * D) * sizeof(float);
    cudaFuncSetAttribute(k_ns_apply<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sma);
    k_ns_apply<D><<<dim3(kMaxM / 16, 2), 256, sma, s>>>(c->hdr, c->ws);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = refine_core<D>(c, s)) != cudaSuccess) return e;
  const size_t sm = (size_t)(kMaxR * (kMaxR + 1) + 2 * kMaxR * D) * sizeof(float);
  cudaFuncSetAttribute(k_trans<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_trans<D><<<2, kChainThreads, sm, s>>>(c->hdr, c->ws);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const size_t smi = (size_t)(D * (2 * D + 1) > 3 * D * D ? D * (2 * D + 1) : 3 * D * D) * sizeof(float);
  cudaFuncSetAttribute(k_inverse<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smi);
  k_inverse<D><<<2, kChainThreads, smi, s>>>(c->hdr, c->ws);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  // the transform products stay on the SIMT units in both precisions: P and P^{-1} accumulate
  // one product per update, and on the tensor cores (TF32, three-term split, accumulation in
  // TMEM) the per-product error of a few 1e-7 drifted the factors by ~1e-3 after 600 d = 128
  // updates, against ~2e-5 for FP32
  {
    constexpr int TS = D < 32 ? D : 32;
    constexpr int NT = D / TS;
    k_products<D><<<4 * NT * NT, 256, 0, s>>>(c->hdr, c->ws, c->PU, c->PUi, c->PV, c->PVi);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  k_commit<D><<<4, 256, 0, s>>>(c->hdr, c->ws, c->PU, c->PUi, c->PV, c->PVi, c->sigma);
  return cudaGetLastError();
}

template <int D>
static cudaError_t scatter_impl(Ctx* c, cudaStream_t s) {
  const size_t sm = (size_t)(D * D + 16 * D + kMaxR * D) * sizeof(float);
  cudaFuncSetAttribute(k_scatter<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_scatter<D><<<dim3(kMaxR / 16, 2), 256, sm, s>>>(c->hdr, c->ws, c->Ub, c->Vb, c->r, c->PUi, c->PVi, c->s0);
  return cudaGetLastError();
}

#define DAMF_DISPATCH_D(fn, ...)                    \
  switch (c->d) {                                   \
    case 16: return fn<16>(__VA_ARGS__);            \
    case 32: return fn<32>(__VA_ARGS__);            \
    case 64: return fn<64>(__VA_ARGS__);            \
    default: return fn<128>(__VA_ARGS__);           \
  }

cudaError_t launch_gather(Ctx* c, cudaStream_t s) { DAMF_DISPATCH_D(gather_impl, c, s) }
cudaError_t launch_chol(Ctx* c, cudaStream_t s) { DAMF_DISPATCH_D(chol_impl, c, s) }
cudaError_t launch_transforms(Ctx* c, cudaStream_t s) { DAMF_DISPATCH_D(trans_impl, c, s) }
cudaError_t launch_scatter(Ctx* c, cudaStream_t s) { DAMF_DISPATCH_D(scatter_impl, c, s) }

template <int D>
static cudaError_t assemble_impl(Ctx* c, cudaStream_t s) {
  k_assemble<D><<<kMaxM, 256, 0, s>>>(c->hdr, c->ws, c->sigma);
  return cudaGetLastError();
}
cudaError_t launch_assemble(Ctx* c, cudaStream_t s) { DAMF_DISPATCH_D(assemble_impl, c, s) }

}  // namespace damf
