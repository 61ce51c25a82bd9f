/*
 * Oracle (test infrastructure only; never linked by the CUDA library).
 *
 * Plain C, sequential, FP64.  Two things live here because Python is too slow
 * for them at the benchmark sizes:
 *
 *  1. A dynamic adjacency structure with set semantics: one growable array of
 *     neighbour ids per node, membership by linear scan.  The graph of Sec. 2
 *     (Preliminaries): A[u][v] = 1 iff v is in row u; deg(u) is the out-degree.
 *
 *  2. The sequential FIFO push for Personalized PageRank (Sec. 4.4, Eq. "ppr").
 *     With P = D^{-1} A and Pi = alpha (I - (1-alpha) P)^{-1}, the pair (Z, r)
 *     keeps the invariant  Pi X = Z + Pi r.  Pushing node u moves alpha r[u]
 *     into Z[u] and adds (1-alpha) A[w][u] / deg(w) * r[u] to r[w] for every
 *     in-neighbour w of u (this follows from Pi = alpha I + (1-alpha) Pi P).
 *     Nodes are pushed in FIFO order until max_j |r[u][j]| <= eps for every u.
 *     Then |Z - Pi X| <= eps elementwise because Pi is row-substochastic.
 *
 * Nothing here is tuned; it is meant to be read against the definitions.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct {
  int32_t n;
  int32_t n_cap;
  int32_t* len;
  int32_t* cap;
  int32_t** nbr;
} og_graph;

og_graph* og_create(int32_t n, int32_t n_cap) {
  if (n_cap < n) n_cap = n;
  og_graph* g = (og_graph*)calloc(1, sizeof(og_graph));
  g->n = n;
  g->n_cap = n_cap;
  g->len = (int32_t*)calloc((size_t)n_cap, sizeof(int32_t));
  g->cap = (int32_t*)calloc((size_t)n_cap, sizeof(int32_t));
  g->nbr = (int32_t**)calloc((size_t)n_cap, sizeof(int32_t*));
  return g;
}

void og_destroy(og_graph* g) {
  if (!g) return;
  for (int32_t i = 0; i < g->n_cap; ++i) free(g->nbr[i]);
  free(g->nbr);
  free(g->len);
  free(g->cap);
  free(g);
}

int32_t og_num_nodes(const og_graph* g) { return g->n; }

/* Append k isolated nodes; returns the new node count or -1 when over capacity. */
int32_t og_add_nodes(og_graph* g, int32_t k) {
  if (g->n + k > g->n_cap) return -1;
  g->n += k;
  return g->n;
}

int32_t og_degree(const og_graph* g, int32_t u) { return g->len[u]; }

int32_t og_has(const og_graph* g, int32_t u, int32_t v) {
  for (int32_t i = 0; i < g->len[u]; ++i)
    if (g->nbr[u][i] == v) return 1;
  return 0;
}

/* Returns 1 when (u, v) was added, 0 when it was already present. */
int32_t og_insert(og_graph* g, int32_t u, int32_t v) {
  if (og_has(g, u, v)) return 0;
  if (g->len[u] == g->cap[u]) {
    int32_t nc = g->cap[u] ? 2 * g->cap[u] : 4;
    g->nbr[u] = (int32_t*)realloc(g->nbr[u], (size_t)nc * sizeof(int32_t));
    g->cap[u] = nc;
  }
  g->nbr[u][g->len[u]++] = v;
  return 1;
}

/* Returns 1 when (u, v) was removed, 0 when it was absent. */
int32_t og_erase(og_graph* g, int32_t u, int32_t v) {
  for (int32_t i = 0; i < g->len[u]; ++i) {
    if (g->nbr[u][i] == v) {
      g->nbr[u][i] = g->nbr[u][g->len[u] - 1];
      g->len[u] -= 1;
      return 1;
    }
  }
  return 0;
}

/* Copies row u into out (caller provides room for og_degree(u) ids). */
int32_t og_neighbors(const og_graph* g, int32_t u, int32_t* out) {
  memcpy(out, g->nbr[u], (size_t)g->len[u] * sizeof(int32_t));
  return g->len[u];
}

/* Bulk load from CSR (rows 0..n-1); existing rows must be empty. */
void og_load_csr(og_graph* g, const int32_t* indptr, const int32_t* indices) {
  for (int32_t u = 0; u < g->n; ++u)
    for (int32_t e = indptr[u]; e < indptr[u + 1]; ++e) og_insert(g, u, indices[e]);
}

/* Total number of stored entries. */
int64_t og_num_entries(const og_graph* g) {
  int64_t s = 0;
  for (int32_t u = 0; u < g->n; ++u) s += g->len[u];
  return s;
}

/* CSR export with rows sorted by column id; indptr has n+1 slots, indices
 * og_num_entries() slots. */
static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}
void og_export_csr(const og_graph* g, int64_t* indptr, int32_t* indices) {
  int64_t pos = 0;
  for (int32_t u = 0; u < g->n; ++u) {
    indptr[u] = pos;
    memcpy(indices + pos, g->nbr[u], (size_t)g->len[u] * sizeof(int32_t));
    qsort(indices + pos, (size_t)g->len[u], sizeof(int32_t), cmp_i32);
    pos += g->len[u];
  }
  indptr[g->n] = pos;
}

static double row_absmax(const double* x, int32_t d) {
  double m = 0.0;
  for (int32_t j = 0; j < d; ++j) {
    double a = fabs(x[j]);
    if (a > m) m = a;
  }
  return m;
}

/*
 * Sequential FIFO push (see header).  in_g holds the in-neighbours of each node
 * (for an undirected graph pass the same structure as out_g); out_g gives the
 * out-degrees deg(w).  Z and r are n x d row-major.  Returns the number of
 * pushes, or -1 when max_pushes was reached before convergence.
 */
/* Threshold of node u: eps (absolute) or eps * max(outdeg(u), 1) (degree-scaled). */
static double push_threshold(const og_graph* out_g, int32_t u, double eps, int32_t deg_scaled) {
  if (!deg_scaled) return eps;
  const int32_t k = out_g->len[u];
  return eps * (double)(k > 1 ? k : 1);
}

int64_t og_push(const og_graph* in_g, const og_graph* out_g, int32_t d, double* Z, double* r,
                double alpha, double eps, int64_t max_pushes, int32_t deg_scaled) {
  const int32_t n = out_g->n;
  int32_t* queue = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  char* queued = (char*)calloc((size_t)n, 1);
  double* rho = (double*)malloc((size_t)d * sizeof(double));
  int64_t head = 0, count = 0; /* ring buffer of capacity n */
  for (int32_t u = 0; u < n; ++u) {
    if (row_absmax(r + (size_t)u * d, d) > push_threshold(out_g, u, eps, deg_scaled)) {
      queue[(head + count) % n] = u;
      queued[u] = 1;
      count++;
    }
  }
  int64_t pushes = 0;
  while (count > 0) {
    if (pushes >= max_pushes) {
      pushes = -1;
      break;
    }
    int32_t u = queue[head];
    head = (head + 1) % n;
    count--;
    queued[u] = 0;
    double* ru = r + (size_t)u * d;
    if (row_absmax(ru, d) <= push_threshold(out_g, u, eps, deg_scaled)) continue;
    double* zu = Z + (size_t)u * d;
    for (int32_t j = 0; j < d; ++j) {
      rho[j] = ru[j];
      ru[j] = 0.0;
      zu[j] += alpha * rho[j];
    }
    pushes++;
    for (int32_t i = 0; i < in_g->len[u]; ++i) {
      int32_t w = in_g->nbr[u][i];
      double c = (1.0 - alpha) / (double)out_g->len[w];
      double* rw = r + (size_t)w * d;
      for (int32_t j = 0; j < d; ++j) rw[j] += c * rho[j];
      if (!queued[w] && row_absmax(rw, d) > push_threshold(out_g, w, eps, deg_scaled)) {
        queue[(head + count) % n] = w;
        queued[w] = 1;
        count++;
      }
    }
  }
  free(queue);
  free(queued);
  free(rho);
  return pushes;
}
