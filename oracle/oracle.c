/*
 * CPU oracle: plain, slow, obviously correct.  TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Cited passages are sections, figures and tables of Pan, Pearce, Owens,
 * "Scalable Breadth-First Search on a GPU Cluster" (arXiv 1803.03922).
 * Nothing here is blocked, fused or reordered beyond the definitions.
 */
#include "oracle.h"

#include <stdlib.h>
#include <string.h>

struct orc_graph {
  int32_t n;
  int64_t nnz;
  int64_t* off; /* n+1 */
  int32_t* col; /* nnz, each row ascending, no duplicates, no self-loops */
};

/* Sec. II-B: the graph is symmetric; Sec. VI-A.3: the undirected graph is made
 * by edge doubling.  Self-loops are dropped and duplicate pairs kept once.
 * Rows are sorted by a two-pass bucket sort: every directed entry u->v is first
 * placed in the bucket of its target v, then the buckets are read in ascending v
 * and each entry appended to row u, so every row receives its targets in
 * ascending order; equal neighbours are then adjacent and kept once. */
orc_graph* orc_graph_build(int32_t n, int64_t m, const int32_t* src, const int32_t* dst) {
  if (n <= 0 || m < 0 || (m > 0 && (!src || !dst))) return NULL;
  for (int64_t e = 0; e < m; ++e)
    if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return NULL;

  /* step 1: entries per vertex; the graph is symmetric, so a vertex is the
   * source of as many entries as it is the target of */
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!cnt) return NULL;
  for (int64_t e = 0; e < m; ++e) {
    int32_t u = src[e], v = dst[e];
    if (u == v) continue;
    cnt[u] += 1;
    cnt[v] += 1;
  }
  int64_t* start = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!start) { free(cnt); return NULL; }
  start[0] = 0;
  for (int32_t u = 0; u < n; ++u) start[u + 1] = start[u] + cnt[u];
  int64_t total = start[n];
  int32_t* bucket = (int32_t*)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
  int32_t* raw = (int32_t*)malloc((size_t)(total > 0 ? total : 1) * sizeof(int32_t));
  if (!bucket || !raw) { free(cnt); free(start); free(bucket); free(raw); return NULL; }
  /* step 2: bucket of target v holds the sources of the entries u->v */
  for (int32_t u = 0; u < n; ++u) cnt[u] = start[u];
  for (int64_t e = 0; e < m; ++e) {
    int32_t u = src[e], v = dst[e];
    if (u == v) continue;
    bucket[cnt[v]++] = u; /* entry u->v */
    bucket[cnt[u]++] = v; /* entry v->u */
  }
  /* step 3: read targets in ascending order, append each entry to its source row */
  for (int32_t u = 0; u < n; ++u) cnt[u] = start[u];
  for (int32_t v = 0; v < n; ++v)
    for (int64_t i = start[v]; i < start[v + 1]; ++i) {
      int32_t u = bucket[i];
      raw[cnt[u]++] = v;
    }
  free(bucket);
  /* step 4: keep each neighbour once (rows are sorted) */
  int64_t* off = (int64_t*)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!off) { free(cnt); free(start); free(raw); return NULL; }
  int64_t w = 0;
  off[0] = 0;
  for (int32_t u = 0; u < n; ++u) {
    int64_t b = start[u], e = start[u + 1];
    for (int64_t i = b; i < e; ++i) {
      if (i > b && raw[i] == raw[i - 1]) continue;
      raw[w++] = raw[i];
    }
    off[u + 1] = w;
  }
  free(cnt);
  free(start);
  orc_graph* g = (orc_graph*)malloc(sizeof(orc_graph));
  if (!g) { free(raw); free(off); return NULL; }
  g->n = n;
  g->nnz = w;
  g->off = off;
  g->col = (int32_t*)realloc(raw, (size_t)(w > 0 ? w : 1) * sizeof(int32_t));
  if (!g->col) g->col = raw;
  return g;
}

void orc_graph_free(orc_graph* g) {
  if (!g) return;
  free(g->off);
  free(g->col);
  free(g);
}

int32_t orc_graph_n(const orc_graph* g) { return g->n; }
int64_t orc_graph_nnz(const orc_graph* g) { return g->nnz; }

void orc_graph_copy(const orc_graph* g, int64_t* off, int32_t* col) {
  if (off) memcpy(off, g->off, ((size_t)g->n + 1) * sizeof(int64_t));
  if (col && g->nnz > 0) memcpy(col, g->col, (size_t)g->nnz * sizeof(int32_t));
}

/* Hop distance (Sec. VI-A.3: the output is the hop distance from the source),
 * by the textbook FIFO-queue BFS. */
static int bfs_depth(const orc_graph* g, int32_t s, int32_t* depth) {
  int32_t n = g->n;
  int32_t* queue = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  if (!queue) return ORC_ERR_OOM;
  for (int32_t v = 0; v < n; ++v) depth[v] = -1;
  int64_t head = 0, tail = 0;
  depth[s] = 0;
  queue[tail++] = s;
  while (head < tail) {
    int32_t u = queue[head++];
    for (int64_t i = g->off[u]; i < g->off[u + 1]; ++i) {
      int32_t v = g->col[i];
      if (depth[v] == -1) {
        depth[v] = depth[u] + 1;
        queue[tail++] = v;
      }
    }
  }
  free(queue);
  return ORC_OK;
}

/* Canonical BFS-tree parent: the smallest-id neighbour one level closer to the
 * source.  Computed as an explicit minimum over the whole row, so it does not
 * rely on the rows being sorted. */
static void canonical_parent(const orc_graph* g, int32_t s, const int32_t* depth, int32_t* parent) {
  for (int32_t v = 0; v < g->n; ++v) {
    parent[v] = -1;
    if (v == s) { parent[v] = s; continue; }
    if (depth[v] <= 0) continue;
    int32_t best = -1;
    for (int64_t i = g->off[v]; i < g->off[v + 1]; ++i) {
      int32_t u = g->col[i];
      if (depth[u] == depth[v] - 1 && (best == -1 || u < best)) best = u;
    }
    parent[v] = best;
  }
}

int orc_bfs(const orc_graph* g, int32_t s, int32_t* depth, int32_t* parent) {
  if (!g || !depth || !parent || s < 0 || s >= g->n) return ORC_ERR_INVALID;
  int rc = bfs_depth(g, s, depth);
  if (rc) return rc;
  canonical_parent(g, s, depth, parent);
  return ORC_OK;
}

int orc_bfs_batch_u8(const orc_graph* g, int32_t k, const int32_t* sources, uint8_t* depth,
                     int32_t* parent) {
  if (!g || k < 0 || (k > 0 && (!sources || !depth || !parent))) return ORC_ERR_INVALID;
  int32_t n = g->n;
  for (int32_t j = 0; j < k; ++j)
    if (sources[j] < 0 || sources[j] >= n) return ORC_ERR_INVALID;
  int32_t* d32 = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  if (!d32) return ORC_ERR_OOM;
  int overflow = 0;
  for (int32_t j = 0; j < k; ++j) {
    int rc = orc_bfs(g, sources[j], d32, parent + (size_t)j * n);
    if (rc) { free(d32); return rc; }
    for (int32_t v = 0; v < n; ++v) {
      int32_t dv = d32[v];
      if (dv > 254) overflow = 1;
      depth[(size_t)j * n + v] = (uint8_t)(dv < 0 ? 255 : (dv > 254 ? 254 : dv));
    }
  }
  free(d32);
  return overflow ? ORC_ERR_OVERFLOW : ORC_OK;
}

int64_t orc_component_edges(const orc_graph* g, const int32_t* depth) {
  int64_t ends = 0;
  for (int32_t v = 0; v < g->n; ++v) {
    if (depth[v] < 0) continue;
    for (int64_t i = g->off[v]; i < g->off[v + 1]; ++i)
      if (depth[g->col[i]] >= 0) ends += 1;
  }
  return ends / 2; /* every undirected edge is stored twice */
}

static int is_edge(const orc_graph* g, int32_t u, int32_t v) {
  for (int64_t i = g->off[u]; i < g->off[u + 1]; ++i)
    if (g->col[i] == v) return 1;
  return 0;
}

static int32_t uf_find(int32_t* p, int32_t x) {
  while (p[x] != x) {
    p[x] = p[p[x]];
    x = p[x];
  }
  return x;
}

int orc_validate(const orc_graph* g, int32_t s, const int32_t* depth, const int32_t* parent) {
  int32_t n = g->n;
  if (s < 0 || s >= n) return 9;
  for (int32_t v = 0; v < n; ++v) {
    if (depth[v] < -1 || depth[v] >= n) return 9;
    if (parent[v] < -1 || parent[v] >= n) return 9;
  }
  if (depth[s] != 0 || parent[s] != s) return 1;
  for (int32_t u = 0; u < n; ++u) {
    for (int64_t i = g->off[u]; i < g->off[u + 1]; ++i) {
      int32_t v = g->col[i];
      if ((depth[u] >= 0) != (depth[v] >= 0)) return 2;
      if (depth[u] >= 0) {
        int32_t diff = depth[u] - depth[v];
        if (diff > 1 || diff < -1) return 3;
      }
    }
  }
  for (int32_t v = 0; v < n; ++v) {
    if (v == s) continue;
    if (depth[v] < 0) {
      if (parent[v] != -1) return 7;
      continue;
    }
    int32_t p = parent[v];
    if (p < 0 || !is_edge(g, p, v)) return 4;
    if (depth[p] != depth[v] - 1) return 5;
    for (int64_t i = g->off[v]; i < g->off[v + 1]; ++i) {
      int32_t u = g->col[i];
      if (u < p && depth[u] == depth[v] - 1) return 6;
    }
  }
  /* reached set == connected component of s, by union-find over all edges */
  int32_t* uf = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  if (!uf) return ORC_ERR_OOM;
  for (int32_t v = 0; v < n; ++v) uf[v] = v;
  for (int32_t u = 0; u < n; ++u)
    for (int64_t i = g->off[u]; i < g->off[u + 1]; ++i) {
      int32_t a = uf_find(uf, u), b = uf_find(uf, g->col[i]);
      if (a != b) uf[a] = b;
    }
  int32_t rs = uf_find(uf, s);
  int bad = 0;
  for (int32_t v = 0; v < n && !bad; ++v)
    if ((uf_find(uf, v) == rs) != (depth[v] >= 0)) bad = 1;
  free(uf);
  return bad ? 8 : 0;
}

/* Sec. III-A: delegates are the vertices with more than TH neighbours, normal
 * vertices the rest; Fig. 2 renumbers delegates in ascending original id.  The
 * device layout places the non-isolated normal vertices next and the isolated
 * ones last, each class in ascending original id. */
void orc_separate(const orc_graph* g, int64_t th, int32_t* internal_of, int32_t* caller_of,
                  int32_t* d_out, int32_t* n_ni_out) {
  int32_t n = g->n;
  int32_t next = 0;
  for (int32_t v = 0; v < n; ++v) /* class 0: delegates */
    if (g->off[v + 1] - g->off[v] > th) internal_of[v] = next++;
  int32_t d = next;
  for (int32_t v = 0; v < n; ++v) { /* class 1: normal vertices with a neighbour */
    int64_t deg = g->off[v + 1] - g->off[v];
    if (deg > 0 && deg <= th) internal_of[v] = next++;
  }
  int32_t n_ni = next;
  for (int32_t v = 0; v < n; ++v) { /* class 2: isolated vertices */
    int64_t deg = g->off[v + 1] - g->off[v];
    if (deg == 0 && deg <= th) internal_of[v] = next++;
  }
  for (int32_t v = 0; v < n; ++v) caller_of[internal_of[v]] = v;
  *d_out = d;
  *n_ni_out = n_ni;
}

/* Sec. IV: nn, nd, dn and dd are the edges from normal/delegate sources to
 * normal/delegate destinations. */
void orc_subgraph_counts(const orc_graph* g, int64_t th, int64_t counts[4]) {
  counts[0] = counts[1] = counts[2] = counts[3] = 0;
  for (int32_t u = 0; u < g->n; ++u) {
    int u_del = (g->off[u + 1] - g->off[u]) > th;
    for (int64_t i = g->off[u]; i < g->off[u + 1]; ++i) {
      int32_t v = g->col[i];
      int v_del = (g->off[v + 1] - g->off[v]) > th;
      counts[(u_del << 1) | v_del] += 1;
    }
  }
}

/* Position (1-based) of v's first neighbour at depth `level`, or its degree. */
static int64_t first_hit(const orc_graph* g, const int32_t* depth, int32_t v, int32_t level) {
  for (int64_t i = g->off[v]; i < g->off[v + 1]; ++i)
    if (depth[g->col[i]] == level) return i - g->off[v] + 1;
  return g->off[v + 1] - g->off[v];
}

int orc_level_counters(const orc_graph* g, int32_t s, const int32_t* depth, int64_t th, int32_t levels,
                       const int32_t* dirs, int64_t* out) {
  if (!g || !depth || !dirs || !out || levels < 0 || s < 0 || s >= g->n) return ORC_ERR_INVALID;
  for (int32_t L = 0; L < levels; ++L) {
    int64_t* o = out + (int64_t)L * 7;
    for (int j = 0; j < 7; ++j) o[j] = 0;
    for (int32_t v = 0; v < g->n; ++v) {
      int64_t deg = g->off[v + 1] - g->off[v];
      if (depth[v] == L) {
        o[0] += 1;
        o[1] += deg;
        if (dirs[L] == 0 && deg > 0 && deg <= th) o[6] += 1;
      }
      if (depth[v] == L + 1) {
        o[2] += 1;
        if (dirs[L] == 0) o[5] += first_hit(g, depth, v, L);
      }
      int unvisited = depth[v] == -1 || depth[v] > L;
      if (dirs[L] == 1 && unvisited && deg > 0) {
        o[3] += 1;
        o[4] += first_hit(g, depth, v, L);
      }
    }
  }
  return ORC_OK;
}

int orc_directions(const orc_graph* g, int32_t s, const int32_t* depth, int32_t rule, int64_t alpha, int64_t beta,
                   double factor0, double factor1, int32_t max_levels, int32_t* dirs) {
  if (!g || !depth || !dirs || s < 0 || s >= g->n || max_levels < 0) return ORC_ERR_INVALID;
  if (rule != ORC_RULE_BEAMER && rule != ORC_RULE_PAPER && rule != ORC_RULE_BEAMER_STAY) return ORC_ERR_INVALID;
  if (g->off[s + 1] == g->off[s]) return 0; /* isolated source: no level runs */
  int32_t levels = 0;
  int64_t n_ni = 0;
  for (int32_t v = 0; v < g->n; ++v) {
    if (g->off[v + 1] > g->off[v]) n_ni += 1;
    if (depth[v] + 1 > levels) levels = depth[v] + 1;
  }
  int64_t* q = calloc((size_t)levels + 1, sizeof(int64_t));
  int64_t* fv = calloc((size_t)levels + 1, sizeof(int64_t));
  if (!q || !fv) {
    free(q);
    free(fv);
    return ORC_ERR_OOM;
  }
  int64_t m_total = 0;
  for (int32_t v = 0; v < g->n; ++v) {
    const int64_t deg = g->off[v + 1] - g->off[v];
    m_total += deg;
    if (depth[v] >= 0) {
      q[depth[v]] += 1;
      fv[depth[v]] += deg;
    }
  }
  int cur = 0;
  int64_t seen_v = 0, seen_m = 0;
  for (int32_t L = 0; L < levels; ++L) {
    seen_v += q[L];
    seen_m += fv[L];
    const int64_t s_u = n_ni - seen_v, m_u = m_total - seen_m;
    const int64_t q_prev = L == 0 ? 1 : q[L - 1];
    int next;
    if (rule == ORC_RULE_PAPER) {
      const double qd = (double)q[L], sd = (double)(s_u > 0 ? s_u : 0);
      const double fvd = (double)fv[L], bv = sd * (qd + sd) / qd;
      next = cur == 0 ? (fvd > factor0 * bv) : !(fvd < factor1 * bv);
    } else if (cur == 0) {
      next = fv[L] * alpha > m_u;
    } else {
      next = !(q[L] * beta < (int64_t)g->n && q[L] < q_prev);
      if (rule == ORC_RULE_BEAMER_STAY && fv[L] * alpha > m_u) next = 1;
    }
    cur = next ? 1 : 0;
    if (L < max_levels) dirs[L] = cur;
  }
  free(q);
  free(fv);
  return levels;
}

/* Sec. IV-B, per subgraph: the dd, dn and nd visits each take their own
 * direction with their own factor pair; nn is always forward.  For a subgraph
 * X with source class S and destination class T (delegate: degree > th):
 *   out_X(u) = neighbours of class T of a vertex u of class S (u's X entries),
 *   in_X(v)  = neighbours of class S of a vertex v of class T (v's entries in
 *              the reversed subgraph; v is a "source" of the reversed one);
 *   q  = vertices of F_L in S with out_X > 0 (the subgraph's input frontier,
 *        zero-out-degree vertices filtered out),  FV = their out_X summed,
 *   U  = unvisited vertices of T with in_X > 0 (sources of the reversed
 *        subgraph: the source list / masks the backward visit starts from),
 *   s  = unvisited vertices of S with out_X > 0,
 *   BV = U (q + s) / q  (in double);
 * forward turns backward when FV > factor0 BV, backward turns forward when
 * FV < factor1 BV; a subgraph with q = 0 has nothing to visit this level and
 * keeps its direction.  "Unvisited" at level L: not in F_0..F_L. */
int orc_subgraph_directions(const orc_graph* g, int32_t s, const int32_t* depth, int64_t th,
                            const double factor0[3], const double factor1[3], int32_t max_levels, int32_t* dirs) {
  if (!g || !depth || !dirs || !factor0 || !factor1 || s < 0 || s >= g->n || max_levels < 0 || th < 0)
    return ORC_ERR_INVALID;
  if (g->off[s + 1] == g->off[s]) return 0; /* isolated source: no level runs */
  const int32_t n = g->n;
  int32_t levels = 0;
  for (int32_t v = 0; v < n; ++v)
    if (depth[v] + 1 > levels) levels = depth[v] + 1;
  /* per vertex: delegate or not, and its delegate / normal neighbours */
  int64_t* ndel = (int64_t*)calloc((size_t)n, sizeof(int64_t));
  if (!ndel) return ORC_ERR_OOM;
  for (int32_t v = 0; v < n; ++v)
    for (int64_t i = g->off[v]; i < g->off[v + 1]; ++i) {
      const int32_t u = g->col[i];
      if (g->off[u + 1] - g->off[u] > th) ndel[v] += 1;
    }
  /* subgraphs in the order dd, dn, nd: source class, destination class (1 = delegate) */
  const int src_del[3] = {1, 1, 0}, dst_del[3] = {1, 0, 1};
  int cur[3] = {0, 0, 0};
  for (int32_t L = 0; L < levels; ++L) {
    for (int x = 0; x < 3; ++x) {
      int64_t q = 0, fv = 0, U = 0, su = 0;
      for (int32_t v = 0; v < n; ++v) {
        const int64_t deg = g->off[v + 1] - g->off[v];
        const int is_del = deg > th;
        const int64_t nb_del = ndel[v], nb_norm = deg - ndel[v];
        const int64_t out_x = is_del == src_del[x] ? (dst_del[x] ? nb_del : nb_norm) : 0;
        const int64_t in_x = is_del == dst_del[x] ? (src_del[x] ? nb_del : nb_norm) : 0;
        const int unvisited = depth[v] == -1 || depth[v] > L;
        if (depth[v] == L && out_x > 0) {
          q += 1;
          fv += out_x;
        }
        if (unvisited && in_x > 0) U += 1;
        if (unvisited && out_x > 0) su += 1;
      }
      if (q > 0) {
        const double qd = (double)q, sd = (double)su, bv = (double)U * (qd + sd) / qd, fvd = (double)fv;
        cur[x] = cur[x] == 0 ? (fvd > factor0[x] * bv) : !(fvd < factor1[x] * bv);
      }
    }
    if (L < max_levels) dirs[L] = cur[0] | (cur[1] << 1) | (cur[2] << 2);
  }
  free(ndel);
  return levels;
}
