/*
 * CPU oracle for single-GPU direction-optimized BFS over a degree-separated graph.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the package smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The GPU product path
 * never links, loads or calls it, and it shares no code with the GPU path.
 *
 * Everything here is the plain definition of the result, written for a reader
 * to check against the paper by eye (Pan, Pearce, Owens, "Scalable Breadth-First
 * Search on a GPU Cluster", arXiv 1803.03922):
 *   - the graph is symmetric: every undirected edge is stored in both directions
 *     (Sec. II-B "Terminology"; Sec. VI-A.3 "edge doubling");
 *   - delegates are vertices whose out-degree is larger than TH, normal vertices
 *     the rest (Sec. II-B; Sec. III-A), renumbered to delegate ids in ascending
 *     original id (Fig. 2: vertices 7 and 8 become delegates 0 and 1);
 *   - the BFS output is the hop distance from the source (Sec. VI-A.3), plus a
 *     canonical BFS-tree parent (smallest-id neighbour one level closer to the
 *     source), the tree the paper discusses in Sec. VI-A.3 but does not build;
 *   - direction optimization changes only which edges are examined, never the
 *     output (Sec. IV-B), so one queue BFS defines the result of every schedule.
 *
 * All ids are the caller's ids.  Offsets are int64, columns int32.
 * Functions returning int return 0 on success and a negative code on error.
 */
#ifndef BFS_ORACLE_H
#define BFS_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_graph orc_graph;

/* Error codes. */
#define ORC_OK 0
#define ORC_ERR_INVALID (-1)
#define ORC_ERR_OOM (-2)
#define ORC_ERR_OVERFLOW (-3)

/* Symmetric simple graph from an edge list (Sec. II-B; Sec. VI-A.3): self-loops
 * are dropped, each remaining pair (u,v) is stored as u->v and v->u, and each
 * row holds its neighbours once, in ascending id.  Returns NULL on bad input
 * (n <= 0, m < 0, an id outside [0,n)) or when memory runs out. */
orc_graph* orc_graph_build(int32_t n, int64_t m, const int32_t* src, const int32_t* dst);
void orc_graph_free(orc_graph* g);
int32_t orc_graph_n(const orc_graph* g);
int64_t orc_graph_nnz(const orc_graph* g); /* directed entries = 2 x unique undirected edges */
/* Copies the row offsets (n+1 entries) and the columns (nnz entries); a NULL
 * destination skips that array. */
void orc_graph_copy(const orc_graph* g, int64_t* off, int32_t* col);

/* Hop distance by a FIFO-queue BFS, then the canonical parent by a separate pass:
 * parent[v] = min{u in N(v) : depth[u] = depth[v]-1}; parent[s] = s; unreached
 * vertices get depth -1 and parent -1 (Sec. VI-A.3). */
int orc_bfs(const orc_graph* g, int32_t s, int32_t* depth, int32_t* parent);

/* Same computation for k sources, with uint8 depth (255 = unreached) laid out
 * [k][n]; parent int32 [k][n].  ORC_ERR_OVERFLOW if some depth exceeds 254. */
int orc_bfs_batch_u8(const orc_graph* g, int32_t k, const int32_t* sources, uint8_t* depth,
                     int32_t* parent);

/* Unique undirected edges whose endpoints are both reached (the traversed
 * component's edge count, used as the numerator of GTEPS). */
int64_t orc_component_edges(const orc_graph* g, const int32_t* depth);

/* Graph500-style check of a (depth, parent) pair.  Returns 0 when every rule
 * holds, otherwise a positive rule number:
 *  1 depth[s] != 0 or parent[s] != s      2 an edge joins a reached and an unreached vertex
 *  3 |depth(u)-depth(v)| > 1 on an edge    4 (parent[v], v) is not an edge
 *  5 depth[parent[v]] != depth[v]-1        6 a smaller-id neighbour sits at depth[v]-1
 *  7 unreached vertex with parent != -1    8 reached set != union-find component of s
 *  9 depth/parent out of range */
int orc_validate(const orc_graph* g, int32_t s, const int32_t* depth, const int32_t* parent);

/* Degree separation (Sec. III-A) and the id layout it implies for the device
 * graph: delegates (degree > th) take ids [0,d) in ascending original id (Fig. 2),
 * non-isolated normal vertices take [d, n_ni) in ascending original id, and
 * isolated vertices (degree 0) take [n_ni, n) in ascending original id.
 * internal_of[caller] and caller_of[internal] are filled (n entries each). */
void orc_separate(const orc_graph* g, int64_t th, int32_t* internal_of, int32_t* caller_of,
                  int32_t* d, int32_t* n_ni);

/* Directed entry counts of the four subgraphs of Sec. IV (nn, nd, dn, dd) for a
 * threshold th: counts[0]=|E_nn|, counts[1]=|E_nd|, counts[2]=|E_dn|, counts[3]=|E_dd|. */
void orc_subgraph_counts(const orc_graph* g, int64_t th, int64_t counts[4]);

/* Per-level work counters of a direction-optimized run with the given per-level
 * directions (dirs[L] = 0 forward, 1 backward), from the final depth of a run
 * from s.  Rows are scanned in ascending neighbour id, so the position of the
 * first visited neighbour is fixed (Sec. II-C: the backward visit stops at the
 * first visited parent).  out[L*7 + j], j =
 *  0 |F_L| (vertices at depth L)         1 m_f = sum of degrees over F_L
 *  2 |F_{L+1}|
 *  3 backward: unvisited vertices with a neighbour at the start of level L
 *  4 backward: sum over those of k_v (first-hit position + 1, or the degree)
 *  5 forward: sum over v in F_{L+1} of the first-hit position + 1 (parent pick)
 *  6 forward: vertices of F_L with 0 < degree <= th (normal-vertex queue). */
int orc_level_counters(const orc_graph* g, int32_t s, const int32_t* depth, int64_t th, int32_t levels,
                       const int32_t* dirs, int64_t* out);

#define ORC_RULE_BEAMER 0
#define ORC_RULE_PAPER 1
#define ORC_RULE_BEAMER_STAY 2

/* Visit directions a direction rule takes on the run from s, given that run's
 * final depth.  The direction of level L (which expands F_L, the vertices at
 * depth L) is decided before it runs, from the current direction (level L-1's,
 * forward before level 0) and these counts:
 *   q   = |F_L|,  FV = sum of degrees over F_L,  q_prev = |F_{L-1}| (1 at L = 0),
 *   s_u = non-isolated vertices not in F_0..F_L (not visited yet),
 *   m_u = sum of their degrees,  n = the number of vertices.
 * ORC_RULE_PAPER (Sec. IV-B): BV = |U| (q + s) / q with U and s both the
 *   unvisited vertices (one symmetric graph), in double as s_u * (q + s_u) / q;
 *   forward turns backward when FV > factor0 * BV, backward turns forward when
 *   FV < factor1 * BV.
 * ORC_RULE_BEAMER (Beamer's rule, which the paper's DO follows, Sec. II-C):
 *   forward turns backward when alpha * FV > m_u; backward turns forward when
 *   beta * q < n and q < q_prev.
 * ORC_RULE_BEAMER_STAY (this build's default; not in the paper): Beamer's rule,
 *   except that backward turns forward only when, besides Beamer's test, the
 *   forward-to-backward test fails too (alpha * FV <= m_u): a level with few
 *   unvisited vertices left stays backward however small its frontier.
 * Writes dirs[L] (0 forward, 1 backward) for L < levels = max depth + 1, at
 * most max_levels of them; returns levels (0 for an isolated source) or an error. */
int orc_directions(const orc_graph* g, int32_t s, const int32_t* depth, int32_t rule, int64_t alpha, int64_t beta,
                   double factor0, double factor1, int32_t max_levels, int32_t* dirs);

/* Per-subgraph visit directions (Sec. IV-B: dd, dn and nd each switch with their
 * own factor pair, nn is always forward) on the run from s with final depth
 * `depth` and delegates of degree > th.  factor0/factor1[x] for x = 0 dd, 1 dn,
 * 2 nd.  dirs[L] = bit 0 dd, bit 1 dn, bit 2 nd backward at level L (the level
 * that expands F_L), for L < levels, at most max_levels of them; returns levels
 * (0 for an isolated source) or an error.  See oracle.c for the quantities. */
int orc_subgraph_directions(const orc_graph* g, int32_t s, const int32_t* depth, int64_t th,
                            const double factor0[3], const double factor1[3], int32_t max_levels, int32_t* dirs);

#ifdef __cplusplus
}
#endif
#endif
