/*
 * bfs_gb300 — direction-optimized breadth-first search over a degree-separated
 * graph on one NVIDIA GB300 (sm_103a).  C ABI: plain pointers and sizes only.
 *
 * Method: Pan, Pearce, Owens, "Scalable Breadth-First Search on a GPU Cluster"
 * (arXiv 1803.03922), single-GPU part:
 *   - degree separation: vertices with more than TH neighbours are delegates,
 *     the rest normal vertices (Sec. II-B, Sec. III-A); delegates are renumbered
 *     into a dense prefix of the id space in ascending original id (Fig. 2);
 *   - compact storage: int32 column indices (Sec. III-C, Table I);
 *   - per level, either a forward (top-down, push) visit with load balancing per
 *     degree class (Sec. IV-A) or a backward (bottom-up, pull) visit that stops
 *     at the first visited parent (Sec. II-C, Sec. IV-B), chosen per level by a
 *     direction heuristic (Sec. IV-B; Beamer's alpha/beta rule by default);
 *   - the output is the hop distance (Sec. VI-A.3) plus a canonical BFS-tree
 *     parent (the smallest-id neighbour one level closer to the source).
 *
 * Ids in every argument and result are the caller's ids.
 *
 * Errors: every int-returning call returns BFS_OK (0) or a negative code; the
 * message of the calling thread's last error is bfs_last_error().  On error the
 * outputs are unspecified and a graph handle passed in stays valid.
 *
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 */
#ifndef BFS_GB300_H
#define BFS_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st; /* cudaStream_t is `struct CUstream_st*` */

#define BFS_OK 0
#define BFS_ERR_INVALID (-1)  /* null pointer, n <= 0, id or source out of range, bad option */
#define BFS_ERR_OOM (-2)      /* device or host allocation failed */
#define BFS_ERR_OVERFLOW (-3) /* a size beyond the int32/int64 layout, or a batched depth > 254 */
#define BFS_ERR_TIMEOUT (-4)  /* a bounded device-side wait expired; the context stays usable */
#define BFS_ERR_CUDA (-5)     /* a CUDA runtime call failed */
#define BFS_ERR_CHECK (-6)    /* a bounds check of a library built with BFS_CHECK failed: an index of a
                                 kernel fell outside its array; the access was skipped (no trap) */

/* Direction schedules.  The output never depends on the schedule (Sec. IV-B:
 * a visit direction changes only the work, not the input or the output). */
#define BFS_SCHED_BEAMER 0    /* TD->BU when m_f*alpha > m_u; BU->TD when n_f*beta < n and shrinking */
#define BFS_SCHED_TOPDOWN 1   /* every level forward (plain BFS) */
#define BFS_SCHED_BOTTOMUP 2  /* level 0 forward, every later level backward */
#define BFS_SCHED_ALTERNATE 3 /* even levels forward, odd levels backward */
#define BFS_SCHED_MASK 4      /* level L backward iff bit min(L,63) of schedule_mask is set */
#define BFS_SCHED_PAPER 5     /* Sec. IV-B workload rule: FV vs factor * BV, BV = |U|(q+s)/q */
#define BFS_SCHED_BEAMER_STAY 7 /* the default: BFS_SCHED_BEAMER, except that BU->TD also needs
                                  m_f*alpha <= m_u (a level with few unvisited vertices left stays
                                  backward however small its frontier); not in the paper */
#define BFS_SCHED_PAPER_SUBGRAPH 6 /* Sec. IV-B per subgraph: the dd, dn and nd visits each take their own
                                      direction by the FV/BV rule with their own factor pair
                                      (subgraph_factor0/1); nn is always forward.  Per subgraph X:
                                      q = frontier vertices of X's source class with an X entry, FV =
                                      their X entries, U = unvisited vertices of X's destination class
                                      with an entry of the reversed subgraph, s = unvisited vertices of
                                      X's source class with an X entry; a subgraph with q = 0 keeps its
                                      direction.  Forward levels take atomicMin parents. */

/* How a forward level picks the canonical parent of a newly reached vertex. */
#define BFS_TD_PARENT_PULL 0      /* after the level, scan its sorted row for the first frontier neighbour */
#define BFS_TD_PARENT_ATOMICMIN 1 /* atomicMin of the frontier neighbour's caller id during the visit */

typedef struct bfs_options {
  int64_t th;               /* degree threshold TH (>= 0): delegates have degree > th. Build-time. */
  int32_t edges_on_device;  /* bfs_build_graph: 1 if src/dst are device pointers, 0 if host. */
  int32_t schedule;         /* BFS_SCHED_* (default BFS_SCHED_BEAMER_STAY) */
  uint64_t schedule_mask;   /* for BFS_SCHED_MASK */
  int32_t alpha;            /* Beamer alpha (default 10) */
  int32_t beta;             /* Beamer beta (default 18) */
  double factor0;           /* BFS_SCHED_PAPER: forward->backward when FV > factor0 * BV (default 0.5) */
  double factor1;           /* BFS_SCHED_PAPER: backward->forward when FV < factor1 * BV (default 1e-7) */
  int32_t td_parent;        /* BFS_TD_PARENT_* (default ATOMICMIN) */
  int32_t blocks_per_sm;    /* level-loop kernel CTAs per SM: 2 = the 64-register build (2 CTAs
                               of 512 threads), 3 = the 40-register build (3 CTAs of 512 threads
                               per SM), 1 = one CTA of 1024 threads per SM (64 registers);
                               0 (default) = 1 above 2^24 non-isolated vertices, else 2 */
  int32_t barrier_timeout_ms; /* bound of every device-side grid-barrier wait (default 2000) */
  int32_t test_skip_barrier;  /* testing only: CTA 0 leaves before the first grid barrier, so the
                                 other CTAs' bounded wait expires and the run reports BFS_ERR_TIMEOUT */
  int32_t run_timeout_ms;     /* bound of one run's device time (default 60000): BFS_ERR_TIMEOUT */
  int32_t tuning;             /* bit 0: forward visits read the discovered word before an atomicOr;
                                 bit 1: record when the first and the last CTA finish each
                                 expansion (bfs_level_log t_first_done_ns / t_last_done_ns) */
  double subgraph_factor0[3]; /* BFS_SCHED_PAPER_SUBGRAPH, for dd, dn, nd: forward->backward when
                                 FV > factor0 * BV (default 0.5, 0.05, 1e-7, Sec. IV-B) */
  double subgraph_factor1[3]; /* the same subgraphs: backward->forward when FV < factor1 * BV
                                 (default 1e-7 each) */
  int32_t reserved[4];
} bfs_options;

/* Fills *opt with the defaults: th 64, host edges, Beamer alpha 15 / beta 18,
 * paper factors 0.5 / 1e-7 (per subgraph 0.5 / 0.05 / 1e-7 and 1e-7), atomicMin
 * parents, 2000 ms barrier bound, 60 s run bound. */
int bfs_options_default(bfs_options* opt);

typedef struct bfs_graph bfs_graph;

/* Builds the device graph (Sec. III; Table I layout with int64 row offsets):
 * drops self-loops, stores every remaining pair in both directions (Sec. II-B),
 * removes duplicates, sorts every row by the neighbour's caller id, separates
 * delegates (degree > th) from normal vertices (Sec. III-A) and renumbers them:
 * internal ids [0,d) are delegates in ascending caller id (Fig. 2), [d,n_ni)
 * non-isolated normal vertices in ascending caller id, [n_ni,n) isolated ones.
 *   src, dst      borrowed, read-only, num_edges int32 ids in [0, num_vertices);
 *                 host memory, or device memory when opt->edges_on_device = 1.
 *   num_vertices  1 .. 2^31-1.   num_edges >= 0 (2*num_edges entries must fit int64).
 *   opt           NULL = defaults.
 *   out           receives a handle owned by the library (release with bfs_free).
 * Synchronizes `stream`.  Errors: INVALID (bad id, n, null), OOM, OVERFLOW, CUDA. */
int bfs_build_graph(const int32_t* src, const int32_t* dst, int64_t num_edges, int32_t num_vertices,
                    const bfs_options* opt, bfs_graph** out, struct CUstream_st* stream);

/* Replaces the run-time options of a graph (everything but th and edges_on_device). */
int bfs_set_options(bfs_graph* g, const bfs_options* opt);

typedef struct bfs_graph_info {
  int32_t n;              /* vertices */
  int32_t n_nonisolated;  /* vertices with degree > 0 (= n_ni) */
  int32_t delegates;      /* d: vertices with degree > th */
  int32_t grid_blocks;    /* CTAs of the level-loop kernel */
  int64_t th;
  int64_t nnz;            /* directed entries = 2 x unique undirected non-loop edges */
  int64_t max_degree;
  int64_t subgraph_edges[4]; /* directed entries of nn, nd, dn, dd (Sec. IV) */
  int64_t chunk_capacity; /* work-list entries reserved for delegate rows */
  int64_t device_bytes;   /* device memory held by the graph */
} bfs_graph_info;

int bfs_graph_get_info(const bfs_graph* g, bfs_graph_info* info);

/* Copies the device graph to caller-owned HOST buffers (synchronous):
 * row_off[n_ni+1] int64 and col[nnz] int32 in internal ids; caller_of[n]
 * (internal -> caller) and internal_of[n] (caller -> internal).  Any pointer may
 * be NULL to skip that array. */
int bfs_graph_export(const bfs_graph* g, int64_t* row_off, int32_t* col, int32_t* caller_of,
                     int32_t* internal_of);

#define BFS_LOG_LEVELS 256

/* One level of a run, as logged by the device. */
typedef struct bfs_level_log {
  int32_t direction;      /* 0 forward (top-down), 1 backward (bottom-up) */
  int32_t converted;      /* 1 if the frontier bitmap was converted to queues first (0 when the
                             sparse backward level before built the queues as it went) */
  int64_t frontier;       /* |F_L|: vertices at depth L */
  int64_t frontier_edges; /* m_f: sum of degrees over F_L */
  int64_t scanned;        /* backward: unvisited non-isolated vertices scanned */
  int64_t edges_examined; /* forward: m_f; backward: sum over scanned v of k_v */
  int64_t parent_edges;   /* forward with PULL parents: row entries read to pick parents */
  int64_t found;          /* |F_{L+1}| */
  int64_t queue_entries;  /* normal-vertex queue entries holding F_L (forward levels) */
  uint64_t t_begin_ns, t_expand_ns, t_end_ns; /* device %globaltimer at the phase edges */
  uint64_t t_first_done_ns, t_last_done_ns;   /* when the first / last CTA finished the expansion
                                                 (with tuning bit 1; else 0) */
  int32_t subgraph_directions; /* BFS_SCHED_PAPER_SUBGRAPH: bit 0 dd, bit 1 dn, bit 2 nd backward
                                  (direction = 1 when any is); 0 otherwise */
  int32_t reserved;
} bfs_level_log;

typedef struct bfs_stats {
  int32_t levels;          /* levels run (= max depth + 1) */
  int32_t logged_levels;   /* min(levels executed, BFS_LOG_LEVELS); 0 for an isolated source */
  int64_t reached;         /* vertices with depth >= 0 */
  int64_t component_edges; /* unique undirected edges in the traversed component (GTEPS numerator) */
  int64_t edges_examined;  /* sum over levels */
  int64_t model_bytes;     /* algorithmic bytes of this run, from the per-level counters: forward
                              levels 8 per frontier vertex + 8 per row entry + 16 per vertex found;
                              backward levels one visited-bitmap pass + 8 per scanned vertex + 8 per
                              examined entry + 12 per vertex found; every level that found something
                              a merge of the delegate and whole bitmaps (read and written) and the
                              next forward level's queue (4 per entry); 8 n of output */
  uint64_t device_ns;      /* %globaltimer span of the whole run (set-up, levels, results) */
  uint64_t setup_ns;       /* part of device_ns spent clearing state before level 0 */
  uint64_t result_ns;      /* part of device_ns spent writing the caller-indexed results */
  bfs_level_log level[BFS_LOG_LEVELS];
} bfs_stats;

/* One BFS from `source` (a caller id).  depth[n] and parent[n] are caller-owned
 * int32 buffers indexed by caller id, both in device memory or both in host
 * memory: depth[v] = hop distance (-1 unreached), parent[v] = canonical parent
 * (parent[source] = source, -1 unreached).  Device buffers: asynchronous on
 * `stream`.  Host buffers: `stream` is synchronized; page-locked (pinned) host
 * buffers are written by the kernel directly, pageable ones through a device
 * copy.
 * stats (optional, host): filled after synchronizing `stream`.
 * One run at a time per graph: runs on one stream are ordered; runs of the same
 * graph on different streams must not overlap.
 * Errors: INVALID (null, source out of range), TIMEOUT, CUDA. */
int bfs_run(bfs_graph* g, int32_t source, int32_t* depth, int32_t* parent, bfs_stats* stats,
            struct CUstream_st* stream);

/* Many BFS runs of one graph, results to host memory, pipelined: while the
 * results of run i cross the host link (copy engine), run i+1 computes on the
 * device.  Not in the paper, which reports device time only.
 * sources[count]: caller ids.  depth[i], parent[i]: caller-owned HOST buffers
 * of n int32 each, laid out as bfs_run's (page-locked buffers overlap the copy
 * with the next run; pageable ones work but without the overlap).  A buffer may
 * appear more than once: the later run's result lands last.
 * status (optional, host [count]): each run's BFS_OK or error code.
 * Ordering: the copies start after the work queued on `stream` before the call;
 * the call returns after `stream` has synchronized, with every result in place.
 * Device memory: two staging pairs (16·n bytes), a copy stream and events,
 * made on first use and kept with the graph.  Same one-run-at-a-time rule as
 * bfs_run.  Errors: INVALID (null, count < 0, source out of range, a device
 * buffer), TIMEOUT (the first failing run's code), CUDA, OOM. */
int bfs_run_many(bfs_graph* g, const int32_t* sources, int32_t count, int32_t* const* depth,
                 int32_t* const* parent, int32_t* status, struct CUstream_st* stream);

/* ---- Batched form: up to 64 queries per launch (64-lane bitset multi-source BFS). ----
 * Not in the paper, which runs one source at a time; the per-query result is the
 * same hop distance and canonical parent as bfs_run, with uint8 depth. */
typedef struct bfs_batch bfs_batch;

#define BFS_BATCH_LOG_LEVELS 64

typedef struct bfs_batch_level {
  int32_t direction;          /* 0 forward (push), 1 backward (pull), for all lanes alike */
  int32_t pulled_lanes;       /* lanes with a frontier at a backward level (they all pull), else 0 */
  int64_t frontier_vertices;  /* vertices in the union of the queries' frontiers */
  int64_t frontier_edges;     /* their degree sum */
  int64_t pairs;              /* (query, vertex) pairs in the frontier */
  uint64_t t_begin_ns, t_expand_ns, t_end_ns;
} bfs_batch_level;

typedef struct bfs_batch_stats {
  int32_t levels;          /* levels run by the batch (max over its queries of max depth + 1) */
  int32_t logged_levels;   /* min(levels, BFS_BATCH_LOG_LEVELS) */
  int64_t pairs_reached;   /* (query, vertex) pairs reached, sources excluded */
  int64_t traversed_edges; /* sum over the queries of the traversed component's undirected edges */
  uint64_t device_ns;      /* %globaltimer span of the launch */
  uint64_t setup_ns;       /* part of device_ns before level 0 */
  uint64_t result_ns;      /* part of device_ns writing the results */
  bfs_batch_level level[BFS_BATCH_LOG_LEVELS];
} bfs_batch_stats;

/* Device state for batches on graph g (about 8*4 + 64 (+256 with parents) bytes per
 * non-isolated vertex).  ctas: CTAs of the context's cooperative launch (0 = two
 * per SM, the whole device).  One batch at a time per context; contexts on
 * different streams may run concurrently only if their ctas add up to at most
 * the device's co-resident capacity (bfs_batch_capacity), so that every launch
 * can be resident at once.  The graph must outlive the context. */
int bfs_batch_create(const bfs_graph* g, int32_t with_parents, int32_t ctas, bfs_batch** out);

/* Co-resident CTA capacity of the batched kernel on the current device (two per SM). */
int bfs_batch_capacity(int32_t* ctas);

/* Device bytes held by a batch context. */
int64_t bfs_batch_device_bytes(const bfs_batch* b);

/* k (1..64) queries from sources[0..k) (host array of caller ids; repeats allowed).
 * depth[k*n] uint8 row-major by query (255 = unreached); parent[k*n] int32 (may be
 * NULL; requires a context created with parents); both device or both host.  Device
 * buffers: asynchronous on `stream` (status via bfs_batch_wait or stats); host
 * buffers (page-locked ones are written by the kernel directly) or stats:
 * synchronizes.  BFS_ERR_OVERFLOW when a depth would exceed 254. */
int bfs_run_batch(bfs_batch* b, const int32_t* sources, int32_t k, uint8_t* depth, int32_t* parent,
                  bfs_batch_stats* stats, struct CUstream_st* stream);

/* Synchronizes `stream`; status of the context's most recent batch. */
int bfs_batch_wait(bfs_batch* b, struct CUstream_st* stream);

/* Groups queries for batching (not in the paper).  Writes to order[0..k) a
 * permutation of 0..k-1 that sorts the sources by the degree sum of their
 * neighbours, largest first (ties keep their order); 0 for an isolated source.
 * That sum is the row entries of a query's second frontier: queries with
 * similar sums reach the graph's big levels at the same level, so batches cut
 * from consecutive runs of the order scan shorter rows in their backward levels.
 * sources: host array of k caller ids (k >= 0); order: host array of k.  Reads
 * the graph on `stream` and synchronizes it.  BFS_ERR_INVALID for a NULL
 * pointer, k < 0 or a source outside [0, n). */
int bfs_batch_order(const bfs_graph* g, const int32_t* sources, int32_t k, int32_t* order,
                    struct CUstream_st* stream);

void bfs_batch_free(bfs_batch* b);

/* ---- Serving loop: continuous batching of queries over device-resident graphs. ----
 * Not in the paper, which runs one source at a time.  A server borrows graph
 * handles and owns a worker thread.  Submitted queries wait in one FIFO per
 * graph.  Whenever fewer than max_concurrent launches are in flight, the worker
 * takes the graph whose oldest waiting query arrived first and launches its
 * waiting queries on a stream of their own: when at most single_max are waiting
 * they run back to back on the single-source level loop (bfs_run's kernel, on
 * the graph's run state, one such launch per graph at a time; with single_path
 * = 1), more are packed, up to max_lanes, into one multi-source launch
 * (bfs_run_batch's kernel).  Either way a
 * query's result is its exact hop distance and canonical parent, the same as
 * alone.  Each query is reported when its launch ends.  Each launch gets capacity / max_concurrent CTAs, so all launches
 * in flight are co-resident.  Batch contexts are created on demand (at most
 * contexts_per_graph per graph); a new context is admitted only when the
 * device's free memory less hbm_reserve_bytes covers it and the bytes of all
 * contexts held stay within hbm_budget_bytes; otherwise idle contexts of other
 * graphs are freed, least recently used first, or the queries keep waiting.
 * The submitting thread, the worker and the polling thread may differ. */
typedef struct bfs_server bfs_server;

typedef struct bfs_server_options {
  int32_t max_concurrent;     /* launches in flight, 1..8 (0 = 2) */
  int32_t max_lanes;          /* queries per launch, 1..64 (0 = 64) */
  int32_t with_parents;       /* 1: every query writes parents as well as depths */
  int32_t contexts_per_graph; /* batch contexts per graph, 1..max_concurrent (0 = max_concurrent) */
  int64_t hbm_reserve_bytes;  /* device memory left free when a context is admitted */
  int64_t hbm_budget_bytes;   /* cap on the device bytes of all contexts held (0 = none) */
  int32_t single_path;        /* 1: few waiting queries of a graph run the single-source level loop */
  int32_t single_max;         /* at most this many waiting queries (1..4; 0 = 3) run back to back on
                                 the level loop rather than as a batch */
  int32_t group_batches;      /* 1 (default): when more than max_lanes queries of a graph wait, a
                                 batch takes the oldest one and the max_lanes-1 nearest it by
                                 bfs_batch_order's key among the oldest 256; 0: arrival order */
  int32_t reserved[5];        /* zero */
} bfs_server_options;

typedef struct bfs_server_done {
  int64_t ticket;       /* as returned by bfs_server_submit */
  int32_t status;       /* BFS_OK, or the negative code of its launch (TIMEOUT, OVERFLOW, CUDA) */
  int32_t graph_id;
  int32_t batch_size;   /* queries in its launch */
  int32_t levels;       /* levels of its launch */
  int64_t t_arrival_ns; /* bfs_server_now_ns() clock throughout */
  int64_t t_launch_ns;
  int64_t t_done_ns;
  int64_t device_ns;    /* %globaltimer span of its launch */
} bfs_server_done;

typedef struct bfs_server_stats {
  int64_t submitted, completed, failed;
  int64_t launches, lanes_launched;
  int64_t contexts_created, contexts_evicted;
  int64_t context_bytes;  /* device bytes of the contexts held now */
  int64_t waiting;        /* queries submitted and not launched */
  int64_t in_flight;      /* launches running */
  int32_t capacity_ctas;  /* co-resident CTAs of the batched kernel on the device */
  int32_t ctas_per_launch;
  int64_t single_launches; /* launches of the single-source level loop (lone queries) */
  int64_t reserved[3];
} bfs_server_stats;

void bfs_server_options_default(bfs_server_options* opt);

/* Creates a server on the current device.  Errors: INVALID (option out of range), CUDA, OOM. */
int bfs_server_create(const bfs_server_options* opt, bfs_server** out);

/* Registers a graph (borrowed: it must outlive the server; the server runs
 * single-source runs on it, so the caller must not call bfs_run on it while the
 * server lives).  *graph_id = 0, 1, ... */
int bfs_server_add_graph(bfs_server* s, bfs_graph* g, int32_t* graph_id);

/* Host monotonic clock in ns (the clock of every bfs_server_done time). */
int64_t bfs_server_now_ns(void);

/* Queues a query from `source` (caller id) on graph graph_id.  depth[n] uint8
 * (255 = unreached) and, for a server with parents, parent[n] int32 (NULL
 * otherwise): caller-owned DEVICE buffers that must stay valid until the query
 * is reported.  t_arrival_ns: the query's arrival on bfs_server_now_ns()'s clock,
 * the start of its latency (0 = now).  *ticket: 1, 2, ... in submission order.
 * Errors: INVALID (bad graph id, source, buffer or a destroyed server). */
int bfs_server_submit(bfs_server* s, int32_t graph_id, int32_t source, uint8_t* depth, int32_t* parent,
                      int64_t t_arrival_ns, int64_t* ticket);

/* Moves up to max_done finished queries into done[] (host array), oldest
 * completion first; waits up to timeout_ms (0 = do not wait, < 0 = until one is
 * done or nothing is queued or running) for the first.  *n_done = the count. */
int bfs_server_poll(bfs_server* s, bfs_server_done* done, int32_t max_done, int32_t timeout_ms, int32_t* n_done);

int bfs_server_get_stats(bfs_server* s, bfs_server_stats* st);

/* Waits for the launches in flight, reports nothing more, frees every context
 * and stops the worker; queries not yet launched are dropped.  NULL is a no-op. */
void bfs_server_destroy(bfs_server* s);

/* sizeof of bfs_server_options, bfs_server_done, bfs_server_stats. */
void bfs_server_abi_sizes(int64_t sizes[3]);

/* Synchronizes `stream` and returns the device-side status of the graph's most
 * recent run: BFS_OK, or BFS_ERR_TIMEOUT when a bounded wait expired (runs with
 * device buffers and no stats do not report it themselves). */
int bfs_wait(bfs_graph* g, struct CUstream_st* stream);

/* BFS for callers that cannot allocate device memory.  The paper has no
 * counterpart: this entry point exists for code that runs where cudaMalloc is
 * not available to it (inside another runtime that owns the device allocator,
 * or under a fixed allocation budget).  It allocates nothing; all its scratch is
 * one fixed-size __device__ array of this library (about 6 MiB, held on every
 * device that loads the library until the process exits).
 *   row_off[n+1] int64, col[row_off[n]] int32: caller-owned DEVICE memory, a
 *     symmetric CSR in the caller's ids with every row sorted ascending and no
 *     self-loops or repeated entries (the graph bfs_build_graph would build).
 *     Checked on every call before any row is read: all four pointers are
 *     device memory, the offsets are non-decreasing within [0, row_off[n]] and
 *     every column lies in [0, n); otherwise BFS_ERR_INVALID.  Not checked:
 *     sorted rows and symmetry (without them the parents need not be canonical).
 *   n: 1 .. 16,777,216 vertices; larger n returns BFS_ERR_OVERFLOW, nothing runs.
 *   depth[n], parent[n]: caller-owned DEVICE int32 buffers; same results as
 *     bfs_run (hop distance, canonical smallest-id parent, -1 unreached).
 * The first call on a device looks up the scratch array's device address (make
 * that first call before any stream capture).  Every call shares the scratch and
 * clears what it needs at its start; calls that overlap on the GPU (for example
 * on two streams) race and must not be issued.  Synchronizes `stream` and
 * returns BFS_OK, BFS_ERR_TIMEOUT (a bounded device wait expired), INVALID,
 * OVERFLOW or CUDA. */
int bfs_run_static(const int64_t* row_off, const int32_t* col, int32_t n, int32_t source, int32_t* depth,
                   int32_t* parent, struct CUstream_st* stream);

/* Degree-class statistics of a built graph for `count` thresholds (Sec. VI-B:
 * TH balances the delegates against the nn edges; Figs. 5 and 7 plot both).  The
 * graph's own TH does not matter: degrees are those of the deduplicated
 * symmetric graph.  For ths[i] (>= 0), out[5*i + j] (host int64) is
 *   j = 0 delegates (vertices of degree > ths[i]), 1 |E_nn|, 2 |E_nd|, 3 |E_dn|,
 *   4 |E_dd| (directed entries whose source/destination are normal (n) or
 *   delegate (d) under ths[i], Sec. IV).
 * Allocates 24 bytes per possible degree on the device for the call and
 * synchronizes `stream`.  Errors: INVALID (null, count < 1, a negative
 * threshold), CUDA. */
int bfs_degree_class_stats(const bfs_graph* g, const int64_t* ths, int32_t count, int64_t* out,
                           struct CUstream_st* stream);

/* Releases every device and host resource of the graph.  NULL is a no-op. */
void bfs_free(bfs_graph* g);

/* Message of the calling thread's last error ("" if none). */
const char* bfs_last_error(void);

/* sizeof of the ABI structs, for bindings to check their layouts:
 * sizes[0] bfs_options, [1] bfs_graph_info, [2] bfs_level_log, [3] bfs_stats,
 * [4] bfs_batch_stats. */
void bfs_abi_sizes(int64_t sizes[5]);

#ifdef __cplusplus
}
#endif
#endif
