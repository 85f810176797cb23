// C ABI of the library: options, graph life cycle, runs, statistics, errors.
#include <cstring>
#include <vector>
#include <new>
#include <string>

#include "bfs_internal.cuh"

namespace bfsgb {

static thread_local std::string t_error;

void set_error(const std::string& msg) { t_error = msg; }

int fail(int code, const std::string& msg) {
  t_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();
  t_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? BFS_ERR_OOM : BFS_ERR_CUDA;
}

int build_graph(const int32_t* src, const int32_t* dst, int64_t m, int32_t n, const bfs_options& opt,
                bfs_graph* g, cudaStream_t s);

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
      cudaSetDevice(dev);
    } else {
      prev = -1;
    }
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

template <class T>
int dmalloc(T** p, size_t count, int64_t* total, const char* what) {
  size_t bytes = count * sizeof(T);
  if (bytes == 0) bytes = sizeof(T);
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, what);
  }
  *total += (int64_t)bytes;
  return BFS_OK;
}

int check_options(const bfs_options& o) {
  if (o.th < 0) return fail(BFS_ERR_INVALID, "th must be >= 0");
  if (o.schedule < BFS_SCHED_BEAMER || o.schedule > BFS_SCHED_BEAMER_STAY)
    return fail(BFS_ERR_INVALID, "unknown schedule");
  for (int i = 0; i < 3; ++i)
    if (!(o.subgraph_factor0[i] >= 0) || !(o.subgraph_factor1[i] >= 0))
      return fail(BFS_ERR_INVALID, "subgraph factors must be >= 0");
  if (o.alpha <= 0 || o.beta <= 0) return fail(BFS_ERR_INVALID, "alpha and beta must be > 0");
  if (o.td_parent != BFS_TD_PARENT_PULL && o.td_parent != BFS_TD_PARENT_ATOMICMIN)
    return fail(BFS_ERR_INVALID, "unknown td_parent");
  if (o.blocks_per_sm < 0 || o.blocks_per_sm > 3)
    return fail(BFS_ERR_INVALID, "blocks_per_sm must be 0, 1, 2 or 3");
  if (o.barrier_timeout_ms <= 0) return fail(BFS_ERR_INVALID, "barrier_timeout_ms must be > 0");
  if (o.run_timeout_ms <= 0) return fail(BFS_ERR_INVALID, "run_timeout_ms must be > 0");
  if (!(o.factor0 >= 0) || !(o.factor1 >= 0)) return fail(BFS_ERR_INVALID, "factors must be >= 0");
  return BFS_OK;
}

int alloc_run_state(bfs_graph* g) {
  int64_t& t = g->device_bytes;
  g->words = ((int64_t)g->n_ni + 31) / 32;
  const size_t words = (size_t)g->words + 32;
  int rc;
  cudaError_t e;
  if ((rc = dmalloc(&g->V, words, &t, "alloc V"))) return rc;
  if ((rc = dmalloc(&g->V1, words, &t, "alloc V1"))) return rc;
  if ((rc = dmalloc(&g->N0, words, &t, "alloc N"))) return rc;
  if ((rc = dmalloc(&g->N1, words, &t, "alloc N"))) return rc;
  // depth nibble planes (4 bits per vertex each, a 16-byte word per visited-bitmap
  // word): enough nibbles for any depth below n_ni
  g->planes_n = 1;
  while (g->planes_n < 8 && ((int64_t)1 << (4 * g->planes_n)) <= (int64_t)g->n_ni) ++g->planes_n;
  g->pstride = (g->words + 1) * 4;
  if ((rc = dmalloc(&g->planes, (size_t)g->pstride * g->planes_n + 4, &t, "alloc depth planes"))) return rc;
  if ((rc = dmalloc(&g->parent_i, (size_t)g->n_ni + 8, &t, "alloc parent"))) return rc;
  if ((rc = dmalloc(&g->Q0, (size_t)g->n_ni + 1, &t, "alloc queue"))) return rc;
  if ((rc = dmalloc(&g->Q1, (size_t)g->n_ni + 1, &t, "alloc queue"))) return rc;
  if ((rc = dmalloc(&g->CL0, (size_t)g->cl_cap, &t, "alloc chunk list"))) return rc;
  if ((rc = dmalloc(&g->CL1, (size_t)g->cl_cap, &t, "alloc chunk list"))) return rc;
  if ((rc = dmalloc(&g->longq, (size_t)g->long_cap, &t, "alloc long-row list"))) return rc;
  if ((rc = dmalloc(&g->slot, (size_t)kSlots, &t, "alloc counters"))) return rc;
  if ((rc = dmalloc(&g->log, (size_t)BFS_LOG_LEVELS, &t, "alloc log"))) return rc;
  if ((rc = dmalloc(&g->hdr, 1, &t, "alloc header"))) return rc;
  if ((rc = dmalloc(&g->arrive, (size_t)kMaxBlocks * 4, &t, "alloc barrier words"))) return rc;
  e = cudaMemset(g->arrive, 0, sizeof(unsigned long long) * kMaxBlocks * 4);
  if (e != cudaSuccess) return cuda_fail(e, "memset barrier words");
  e = cudaMemset(g->hdr, 0, sizeof(RunHeader));
  if (e != cudaSuccess) return cuda_fail(e, "memset header");
  e = cudaMemset(g->slot, 0, sizeof(LevelSlot) * kSlots);
  if (e != cudaSuccess) return cuda_fail(e, "memset counters");
  return BFS_OK;
}

void free_all(bfs_graph* g) {
  void* ptrs[] = {g->off, g->col, g->caller_of, g->internal_of, g->head, g->deg, g->lead, g->V, g->V1, g->N0, g->N1, g->planes, g->crank,
                  g->parent_i, g->Q0, g->Q1, g->CL0, g->CL1, g->longq, g->slot, g->log, g->hdr, g->arrive, g->out_scratch,
                  g->deg_del, g->sub_tot};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (g->stage) cudaFree(g->stage);
  for (int i = 0; i < 2; ++i) {
    if (g->ev_run[i]) cudaEventDestroy(g->ev_run[i]);
    if (g->ev_copy[i]) cudaEventDestroy(g->ev_copy[i]);
  }
  if (g->ev_join) cudaEventDestroy(g->ev_join);
  if (g->copy_stream) cudaStreamDestroy(g->copy_stream);
  if (g->hdr_many) cudaFreeHost(g->hdr_many);
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Status of the most recent run (needs the stream to be synchronized).
int run_status(bfs_graph* g, RunHeader* h) {
  cudaError_t e = cudaMemcpy(h, g->hdr, sizeof(RunHeader), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read run header");
  if (h->err != 0 && (h->err >> 4) == (g->epoch & 0x0FFFFFFFu)) {
    int code = -(int)(h->err & 0xFu);
    if (code == BFS_ERR_TIMEOUT) return fail(code, "a device-side grid barrier wait passed its deadline");
    if (code == BFS_ERR_CHECK) return fail(code, "a bounds check of the BFS_CHECK build failed in the level loop");
    return fail(code, "the level-loop kernel reported an error");
  }
  return BFS_OK;
}

}  // namespace

// Device address of page-locked host memory (written by kernels directly over the
// host link), or null for device or pageable memory.
void* pinned_device_ptr(void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}


// Algorithmic bytes of one run, from its per-level counters: what the method
// must move level by level (Sec. IV-A forward visit, Sec. II-C / IV-B backward
// visit, Sec. VI-A.3 output), whatever the kernel moves beyond it.  With B = one
// pass over the visited bitmap (4 * words) and D = over its delegate prefix:
//   forward level:  8 per frontier vertex (offset pair), 8 per row entry (the
//                   column and one state probe), 16 per vertex found (depth,
//                   parent, queue entry written now and read next level);
//   backward level: B, 8 per scanned vertex (offset pair), 8 per examined entry
//                   (column and frontier probe), 12 per vertex found (depth,
//                   parent, frontier bit);
//   level end (a level that found something): 2 (D + B) for the bitmap merge,
//                   and 4 per queue entry of the next level when it is forward;
//   output: 8 n (depth and parent of every vertex), once.
int64_t model_bytes_from_log(const bfs_graph* g, const bfs_stats* st) {
  const int64_t B = g->words * 4, D = ((int64_t)g->d + 31) / 32 * 4;
  int64_t b = 8 * (int64_t)g->n;
  for (int L = 0; L < st->logged_levels; ++L) {
    const bfs_level_log& l = st->level[L];
    if (l.direction == 0)
      b += 8 * l.frontier + 8 * l.frontier_edges + 16 * l.found;
    else
      b += B + 8 * l.scanned + 8 * l.edges_examined + 12 * l.found;
    if (l.found > 0) {
      b += 2 * (D + B);
      if (L + 1 < st->logged_levels && st->level[L + 1].direction == 0) b += 4 * st->level[L + 1].queue_entries;
    }
  }
  return b;
}

}  // namespace bfsgb

using namespace bfsgb;

extern "C" int bfs_options_default(bfs_options* opt) {
  if (!opt) return fail(BFS_ERR_INVALID, "opt is NULL");
  std::memset(opt, 0, sizeof(*opt));
  opt->th = 64;
  opt->edges_on_device = 0;
  opt->schedule = BFS_SCHED_BEAMER_STAY;
  opt->schedule_mask = 0;
  opt->alpha = 10;
  opt->beta = 18;
  opt->factor0 = 0.5;
  opt->factor1 = 1e-7;
  opt->td_parent = BFS_TD_PARENT_ATOMICMIN;
  opt->blocks_per_sm = 0;
  opt->barrier_timeout_ms = 2000;
  opt->run_timeout_ms = 60000;
  opt->subgraph_factor0[0] = 0.5;
  opt->subgraph_factor0[1] = 0.05;
  opt->subgraph_factor0[2] = 1e-7;
  for (int i = 0; i < 3; ++i) opt->subgraph_factor1[i] = 1e-7;
  return BFS_OK;
}

extern "C" int bfs_build_graph(const int32_t* src, const int32_t* dst, int64_t num_edges, int32_t num_vertices,
                               const bfs_options* opt, bfs_graph** out, struct CUstream_st* stream) {
  if (!out) return fail(BFS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (num_vertices <= 0) return fail(BFS_ERR_INVALID, "num_vertices must be >= 1");
  if (num_edges < 0) return fail(BFS_ERR_INVALID, "num_edges must be >= 0");
  if (num_edges > 0 && (!src || !dst)) return fail(BFS_ERR_INVALID, "src or dst is NULL");
  bfs_options o;
  bfs_options_default(&o);
  if (opt) o = *opt;
  int rc = check_options(o);
  if (rc) return rc;
  bfs_graph* g = new (std::nothrow) bfs_graph();
  if (!g) return fail(BFS_ERR_OOM, "host allocation failed");
  cudaStream_t s = (cudaStream_t)stream;
  rc = build_graph(src, dst, num_edges, num_vertices, o, g, s);
  if (!rc) rc = alloc_run_state(g);
  if (!rc) rc = configure_run(g);
  if (rc) {
    std::string msg = bfs_last_error();
    cudaStreamSynchronize(s);
    free_all(g);
    delete g;
    set_error(msg);
    return rc;
  }
  *out = g;
  return BFS_OK;
}

extern "C" int bfs_set_options(bfs_graph* g, const bfs_options* opt) {
  if (!g || !opt) return fail(BFS_ERR_INVALID, "graph or opt is NULL");
  bfs_options o = *opt;
  o.th = g->opt.th;
  o.edges_on_device = g->opt.edges_on_device;
  int rc = check_options(o);
  if (rc) return rc;
  const int old_bps = g->opt.blocks_per_sm;
  g->opt = o;
  if (o.blocks_per_sm != old_bps) {
    DeviceGuard dg(g->device);
    rc = configure_run(g);
    if (rc) return rc;
  }
  return BFS_OK;
}

extern "C" int bfs_graph_get_info(const bfs_graph* g, bfs_graph_info* info) {
  if (!g || !info) return fail(BFS_ERR_INVALID, "graph or info is NULL");
  std::memset(info, 0, sizeof(*info));
  info->n = g->n;
  info->n_nonisolated = g->n_ni;
  info->delegates = g->d;
  info->grid_blocks = g->grid_blocks;
  info->th = g->th;
  info->nnz = g->nnz;
  info->max_degree = g->max_deg;
  for (int j = 0; j < 4; ++j) info->subgraph_edges[j] = g->sub[j];
  info->chunk_capacity = g->cl_cap;
  info->device_bytes = g->device_bytes;
  return BFS_OK;
}

extern "C" int bfs_graph_export(const bfs_graph* g, int64_t* row_off, int32_t* col, int32_t* caller_of,
                                int32_t* internal_of) {
  if (!g) return fail(BFS_ERR_INVALID, "graph is NULL");
  DeviceGuard dg(g->device);
  cudaError_t e = cudaSuccess;
  if (row_off) e = cudaMemcpy(row_off, g->off, ((size_t)g->n_ni + 1) * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && col && g->nnz > 0) e = cudaMemcpy(col, g->col, (size_t)g->nnz * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && caller_of) e = cudaMemcpy(caller_of, g->caller_of, (size_t)g->n * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && internal_of)
    e = cudaMemcpy(internal_of, g->internal_of, (size_t)g->n * 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "export");
  return BFS_OK;
}

static int fill_stats(bfs_graph* g, bfs_stats* st, const RunHeader& h) {
  std::memset(st, 0, sizeof(*st));
  st->levels = h.levels;
  st->logged_levels = h.levels_run < BFS_LOG_LEVELS ? h.levels_run : BFS_LOG_LEVELS;
  st->reached = (int64_t)h.reached;
  st->component_edges = (int64_t)(h.reached_edges / 2);
  st->device_ns = h.t1 - h.t0;
  st->setup_ns = h.t_init - h.t0;
  st->result_ns = h.t1 - h.t_loop;
  if (st->logged_levels > 0) {
    LevelLogDev lg[BFS_LOG_LEVELS];
    cudaError_t e = cudaMemcpy(lg, g->log, sizeof(LevelLogDev) * st->logged_levels, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "read level log");
    for (int L = 0; L < st->logged_levels; ++L) {
      bfs_level_log& o = st->level[L];
      o.direction = lg[L].dir;
      o.converted = lg[L].converted;
      o.frontier = (int64_t)lg[L].n_f;
      o.frontier_edges = (int64_t)lg[L].m_f;
      o.scanned = (int64_t)lg[L].scanned;
      o.edges_examined = (int64_t)lg[L].edges;
      o.parent_edges = (int64_t)lg[L].fix_edges;
      o.found = (int64_t)lg[L].found;
      o.queue_entries = (int64_t)lg[L].qn;
      o.t_begin_ns = lg[L].t_begin;
      o.t_expand_ns = lg[L].t_expand;
      o.t_end_ns = lg[L].t_end;
      o.t_first_done_ns = lg[L].t_first;
      o.t_last_done_ns = lg[L].t_last;
      o.subgraph_directions = lg[L].subdirs;
      st->edges_examined += o.edges_examined;
    }
  }
  st->model_bytes = model_bytes_from_log(g, st);
  return BFS_OK;
}

extern "C" int bfs_run(bfs_graph* g, int32_t source, int32_t* depth, int32_t* parent, bfs_stats* stats,
                       struct CUstream_st* stream) {
  if (!g) return fail(BFS_ERR_INVALID, "graph is NULL");
  if (!depth || !parent) return fail(BFS_ERR_INVALID, "depth or parent is NULL");
  if (source < 0 || source >= g->n) return fail(BFS_ERR_INVALID, "source out of range");
  DeviceGuard dg(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  const bool dd = is_device_ptr(depth), dp = is_device_ptr(parent);
  if (dd != dp) return fail(BFS_ERR_INVALID, "depth and parent must both be device or both be host memory");
  int rc;
  int32_t* pd = dd ? nullptr : static_cast<int32_t*>(pinned_device_ptr(depth));
  int32_t* pp = dd ? nullptr : static_cast<int32_t*>(pinned_device_ptr(parent));
  if (dd) {
    rc = launch_run(g, source, depth, parent, s);
    if (rc) return rc;
  } else if (pd && pp) {  // page-locked host buffers: the result pass writes them directly
    rc = launch_run(g, source, pd, pp, s);
    if (rc) return rc;
  } else {
    if (!g->out_scratch) {
      cudaError_t e = cudaMalloc(&g->out_scratch, (size_t)g->n * 8);
      if (e != cudaSuccess) {
        g->out_scratch = nullptr;
        return cuda_fail(e, "alloc output scratch");
      }
      g->device_bytes += (int64_t)g->n * 8;
    }
    rc = launch_run(g, source, g->out_scratch, g->out_scratch + g->n, s);
    if (rc) return rc;
    cudaError_t e = cudaMemcpyAsync(depth, g->out_scratch, (size_t)g->n * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(parent, g->out_scratch + g->n, (size_t)g->n * 4, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_fail(e, "copy results");
  }
  if (!dd || stats) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "bfs_run");
    RunHeader h;
    rc = run_status(g, &h);
    if (rc) return rc;
    if (stats) return fill_stats(g, stats, h);
  }
  return BFS_OK;
}

namespace {

// Staging buffers, copy stream, events and header copies of bfs_run_many.
int many_state(bfs_graph* g, int32_t count) {
  const int64_t n4 = ((int64_t)g->n + 3) & ~(int64_t)3;
  cudaError_t e = cudaSuccess;
  if (!g->stage) {
    e = cudaMalloc(&g->stage, (size_t)n4 * 4 * 4);
    if (e != cudaSuccess) {
      g->stage = nullptr;
      return cuda_fail(e, "alloc staging buffers");
    }
    g->device_bytes += n4 * 16;
  }
  if (!g->copy_stream && (e = cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking)) != cudaSuccess) {
    g->copy_stream = nullptr;
    return cuda_fail(e, "create copy stream");
  }
  for (int i = 0; i < 2; ++i) {
    if (!g->ev_run[i] && (e = cudaEventCreateWithFlags(&g->ev_run[i], cudaEventDisableTiming)) != cudaSuccess) {
      g->ev_run[i] = nullptr;
      return cuda_fail(e, "create event");
    }
    if (!g->ev_copy[i] && (e = cudaEventCreateWithFlags(&g->ev_copy[i], cudaEventDisableTiming)) != cudaSuccess) {
      g->ev_copy[i] = nullptr;
      return cuda_fail(e, "create event");
    }
  }
  if (!g->ev_join && (e = cudaEventCreateWithFlags(&g->ev_join, cudaEventDisableTiming)) != cudaSuccess) {
    g->ev_join = nullptr;
    return cuda_fail(e, "create event");
  }
  if (g->hdr_many_cap < count) {
    if (g->hdr_many) cudaFreeHost(g->hdr_many);
    g->hdr_many = nullptr;
    g->hdr_many_cap = 0;
    if ((e = cudaMallocHost((void**)&g->hdr_many, (size_t)count * sizeof(RunHeader))) != cudaSuccess) {
      g->hdr_many = nullptr;
      return cuda_fail(e, "alloc header copies");
    }
    g->hdr_many_cap = count;
  }
  return BFS_OK;
}

}  // namespace

extern "C" int bfs_run_many(bfs_graph* g, const int32_t* sources, int32_t count, int32_t* const* depth,
                            int32_t* const* parent, int32_t* status, struct CUstream_st* stream) {
  if (!g) return fail(BFS_ERR_INVALID, "graph is NULL");
  if (count < 0) return fail(BFS_ERR_INVALID, "count must be >= 0");
  if (count == 0) return BFS_OK;
  if (!sources || !depth || !parent) return fail(BFS_ERR_INVALID, "sources, depth or parent is NULL");
  for (int32_t i = 0; i < count; ++i) {
    if (sources[i] < 0 || sources[i] >= g->n) return fail(BFS_ERR_INVALID, "source out of range");
    if (!depth[i] || !parent[i]) return fail(BFS_ERR_INVALID, "a depth or parent buffer is NULL");
  }
  DeviceGuard dg(g->device);
  for (int32_t i = 0; i < count; ++i)
    if (is_device_ptr(depth[i]) || is_device_ptr(parent[i]))
      return fail(BFS_ERR_INVALID, "bfs_run_many writes host buffers (use bfs_run for device buffers)");
  int rc = many_state(g, count);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream, x = g->copy_stream;
  const int64_t n4 = ((int64_t)g->n + 3) & ~(int64_t)3;
  const size_t bytes = (size_t)g->n * 4;
  std::vector<unsigned> epoch((size_t)count, 0u);
  // the copies start after the work already queued on `stream`
  cudaError_t e = cudaEventRecord(g->ev_join, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(x, g->ev_join, 0);
  int32_t launched = 0;
  for (int32_t i = 0; i < count && e == cudaSuccess && rc == BFS_OK; ++i) {
    const int slot = i & 1;
    int32_t* sd = g->stage + (int64_t)slot * 2 * n4;
    int32_t* sp = sd + n4;
    if (i >= 2) e = cudaStreamWaitEvent(s, g->ev_copy[slot], 0);  // run i-2's copy has left the slot
    if (e != cudaSuccess) break;
    rc = launch_run(g, sources[i], sd, sp, s);
    if (rc) break;
    launched = i + 1;
    epoch[(size_t)i] = g->epoch & 0x0FFFFFFFu;
    e = cudaMemcpyAsync(g->hdr_many + i, g->hdr, sizeof(RunHeader), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(g->ev_run[slot], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(x, g->ev_run[slot], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(depth[i], sd, bytes, cudaMemcpyDeviceToHost, x);
    if (e == cudaSuccess) e = cudaMemcpyAsync(parent[i], sp, bytes, cudaMemcpyDeviceToHost, x);
    if (e == cudaSuccess) e = cudaEventRecord(g->ev_copy[slot], x);
  }
  // `stream` ends after the last copy; then every run's header is in place
  cudaError_t e2 = cudaEventRecord(g->ev_join, x);
  if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, g->ev_join, 0);
  const cudaError_t e3 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2 != cudaSuccess ? e2 : e3;
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "bfs_run_many");
  int first = BFS_OK;
  for (int32_t i = 0; i < launched; ++i) {
    const RunHeader& h = g->hdr_many[i];
    int st = BFS_OK;
    if (h.err != 0 && (h.err >> 4) == epoch[(size_t)i]) st = -(int)(h.err & 0xFu);
    if (status) status[i] = st;
    if (st != BFS_OK && first == BFS_OK) first = st;
  }
  if (first == BFS_ERR_TIMEOUT) return fail(first, "a device-side grid barrier wait passed its deadline");
  if (first != BFS_OK) return fail(first, "the level-loop kernel reported an error");
  return BFS_OK;
}

extern "C" int bfs_wait(bfs_graph* g, struct CUstream_st* stream) {
  if (!g) return fail(BFS_ERR_INVALID, "graph is NULL");
  DeviceGuard dg(g->device);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "bfs_wait");
  RunHeader h;
  return run_status(g, &h);
}

extern "C" void bfs_free(bfs_graph* g) {
  if (!g) return;
  DeviceGuard dg(g->device);
  cudaDeviceSynchronize();
  free_all(g);
  delete g;
}

extern "C" const char* bfs_last_error(void) { return t_error.c_str(); }

extern "C" void bfs_abi_sizes(int64_t sizes[5]) {
  sizes[0] = (int64_t)sizeof(bfs_options);
  sizes[1] = (int64_t)sizeof(bfs_graph_info);
  sizes[2] = (int64_t)sizeof(bfs_level_log);
  sizes[3] = (int64_t)sizeof(bfs_stats);
  sizes[4] = (int64_t)sizeof(bfs_batch_stats);
}
