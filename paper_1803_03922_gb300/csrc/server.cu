// Serving loop: continuous batching of BFS queries over device-resident graphs
// (the bfs_server_* entry points).  The paper runs one source at a time; this is
// the runtime that turns the 64-lane multi-source kernel into a query server.
//
// Threads: callers submit and poll under `mu`; one worker thread owns the batch
// contexts and does every CUDA call of the server.  An event recorded after each
// launch marks its end: while launches are in flight the worker polls their
// events and the submission queue without sleeping (a query's completion and a
// new query's launch cost no thread wake-up); with nothing in flight it waits for
// a submission.  The worker never holds `mu` across a CUDA call.
//
// Scheduling: one FIFO per graph.  While fewer than max_concurrent launches run,
// the graph whose oldest waiting query arrived first gets one launch of up to
// max_lanes of its waiting queries: when at most single_max are waiting they run
// back to back on the single-source level loop on the graph's own run state
// (when no other single run of that graph is in flight), more share a
// multi-source batch on an idle batch context (or a
// new one, if free device memory and the budget admit it, after freeing idle
// contexts of other graphs least recently used first).  Every launch has
// capacity / max_concurrent CTAs, so the cooperative launches in flight always
// fit on the device together.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "bfs_internal.cuh"

using bfsgb::cuda_fail;
using bfsgb::fail;
using bfsgb::RunHeader;

namespace bfsgb {
// msbfs.cu: the keys of bfs_batch_order for k device-resident sources.
int order_keys_async(const bfs_graph* g, const int32_t* dsrc, int32_t k, unsigned long long* dkey, cudaStream_t s);
}  // namespace bfsgb

namespace {

constexpr int kMaxLanes = 64;
constexpr int kMaxConcurrent = 8;
constexpr int kMaxSingle = 4;  // single-source runs per launch of a graph's level-loop context
constexpr int kGroupWindow = 256;  // oldest waiting queries of a graph that a grouped batch picks from

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Query {
  int64_t ticket;
  int32_t source;
  uint8_t* depth;
  int32_t* parent;
  int64_t t_arrival;
};

struct GraphEntry {
  bfs_graph* g;
  std::deque<Query> waiting;
};

struct Context {
  bfs_server* srv = nullptr;
  int gid = 0;
  bool single = false;     // runs the single-source level loop on the graph's run state
  bfs_batch* b = nullptr;  // batch contexts only
  cudaStream_t stream = nullptr;
  RunHeader* hdr = nullptr;  // pinned host copies of the launch's run headers [kMaxSingle]
  int64_t bytes = 0;
  int ctas = 0;  // CTAs of the launch in flight
  bool busy = false;
  int64_t last_used = 0;
  std::vector<Query> q;  // the queries of the launch in flight
  unsigned epoch[kMaxSingle] = {0, 0, 0, 0};
  int64_t t_launch = 0;
  cudaEvent_t ev = nullptr;  // recorded after the launch: its end
};

bool device_ptr(const void* q) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

struct bfs_server {
  bfs_server_options opt{};
  int device = 0;
  int capacity = 0, slice = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  // guarded by mu
  std::deque<GraphEntry> graphs;
  std::deque<bfs_server_done> done;
  int64_t next_ticket = 1;
  int64_t waiting = 0;
  int in_flight = 0;
  bool stop = false, wake = false;
  int64_t submitted = 0, completed = 0, failed = 0, launches = 0, lanes = 0, single_launches = 0;
  int64_t created = 0, evicted = 0, ctx_bytes = 0;
  // worker thread only
  std::vector<std::unique_ptr<Context>> ctx;
  int ctas_in_use = 0;
  std::thread worker;
  // grouped batches: a stream and buffers for the keys of a window of waiting queries
  cudaStream_t order_stream = nullptr;
  int32_t* order_src_h = nullptr;              // pinned [kGroupWindow]
  unsigned long long* order_key_h = nullptr;   // pinned [kGroupWindow]
  int32_t* order_src_d = nullptr;              // device [kGroupWindow]
  unsigned long long* order_key_d = nullptr;   // device [kGroupWindow]
};

namespace {

// Moves the queries of a finished launch to the done list.  status: the launch's
// own failure, or BFS_OK to take each query's status from its run header (one
// header per single-source run, one for a whole batch).
void finish(bfs_server* s, Context& c, int status, int64_t t_done) {
  const int k = (int)c.q.size();
  int failed = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (int i = 0; i < k; ++i) {
      const Query& q = c.q[i];
      const int hi = c.single ? i : 0;
      const RunHeader& h = c.hdr[hi];
      const int st = status != BFS_OK ? status : bfsgb::ms_header_status(h, c.epoch[hi]);
      failed += st != BFS_OK;
      bfs_server_done d;
      std::memset(&d, 0, sizeof(d));
      d.ticket = q.ticket;
      d.status = st;
      d.graph_id = c.gid;
      d.batch_size = c.single ? 1 : k;
      d.levels = st == BFS_OK ? h.levels : 0;
      d.t_arrival_ns = q.t_arrival;
      d.t_launch_ns = c.t_launch;
      d.t_done_ns = t_done;
      d.device_ns = st == BFS_OK ? (int64_t)(h.t1 - h.t0) : 0;
      s->done.push_back(d);
    }
    s->completed += k;
    s->failed += failed;
    s->in_flight -= 1;
  }
  c.q.clear();
  c.busy = false;
  c.last_used = t_done;
  s->ctas_in_use -= c.ctas;
  c.ctas = 0;
  s->cv_done.notify_all();
}

// Finishes every launch whose end event has completed; returns how many.
int reap(bfs_server* s) {
  int n = 0;
  for (auto& cp : s->ctx) {
    Context& c = *cp;
    if (!c.busy) continue;
    const cudaError_t e = cudaEventQuery(c.ev);
    if (e == cudaErrorNotReady) continue;
    if (e == cudaSuccess)
      finish(s, c, BFS_OK, now_ns());
    else
      finish(s, c, cuda_fail(e, "serving launch"), now_ns());
    ++n;
  }
  return n;
}

bool admit(bfs_server* s, int64_t bytes) {
  int64_t held;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    held = s->ctx_bytes;
  }
  if (s->opt.hbm_budget_bytes > 0 && held + bytes > s->opt.hbm_budget_bytes) return false;
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (int64_t)free_b >= bytes + s->opt.hbm_reserve_bytes;
}

void drop_context(bfs_server* s, size_t i) {
  Context& c = *s->ctx[i];
  if (c.b) bfs_batch_free(c.b);
  if (c.ev) cudaEventDestroy(c.ev);
  if (c.stream) cudaStreamDestroy(c.stream);
  if (c.hdr) cudaFreeHost(c.hdr);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->ctx_bytes -= c.bytes;
  }
  s->ctx.erase(s->ctx.begin() + (std::ptrdiff_t)i);
}

Context* new_context(bfs_server* s, int gid) {
  std::unique_ptr<Context> c(new (std::nothrow) Context());
  if (!c) return nullptr;
  c->srv = s;
  c->gid = gid;
  if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost((void**)&c->hdr, kMaxSingle * sizeof(RunHeader)) != cudaSuccess) {
    cudaGetLastError();
    if (c->ev) cudaEventDestroy(c->ev);
    if (c->stream) cudaStreamDestroy(c->stream);
    return nullptr;
  }
  std::memset(c->hdr, 0, kMaxSingle * sizeof(RunHeader));
  s->ctx.push_back(std::move(c));
  return s->ctx.back().get();
}

// The graph's single-source context if it is idle (made on first use), else null.
Context* acquire_single(bfs_server* s, int gid) {
  for (auto& cp : s->ctx)
    if (cp->gid == gid && cp->single) return cp->busy ? nullptr : cp.get();
  Context* c = new_context(s, gid);
  if (c) c->single = true;
  return c;
}

// An idle batch context of graph gid, a new one, or null (the graph's queries wait).
Context* acquire_context(bfs_server* s, int gid, const bfs_graph* g) {
  int count = 0;
  Context* idle = nullptr;
  for (auto& cp : s->ctx)
    if (cp->gid == gid && !cp->single) {
      ++count;
      if (!cp->busy && (!idle || cp->last_used > idle->last_used)) idle = cp.get();
    }
  if (idle) return idle;
  if (count >= s->opt.contexts_per_graph) return nullptr;
  const int64_t need = bfsgb::ms_batch_bytes(g, s->opt.with_parents);
  while (!admit(s, need)) {
    // free the least recently used idle context of another graph
    size_t victim = s->ctx.size();
    for (size_t i = 0; i < s->ctx.size(); ++i) {
      const Context& c = *s->ctx[i];
      if (c.busy || c.gid == gid || c.single) continue;
      if (victim == s->ctx.size() || c.last_used < s->ctx[victim]->last_used) victim = i;
    }
    if (victim == s->ctx.size()) return nullptr;
    drop_context(s, victim);
    std::lock_guard<std::mutex> lk(s->mu);
    s->evicted += 1;
  }
  bfs_batch* b = nullptr;
  if (bfs_batch_create(g, s->opt.with_parents, s->slice, &b) != BFS_OK) return nullptr;
  Context* c = new_context(s, gid);
  if (!c) {
    bfs_batch_free(b);
    return nullptr;
  }
  c->b = b;
  c->bytes = bfs_batch_device_bytes(b);
  std::lock_guard<std::mutex> lk(s->mu);
  s->ctx_bytes += c->bytes;
  s->created += 1;
  return c;
}

void launch(bfs_server* s, Context& c) {
  const int k = (int)c.q.size();
  int32_t src[kMaxLanes];
  uint8_t* dl[kMaxLanes];
  int32_t* pl[kMaxLanes];
  for (int j = 0; j < k; ++j) {
    src[j] = c.q[j].source;
    dl[j] = c.q[j].depth;
    pl[j] = c.q[j].parent;
  }
  c.busy = true;
  c.t_launch = now_ns();
  int rc;
  if (c.single) {
    bfs_graph* g;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      g = s->graphs[c.gid].g;
    }
    // back-to-back runs on the graph's run state, each header copied after its run
    rc = BFS_OK;
    for (int i = 0; i < k && rc == BFS_OK; ++i) {
      rc = bfsgb::launch_run(g, src[i], nullptr, s->opt.with_parents ? pl[i] : nullptr, c.stream, c.ctas, dl[i]);
      c.epoch[i] = g->epoch & 0x0FFFFFFFu;
      if (rc == BFS_OK) {
        const cudaError_t e =
            cudaMemcpyAsync(c.hdr + i, g->hdr, sizeof(RunHeader), cudaMemcpyDeviceToHost, c.stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "copy run header");
      }
    }
  } else {
    rc = bfsgb::ms_launch(c.b, src, k, dl, s->opt.with_parents ? pl : nullptr, c.stream, c.hdr, &c.epoch[0]);
  }
  if (rc == BFS_OK) {
    const cudaError_t e = cudaEventRecord(c.ev, c.stream);
    if (e == cudaSuccess) return;
    rc = cuda_fail(e, "record the launch's end");
  }
  cudaStreamSynchronize(c.stream);  // runs already queued finish before the context is reused
  finish(s, c, rc, now_ns());
}

void release_order(bfs_server* s) {
  if (s->order_stream) cudaStreamDestroy(s->order_stream);
  if (s->order_src_h) cudaFreeHost(s->order_src_h);
  if (s->order_key_h) cudaFreeHost(s->order_key_h);
  if (s->order_src_d) cudaFree(s->order_src_d);
  if (s->order_key_d) cudaFree(s->order_key_d);
  s->order_stream = nullptr;
  s->order_src_h = nullptr;
  s->order_key_h = nullptr;
  s->order_src_d = nullptr;
  s->order_key_d = nullptr;
}

// Grouped batch of graph gid when more than cap queries wait: the oldest waiting
// query and the cap-1 queries whose grouping keys (bfs_batch_order's) lie nearest
// it among the oldest kGroupWindow, as ascending positions in the waiting queue.
// Empty: take the queue in arrival order.  Only the worker removes waiting
// queries, so the window's positions hold while the lock is released.
std::vector<int> group_pick(bfs_server* s, int gid, int cap) {
  std::vector<int> pick;
  if (!s->order_stream) return pick;
  int W = 0;
  const bfs_graph* g = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    const std::deque<Query>& w = s->graphs[gid].waiting;
    if ((int)w.size() <= cap) return pick;
    W = (int)std::min<size_t>(w.size(), (size_t)kGroupWindow);
    for (int i = 0; i < W; ++i) s->order_src_h[i] = w[(size_t)i].source;
    g = s->graphs[gid].g;
  }
  cudaError_t e = cudaMemcpyAsync(s->order_src_d, s->order_src_h, sizeof(int32_t) * W, cudaMemcpyHostToDevice,
                                  s->order_stream);
  if (e != cudaSuccess || bfsgb::order_keys_async(g, s->order_src_d, W, s->order_key_d, s->order_stream) != BFS_OK)
    return pick;
  e = cudaMemcpyAsync(s->order_key_h, s->order_key_d, sizeof(unsigned long long) * W, cudaMemcpyDeviceToHost,
                      s->order_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->order_stream);
  if (e != cudaSuccess) return pick;
  std::vector<int> idx((size_t)W);
  for (int i = 0; i < W; ++i) idx[(size_t)i] = i;
  std::stable_sort(idx.begin(), idx.end(),
                   [&](int a, int b) { return s->order_key_h[a] > s->order_key_h[b]; });
  int pos = 0;
  while (idx[(size_t)pos] != 0) ++pos;
  int start = pos - cap / 2;
  if (start > W - cap) start = W - cap;
  if (start < 0) start = 0;
  pick.assign(idx.begin() + start, idx.begin() + start + cap);
  std::sort(pick.begin(), pick.end());
  return pick;
}

void schedule(bfs_server* s) {
  for (;;) {
    std::vector<int> order;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->stop || s->in_flight >= s->opt.max_concurrent) return;
      for (int i = 0; i < (int)s->graphs.size(); ++i)
        if (!s->graphs[i].waiting.empty()) order.push_back(i);
      std::sort(order.begin(), order.end(), [&](int a, int b) {
        const Query& qa = s->graphs[a].waiting.front();
        const Query& qb = s->graphs[b].waiting.front();
        return qa.t_arrival != qb.t_arrival ? qa.t_arrival < qb.t_arrival : qa.ticket < qb.ticket;
      });
    }
    // CTAs: a batch takes its slice; single-source runs take the whole device when
    // nothing else runs, else a slice; launches start only while they all fit
    const int free_ctas = s->capacity - s->ctas_in_use;
    Context* c = nullptr;
    int ctas = 0;
    for (int gid : order) {
      const bfs_graph* g;
      size_t waiting;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        g = s->graphs[gid].g;
        waiting = s->graphs[gid].waiting.size();
      }
      if (free_ctas < s->slice) break;
      if ((int)waiting <= s->opt.single_max && (c = acquire_single(s, gid))) {
        ctas = s->ctas_in_use == 0 ? s->capacity : s->slice;
        break;
      }
      if ((c = acquire_context(s, gid, g))) {
        ctas = s->slice;
        break;
      }
    }
    if (!c) return;
    c->ctas = ctas;
    s->ctas_in_use += ctas;
    const int cap = c->single ? s->opt.single_max : s->opt.max_lanes;
    const std::vector<int> pick = c->single ? std::vector<int>() : group_pick(s, c->gid, cap);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      std::deque<Query>& w = s->graphs[c->gid].waiting;
      if (!pick.empty()) {
        for (int i : pick) c->q.push_back(w[(size_t)i]);
        for (size_t j = pick.size(); j-- > 0;) w.erase(w.begin() + pick[j]);
      }
      while (!w.empty() && (int)c->q.size() < cap) {
        c->q.push_back(w.front());
        w.pop_front();
      }
      s->waiting -= (int64_t)c->q.size();
      s->in_flight += 1;
      s->launches += 1;
      s->lanes += (int64_t)c->q.size();
      if (c->single) s->single_launches += 1;
    }
    launch(s, *c);
  }
}

void worker_main(bfs_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    reap(s);
    schedule(s);
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop && s->in_flight == 0) break;
    if (s->in_flight > 0) {  // poll the launches' end events and the queue
      s->wake = false;
      lk.unlock();
      std::this_thread::yield();
      continue;
    }
    s->cv_work.wait_for(lk, std::chrono::milliseconds(50), [&] { return s->wake; });
    s->wake = false;
  }
  s->cv_done.notify_all();
}

}  // namespace

extern "C" void bfs_server_options_default(bfs_server_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->max_concurrent = 2;
  opt->max_lanes = kMaxLanes;
  opt->with_parents = 1;
  opt->contexts_per_graph = 2;
  opt->single_path = 1;
  opt->single_max = 3;
  opt->group_batches = 1;
}

extern "C" int64_t bfs_server_now_ns(void) { return now_ns(); }

extern "C" int bfs_server_create(const bfs_server_options* opt, bfs_server** out) {
  if (!out) return fail(BFS_ERR_INVALID, "out is NULL");
  *out = nullptr;
  bfs_server_options o;
  if (opt) o = *opt;
  else bfs_server_options_default(&o);
  if (o.max_concurrent == 0) o.max_concurrent = 2;
  if (o.max_lanes == 0) o.max_lanes = kMaxLanes;
  if (o.contexts_per_graph == 0) o.contexts_per_graph = o.max_concurrent;
  if (o.max_concurrent < 1 || o.max_concurrent > kMaxConcurrent) return fail(BFS_ERR_INVALID, "max_concurrent must be 1..8");
  if (o.max_lanes < 1 || o.max_lanes > kMaxLanes) return fail(BFS_ERR_INVALID, "max_lanes must be 1..64");
  if (o.contexts_per_graph < 1 || o.contexts_per_graph > o.max_concurrent)
    return fail(BFS_ERR_INVALID, "contexts_per_graph must be 1..max_concurrent");
  if (o.with_parents != 0 && o.with_parents != 1) return fail(BFS_ERR_INVALID, "with_parents must be 0 or 1");
  if (o.single_path != 0 && o.single_path != 1) return fail(BFS_ERR_INVALID, "single_path must be 0 or 1");
  if (o.single_max < 0 || o.single_max > kMaxSingle) return fail(BFS_ERR_INVALID, "single_max must be 0..4");
  if (!o.single_path) o.single_max = 0;
  else if (o.single_max == 0) o.single_max = 3;
  if (o.hbm_reserve_bytes < 0 || o.hbm_budget_bytes < 0) return fail(BFS_ERR_INVALID, "byte limits must be >= 0");
  if (o.group_batches != 0 && o.group_batches != 1) return fail(BFS_ERR_INVALID, "group_batches must be 0 or 1");
  int dev = 0, cap = 0;
  const cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "bfs_server_create");
  int rc = bfs_batch_capacity(&cap);
  if (rc) return rc;
  if (cap / o.max_concurrent < 1) return fail(BFS_ERR_INVALID, "max_concurrent exceeds the device's CTA capacity");
  bfs_server* s = new (std::nothrow) bfs_server();
  if (!s) return fail(BFS_ERR_OOM, "host allocation failed");
  s->opt = o;
  s->device = dev;
  s->capacity = cap;
  s->slice = cap / o.max_concurrent;
  if (o.group_batches) {
    cudaError_t ge = cudaStreamCreateWithFlags(&s->order_stream, cudaStreamNonBlocking);
    if (ge == cudaSuccess) ge = cudaMallocHost((void**)&s->order_src_h, sizeof(int32_t) * kGroupWindow);
    if (ge == cudaSuccess) ge = cudaMallocHost((void**)&s->order_key_h, sizeof(unsigned long long) * kGroupWindow);
    if (ge == cudaSuccess) ge = cudaMalloc((void**)&s->order_src_d, sizeof(int32_t) * kGroupWindow);
    if (ge == cudaSuccess) ge = cudaMalloc((void**)&s->order_key_d, sizeof(unsigned long long) * kGroupWindow);
    if (ge != cudaSuccess) {
      release_order(s);
      delete s;
      return cuda_fail(ge, "server grouping buffers");
    }
  }
  try {
    s->worker = std::thread(worker_main, s);
  } catch (...) {
    release_order(s);
    delete s;
    return fail(BFS_ERR_OOM, "cannot start the worker thread");
  }
  *out = s;
  return BFS_OK;
}

extern "C" int bfs_server_add_graph(bfs_server* s, bfs_graph* g, int32_t* graph_id) {
  if (!s || !g || !graph_id) return fail(BFS_ERR_INVALID, "server, graph or graph_id is NULL");
  if (g->device != s->device) return fail(BFS_ERR_INVALID, "the graph lives on another device than the server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return fail(BFS_ERR_INVALID, "the server is stopping");
  s->graphs.push_back(GraphEntry{g, {}});
  *graph_id = (int32_t)s->graphs.size() - 1;
  return BFS_OK;
}

extern "C" int bfs_server_submit(bfs_server* s, int32_t graph_id, int32_t source, uint8_t* depth, int32_t* parent,
                                 int64_t t_arrival_ns, int64_t* ticket) {
  if (!s || !depth || !ticket) return fail(BFS_ERR_INVALID, "server, depth or ticket is NULL");
  if ((parent != nullptr) != (s->opt.with_parents == 1))
    return fail(BFS_ERR_INVALID, s->opt.with_parents ? "this server needs a parent buffer" : "this server writes no parents");
  if (!device_ptr(depth) || (parent && !device_ptr(parent)))
    return fail(BFS_ERR_INVALID, "depth and parent must be device buffers");
  const int64_t t = t_arrival_ns ? t_arrival_ns : now_ns();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return fail(BFS_ERR_INVALID, "the server is stopping");
    if (graph_id < 0 || graph_id >= (int32_t)s->graphs.size()) return fail(BFS_ERR_INVALID, "unknown graph id");
    GraphEntry& ge = s->graphs[graph_id];
    if (source < 0 || source >= ge.g->n) return fail(BFS_ERR_INVALID, "source out of range");
    *ticket = s->next_ticket++;
    ge.waiting.push_back(Query{*ticket, source, depth, parent, t});
    s->waiting += 1;
    s->submitted += 1;
    s->wake = true;
  }
  s->cv_work.notify_one();
  return BFS_OK;
}

extern "C" int bfs_server_poll(bfs_server* s, bfs_server_done* done, int32_t max_done, int32_t timeout_ms,
                               int32_t* n_done) {
  if (!s || !n_done || (max_done > 0 && !done)) return fail(BFS_ERR_INVALID, "server, done or n_done is NULL");
  *n_done = 0;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && timeout_ms != 0) {
    auto ready = [&] { return !s->done.empty() || (s->waiting == 0 && s->in_flight == 0) || s->stop; };
    if (timeout_ms < 0) s->cv_done.wait(lk, ready);
    else s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  }
  int32_t n = 0;
  while (n < max_done && !s->done.empty()) {
    done[n++] = s->done.front();
    s->done.pop_front();
  }
  *n_done = n;
  return BFS_OK;
}

extern "C" int bfs_server_get_stats(bfs_server* s, bfs_server_stats* st) {
  if (!s || !st) return fail(BFS_ERR_INVALID, "server or stats is NULL");
  std::memset(st, 0, sizeof(*st));
  std::lock_guard<std::mutex> lk(s->mu);
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->failed = s->failed;
  st->launches = s->launches;
  st->lanes_launched = s->lanes;
  st->single_launches = s->single_launches;
  st->contexts_created = s->created;
  st->contexts_evicted = s->evicted;
  st->context_bytes = s->ctx_bytes;
  st->waiting = s->waiting;
  st->in_flight = s->in_flight;
  st->capacity_ctas = s->capacity;
  st->ctas_per_launch = s->slice;
  return BFS_OK;
}

extern "C" void bfs_server_destroy(bfs_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->wake = true;
  }
  s->cv_work.notify_all();
  s->cv_done.notify_all();
  if (s->worker.joinable()) s->worker.join();
  while (!s->ctx.empty()) drop_context(s, s->ctx.size() - 1);
  release_order(s);
  delete s;
}

extern "C" void bfs_server_abi_sizes(int64_t sizes[3]) {
  if (!sizes) return;
  sizes[0] = (int64_t)sizeof(bfs_server_options);
  sizes[1] = (int64_t)sizeof(bfs_server_done);
  sizes[2] = (int64_t)sizeof(bfs_server_stats);
}
