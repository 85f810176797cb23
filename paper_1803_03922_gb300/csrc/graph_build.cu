// Device graph builder (one-time set-up, not part of a BFS run).
//
// Sec. II-B / VI-A.3: the graph is symmetric (each undirected pair stored both
// ways, self-loops dropped, duplicates removed).  Sec. III-A: vertices with more
// than TH neighbours are delegates.  Fig. 2: delegates get dense ids in ascending
// original id.  Sec. III-C / Table I: int32 column indices.  Every row is sorted
// by the neighbour's caller id so that a backward visit that stops at its first
// visited neighbour returns the smallest-id parent.
//
// The one-time sort, unique and prefix sums use CUB (open-source CCCL headers);
// the classification, renumbering and column scatter are the kernels below.
#include <cub/cub.cuh>

#include <algorithm>
#include <vector>

#include "bfs_internal.cuh"

namespace bfsgb {
namespace {

constexpr int kB = 256;

int grid_for(int64_t items) {
  int64_t b = (items + kB - 1) / kB;
  if (b > 152LL * 32) b = 152LL * 32;
  return b < 1 ? 1 : (int)b;
}

__global__ void k_check_ids(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                            int32_t n, int* __restrict__ bad) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = src[e], v = dst[e];
    if (u < 0 || u >= n || v < 0 || v >= n) atomicExch(bad, 1);
  }
}

// Both directions of every pair as (u << 32 | v); a self-loop becomes the
// sentinel (n << 32), which sorts after every real key and is dropped.
__global__ void k_make_keys(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                            uint64_t sentinel, uint64_t* __restrict__ keys) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    uint64_t u = (uint32_t)src[e], v = (uint32_t)dst[e];
    bool loop = u == v;
    keys[2 * e] = loop ? sentinel : ((u << 32) | v);
    keys[2 * e + 1] = loop ? sentinel : ((v << 32) | u);
  }
}

// Row bounds in the sorted unique key array, by caller id.
__global__ void k_row_bounds(const uint64_t* __restrict__ keys, int64_t M, int64_t* __restrict__ start_c,
                             int64_t* __restrict__ end_c) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t u = (uint32_t)(keys[i] >> 32);
    if (i == 0 || (uint32_t)(keys[i - 1] >> 32) != u) start_c[u] = i;
    if (i == M - 1 || (uint32_t)(keys[i + 1] >> 32) != u) end_c[u] = i + 1;
  }
}

__global__ void k_classify(const int64_t* __restrict__ start_c, const int64_t* __restrict__ end_c, int32_t n,
                           int64_t th, int32_t* __restrict__ fdel, int32_t* __restrict__ fnor) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    int64_t deg = end_c[c] - start_c[c];
    fdel[c] = deg > th ? 1 : 0;
    fnor[c] = (deg > 0 && deg <= th) ? 1 : 0;
  }
}

// Sec. III-A / Fig. 2 renumbering: delegates [0,d), non-isolated normal vertices
// [d,n_ni), isolated vertices [n_ni,n); each class keeps ascending caller order.
__global__ void k_internal_ids(const int32_t* __restrict__ fdel, const int32_t* __restrict__ fnor,
                               const int32_t* __restrict__ sdel, const int32_t* __restrict__ snor,
                               const int64_t* __restrict__ start_c, const int64_t* __restrict__ end_c, int32_t n,
                               int32_t d, int32_t n_ni, int32_t* __restrict__ internal_of,
                               int32_t* __restrict__ caller_of, int64_t* __restrict__ deg_int) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
    int32_t id;
    if (fdel[c])
      id = sdel[c];
    else if (fnor[c])
      id = d + snor[c];
    else
      id = n_ni + (int32_t)(c - sdel[c] - snor[c]);
    internal_of[c] = id;
    caller_of[id] = (int32_t)c;
    if (id < n_ni) deg_int[id] = end_c[c] - start_c[c];
  }
}

// Caller-rank words: for caller ids [32w, 32w+32), which are delegates and which
// non-isolated normal vertices, and how many of each precede 32w.  Both classes
// are numbered in caller order, so a caller id's internal id is its class base
// plus its rank: the level loop's result pass reads 16 bytes per 32 caller ids
// instead of internal_of.
__global__ void k_caller_rank(const int32_t* __restrict__ fdel, const int32_t* __restrict__ fnor,
                              const int32_t* __restrict__ sdel, const int32_t* __restrict__ snor, int32_t n,
                              int4* __restrict__ crank) {
  const int64_t nw = ((int64_t)n + 31) / 32;
  for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < nw; w += (int64_t)gridDim.x * blockDim.x) {
    unsigned md = 0, mn = 0;
    const int64_t c0 = w * 32;
    for (int b = 0; b < 32 && c0 + b < n; ++b) {
      md |= (unsigned)(fdel[c0 + b] != 0) << b;
      mn |= (unsigned)(fnor[c0 + b] != 0) << b;
    }
    crank[w] = make_int4((int)md, (int)mn, sdel[c0], snor[c0]);
  }
}

// Column scatter: entry i of caller row u lands at off[internal(u)] + (i - start_c[u])
// and stores internal(v); rows stay in ascending caller id of the neighbour.
// Also counts the nn/nd/dn/dd entries (Sec. IV) with the class of each endpoint.
__global__ void k_scatter_cols(const uint64_t* __restrict__ keys, int64_t M, const int64_t* __restrict__ start_c,
                               const int32_t* __restrict__ internal_of, const int64_t* __restrict__ off, int32_t d,
                               int32_t* __restrict__ col, unsigned long long* __restrict__ sub) {
  __shared__ unsigned long long s[4];
  if (threadIdx.x < 4) s[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long loc[4] = {0, 0, 0, 0};
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = keys[i];
    uint32_t u = (uint32_t)(k >> 32), v = (uint32_t)(k & 0xFFFFFFFFu);
    int32_t ui = internal_of[u], vi = internal_of[v];
    col[off[ui] + (i - start_c[u])] = vi;
    loc[((ui < d) << 1) | (vi < d)] += 1;
  }
  for (int j = 0; j < 4; ++j)
    if (loc[j]) atomicAdd(&s[j], loc[j]);
  __syncthreads();
  if (threadIdx.x < 4 && s[threadIdx.x]) atomicAdd(&sub[threadIdx.x], s[threadIdx.x]);
}

// Largest degree, the chunk-list capacity sum_{v<d} ceil(deg(v)/kChunk), and the
// number of rows longer than kHead + kShort (capacity of the long-row list).
__global__ void k_degree_stats(const int64_t* __restrict__ off, int32_t n_ni, int32_t d,
                               unsigned long long* __restrict__ out /* [0]=max deg, [1]=chunks, [2]=long rows */) {
  unsigned long long mx = 0, ch = 0, lg = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n_ni; v += (int64_t)gridDim.x * blockDim.x) {
    int64_t deg = off[v + 1] - off[v];
    mx = deg > (int64_t)mx ? (unsigned long long)deg : mx;
    if (v < d) ch += (deg + kChunk - 1) / kChunk;
    if (deg > kHead + kShort) lg += 1;
  }
  atomicMax(&out[0], mx);
  if (ch) atomicAdd(&out[1], ch);
  if (lg) atomicAdd(&out[2], lg);
}

// Per-vertex head record: the first kHead row entries (internal ids, -1 past the
// end) and their caller ids (with kHead = 4 one 32-byte sector per vertex; with
// 2 the four ints share one 16-byte word), plus an int32 degree array.  A backward scan that settles within the first entries reads only this
// sector, indexed by the vertex itself (coalesced across a warp).  The lead
// record is the first entry and its caller id alone (8 bytes): dense backward
// levels, where the first entry settles most vertices, read only that.
__global__ void k_heads(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                        const int32_t* __restrict__ caller_of, int32_t n_ni, int4* __restrict__ head,
                        int32_t* __restrict__ deg, int2* __restrict__ lead) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n_ni; v += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = off[v], e = off[v + 1];
    int nb[kHead], cid[kHead];
#pragma unroll
    for (int t = 0; t < kHead; ++t) {
      nb[t] = (b + t < e) ? col[b + t] : -1;
      cid[t] = nb[t] >= 0 ? caller_of[nb[t]] : -1;
    }
    if constexpr (kHead == 2) {
      head[v] = make_int4(nb[0], nb[1], cid[0], cid[1]);
    } else {
#pragma unroll
      for (int t = 0; t < kHead; t += 4) {
        head[kHeadVecs * v + t / 4] = make_int4(nb[t], nb[t + 1], nb[t + 2], nb[t + 3]);
        head[kHeadVecs * v + kHead / 4 + t / 4] = make_int4(cid[t], cid[t + 1], cid[t + 2], cid[t + 3]);
      }
    }
    deg[v] = (int32_t)(e - b);
    lead[v] = make_int2(nb[0], cid[0]);
  }
}

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { reset(); }
  void reset() {
    if (p) cudaFree(p);
    p = nullptr;
  }
  template <class T>
  T* as() const { return (T*)p; }
};

int dalloc(DevBuf& b, size_t bytes, const char* what) {
  cudaError_t e = cudaMalloc(&b.p, bytes > 0 ? bytes : 1);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return fail(BFS_ERR_OOM, std::string("device allocation failed: ") + what + " (" +
                                 std::to_string(bytes) + " bytes)");
  }
  return BFS_OK;
}

#define BFS_TRY(x)        \
  do {                    \
    int _rc = (x);        \
    if (_rc) return _rc;  \
  } while (0)
#define BFS_CUDA(x, what)                         \
  do {                                            \
    cudaError_t _e = (x);                         \
    if (_e != cudaSuccess) return cuda_fail(_e, what); \
  } while (0)

int bitlen(uint32_t x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

}  // namespace

int build_graph(const int32_t* src, const int32_t* dst, int64_t m, int32_t n, const bfs_options& opt,
                bfs_graph* g, cudaStream_t s) {
  if (m > (INT64_MAX / 2) - 1) return fail(BFS_ERR_OVERFLOW, "num_edges too large");
  const int64_t M2 = 2 * m;
  BFS_CUDA(cudaGetDevice(&g->device), "cudaGetDevice");
  g->n = n;
  g->th = opt.th;
  g->opt = opt;

  // 1. edges on the device
  DevBuf esrc, edst;
  const int32_t* dsrc = src;
  const int32_t* ddst = dst;
  if (!opt.edges_on_device && m > 0) {
    BFS_TRY(dalloc(esrc, (size_t)m * 4, "edge src"));
    BFS_TRY(dalloc(edst, (size_t)m * 4, "edge dst"));
    BFS_CUDA(cudaMemcpyAsync(esrc.p, src, (size_t)m * 4, cudaMemcpyHostToDevice, s), "copy edges");
    BFS_CUDA(cudaMemcpyAsync(edst.p, dst, (size_t)m * 4, cudaMemcpyHostToDevice, s), "copy edges");
    dsrc = esrc.as<int32_t>();
    ddst = edst.as<int32_t>();
  }
  // 2. ids in range
  DevBuf bad;
  BFS_TRY(dalloc(bad, sizeof(int) * 4, "flag"));
  BFS_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int) * 4, s), "memset");
  if (m > 0) k_check_ids<<<grid_for(m), kB, 0, s>>>(dsrc, ddst, m, n, bad.as<int>());
  int hbad = 0;
  BFS_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s), "copy flag");
  BFS_CUDA(cudaStreamSynchronize(s), "check ids");
  if (hbad) return fail(BFS_ERR_INVALID, "an edge endpoint lies outside [0, num_vertices)");

  // 3. keys, sort, unique
  DevBuf ka, kb, nsel, tmp;
  int64_t M = 0;
  if (M2 > 0) {
    BFS_TRY(dalloc(ka, (size_t)M2 * 8, "sort keys"));
    BFS_TRY(dalloc(kb, (size_t)M2 * 8, "sort keys"));
    BFS_TRY(dalloc(nsel, 16, "count"));
    const uint64_t sentinel = (uint64_t)(uint32_t)n << 32;
    k_make_keys<<<grid_for(m), kB, 0, s>>>(dsrc, ddst, m, sentinel, ka.as<uint64_t>());
    BFS_CUDA(cudaGetLastError(), "k_make_keys");
    esrc.reset();
    edst.reset();
    const int end_bit = 32 + bitlen((uint32_t)n);
    cub::DoubleBuffer<uint64_t> db(ka.as<uint64_t>(), kb.as<uint64_t>());
    size_t t_sort = 0, t_uniq = 0;
    BFS_CUDA(cub::DeviceRadixSort::SortKeys(nullptr, t_sort, db, M2, 0, end_bit, s), "sort size");
    BFS_CUDA(cub::DeviceSelect::Unique(nullptr, t_uniq, ka.as<uint64_t>(), kb.as<uint64_t>(),
                                       nsel.as<int64_t>(), M2, s),
             "unique size");
    BFS_TRY(dalloc(tmp, std::max(t_sort, t_uniq), "cub temp"));
    BFS_CUDA(cub::DeviceRadixSort::SortKeys(tmp.p, t_sort, db, M2, 0, end_bit, s), "sort");
    uint64_t* sorted = db.Current();
    uint64_t* other = db.Alternate();
    BFS_CUDA(cub::DeviceSelect::Unique(tmp.p, t_uniq, sorted, other, nsel.as<int64_t>(), M2, s), "unique");
    int64_t cnt = 0;
    BFS_CUDA(cudaMemcpyAsync(&cnt, nsel.p, 8, cudaMemcpyDeviceToHost, s), "copy count");
    BFS_CUDA(cudaStreamSynchronize(s), "unique");
    M = cnt;
    if (M > 0) {
      uint64_t last = 0;
      BFS_CUDA(cudaMemcpy(&last, other + (M - 1), 8, cudaMemcpyDeviceToHost), "copy key");
      if (last == sentinel) --M;
    }
    // keep the unique keys in ka
    if (other != ka.as<uint64_t>()) std::swap(ka.p, kb.p);
  }
  kb.reset();
  tmp.reset();
  g->nnz = M;

  // 4. degrees and classes
  DevBuf start_c, end_c, fdel, fnor, sdel, snor;
  BFS_TRY(dalloc(start_c, (size_t)n * 8, "row starts"));
  BFS_TRY(dalloc(end_c, (size_t)n * 8, "row ends"));
  BFS_CUDA(cudaMemsetAsync(start_c.p, 0, (size_t)n * 8, s), "memset");
  BFS_CUDA(cudaMemsetAsync(end_c.p, 0, (size_t)n * 8, s), "memset");
  if (M > 0) k_row_bounds<<<grid_for(M), kB, 0, s>>>(ka.as<uint64_t>(), M, start_c.as<int64_t>(), end_c.as<int64_t>());
  BFS_TRY(dalloc(fdel, (size_t)n * 4, "flags"));
  BFS_TRY(dalloc(fnor, (size_t)n * 4, "flags"));
  BFS_TRY(dalloc(sdel, (size_t)n * 4, "scan"));
  BFS_TRY(dalloc(snor, (size_t)n * 4, "scan"));
  k_classify<<<grid_for(n), kB, 0, s>>>(start_c.as<int64_t>(), end_c.as<int64_t>(), n, opt.th, fdel.as<int32_t>(),
                                        fnor.as<int32_t>());
  {
    size_t t1 = 0;
    BFS_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, t1, fdel.as<int32_t>(), sdel.as<int32_t>(), n, s), "scan size");
    DevBuf t;
    BFS_TRY(dalloc(t, t1, "scan temp"));
    BFS_CUDA(cub::DeviceScan::ExclusiveSum(t.p, t1, fdel.as<int32_t>(), sdel.as<int32_t>(), n, s), "scan");
    BFS_CUDA(cub::DeviceScan::ExclusiveSum(t.p, t1, fnor.as<int32_t>(), snor.as<int32_t>(), n, s), "scan");
    int32_t h[4];
    BFS_CUDA(cudaMemcpyAsync(&h[0], sdel.as<int32_t>() + (n - 1), 4, cudaMemcpyDeviceToHost, s), "copy");
    BFS_CUDA(cudaMemcpyAsync(&h[1], fdel.as<int32_t>() + (n - 1), 4, cudaMemcpyDeviceToHost, s), "copy");
    BFS_CUDA(cudaMemcpyAsync(&h[2], snor.as<int32_t>() + (n - 1), 4, cudaMemcpyDeviceToHost, s), "copy");
    BFS_CUDA(cudaMemcpyAsync(&h[3], fnor.as<int32_t>() + (n - 1), 4, cudaMemcpyDeviceToHost, s), "copy");
    BFS_CUDA(cudaStreamSynchronize(s), "class counts");
    g->d = h[0] + h[1];
    g->n_ni = g->d + h[2] + h[3];
  }

  // 5. renumbering, offsets, columns
  int64_t dev_bytes = 0;
  BFS_CUDA(cudaMalloc(&g->internal_of, ((size_t)n + 4) * 4), "alloc internal_of");
  BFS_CUDA(cudaMemsetAsync(g->internal_of, 0x7F, ((size_t)n + 4) * 4, s), "memset");
  BFS_CUDA(cudaMalloc(&g->caller_of, (size_t)n * 4), "alloc caller_of");
  BFS_CUDA(cudaMalloc(&g->off, ((size_t)g->n_ni + 1) * 8), "alloc row offsets");
  dev_bytes += (int64_t)n * 8 + ((int64_t)g->n_ni + 1) * 8;
  DevBuf deg_int;
  BFS_TRY(dalloc(deg_int, ((size_t)g->n_ni + 1) * 8, "degrees"));
  BFS_CUDA(cudaMemsetAsync(deg_int.p, 0, ((size_t)g->n_ni + 1) * 8, s), "memset");
  k_internal_ids<<<grid_for(n), kB, 0, s>>>(fdel.as<int32_t>(), fnor.as<int32_t>(), sdel.as<int32_t>(),
                                            snor.as<int32_t>(), start_c.as<int64_t>(), end_c.as<int64_t>(), n, g->d,
                                            g->n_ni, g->internal_of, g->caller_of, deg_int.as<int64_t>());
  BFS_CUDA(cudaMalloc(&g->crank, (((size_t)n + 31) / 32 + 1) * sizeof(int4)), "alloc caller ranks");
  dev_bytes += (((int64_t)n + 31) / 32 + 1) * 16;
  k_caller_rank<<<grid_for(((int64_t)n + 31) / 32), kB, 0, s>>>(fdel.as<int32_t>(), fnor.as<int32_t>(), sdel.as<int32_t>(),
                                                               snor.as<int32_t>(), n, g->crank);
  {
    size_t t1 = 0;
    BFS_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, t1, deg_int.as<int64_t>(), g->off, (int64_t)g->n_ni + 1, s),
             "scan size");
    DevBuf t;
    BFS_TRY(dalloc(t, t1, "scan temp"));
    BFS_CUDA(cub::DeviceScan::ExclusiveSum(t.p, t1, deg_int.as<int64_t>(), g->off, (int64_t)g->n_ni + 1, s), "scan");
  }
  BFS_CUDA(cudaMalloc(&g->col, ((size_t)M + kColPad) * 4), "alloc columns");
  BFS_CUDA(cudaMemsetAsync(g->col, 0, ((size_t)M + kColPad) * 4, s), "memset");
  dev_bytes += ((int64_t)M + kColPad) * 4;
  DevBuf sub;
  BFS_TRY(dalloc(sub, 8 * 8, "counts"));
  BFS_CUDA(cudaMemsetAsync(sub.p, 0, 8 * 8, s), "memset");
  if (M > 0)
    k_scatter_cols<<<grid_for(M), kB, 0, s>>>(ka.as<uint64_t>(), M, start_c.as<int64_t>(), g->internal_of, g->off,
                                              g->d, g->col, sub.as<unsigned long long>());
  BFS_CUDA(cudaMalloc(&g->head, ((size_t)g->n_ni + 1) * kHeadVecs * sizeof(int4)), "alloc head records");
  BFS_CUDA(cudaMalloc(&g->deg, ((size_t)g->n_ni + 4) * 4), "alloc degrees");
  BFS_CUDA(cudaMalloc(&g->lead, ((size_t)g->n_ni + 1) * sizeof(int2)), "alloc lead records");
  dev_bytes += ((int64_t)g->n_ni + 1) * kHeadVecs * 16 + ((int64_t)g->n_ni + 4) * 4 + ((int64_t)g->n_ni + 1) * 8;
  if (g->n_ni > 0) {
    k_degree_stats<<<grid_for(g->n_ni), kB, 0, s>>>(g->off, g->n_ni, g->d, sub.as<unsigned long long>() + 4);
    k_heads<<<grid_for(g->n_ni), kB, 0, s>>>(g->off, g->col, g->caller_of, g->n_ni, g->head, g->deg, g->lead);
  }
  BFS_CUDA(cudaGetLastError(), "builder kernels");
  unsigned long long hs[8];
  BFS_CUDA(cudaMemcpyAsync(hs, sub.p, sizeof(hs), cudaMemcpyDeviceToHost, s), "copy counts");
  BFS_CUDA(cudaStreamSynchronize(s), "build");
  for (int j = 0; j < 4; ++j) g->sub[j] = (int64_t)hs[j];
  g->max_deg = (int64_t)hs[4];
  g->cl_cap = (int64_t)hs[5] + 1;
  g->long_cap = (int64_t)hs[6] + 1;
  g->device_bytes = dev_bytes;
  return BFS_OK;
}

}  // namespace bfsgb
