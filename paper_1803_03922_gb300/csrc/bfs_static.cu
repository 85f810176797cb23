// bfs_run_static: a BFS entry point that allocates nothing.
//
// Some callers cannot call cudaMalloc: code running inside another runtime
// that owns the device allocator (a plugin or an embedding host with its own
// memory pool), or a process whose allocation budget is fixed before it starts.
// For them this file provides one level-loop variant whose scratch (visited and
// discovered bitmaps, counters, the grid-barrier words) lives in a file-scope
// __device__ array of fixed size, loaded with the module.  The caller passes
// its own symmetric CSR and its own result buffers.
//
// The variant runs the same direction-optimized loop as bfs_run (forward
// levels with atomicMin canonical parents, backward levels that stop at the
// first visited neighbour of a sorted row, Beamer alpha = 15 / beta = 18), but
// on the caller's ids directly: no degree separation and no renumbering.
#include <climits>
#include <mutex>

#include "bfs_internal.cuh"

namespace bfsgb {
namespace {

constexpr int64_t kStaticMaxVertices = (int64_t)1 << 24;
constexpr int64_t kStaticWords = kStaticMaxVertices / 32;
constexpr int kStaticThreads = 512;

struct StaticHeader {
  unsigned int bar_count;
  unsigned int bar_gen;
  unsigned int err;     // (epoch << 4) | -BFS_ERR_*
  unsigned int exited;  // CTAs that left the kernel
  unsigned long long n_f[2], m_f[2];  // next-frontier counters, by level parity
  unsigned long long pad[10];
};
// rows longer than this are walked by the whole warp (forward) or scanned by it (backward)
constexpr int64_t kStaticWarpRow = 32;
static_assert(sizeof(StaticHeader) <= 256, "header fits its slot");

// Scratch shared by every call on this device: a 256-byte header, then the
// visited bitmap V and two frontier bitmaps A and B (kStaticWords words each).
constexpr size_t kStaticBytes = 256 + 3 * (size_t)kStaticWords * 4;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

struct StaticParams {
  const int64_t* off;
  const int32_t* col;
  int32_t* depth;
  int32_t* parent;
  unsigned char* scratch;  // device address of g_static_scratch
  int32_t n, src;
  int64_t nnz;
  unsigned int epoch;
  unsigned long long timeout_ns;
};

__device__ __forceinline__ unsigned long long st_timer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned st_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ bool st_failed(const StaticParams& p, StaticHeader* h) {
  const unsigned e = *(volatile unsigned*)&h->err;
  return e != 0 && (e >> 4) == (p.epoch & 0x0FFFFFFFu);
}

// Grid barrier with a %globaltimer deadline (cooperative launch).
__device__ bool st_sync(const StaticParams& p, StaticHeader* h) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g0 = st_acquire(&h->bar_gen);
    __threadfence();
    if (atomicAdd(&h->bar_count, 1u) == gridDim.x - 1) {
      atomicExch(&h->bar_count, 0u);
      __threadfence();
      atomicAdd(&h->bar_gen, 1u);
    } else {
      const unsigned long long t0 = st_timer();
      while (st_acquire(&h->bar_gen) == g0) {
        if (st_failed(p, h)) {
          ok = 0;
          break;
        }
        if (st_timer() - t0 > p.timeout_ns) {
          atomicExch(&h->err, ((p.epoch & 0x0FFFFFFFu) << 4) | (unsigned)(-BFS_ERR_TIMEOUT));
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (ok && st_failed(p, h)) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// One forward row entry u->v: an unvisited target offers u as its parent
// (atomicMin keeps the smallest) and sets its bit in N.
__device__ __forceinline__ void st_push(const StaticParams& p, const uint32_t* V, uint32_t* N, int u, int v) {
  if ((V[v >> 5] >> (v & 31)) & 1u) return;
  atomicMin(p.parent + v, u);
  atomicOr(N + (v >> 5), 1u << (v & 31));
}

__device__ void st_body(const StaticParams& p) {
  StaticHeader* h = reinterpret_cast<StaticHeader*>(p.scratch);
  uint32_t* V = reinterpret_cast<uint32_t*>(p.scratch + 256);
  uint32_t* A = V + kStaticWords;
  uint32_t* B = A + kStaticWords;
  __shared__ int s_dir, s_done;
  __shared__ long long s_mu;
  __shared__ unsigned long long s_prev;
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gth = (int64_t)gridDim.x * blockDim.x;
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = gtid >> 5, nwarps = gth >> 5;
  const int64_t W = ((int64_t)p.n + 31) / 32;
  const int sw = p.src >> 5;
  const unsigned sbit = 1u << (p.src & 31);

  // set-up: bitmaps (the source is the frontier of level 0, held in A), results
  for (int64_t w = gtid; w < W; w += gth) {
    V[w] = w == sw ? sbit : 0u;
    A[w] = w == sw ? sbit : 0u;
    B[w] = 0u;
  }
  for (int64_t v = gtid; v < p.n; v += gth) {
    p.depth[v] = v == p.src ? 0 : -1;
    p.parent[v] = v == p.src ? p.src : INT_MAX;
  }
  // the caller's CSR: offsets non-decreasing within [0, nnz], columns in [0, n);
  // anything else ends the run with BFS_ERR_INVALID before a row is read
  bool bad = false;
  for (int64_t v = gtid; v < p.n; v += gth) {
    const int64_t o0 = p.off[v], o1 = p.off[v + 1];
    bad |= o0 < 0 || o0 > o1 || o1 > p.nnz;
  }
  if (__syncthreads_or(bad)) {
    if (threadIdx.x == 0) atomicExch(&h->err, ((p.epoch & 0x0FFFFFFFu) << 4) | (unsigned)(-BFS_ERR_INVALID));
  } else {
    for (int64_t j = gtid; j < p.nnz; j += gth) {
      const int c = p.col[j];
      bad |= c < 0 || c >= p.n;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0)
      atomicExch(&h->err, ((p.epoch & 0x0FFFFFFFu) << 4) | (unsigned)(-BFS_ERR_INVALID));
  }
  if (!st_sync(p, h)) return;
  const long long sdeg = (long long)(p.off[p.src + 1] - p.off[p.src]);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    h->n_f[0] = h->n_f[1] = h->m_f[0] = h->m_f[1] = 0;
  }
  if (threadIdx.x == 0) {
    s_dir = 0;
    s_done = sdeg == 0;
    s_mu = (long long)p.nnz - sdeg;
    s_prev = 1;
  }
  if (!st_sync(p, h)) return;

  for (int L = 0; !s_done; ++L) {
    if (threadIdx.x == 0 && L > p.n + 1)
      atomicExch(&h->err, ((p.epoch & 0x0FFFFFFFu) << 4) | (unsigned)(-BFS_ERR_TIMEOUT));
    uint32_t* F = (L & 1) ? B : A;  // frontier F_L
    uint32_t* N = (L & 1) ? A : B;  // discovered in level L (cleared)
    const int dir = s_dir;
    unsigned long long nf = 0, mf = 0;
    if (dir == 0) {
      // forward: the set bits of F, 32 words per warp (lane i owns word i); a
      // lane walks a short row alone, the warp walks long rows together
      for (int64_t w0 = gwarp * 32; w0 < W; w0 += nwarps * 32) {
        const int64_t w = w0 + lane;
        unsigned fb = w < W ? F[w] : 0u;
        while (__any_sync(kFull, fb != 0)) {
          int u = -1;
          int64_t b = 0, e = 0;
          if (fb) {
            u = (int)(w * 32 + __ffs(fb) - 1);
            fb &= fb - 1;
            b = p.off[u];
            e = p.off[u + 1];
          }
          const bool wide = u >= 0 && e - b > kStaticWarpRow;
          if (u >= 0 && !wide)
            for (int64_t j = b; j < e; ++j) st_push(p, V, N, u, p.col[j]);
          for (unsigned lm = __ballot_sync(kFull, wide); lm; lm &= lm - 1) {
            const int l = __ffs(lm) - 1;
            const int uu = __shfl_sync(kFull, u, l);
            const int64_t rb = __shfl_sync(kFull, b, l), re = __shfl_sync(kFull, e, l);
            for (int64_t j0 = rb; j0 < re; j0 += 128) {  // four loads in flight per lane
              int c[4];
#pragma unroll
              for (int t = 0; t < 4; ++t) {
                const int64_t j = j0 + lane + 32 * t;
                c[t] = j < re ? p.col[j] : -1;
              }
#pragma unroll
              for (int t = 0; t < 4; ++t)
                if (c[t] >= 0) st_push(p, V, N, uu, c[t]);
            }
          }
        }
      }
    } else {
      // backward: every unvisited vertex scans its sorted row to the first
      // visited neighbour; 32 words per warp, long rows scanned by the warp
      for (int64_t w0 = gwarp * 32; w0 < W; w0 += nwarps * 32) {
        const int64_t w = w0 + lane;
        unsigned unv = 0;
        if (w < W) {
          unv = ~V[w];
          if (w == W - 1 && (p.n & 31)) unv &= (1u << (p.n & 31)) - 1u;
        }
        unsigned found = 0;
        while (__any_sync(kFull, unv != 0)) {
          int v = -1, i = 0, hit = -1;
          int64_t b = 0, e = 0;
          if (unv) {
            i = __ffs(unv) - 1;
            unv &= unv - 1;
            v = (int)(w * 32 + i);
            b = p.off[v];
            e = p.off[v + 1];
          }
          const bool wide = v >= 0 && e - b > kStaticWarpRow;
          if (v >= 0 && !wide)
            for (int64_t j = b; j < e; ++j) {
              const int c = p.col[j];
              if ((V[c >> 5] >> (c & 31)) & 1u) {
                hit = c;
                break;
              }
            }
          for (unsigned lm = __ballot_sync(kFull, wide); lm; lm &= lm - 1) {
            const int l = __ffs(lm) - 1;
            const int64_t rb = __shfl_sync(kFull, b, l), re = __shfl_sync(kFull, e, l);
            int h2 = -1;
            for (int64_t j0 = rb; j0 < re; j0 += 32) {  // the first visited entry in row order
              const int64_t j = j0 + lane;
              const int c = j < re ? p.col[j] : -1;
              const unsigned hb = __ballot_sync(kFull, c >= 0 && ((V[c >> 5] >> (c & 31)) & 1u));
              if (hb) {
                h2 = __shfl_sync(kFull, c, __ffs(hb) - 1);
                break;
              }
            }
            if (lane == l) hit = h2;
          }
          if (hit >= 0) {
            p.parent[v] = hit;
            p.depth[v] = L + 1;
            found |= 1u << i;
            nf += 1;
            mf += (unsigned long long)(e - b);
          }
        }
        if (found) N[w] = found;
      }
    }
    if (!st_sync(p, h)) return;
    // level end: merge N into V, clear F for reuse, count and (forward) write depths
    for (int64_t w = gtid; w < W; w += gth) {
      const unsigned nb = __ldcg(N + w);
      F[w] = 0u;
      if (!nb) continue;
      V[w] |= nb;
      if (dir == 0) {
        unsigned x = nb;
        while (x) {
          const int v = (int)(w * 32 + __ffs(x) - 1);
          x &= x - 1;
          p.depth[v] = L + 1;
          nf += 1;
          mf += (unsigned long long)(p.off[v + 1] - p.off[v]);
        }
      }
    }
    if (nf) atomicAdd(&h->n_f[L & 1], nf);
    if (mf) atomicAdd(&h->m_f[L & 1], mf);
    if (!st_sync(p, h)) return;
    if (threadIdx.x == 0) {
      const unsigned long long n1 = __ldcg(&h->n_f[L & 1]), m1 = __ldcg(&h->m_f[L & 1]);
      s_mu -= (long long)m1;
      if (n1 == 0) {
        s_done = 1;
      } else if (dir == 0) {
        s_dir = (long long)(m1 * 15ull) > s_mu ? 1 : 0;
      } else {
        s_dir = (n1 * 18ull < (unsigned long long)p.n && n1 < s_prev) ? 0 : 1;
      }
      s_prev = n1;
    }
    // the other parity's counters were last read before this level: clear them for level L+1
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      h->n_f[(L + 1) & 1] = 0;
      h->m_f[(L + 1) & 1] = 0;
    }
    __syncthreads();
  }
  for (int64_t v = gtid; v < p.n; v += gth)
    if (p.parent[v] == INT_MAX) p.parent[v] = -1;
}

__global__ void __launch_bounds__(kStaticThreads, 2) bfs_static_loop(StaticParams p) {
  st_body(p);
  __syncthreads();
  if (threadIdx.x == 0) {
    StaticHeader* h = reinterpret_cast<StaticHeader*>(p.scratch);
    __threadfence();
    if (atomicAdd(&h->exited, 1u) == gridDim.x - 1) {
      atomicExch(&h->bar_count, 0u);
      atomicExch(&h->exited, 0u);
      __threadfence();
    }
  }
}

// Device address of the scratch array and the grid size, per device, set up by
// the first call on that device.
struct StaticDeviceState {
  unsigned char* scratch = nullptr;
  int grid = 0;
};
std::mutex g_static_mu;
StaticDeviceState g_static_dev[64];
unsigned int g_static_epoch = 0;

}  // namespace
}  // namespace bfsgb

using namespace bfsgb;

extern "C" int bfs_run_static(const int64_t* row_off, const int32_t* col, int32_t n, int32_t source, int32_t* depth,
                              int32_t* parent, struct CUstream_st* stream) {
  if (!row_off || !col || !depth || !parent) return fail(BFS_ERR_INVALID, "a pointer argument is NULL");
  if (n <= 0) return fail(BFS_ERR_INVALID, "n must be >= 1");
  if ((int64_t)n > kStaticMaxVertices)
    return fail(BFS_ERR_OVERFLOW, "bfs_run_static supports at most 16777216 vertices (its fixed scratch size)");
  if (source < 0 || source >= n) return fail(BFS_ERR_INVALID, "source out of range");
  {
    const void* ptrs[4] = {row_off, col, depth, parent};
    for (const void* q : ptrs) {
      cudaPointerAttributes a;
      if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
        cudaGetLastError();
        return fail(BFS_ERR_INVALID, "bfs_run_static takes device pointers only");
      }
      if (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)
        return fail(BFS_ERR_INVALID, "bfs_run_static takes device pointers only");
    }
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) return fail(BFS_ERR_INVALID, "device ordinal above 63");
  StaticParams p;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    StaticDeviceState& st = g_static_dev[dev];
    if (!st.scratch) {
      // host code cannot use g_static_scratch's name as a device address: ask the runtime
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_static_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
      int sms = 0, per_sm = 0, coop = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return cuda_fail(e, "device attributes");
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
      if (!coop) return fail(BFS_ERR_CUDA, "device does not support cooperative launch");
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bfs_static_loop, kStaticThreads, 0);
      if (e != cudaSuccess) return cuda_fail(e, "occupancy");
      if (per_sm < 1) return fail(BFS_ERR_CUDA, "static level-loop kernel does not fit on an SM");
      st.scratch = (unsigned char*)ptr;
      st.grid = sms * (per_sm < 2 ? per_sm : 2);
    }
    p.scratch = st.scratch;
    p.epoch = (++g_static_epoch) & 0x0FFFFFFFu;
    if (p.epoch == 0) p.epoch = (++g_static_epoch) & 0x0FFFFFFFu;
  }
  int64_t nnz = 0;
  e = cudaMemcpyAsync(&nnz, row_off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "read row_off[n]");
  if (nnz < 0) return fail(BFS_ERR_INVALID, "row_off[n] is negative");
  p.off = row_off;
  p.col = col;
  p.depth = depth;
  p.parent = parent;
  p.n = n;
  p.src = source;
  p.nnz = nnz;
  // every barrier wait is bounded: 2 s, plus 4 ns per row entry so that a valid
  // graph with very long rows cannot reach the bound
  p.timeout_ns = 2000ull * 1000000ull + 4ull * (unsigned long long)nnz;
  void* args[] = {&p};
  const int grid = g_static_dev[dev].grid;
  e = cudaLaunchCooperativeKernel((const void*)bfs_static_loop, dim3(grid), dim3(kStaticThreads), args, 0,
                                  (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "static level-loop launch");
  unsigned int err = 0;
  e = cudaMemcpyAsync(&err, p.scratch + 8, sizeof(unsigned int), cudaMemcpyDeviceToHost, (cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "bfs_run_static");
  if (err != 0 && (err >> 4) == p.epoch) {
    const int code = -(int)(err & 0xFu);
    return fail(code, code == BFS_ERR_TIMEOUT   ? "a device-side wait of bfs_run_static passed its deadline"
                      : code == BFS_ERR_INVALID ? "bfs_run_static: row offsets not non-decreasing within "
                                                  "[0, row_off[n]], or a column outside [0, n)"
                                                : "bfs_run_static reported an error");
  }
  return BFS_OK;
}
