// Degree-class statistics for a sweep of thresholds (Sec. VI-B, Figs. 5 and 7):
// for each TH, the number of delegates (degree > TH, Sec. III-A) and the
// directed entries of the four subgraphs nn, nd, dn, dd (Sec. IV).  Degrees do
// not depend on TH, so one pass over the built graph makes three histograms:
// vertex degree, and for every entry (v, u) the larger and the smaller of
// deg(v) and deg(u).  Then, for any TH,
//   delegates = #{v : deg(v) > TH},
//   |E_nn| = #{entries : max <= TH},  |E_dd| = #{entries : min > TH},
//   |E_nd| = |E_dn| = (nnz - |E_nn| - |E_dd|) / 2   (each pair is stored both ways).
#include <cstring>
#include <vector>

#include "bfs_internal.cuh"
#include "device_common.cuh"

namespace bfsgb {
namespace {

constexpr int kSmallBins = 1024;  // low degrees, counted in shared memory first

__device__ __forceinline__ void hist_add(unsigned int* s, unsigned long long* g, int64_t bin) {
  if (bin < kSmallBins) atomicAdd(s + bin, 1u);
  else atomicAdd(g + bin, 1ull);
}

// One warp per 32 consecutive vertices; their rows are contiguous, so the warp
// walks the entries 32 per step and finds each entry's row by a binary search
// over the lanes' row ends.
__global__ void __launch_bounds__(512) k_class_hist(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                                                    const int32_t* __restrict__ deg, int32_t n_ni, int64_t nbins,
                                                    unsigned long long* __restrict__ hdeg,
                                                    unsigned long long* __restrict__ hmax,
                                                    unsigned long long* __restrict__ hmin) {
  __shared__ unsigned int s_deg[kSmallBins], s_max[kSmallBins], s_min[kSmallBins];
  for (int i = threadIdx.x; i < kSmallBins; i += blockDim.x) s_deg[i] = s_max[i] = s_min[i] = 0;
  __syncthreads();
  const int lane = lane_id();
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nbatch = ((int64_t)n_ni + 31) / 32;
  for (int64_t b = gwarp; b < nbatch; b += nwarps) {
    const int64_t v0 = b * 32, v = v0 + lane;
    const int64_t vend = min(v0 + 32, (int64_t)n_ni);
    const int dv = v < n_ni ? deg[v] : 0;
    if (v < n_ni) hist_add(s_deg, hdeg, dv);
    const int64_t base = off[v0], end = off[vend];
    const int64_t incl = (v < n_ni ? off[v] + dv : end) - base;  // this lane's row end, relative
    for (int64_t s0 = base; s0 < end; s0 += 32) {
      const int64_t rel = s0 - base + lane;
      int pos = 0;
#pragma unroll
      for (int sh = 16; sh >= 1; sh >>= 1) {
        const int64_t t = __shfl_sync(kFull, incl, pos + sh - 1);
        if (t <= rel) pos += sh;
      }
      const int da = __shfl_sync(kFull, dv, pos);
      if (s0 + lane < end) {
        const int du = deg[col[s0 + lane]];
        hist_add(s_max, hmax, da > du ? da : du);
        hist_add(s_min, hmin, da < du ? da : du);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kSmallBins && i < nbins; i += blockDim.x) {
    if (s_deg[i]) atomicAdd(hdeg + i, (unsigned long long)s_deg[i]);
    if (s_max[i]) atomicAdd(hmax + i, (unsigned long long)s_max[i]);
    if (s_min[i]) atomicAdd(hmin + i, (unsigned long long)s_min[i]);
  }
}

}  // namespace
}  // namespace bfsgb

using namespace bfsgb;

extern "C" int bfs_degree_class_stats(const bfs_graph* g, const int64_t* ths, int32_t count, int64_t* out,
                                      struct CUstream_st* stream) {
  if (!g || !ths || !out || count < 1) return fail(BFS_ERR_INVALID, "graph, ths or out is NULL, or count < 1");
  for (int32_t i = 0; i < count; ++i)
    if (ths[i] < 0) return fail(BFS_ERR_INVALID, "thresholds must be >= 0");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != g->device) cudaSetDevice(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nbins = (g->max_deg > kSmallBins ? g->max_deg : kSmallBins) + 1;
  unsigned long long* h = nullptr;
  int rc = BFS_OK;
  cudaError_t e = cudaMalloc((void**)&h, 3 * (size_t)nbins * 8);
  if (e == cudaSuccess) e = cudaMemsetAsync(h, 0, 3 * (size_t)nbins * 8, s);
  if (e == cudaSuccess && g->n_ni > 0) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    k_class_hist<<<sms * 2, 512, 0, s>>>(g->off, g->col, g->deg, g->n_ni, nbins, h, h + nbins, h + 2 * nbins);
    e = cudaGetLastError();
  }
  std::vector<unsigned long long> hh;
  if (e == cudaSuccess) {
    hh.resize(3 * (size_t)nbins);
    e = cudaMemcpyAsync(hh.data(), h, 3 * (size_t)nbins * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (h) cudaFree(h);
  if (e != cudaSuccess) rc = cuda_fail(e, "bfs_degree_class_stats");
  if (!rc) {
    const unsigned long long* hdeg = hh.data();
    const unsigned long long* hmax = hdeg + nbins;
    const unsigned long long* hmin = hdeg + 2 * nbins;
    // cumulative counts up to bin k (inclusive)
    std::vector<int64_t> cdeg(nbins), cmax(nbins), cmin(nbins);
    int64_t a = 0, b = 0, c = 0;
    for (int64_t k = 0; k < nbins; ++k) {
      a += (int64_t)hdeg[k];
      b += (int64_t)hmax[k];
      c += (int64_t)hmin[k];
      cdeg[k] = a;
      cmax[k] = b;
      cmin[k] = c;
    }
    const int64_t n_counted = a, nnz = b;  // vertices [0, n_ni), entries
    for (int32_t i = 0; i < count; ++i) {
      const int64_t k = ths[i] < nbins - 1 ? ths[i] : nbins - 1;
      const int64_t del = n_counted - cdeg[k];  // isolated vertices (degree 0) are never delegates
      const int64_t nn = cmax[k], dd = nnz - cmin[k];
      const int64_t mixed = nnz - nn - dd;
      int64_t* o = out + (int64_t)i * 5;
      o[0] = del;
      o[1] = nn;
      o[2] = mixed / 2;
      o[3] = mixed / 2;
      o[4] = dd;
    }
  }
  if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
  return rc;
}
