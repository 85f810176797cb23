// Device twin of the seeded graph generator (input generation only; see gg_core.h).
#include <cuda_runtime.h>
#include <stdint.h>

#include "gg_core.h"

__global__ void gg_rmat_kernel(int scale, uint64_t seed, int64_t m, int32_t* __restrict__ src,
                               int32_t* __restrict__ dst) {
  const uint64_t stream = gg_stream(seed, GG_TAG_RMAT);
  const gg_perm p = gg_perm_make(seed, scale);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t u, v;
    gg_rmat_edge(stream, scale, (uint64_t)e, &u, &v);
    src[e] = (int32_t)gg_perm_apply(&p, u);
    dst[e] = (int32_t)gg_perm_apply(&p, v);
  }
}

__global__ void gg_er_kernel(uint32_t n, uint64_t seed, int64_t m, int32_t* __restrict__ src,
                             int32_t* __restrict__ dst) {
  const uint64_t stream = gg_stream(seed, GG_TAG_ER);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t u, v;
    gg_er_edge(stream, n, (uint64_t)e, &u, &v);
    src[e] = (int32_t)u;
    dst[e] = (int32_t)v;
  }
}

__global__ void gg_mark_kernel(int64_t m, const int32_t* __restrict__ src,
                               const int32_t* __restrict__ dst, uint8_t* __restrict__ mask) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = src[e], v = dst[e];
    if (u != v) {
      mask[u] = 1;
      mask[v] = 1;
    }
  }
}

static int gg_grid(int64_t m) {
  int64_t b = (m + 255) / 256;
  if (b > 152 * 64) b = 152 * 64;
  return b < 1 ? 1 : (int)b;
}

extern "C" int gg_rmat_device(int scale, int edge_factor, uint64_t seed, int32_t* src, int32_t* dst,
                              void* stream) {
  if (scale < 0 || scale > 30 || edge_factor < 0 || !src || !dst) return -1;
  int64_t m = (int64_t)edge_factor << scale;
  if (m == 0) return 0;
  gg_rmat_kernel<<<gg_grid(m), 256, 0, (cudaStream_t)stream>>>(scale, seed, m, src, dst);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

extern "C" int gg_er_device(int32_t n, int64_t m, uint64_t seed, int32_t* src, int32_t* dst,
                            void* stream) {
  if (n <= 0 || m < 0 || !src || !dst) return -1;
  if (m == 0) return 0;
  gg_er_kernel<<<gg_grid(m), 256, 0, (cudaStream_t)stream>>>((uint32_t)n, seed, m, src, dst);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}

// mask must hold n zeroed bytes on the device.
extern "C" int gg_mark_nonisolated_device(int64_t m, const int32_t* src, const int32_t* dst,
                                          uint8_t* mask, void* stream) {
  if (m < 0 || !mask) return -1;
  if (m == 0) return 0;
  gg_mark_kernel<<<gg_grid(m), 256, 0, (cudaStream_t)stream>>>(m, src, dst, mask);
  return cudaGetLastError() == cudaSuccess ? 0 : -2;
}
