// Device helpers shared by the level-loop kernels: warp primitives, the run
// status word, and the bounded grid barrier.  P is a kernel parameter struct
// with `hdr` (RunHeader*), `arrive`, `epoch` and `timeout_ns`.
#pragma once

#include "bfs_internal.cuh"

namespace bfsgb {

__device__ __forceinline__ int lane_id() { return (int)(threadIdx.x & 31u); }

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long warp_sum(unsigned long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

__device__ __forceinline__ int64_t warp_incl_scan(int64_t x) {
  const int lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += t;
  }
  return x;
}

// Status word: (epoch << 4) | code, code = -BFS_ERR_*.
template <class P>
__device__ __forceinline__ bool run_failed(const P& p) {
  unsigned e = *(volatile unsigned*)&p.hdr->err;
  return e != 0 && (e >> 4) == (p.epoch & 0x0FFFFFFFu);
}

template <class P>
__device__ __forceinline__ void set_failed(const P& p, int code) {
  atomicExch((unsigned*)&p.hdr->err, ((p.epoch & 0x0FFFFFFFu) << 4) | (unsigned)(-code));
}

// Bounds checks of a BFS_CHECK build: an index outside [0, n) records
// BFS_ERR_CHECK in the run's status word (never a trap) and the caller skips the
// access; other builds compile every check to `true`.
template <class P>
__device__ __forceinline__ bool check_index(const P& p, long long i, long long n) {
  if (i >= 0 && i < n) return true;
  set_failed(p, BFS_ERR_CHECK);
  return false;
}
#ifdef BFS_CHECK
#define BFS_IN(p, i, n) ::bfsgb::check_index((p), (long long)(i), (long long)(n))
#else
#define BFS_IN(p, i, n) true
#endif

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Grid-wide barrier over co-resident CTAs (cooperative launch), without a shared
// atomic counter: every CTA release-stores its own arrival word (epoch-tagged,
// so words left by earlier runs never match; its low 8 bits carry the OR of the
// CTA's `flags`), CTA 0's threads acquire-poll all arrival words in parallel,
// CTA 0's thread 0 runs master(OR of all CTAs' flags) (which may read everything
// written before the barrier) and release-stores one word that carries the
// barrier tag and master's 8 result bits; every CTA acquire-polls that word.
// Every wait has a %globaltimer deadline.  Returns master's bits to every
// thread of every CTA, or -1 (uniformly per CTA) if the run failed.
template <class P, class F>
__device__ int grid_sync(const P& p, unsigned& seq, F&& master, int flags = 0) {
  __shared__ int s_res, s_flags;
  ++seq;
  const unsigned long long tag =
      ((unsigned long long)(p.epoch & 0x0FFFFFFFu) << 36) | ((unsigned long long)(seq & 0x0FFFFFFFu) << 8);
  if (threadIdx.x == 0) s_flags = 0;
  __syncthreads();
  if (flags) atomicOr(&s_flags, flags);
  __syncthreads();
  if (threadIdx.x == 0) st_release64(p.arrive + 4 * blockIdx.x, tag | (unsigned)(s_flags & 0xFF));
  if (blockIdx.x == 0) {
    int ok = 1, fl = 0;
    const unsigned long long t0 = gtimer();
    for (int t = threadIdx.x; t < (int)gridDim.x && ok; t += blockDim.x) {
      unsigned long long a;
      while ((a = ld_acquire64(p.arrive + 4 * t)) < tag) {
        if (run_failed(p)) {
          ok = 0;
          break;
        }
        if (gtimer() - t0 > p.timeout_ns) {
          set_failed(p, BFS_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(20);
      }
      fl |= (int)(a & 0xFFu);
    }
    ok = __syncthreads_and(ok);
    if (fl) atomicOr(&s_flags, fl);  // every CTA 0 thread has finished with s_flags above
    __syncthreads();
    if (threadIdx.x == 0 && ok) st_release64(&p.hdr->release, tag | (unsigned)(master(s_flags) & 0xFF));
  }
  if (threadIdx.x == 0) {
    int res = -1;
    const unsigned long long t0 = gtimer();
    for (;;) {
      const unsigned long long r = ld_acquire64(&p.hdr->release);
      if (r >= tag) {
        res = (int)(r & 0xFFu);
        break;
      }
      if (run_failed(p)) break;
      if (gtimer() - t0 > p.timeout_ns) {
        set_failed(p, BFS_ERR_TIMEOUT);
        break;
      }
      __nanosleep(20);
    }
    if (res >= 0 && run_failed(p)) res = -1;
    s_res = res;
  }
  __syncthreads();
  return s_res;
}

__device__ __forceinline__ int no_master(int) { return 0; }

// A warp's index for static work splits, numbered CTA-interleaved (warp 0 of
// every CTA first, then warp 1, ...), so that a level with fewer items than warps
// spreads them over all SMs instead of filling the first CTAs.
__device__ __forceinline__ int64_t spread_warp() {
  return (int64_t)(threadIdx.x >> 5) * gridDim.x + blockIdx.x;
}


// Exclusive prefix sum over the CTA of two per-thread counts; returns the
// CTA totals.  Called by all threads of the CTA.
__device__ inline void block_scan2(unsigned long long a, unsigned long long b, unsigned long long& ea,
                            unsigned long long& eb, unsigned long long& ta, unsigned long long& tb) {
  __shared__ unsigned long long s_a[kMaxWarpsPerBlock], s_b[kMaxWarpsPerBlock];
  const int lane = lane_id(), wid = threadIdx.x >> 5;
  unsigned long long ia = a, ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long xa = __shfl_up_sync(kFull, ia, o), xb = __shfl_up_sync(kFull, ib, o);
    if (lane >= o) {
      ia += xa;
      ib += xb;
    }
  }
  if (lane == 31) {
    s_a[wid] = ia;
    s_b[wid] = ib;
  }
  __syncthreads();
  unsigned long long pa = 0, pb = 0;
  ta = tb = 0;
  const int nw = (int)(blockDim.x >> 5);
  for (int w = 0; w < nw; ++w) {
    if (w < wid) {
      pa += s_a[w];
      pb += s_b[w];
    }
    ta += s_a[w];
    tb += s_b[w];
  }
  ea = pa + ia - a;
  eb = pb + ib - b;
  __syncthreads();
}

}  // namespace bfsgb
