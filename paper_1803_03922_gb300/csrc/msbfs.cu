// 64-lane multi-source BFS: up to 64 queries per launch over one degree-separated
// graph, one bit per query ("lane") in a 64-bit word per vertex.
//
// State per internal vertex v: visit[v] (lanes that reached v) and three
// frontier words F[L%3][v] (lanes for which v is at depth L).  Per level, on
// the union of the lanes' frontiers:
//   forward (push): every frontier vertex u pushes F[u] & ~visit[v] into
//     F_next[v] with a 64-bit atomicOr; delegate rows come from 512-entry chunks
//     (as in the single-source loop) so a hub spreads over many warps; each new
//     (lane, v) takes the smallest frontier caller id by atomicMin;
//   backward (pull): every vertex still missing some lane scans its row (sorted
//     by caller id) 32 entries at a time; an inclusive OR-scan of
//     F[u] & need along the row gives, for every lane at once, its first hit,
//     i.e. its canonical parent; the scan stops when no needed lane is left.
// The level end merges F_next into visit, writes depths (forward levels), builds
// the next delegate chunk list and counts the frontier for the direction choice
// (Beamer alpha on vertex counts).  Depth is uint8 per (query, vertex), 255 =
// unreached; a depth above 254 is an overflow error.
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>
#include <new>

#include "bfs_internal.cuh"
#include "device_common.cuh"

namespace bfsgb {
namespace {

constexpr int kMsLanes = 64;

struct __align__(64) MsSlot {
  unsigned long long nfv;    // frontier vertices (any lane)
  unsigned long long mfv;    // degree sum over frontier vertices
  unsigned long long pairs;  // (lane, vertex) pairs in the frontier
  unsigned long long pdeg;   // sum over those pairs of the degree
  unsigned long long nch;    // delegate chunk entries of the frontier
  unsigned long long mdone;  // degree of vertices every active lane has now reached
  unsigned long long ndl;    // deferred row chunks of the backward level
  unsigned long long aux;    // lanes present in this level's frontier (slot 0: lanes with a non-isolated source)
};

// A chunk of a long row whose first kMsHead entries left some lane without a
// parent: entries [head end + c * kChunk, + kChunk) of v's row, for lanes `need`.
struct __align__(16) MsDefer {
  int32_t v, c;
  unsigned long long need;
};

constexpr int kMsHead = 512;

struct MsLog {
  int32_t dir, pad;  // pad: lanes that pull at a backward level
  unsigned long long nfv, mfv, pairs, t_begin, t_expand, t_end;
};

struct MsParams {
  const int64_t* off;
  const int32_t* col;
  const int32_t* deg;
  const int32_t* caller_of;
  const int32_t* internal_of;
  unsigned long long* visit;
  unsigned long long* F0;
  unsigned long long* F1;
  unsigned long long* F2;
  uint8_t* depth_i;   // [n_ni][ls] (vertex-major: a vertex's lanes share cache lines)
  int32_t* parent_i;  // [n_ni][ls] or null
  int2* CL0;
  int2* CL1;
  MsDefer* DL;        // deferred row chunks of a backward level [cl_cap]
  MsSlot* slot;       // [4]
  MsLog* log;         // [BFS_BATCH_LOG_LEVELS]
  RunHeader* hdr;
  unsigned long long* arrive;
  int64_t nnz;
  int32_t n, n_ni, d, k;
  int32_t ls;           // lane stride of depth_i / parent_i: k rounded up to a multiple of 4
  int32_t out_parents;  // 1: out_p[j] are written
  int32_t alpha;
  unsigned int epoch;
  unsigned long long timeout_ns;
  unsigned long long run_timeout_ns;
  int32_t src_c[kMsLanes];
  uint8_t* out_d[kMsLanes];  // lane j's depth row, n entries in caller ids
  int32_t* out_p[kMsLanes];  // lane j's parent row (when out_parents)
};

// Lane words: one bit per query, 64 lanes in an unsigned long long, or 32 in an
// unsigned int for batches of at most 32 queries (half the per-vertex state
// traffic of every sweep).  The state arrays hold 64-bit slots either way.
template <typename W>
__device__ __forceinline__ W* Fbuf(const MsParams& p, int i) {
  return reinterpret_cast<W*>(i == 0 ? p.F0 : (i == 1 ? p.F1 : p.F2));
}
template <typename W>
__device__ __forceinline__ W* visit_of(const MsParams& p) {
  return reinterpret_cast<W*>(p.visit);
}
__device__ __forceinline__ int ffs_w(unsigned long long x) { return __ffsll((long long)x); }
__device__ __forceinline__ int ffs_w(unsigned x) { return __ffs((int)x); }
__device__ __forceinline__ int popc_w(unsigned long long x) { return __popcll(x); }
__device__ __forceinline__ int popc_w(unsigned x) { return __popc(x); }
__device__ __forceinline__ unsigned long long warp_or(unsigned long long x) {
  const unsigned lo = __reduce_or_sync(kFull, (unsigned)x), hi = __reduce_or_sync(kFull, (unsigned)(x >> 32));
  return ((unsigned long long)hi << 32) | lo;
}
__device__ __forceinline__ unsigned long long warp_or(unsigned x) { return __reduce_or_sync(kFull, x); }

// Offers caller id pc as parent of v to every lane of nb (forward levels).
template <typename W>
__device__ __forceinline__ void ms_offer(const MsParams& p, int v, W nb, int pc) {
  while (nb) {
    const int b = ffs_w(nb) - 1;
    nb &= nb - 1;
    atomicMin(p.parent_i + (int64_t)v * p.ls + b, pc);
  }
}

template <typename W>
__device__ __forceinline__ void ms_push(const MsParams& p, W fu, int pc, int v, W* __restrict__ Fn) {
  const W nb = fu & ~visit_of<W>(p)[v];
  if (!nb) return;
  atomicOr(Fn + v, nb);
  if (p.parent_i) ms_offer(p, v, nb, pc);
}

// Forward level: delegate chunks, then the normal frontier vertices gathered 32
// per warp (lane i owns vertex w0+i when its frontier word is nonzero; the warp
// walks the owned rows' entries 32 at a time).
template <typename W>
__device__ void ms_expand_td(const MsParams& p, int L) {
  const MsSlot* sc = p.slot + (L & 3);
  const W* Fc = Fbuf<W>(p, L % 3);
  W* Fn = Fbuf<W>(p, (L + 1) % 3);
  const int2* CL = (L & 1) ? p.CL1 : p.CL0;
  const int lane = lane_id();
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nch = (int64_t)__ldcg(&sc->nch);
  const int64_t nbatch = ((int64_t)p.n_ni - p.d + 31) / 32;
  for (int64_t it = gwarp; it < nch + nbatch; it += nwarps) {
    if (it < nch) {
      const int2 ck = CL[it];
      const int u = ck.x;
      const W fu = Fc[u];
      const int pc = p.parent_i ? p.caller_of[u] : 0;
      const int64_t rb = p.off[u], re = rb + p.deg[u];
      const int64_t beg = rb + (int64_t)ck.y * kChunk, end = min(beg + kChunk, re);
      for (int64_t j = beg + lane; j < end; j += 32) ms_push(p, fu, pc, __ldcs(p.col + j), Fn);
      continue;
    }
    const int64_t u0 = p.d + (it - nch) * 32;
    const int64_t u = u0 + lane;
    W fu = 0;
    int64_t beg = 0, deg = 0;
    int pc = 0;
    if (u < p.n_ni) {
      fu = Fc[u];
      if (fu) {
        beg = p.off[u];
        deg = p.deg[u];
        if (p.parent_i) pc = p.caller_of[u];
      }
    }
    const int64_t incl = warp_incl_scan(deg);
    const int64_t total = __shfl_sync(kFull, incl, 31);
    const int64_t excl = incl - deg;
    for (int64_t base = 0; base < total; base += 32) {
      const int64_t e = base + lane;
      int pos = 0;
#pragma unroll
      for (int s = 16; s >= 1; s >>= 1) {
        const int64_t t = __shfl_sync(kFull, incl, pos + s - 1);
        if (t <= e) pos += s;
      }
      const int64_t ob = __shfl_sync(kFull, beg, pos);
      const int64_t ox = __shfl_sync(kFull, excl, pos);
      const W ofu = __shfl_sync(kFull, fu, pos);
      const int opc = __shfl_sync(kFull, pc, pos);
      if (e < total) ms_push(p, ofu, opc, __ldcs(p.col + ob + (e - ox)), Fn);
    }
  }
}

// Backward level.  A vertex still missing some lane looks for each missing lane's
// first frontier neighbour in its row (sorted by caller id): that neighbour is
// the lane's canonical parent.  Normal vertices (rows of at most TH entries):
// one thread per vertex walks its row in order, keeping the lanes already
// found, and stops when no needed lane is left.  Delegates (long rows): the
// whole warp takes 32 entries per step, and an inclusive OR-scan of
// h_i = F[u_i] & need gives each lane's first hit (bits set in h_i and not
// before).  Column reads are streaming loads so they do not evict the frontier
// words from L2.
// Parents are stored as caller ids, as forward levels need for atomicMin; one
// caller_of gather serves every lane an entry settles.
template <typename W>
__device__ __forceinline__ void ms_found(const MsParams& p, int v, W nb, int u, int L) {
  const int pc = p.parent_i ? p.caller_of[u] : 0;
  while (nb) {
    const int b = ffs_w(nb) - 1;
    nb &= nb - 1;
    if (p.parent_i) p.parent_i[(int64_t)v * p.ls + b] = pc;
    p.depth_i[(int64_t)v * p.ls + b] = (uint8_t)(L + 1);
  }
}

// Returns 1 in a thread that deferred row chunks.
template <typename W>
__device__ int ms_expand_bu(const MsParams& p, int L, W lanes) {
  MsSlot* sc = p.slot + (L & 3);
  int deferred = 0;
  const W* Fc = Fbuf<W>(p, L % 3);
  W* Fn = Fbuf<W>(p, (L + 1) % 3);
  const int lane = lane_id();
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t gwarp = gtid >> 5, nwarps = gthreads >> 5;
  // normal vertices, 32 per warp (lane i owns vertex v0 + i).  Head: each owner
  // checks the first four entries of its row.  Rest: the warp walks the rows'
  // remaining entries 32 per step (consecutive rows are contiguous, so the column
  // loads coalesce); a segmented OR-scan along the lanes gives each entry's new
  // first hits, and an owner carries its vertex's found lanes from step to step.
  const int64_t nbatch = ((int64_t)p.n_ni - p.d + 31) / 32;
  for (int64_t it = gwarp; it < nbatch; it += nwarps) {  // warp-uniform
    const int64_t v0 = p.d + it * 32;
    const int64_t v = v0 + lane;
    W need = 0, found = 0;
    int64_t beg = 0, end = 0;
    if (v < p.n_ni) {
      need = lanes & ~visit_of<W>(p)[v];
      if (need) {
        beg = p.off[v];
        end = beg + p.deg[v];
      }
    }
    if (need) {
      int u[4];
      W h[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) u[t] = beg + t < end ? __ldcs(p.col + beg + t) : -1;
#pragma unroll
      for (int t = 0; t < 4; ++t) h[t] = u[t] >= 0 ? Fc[u[t]] : (W)0;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const W x = h[t] & need;
        if (x) {
          ms_found(p, (int)v, x, u[t], L);
          found |= x;
          need &= ~x;
        }
      }
    }
    const int64_t rb = beg + 4;
    const int64_t rest = (need && end > rb) ? end - rb : 0;
    const int64_t incl = warp_incl_scan(rest);
    const int64_t total = __shfl_sync(kFull, incl, 31);
    const int64_t excl = incl - rest;
    // four 32-entry rounds per step: their column loads and frontier words are
    // all in flight before the first round's scan
    constexpr int kRounds = 4;
    for (int64_t base = 0; base < total; base += 32 * kRounds) {
      if (!__any_sync(kFull, need != 0 && excl + rest > base)) break;
      int pos[kRounds], u[kRounds];
      W h[kRounds];
#pragma unroll
      for (int r = 0; r < kRounds; ++r) {
        const int64_t e = base + 32 * r + lane;
        int ps = 0;
#pragma unroll
        for (int sh = 16; sh >= 1; sh >>= 1) {
          const int64_t t = __shfl_sync(kFull, incl, ps + sh - 1);
          if (t <= e) ps += sh;
        }
        pos[r] = ps;
        const int64_t orb = __shfl_sync(kFull, rb, ps);
        const int64_t oex = __shfl_sync(kFull, excl, ps);
        const W oneed = __shfl_sync(kFull, need, ps);
        u[r] = (e < total && oneed) ? __ldcs(p.col + orb + (e - oex)) : -1;
      }
#pragma unroll
      for (int r = 0; r < kRounds; ++r) h[r] = u[r] >= 0 ? Fc[u[r]] : (W)0;
#pragma unroll
      for (int r = 0; r < kRounds; ++r) {
        const int64_t rbase = base + 32 * r;
        const W hh = h[r] & __shfl_sync(kFull, need, pos[r]);  // the owner's current need
        W sc = hh;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const W t = __shfl_up_sync(kFull, sc, o);
          const int ps = __shfl_up_sync(kFull, pos[r], o);
          if (lane >= o && ps == pos[r]) sc |= t;
        }
        W before = __shfl_up_sync(kFull, sc, 1);
        const int pprev = __shfl_up_sync(kFull, pos[r], 1);
        if (lane == 0 || pprev != pos[r]) before = 0;
        const W nb = hh & ~before;
        if (nb) ms_found(p, (int)(v0 + pos[r]), nb, u[r], L);
        // this round's part of the owner's row: lanes [lo, hi) - rbase; its last
        // lane holds the OR of the part
        const int64_t lo = max(excl, rbase), hi = min(excl + rest, rbase + 32);
        const W tot = __shfl_sync(kFull, sc, hi > lo ? (int)(hi - 1 - rbase) : lane);
        if (hi > lo) {
          found |= tot;
          need &= ~tot;
        }
      }
    }
    if (found) Fn[v] = found;
  }
  // delegates: one warp per vertex over the first kMsHead entries of its row;
  // what is left of a row with lanes still missing goes to the deferred list
  const int64_t items = ((int64_t)p.d + 31) / 32;
  for (int64_t it = gwarp; it < items; it += nwarps) {
    const int64_t v = it * 32 + lane;
    const W need_l = v < p.d ? (lanes & ~visit_of<W>(p)[v]) : (W)0;
    unsigned pend = __ballot_sync(kFull, need_l != 0);
    while (pend) {
      const int j = __ffs(pend) - 1;
      pend &= pend - 1;
      const int vv = (int)(it * 32 + j);
      W need = __shfl_sync(kFull, need_l, j);
      const int64_t beg = p.off[vv], end = beg + p.deg[vv];
      W found = 0;
      const int64_t al = beg & ~(int64_t)3, hend = min(end, al + kMsHead);
      // 128 entries per step: lane l holds entries 4l..4l+3 of the step (one
      // 128-bit load), in row order within the lane, lanes in order along the row
      for (int64_t j0 = al; j0 < hend && need; j0 += 128) {
        const int64_t jj = j0 + 4 * lane;
        int4 c4 = make_int4(-1, -1, -1, -1);
        if (jj < hend) c4 = __ldcs(reinterpret_cast<const int4*>(p.col + jj));
        const int u[4] = {jj >= beg ? c4.x : -1, (jj + 1 >= beg && jj + 1 < hend) ? c4.y : -1,
                          (jj + 2 >= beg && jj + 2 < hend) ? c4.z : -1, (jj + 3 >= beg && jj + 3 < hend) ? c4.w : -1};
        W h[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) h[t] = u[t] >= 0 ? (Fc[u[t]] & need) : (W)0;
        const W mine = h[0] | h[1] | h[2] | h[3];
        W incl = mine;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const W t = __shfl_up_sync(kFull, incl, o);
          if (lane >= o) incl |= t;
        }
        W before = __shfl_up_sync(kFull, incl, 1);
        if (lane == 0) before = 0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const W nb = h[t] & ~before;
          if (nb) ms_found(p, vv, nb, u[t], L);
          before |= h[t];
        }
        const W tot = __shfl_sync(kFull, incl, 31);
        found |= tot;
        need &= ~tot;
      }
      if (lane == 0 && found) Fn[vv] = found;
      if (need && hend < end) {
        const int nc = (int)((end - hend + kChunk - 1) / kChunk);
        W dbase = 0;
        if (lane == 0) dbase = atomicAdd(&sc->ndl, (W)nc);
        dbase = __shfl_sync(kFull, dbase, 0);
        for (int c = lane; c < nc; c += 32) {
          MsDefer e;
          e.v = vv;
          e.c = c;
          e.need = need;
          p.DL[dbase + c] = e;
        }
        deferred = 1;
      }
    }
  }
  return deferred;
}

// Deferred chunks of a backward level, after a grid barrier (the head scans'
// found bits are in F_next).  Chunks of one row run on different warps, so a
// lane's canonical parent (first hit in row order = smallest caller id) is the
// atomicMin of the chunks' first hits, in caller ids as in forward levels.
template <typename W>
__device__ void ms_drain_bu(const MsParams& p, int L) {
  const MsSlot* sc = p.slot + (L & 3);
  const W* Fc = Fbuf<W>(p, L % 3);
  W* Fn = Fbuf<W>(p, (L + 1) % 3);
  const int lane = lane_id();
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nd = (int64_t)__ldcg(&sc->ndl);
  for (int64_t it = gwarp; it < nd; it += nwarps) {
    const MsDefer e = p.DL[it];
    const int v = e.v;
    W need = (W)e.need, found = 0;
    const int64_t beg = p.off[v], end = beg + p.deg[v];
    const int64_t c0 = (beg & ~(int64_t)3) + kMsHead + (int64_t)e.c * kChunk;
    const int64_t c1 = min(c0 + kChunk, end);
    for (int64_t j0 = c0; j0 < c1 && need; j0 += 128) {
      const int64_t jj = j0 + 4 * lane;
      int4 c4 = make_int4(-1, -1, -1, -1);
      if (jj < c1) c4 = __ldcs(reinterpret_cast<const int4*>(p.col + jj));
      const int u[4] = {c4.x, jj + 1 < c1 ? c4.y : -1, jj + 2 < c1 ? c4.z : -1, jj + 3 < c1 ? c4.w : -1};
      W h[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) h[t] = u[t] >= 0 ? (Fc[u[t]] & need) : 0ull;
      W incl = h[0] | h[1] | h[2] | h[3];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const W t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl |= t;
      }
      W before = __shfl_up_sync(kFull, incl, 1);
      if (lane == 0) before = 0;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        W nb = h[t] & ~before;
        before |= h[t];
        if (!nb) continue;
        const int pc = p.parent_i ? p.caller_of[u[t]] : 0;
        while (nb) {
          const int b = ffs_w(nb) - 1;
          nb &= nb - 1;
          if (p.parent_i) atomicMin(p.parent_i + (int64_t)v * p.ls + b, pc);
          p.depth_i[(int64_t)v * p.ls + b] = (uint8_t)(L + 1);
        }
      }
      const W tot = __shfl_sync(kFull, incl, 31);
      found |= tot;
      need &= ~tot;
    }
    if (lane == 0 && found) atomicOr(Fn + v, found);
  }
}

// Level end: merge F_next into visit, clear the frontier word two levels back,
// (forward) write depths, count the next frontier and list its delegate chunks.
template <typename W>
__device__ void ms_level_end(const MsParams& p, int L, bool td, W lanes) {
  __shared__ unsigned long long s_red[6];
  __shared__ unsigned long long s_base;
  W* Fn = Fbuf<W>(p, (L + 1) % 3);
  W* Fo = Fbuf<W>(p, (L + 2) % 3);
  W* visit = visit_of<W>(p);
  int2* CLn = (L & 1) ? p.CL0 : p.CL1;
  MsSlot* sn = p.slot + ((L + 1) & 3);
  const int tid = threadIdx.x;
  if (tid < 6) s_red[tid] = 0;
  __syncthreads();
  unsigned long long nfv = 0, mfv = 0, pairs = 0, pdeg = 0, mdone = 0;
  W act = 0;
  bool overflow = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b0 = (int64_t)blockIdx.x * blockDim.x; b0 < p.n_ni; b0 += stride) {  // CTA-uniform
    const int64_t v = b0 + tid;
    W fn = 0;
    unsigned long long nch = 0;
    int dg = 0;
    if (v < p.n_ni) {
      Fo[v] = 0;
      fn = __ldcg(Fn + v);
      if (fn) {
        act |= fn;
        const W old = visit[v];
        visit[v] = old | fn;
        dg = p.deg[v];
        nfv += 1;
        mfv += (unsigned long long)dg;
        pairs += (unsigned long long)popc_w(fn);
        pdeg += (unsigned long long)popc_w(fn) * (unsigned long long)dg;
        if ((old | fn) == lanes && old != lanes) mdone += (unsigned long long)dg;
        if (L + 1 > 254) overflow = true;
        if (td) {
          W x = fn;
          while (x) {
            const int b = ffs_w(x) - 1;
            x &= x - 1;
            p.depth_i[(int64_t)v * p.ls + b] = (uint8_t)(L + 1);
          }
        }
        if (v < p.d) nch = ((unsigned long long)dg + kChunk - 1) / kChunk;
      }
    }
    // delegate chunk list of the next frontier (only the CTAs' tiles below d hold delegates)
    if (b0 < p.d) {
      unsigned long long e0, e1, t0, t1;
      block_scan2(nch, 0ull, e0, e1, t0, t1);
      if (tid == 0) s_base = t0 ? atomicAdd(&sn->nch, t0) : 0ull;
      __syncthreads();
      unsigned long long cb = s_base + e0;
      for (unsigned long long c = 0; c < nch; ++c) CLn[cb++] = make_int2((int)v, (int)c);
      __syncthreads();
    }
  }
  if (overflow) set_failed(p, BFS_ERR_OVERFLOW);
  {  // lanes present in the next frontier
    __shared__ unsigned long long s_act;
    if (tid == 0) s_act = 0ull;
    __syncthreads();
    const unsigned long long w = warp_or(act);
    if (lane_id() == 0 && w) atomicOr(&s_act, w);
    __syncthreads();
    if (tid == 0 && s_act) atomicOr(&sn->aux, s_act);
  }
  const unsigned long long x[5] = {warp_sum(nfv), warp_sum(mfv), warp_sum(pairs), warp_sum(pdeg), warp_sum(mdone)};
  if (lane_id() == 0)
    for (int i = 0; i < 5; ++i)
      if (x[i]) atomicAdd(&s_red[i], x[i]);
  __syncthreads();
  if (tid == 0) {
    if (s_red[0]) atomicAdd(&sn->nfv, s_red[0]);
    if (s_red[1]) atomicAdd(&sn->mfv, s_red[1]);
    if (s_red[2]) atomicAdd(&sn->pairs, s_red[2]);
    if (s_red[3]) atomicAdd(&sn->pdeg, s_red[3]);
    if (s_red[4]) atomicAdd(&sn->mdone, s_red[4]);
  }
}

constexpr int kMsBackward = 1, kMsDone = 2, kMsDrain = 4;

template <typename W>
__global__ void __launch_bounds__(kThreads, 2) ms_bfs_loop(MsParams p) {
  W* visit = visit_of<W>(p);
  W* F0 = Fbuf<W>(p, 0);
  __shared__ long long s_mu;
  __shared__ unsigned long long s_pairs, s_pdeg;
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  unsigned seq = 0;
  // set-up: state words, parent slots
  {
    W* F1 = Fbuf<W>(p, 1);
    W* F2 = Fbuf<W>(p, 2);
    for (int64_t v = gtid; v < p.n_ni; v += gthreads) {
      visit[v] = 0;
      F0[v] = 0;
      F1[v] = 0;
      F2[v] = 0;
    }
  }
  if (p.parent_i) {
    const int64_t P4 = (int64_t)p.n_ni * (p.ls / 4);
    for (int64_t i = gtid; i < P4; i += gthreads)
      reinterpret_cast<int4*>(p.parent_i)[i] = make_int4(INT_MAX, INT_MAX, INT_MAX, INT_MAX);
  }
  if (leader) {
    for (int i = 0; i < 4; ++i) p.slot[i] = MsSlot();
    p.hdr->t0 = gtimer();
  }
  if (grid_sync(p, seq, no_master) < 0) return;
  if (leader) {  // seed the k sources (a source may repeat across lanes)
    unsigned long long nfv = 0, mfv = 0, nch = 0, pdeg = 0;
    W act = 0;
    for (int j = 0; j < p.k; ++j) {
      const int v = p.internal_of[p.src_c[j]];
      if (v >= p.n_ni) continue;  // an isolated source: its lane is finished
      const W bit = (W)1 << j;
      act |= bit;
      const int dg = p.deg[v];
      if (F0[v] == 0) {
        nfv += 1;
        mfv += (unsigned long long)dg;
        if (v < p.d)
          for (int64_t c = 0; c < ((int64_t)dg + kChunk - 1) / kChunk; ++c) p.CL0[nch++] = make_int2(v, (int)c);
      }
      F0[v] |= bit;
      visit[v] |= bit;
      p.depth_i[(int64_t)v * p.ls + j] = 0;
      if (p.parent_i) p.parent_i[(int64_t)v * p.ls + j] = p.src_c[j];
      pdeg += (unsigned long long)dg;
    }
    p.slot[0].nfv = nfv;
    p.slot[0].mfv = mfv;
    p.slot[0].nch = nch;
    p.slot[0].aux = act;
    s_mu = (long long)p.nnz;
    s_pairs = 0;
    s_pdeg = pdeg;
  }
  int bits = grid_sync(p, seq, [&](int) { return p.slot[0].nfv ? 0 : kMsDone; });
  if (bits < 0) return;
  __shared__ unsigned long long s_tb, s_te;
  const W lanes = (W)__ldcg(&p.slot[0].aux);  // lanes with a non-isolated source
  const unsigned long long t_start = gtimer();
  if (leader) p.hdr->t_init = t_start;
  int L = 0;
  while (!(bits & kMsDone)) {
    if (leader) s_tb = gtimer();
    if (threadIdx.x == 0 && (L > 300 || gtimer() - t_start > p.run_timeout_ns)) set_failed(p, BFS_ERR_TIMEOUT);
    const bool bu = (bits & kMsBackward) != 0;
    if (bu) {
      // lanes whose frontier is empty can find no parent: they are not searched for
      const int fl = ms_expand_bu<W>(p, L, (W)__ldcg(&p.slot[L & 3].aux));
      const int b2 = grid_sync(p, seq, [](int f) { return (f & 1) ? kMsDrain : 0; }, fl);
      if (b2 < 0) return;
      if (b2 & kMsDrain) {
        ms_drain_bu<W>(p, L);
        if (grid_sync(p, seq, no_master) < 0) return;
      }
    } else {
      ms_expand_td<W>(p, L);
      if (grid_sync(p, seq, no_master) < 0) return;
    }
    if (leader) s_te = gtimer();
    ms_level_end<W>(p, L, !bu, lanes);
    if (leader) p.slot[(L + 2) & 3] = MsSlot();
    bits = grid_sync(p, seq, [&](int) {
      const MsSlot* sc = p.slot + (L & 3);
      if (L < BFS_BATCH_LOG_LEVELS) {
        MsLog& lg = p.log[L];
        lg.dir = bu ? 1 : 0;
        lg.pad = bu ? popc_w((W)__ldcg(&sc->aux)) : 0;
        lg.nfv = __ldcg(&sc->nfv);
        lg.mfv = __ldcg(&sc->mfv);
        lg.pairs = __ldcg(&sc->pairs);
        lg.t_begin = s_tb;
        lg.t_expand = s_te;
        lg.t_end = gtimer();
      }
      const MsSlot* sn = p.slot + ((L + 1) & 3);
      const unsigned long long nfv = __ldcg(&sn->nfv), mfv = __ldcg(&sn->mfv);
      s_mu -= (long long)__ldcg(&sn->mdone);
      s_pairs += __ldcg(&sn->pairs);
      s_pdeg += __ldcg(&sn->pdeg);
      if (nfv == 0) return kMsDone;
      // Beamer's alpha on the union frontier; once backward, stay backward (lanes
      // that are done cost one visit-word read per vertex)
      return (bu || (long long)(mfv * (unsigned long long)p.alpha) > s_mu) ? kMsBackward : 0;
    });
    if (bits < 0) return;
    ++L;
  }
  // results in caller ids: out_d[j][c] for the k lanes, a vertex's lanes read
  // four at a time (its depth bytes and parents are contiguous)
  if (leader) p.hdr->t_loop = gtimer();
  for (int64_t c = gtid; c < p.n; c += gthreads) {
    const int v = p.internal_of[c];
    const bool in = v < p.n_ni;
    const W vis = in ? visit[v] : (W)0;
    for (int j0 = 0; j0 < p.k; j0 += 4) {
      unsigned dq = 0xFFFFFFFFu;
      int4 pq = make_int4(-1, -1, -1, -1);
      if (in && ((vis >> j0) & 0xFu)) {
        dq = *reinterpret_cast<const unsigned*>(p.depth_i + (int64_t)v * p.ls + j0);
        if (p.out_parents) pq = *reinterpret_cast<const int4*>(p.parent_i + (int64_t)v * p.ls + j0);
      }
      const int pv4[4] = {pq.x, pq.y, pq.z, pq.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int j = j0 + t;
        if (j >= p.k) break;
        const bool r = (vis >> j) & 1ull;
        uint8_t dv = r ? (uint8_t)((dq >> (8 * t)) & 0xFFu) : (uint8_t)255;
        int pv = -1;
        if (r) pv = pv4[t];
        if (c == p.src_c[j]) {
          dv = 0;
          pv = p.src_c[j];
        }
        p.out_d[j][c] = dv;
        if (p.out_parents) p.out_p[j][c] = pv;
      }
    }
  }
  if (leader) {  // every query reaches its source: max depth + 1 >= 1 even if all sources are isolated
    p.hdr->levels = L > 0 ? L : 1;
    p.hdr->levels_run = L;
    p.hdr->t1 = gtimer();
    p.hdr->reached = s_pairs;
    p.hdr->reached_edges = s_pdeg;
  }
}

}  // namespace
}  // namespace bfsgb

struct bfs_batch {
  const bfs_graph* g = nullptr;
  int with_parents = 0;
  unsigned long long* visit = nullptr;
  unsigned long long* F = nullptr;  // 3 x n_ni
  uint8_t* depth_i = nullptr;
  int32_t* parent_i = nullptr;
  int2* CL = nullptr;  // 2 x cl_cap
  bfsgb::MsDefer* DL = nullptr;  // cl_cap
  bfsgb::MsSlot* slot = nullptr;
  bfsgb::MsLog* log = nullptr;
  bfsgb::RunHeader* hdr = nullptr;
  unsigned long long* arrive = nullptr;
  uint8_t* out_depth = nullptr;  // scratch for host result buffers [64 n]
  int32_t* out_parent = nullptr;
  int grid = 0;
  unsigned int epoch = 0;
  int64_t device_bytes = 0;
};

using namespace bfsgb;

namespace {

void batch_free_all(bfs_batch* b) {
  void* ptrs[] = {b->visit, b->F, b->depth_i, b->parent_i, b->CL, b->DL, b->slot, b->log, b->hdr, b->arrive,
                  b->out_depth, b->out_parent};
  for (void* q : ptrs)
    if (q) cudaFree(q);
}

int balloc(void** p, size_t bytes, bfs_batch* b, const char* what) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, what);
  }
  b->device_bytes += (int64_t)bytes;
  return BFS_OK;
}

// Resident CTAs per SM of the batched kernel: the smaller of its two lane widths.
cudaError_t ms_occupancy(int* per_sm) {
  int a = 0, b = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, ms_bfs_loop<unsigned long long>, kThreads, 0);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, ms_bfs_loop<unsigned>, kThreads, 0);
  *per_sm = a < b ? a : b;
  return e;
}

bool dev_ptr(const void* q) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, q) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int bfs_batch_capacity(int32_t* ctas) {
  if (!ctas) return fail(BFS_ERR_INVALID, "ctas is NULL");
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = ms_occupancy(&per_sm);
  if (e != cudaSuccess) return cuda_fail(e, "bfs_batch_capacity");
  *ctas = sms * (per_sm < 2 ? per_sm : 2);
  return BFS_OK;
}

extern "C" int64_t bfs_batch_device_bytes(const bfs_batch* b) { return b ? b->device_bytes : 0; }

extern "C" int bfs_batch_create(const bfs_graph* g, int32_t with_parents, int32_t ctas, bfs_batch** out) {
  if (!g || !out) return fail(BFS_ERR_INVALID, "graph or out is NULL");
  if (ctas < 0) return fail(BFS_ERR_INVALID, "ctas must be >= 0");
  *out = nullptr;
  bfs_batch* b = new (std::nothrow) bfs_batch();
  if (!b) return fail(BFS_ERR_OOM, "host allocation failed");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != g->device) cudaSetDevice(g->device);
  b->g = g;
  b->with_parents = with_parents ? 1 : 0;
  const size_t nn = (size_t)g->n_ni + 1;
  int rc = BFS_OK;
  if (!rc) rc = balloc((void**)&b->visit, nn * 8, b, "alloc visit words");
  if (!rc) rc = balloc((void**)&b->F, 3 * nn * 8, b, "alloc frontier words");
  if (!rc) rc = balloc((void**)&b->depth_i, (size_t)kMsLanes * nn, b, "alloc batch depths");
  if (!rc && with_parents) rc = balloc((void**)&b->parent_i, (size_t)kMsLanes * nn * 4, b, "alloc batch parents");
  if (!rc) rc = balloc((void**)&b->CL, 2 * (size_t)g->cl_cap * sizeof(int2), b, "alloc chunk lists");
  if (!rc) rc = balloc((void**)&b->DL, (size_t)g->cl_cap * sizeof(MsDefer), b, "alloc deferred chunks");
  if (!rc) rc = balloc((void**)&b->slot, 4 * sizeof(MsSlot), b, "alloc counters");
  if (!rc) rc = balloc((void**)&b->log, BFS_BATCH_LOG_LEVELS * sizeof(MsLog), b, "alloc batch log");
  if (!rc) rc = balloc((void**)&b->hdr, sizeof(RunHeader), b, "alloc header");
  if (!rc) rc = balloc((void**)&b->arrive, (size_t)kMaxBlocks * 4 * 8, b, "alloc barrier words");
  if (!rc) {
    cudaError_t e = cudaMemset(b->hdr, 0, sizeof(RunHeader));
    if (e == cudaSuccess) e = cudaMemset(b->arrive, 0, (size_t)kMaxBlocks * 4 * 8);
    if (e != cudaSuccess) rc = cuda_fail(e, "memset batch header");
  }
  if (!rc) {
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
    cudaError_t e = ms_occupancy(&per_sm);
    if (e != cudaSuccess) rc = cuda_fail(e, "occupancy");
    else if (per_sm < 1) rc = fail(BFS_ERR_CUDA, "multi-source kernel does not fit on an SM");
    else {
      const int cap = sms * (per_sm < 2 ? per_sm : 2);
      if (ctas > cap) rc = fail(BFS_ERR_INVALID, "ctas exceeds the co-resident capacity");
      b->grid = ctas > 0 ? ctas : cap;
    }
  }
  if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
  if (rc) {
    std::string msg = bfs_last_error();
    batch_free_all(b);
    delete b;
    set_error(msg);
    return rc;
  }
  *out = b;
  return BFS_OK;
}

namespace bfsgb {

int64_t ms_batch_bytes(const bfs_graph* g, int with_parents) {
  const int64_t nn = (int64_t)g->n_ni + 1;
  return nn * 8 * 4 + (int64_t)kMsLanes * nn * (with_parents ? 5 : 1) + 2 * (int64_t)g->cl_cap * 8 +
         (int64_t)g->cl_cap * (int64_t)sizeof(MsDefer) +
         4 * (int64_t)sizeof(MsSlot) + BFS_BATCH_LOG_LEVELS * (int64_t)sizeof(MsLog) + (int64_t)sizeof(RunHeader) +
         (int64_t)kMaxBlocks * 32;
}

int ms_header_status(const RunHeader& h, unsigned epoch) {
  if (h.err != 0 && (h.err >> 4) == (epoch & 0x0FFFFFFFu)) {
    const int code = -(int)(h.err & 0xFu);
    return fail(code, code == BFS_ERR_OVERFLOW ? "a depth exceeds 254 (uint8 depth of the batched form)"
                                               : "a device-side wait of the multi-source loop passed its deadline");
  }
  return BFS_OK;
}

int ms_launch(bfs_batch* b, const int32_t* sources, int k, uint8_t* const* depth, int32_t* const* parent,
              cudaStream_t s, RunHeader* hdr_out, unsigned* epoch_out) {
  const bfs_graph* g = b->g;
  MsParams p;
  std::memset(&p, 0, sizeof(p));
  p.off = g->off;
  p.col = g->col;
  p.deg = g->deg;
  p.caller_of = g->caller_of;
  p.internal_of = g->internal_of;
  const size_t nn = (size_t)g->n_ni + 1;
  p.visit = b->visit;
  p.F0 = b->F;
  p.F1 = b->F + nn;
  p.F2 = b->F + 2 * nn;
  p.depth_i = b->depth_i;
  p.parent_i = parent ? b->parent_i : nullptr;
  p.CL0 = b->CL;
  p.CL1 = b->CL + g->cl_cap;
  p.DL = b->DL;
  p.slot = b->slot;
  p.log = b->log;
  p.hdr = b->hdr;
  p.arrive = b->arrive;
  p.nnz = g->nnz;
  p.n = g->n;
  p.n_ni = g->n_ni;
  p.d = g->d;
  p.k = k;
  p.ls = (k + 3) & ~3;
  p.out_parents = parent ? 1 : 0;
  p.alpha = g->opt.alpha;
  p.timeout_ns = (unsigned long long)g->opt.barrier_timeout_ms * 1000000ull;
  p.run_timeout_ns = (unsigned long long)g->opt.run_timeout_ms * 1000000ull;
  for (int j = 0; j < k; ++j) {
    p.src_c[j] = sources[j];
    p.out_d[j] = depth[j];
    p.out_p[j] = parent ? parent[j] : nullptr;
  }
  p.epoch = ++b->epoch & 0x0FFFFFFFu;
  if (p.epoch == 0) p.epoch = ++b->epoch & 0x0FFFFFFFu;
  cudaError_t e = cudaSuccess;
  if (p.epoch == 1) {
    e = cudaMemsetAsync(b->arrive, 0, (size_t)kMaxBlocks * 4 * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(&b->hdr->release, 0, 8, s);
  }
  void* args[] = {&p};
  if (e == cudaSuccess)
    e = cudaLaunchCooperativeKernel(k <= 32 ? (const void*)ms_bfs_loop<unsigned> : (const void*)ms_bfs_loop<unsigned long long>,
                                    dim3(b->grid), dim3(kThreads), args, 0, s);
  if (e == cudaSuccess && hdr_out) e = cudaMemcpyAsync(hdr_out, b->hdr, sizeof(RunHeader), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "multi-source launch");
  if (epoch_out) *epoch_out = p.epoch;
  return BFS_OK;
}

}  // namespace bfsgb

extern "C" int bfs_run_batch(bfs_batch* b, const int32_t* sources, int32_t k, uint8_t* depth, int32_t* parent,
                             bfs_batch_stats* stats, struct CUstream_st* stream) {
  if (!b || !sources || !depth) return fail(BFS_ERR_INVALID, "batch, sources or depth is NULL");
  if (k < 1 || k > kMsLanes) return fail(BFS_ERR_INVALID, "k must be 1..64");
  if (parent && !b->with_parents) return fail(BFS_ERR_INVALID, "the batch context was created without parents");
  const bfs_graph* g = b->g;
  for (int j = 0; j < k; ++j)
    if (sources[j] < 0 || sources[j] >= g->n) return fail(BFS_ERR_INVALID, "source out of range");
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != g->device) cudaSetDevice(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  const bool dd = dev_ptr(depth);
  if (parent && dev_ptr(parent) != dd) {
    if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
    return fail(BFS_ERR_INVALID, "depth and parent must both be device or both be host memory");
  }
  int rc = BFS_OK;
  uint8_t* od = depth;
  int32_t* op = parent;
  uint8_t* pd = dd ? nullptr : static_cast<uint8_t*>(pinned_device_ptr(depth));
  int32_t* pp = (dd || !parent) ? nullptr : static_cast<int32_t*>(pinned_device_ptr(parent));
  const bool direct = !dd && pd && (!parent || pp);  // page-locked host buffers, written directly
  if (direct) {
    od = pd;
    op = pp;
  } else if (!dd) {
    if (!b->out_depth) rc = balloc((void**)&b->out_depth, (size_t)kMsLanes * g->n, b, "alloc batch output");
    if (!rc && b->with_parents && !b->out_parent)
      rc = balloc((void**)&b->out_parent, (size_t)kMsLanes * g->n * 4, b, "alloc batch output");
    od = b->out_depth;
    op = parent ? b->out_parent : nullptr;
  }
  unsigned epoch = 0;
  if (!rc) {
    uint8_t* dl[kMsLanes];
    int32_t* pl[kMsLanes];
    for (int j = 0; j < k; ++j) {
      dl[j] = od + (int64_t)j * g->n;
      pl[j] = op ? op + (int64_t)j * g->n : nullptr;
    }
    rc = ms_launch(b, sources, k, dl, op ? pl : nullptr, s, nullptr, &epoch);
  }
  cudaError_t e = cudaSuccess;
  if (!rc && !dd && !direct) {
    e = cudaMemcpyAsync(depth, od, (size_t)k * g->n, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && parent) e = cudaMemcpyAsync(parent, op, (size_t)k * g->n * 4, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) rc = cuda_fail(e, "copy batch results");
  }
  if (!rc && (!dd || stats)) {
    e = cudaStreamSynchronize(s);
    RunHeader h;
    if (e == cudaSuccess) e = cudaMemcpy(&h, b->hdr, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
      rc = cuda_fail(e, "bfs_run_batch");
    } else {
      rc = ms_header_status(h, epoch);
      if (!rc && stats) {
        std::memset(stats, 0, sizeof(*stats));
        stats->levels = h.levels;
        stats->pairs_reached = (int64_t)h.reached;
        stats->traversed_edges = (int64_t)(h.reached_edges / 2);
        stats->device_ns = h.t1 - h.t0;
        stats->setup_ns = h.t_init - h.t0;
        stats->result_ns = h.t1 - h.t_loop;
        stats->logged_levels = h.levels_run < BFS_BATCH_LOG_LEVELS ? h.levels_run : BFS_BATCH_LOG_LEVELS;
        MsLog lg[BFS_BATCH_LOG_LEVELS];
        if (stats->logged_levels > 0 &&
            cudaMemcpy(lg, b->log, sizeof(MsLog) * stats->logged_levels, cudaMemcpyDeviceToHost) == cudaSuccess) {
          for (int L = 0; L < stats->logged_levels; ++L) {
            bfs_batch_level& o = stats->level[L];
            o.direction = lg[L].dir;
            o.pulled_lanes = lg[L].pad;
            o.frontier_vertices = (int64_t)lg[L].nfv;
            o.frontier_edges = (int64_t)lg[L].mfv;
            o.pairs = (int64_t)lg[L].pairs;
            o.t_begin_ns = lg[L].t_begin;
            o.t_expand_ns = lg[L].t_expand;
            o.t_end_ns = lg[L].t_end;
          }
        }
      }
    }
  }
  if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
  return rc;
}

extern "C" int bfs_batch_wait(bfs_batch* b, struct CUstream_st* stream) {
  if (!b) return fail(BFS_ERR_INVALID, "batch is NULL");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "bfs_batch_wait");
  RunHeader h;
  e = cudaMemcpy(&h, b->hdr, sizeof(h), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read batch header");
  return ms_header_status(h, b->epoch);
}

extern "C" void bfs_batch_free(bfs_batch* b) {
  if (!b) return;
  cudaDeviceSynchronize();
  batch_free_all(b);
  delete b;
}

namespace bfsgb {
namespace {

// One warp per query: the degree sum of the source's neighbours (0 for an
// isolated source), the size of the query's second frontier in entries.
__global__ void k_order_keys(const int64_t* __restrict__ off, const int32_t* __restrict__ col,
                             const int32_t* __restrict__ deg, const int32_t* __restrict__ internal_of, int32_t n_ni,
                             const int32_t* __restrict__ src, int32_t k, unsigned long long* __restrict__ key) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; j < k; j += nwarps) {
    const int u = internal_of[src[j]];
    unsigned long long s = 0;
    if (u >= 0 && u < n_ni)
      for (int64_t e = off[u] + lane; e < off[u + 1]; e += 32) s += (unsigned long long)deg[col[e]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if (lane == 0) key[j] = s;
  }
}

}  // namespace

// Keys of bfs_batch_order for k sources already on the device (dsrc), into the
// device array dkey; asynchronous on s.
int order_keys_async(const bfs_graph* g, const int32_t* dsrc, int32_t k, unsigned long long* dkey, cudaStream_t s) {
  if (k <= 0) return BFS_OK;
  const int blocks = (int)std::min<int64_t>(((int64_t)k * 32 + 255) / 256, 4096);
  k_order_keys<<<blocks, 256, 0, s>>>(g->off, g->col, g->deg, g->internal_of, g->n_ni, dsrc, k, dkey);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BFS_OK : cuda_fail(e, "order keys");
}

}  // namespace bfsgb

extern "C" int bfs_batch_order(const bfs_graph* g, const int32_t* sources, int32_t k, int32_t* order,
                               struct CUstream_st* stream) {
  using namespace bfsgb;
  if (!g || (k > 0 && (!sources || !order))) return fail(BFS_ERR_INVALID, "graph, sources or order is NULL");
  if (k < 0) return fail(BFS_ERR_INVALID, "k must be >= 0");
  for (int32_t j = 0; j < k; ++j)
    if (sources[j] < 0 || sources[j] >= g->n) return fail(BFS_ERR_INVALID, "source out of range");
  if (k == 0) return BFS_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  if (prev != g->device) cudaSetDevice(g->device);
  cudaStream_t s = (cudaStream_t)stream;
  int32_t* dsrc = nullptr;
  unsigned long long* dkey = nullptr;
  std::vector<unsigned long long> key((size_t)k);
  cudaError_t e = cudaMalloc(&dsrc, sizeof(int32_t) * (size_t)k);
  if (e == cudaSuccess) e = cudaMalloc(&dkey, sizeof(unsigned long long) * (size_t)k);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dsrc, sources, sizeof(int32_t) * (size_t)k, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && order_keys_async(g, dsrc, k, dkey, s) != BFS_OK) e = cudaErrorLaunchFailure;
  if (e == cudaSuccess) e = cudaMemcpyAsync(key.data(), dkey, sizeof(unsigned long long) * (size_t)k,
                                            cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (dsrc) cudaFree(dsrc);
  if (dkey) cudaFree(dkey);
  if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
  if (e != cudaSuccess) return cuda_fail(e, "bfs_batch_order");
  std::vector<int32_t> idx((size_t)k);
  for (int32_t j = 0; j < k; ++j) idx[(size_t)j] = j;
  std::stable_sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) { return key[(size_t)a] > key[(size_t)b]; });
  std::memcpy(order, idx.data(), sizeof(int32_t) * (size_t)k);
  return BFS_OK;
}
