// Level loop of direction-optimized BFS over a degree-separated graph: one
// persistent cooperative kernel per BFS run, so no level ever returns to the host.
//
// Per level L (frontier F_L = vertices at depth L):
//   forward (top-down, push; Sec. IV-A): normal vertices of F_L come from an int32
//     queue and are expanded a warp-batch at a time (one lane owns a vertex, the
//     warp gathers the 32 rows' entries together); delegates of F_L come from a
//     list of 512-entry row chunks, so a very high-degree row is spread over many
//     warps (merge-style partitioning, Sec. IV-A) and read with 128-bit loads.
//     Every unvisited target sets its bit in the discovered bitmap N, and (the
//     default) offers the frontier vertex's caller id to its parent by atomicMin.
//   backward (bottom-up, pull; Sec. II-C, IV-B): every unvisited non-isolated
//     vertex scans its row, which is sorted by caller id, and stops at the first
//     neighbour already visited; that neighbour is the canonical parent.
//   level end (fused): N is merged into the visited bitmap V; after a forward
//     level the same pass converts N into the next queue and chunk list, writes
//     the depths and counts the new frontier.
//   direction (Sec. IV-B): chosen from the frontier counters by every CTA alike.
// When a backward level is followed by a forward one, the bitmap of the new
// frontier is converted into the queue and chunk list first.  Work is assigned
// statically (warp w takes items w, w + warps, ...) and counters are added once
// per CTA, so no single global counter is contended.
//
// Every grid-barrier wait is bounded by a %globaltimer deadline; on expiry the
// kernel records BFS_ERR_TIMEOUT and every CTA returns.
#include <climits>

#include "bfs_internal.cuh"
#include "device_common.cuh"

namespace bfsgb {
namespace {

struct Acc {
  unsigned long long nf = 0, mf = 0, edges = 0, scanned = 0, fix = 0;
};

// Adds every thread's Acc into global counters with one atomic per CTA and
// counter (the targets may be null).  Called by all threads of the CTA.
__device__ void flush_block(Acc& a, unsigned long long* nf, unsigned long long* mf, unsigned long long* edges,
                            unsigned long long* scanned, unsigned long long* fix) {
  __shared__ unsigned long long s_red[5];
  if (threadIdx.x < 5) s_red[threadIdx.x] = 0;
  __syncthreads();
  const unsigned long long x[5] = {warp_sum(a.nf), warp_sum(a.mf), warp_sum(a.edges), warp_sum(a.scanned),
                                   warp_sum(a.fix)};
  if (lane_id() == 0)
#pragma unroll
    for (int i = 0; i < 5; ++i)
      if (x[i]) atomicAdd(&s_red[i], x[i]);
  __syncthreads();
  unsigned long long* t[5] = {nf, mf, edges, scanned, fix};
  if (threadIdx.x < 5 && s_red[threadIdx.x] && t[threadIdx.x]) atomicAdd(t[threadIdx.x], s_red[threadIdx.x]);
  a = Acc();
}

// Depth is kept as 4-bit nibbles, eight vertices per 32-bit word (nibble
// plane k holds bits 4k..4k+3 of every vertex's depth; plane 0 alone covers
// depths below 16).  The owner of a visited-bitmap word w writes the nibbles of
// the word's vertices f found at depth D as one 16-byte store or OR, instead of
// a 4-byte store per vertex, and the result pass reads one word per 8 vertices.
// Plane 0 is cleared by the run's set-up; plane k >= 1 is first needed at
// D = 16^k, and that level's word owners store there, clearing what an earlier
// run left.  A vertex's depth is nonzero unless it is the source or unreached.

// The 32 bits of f spread to 32 nibbles (four words of eight), each nibble = x
// (0..15) where its bit is set.
__device__ __forceinline__ uint4 spread_nibbles(unsigned f, unsigned x) {
  unsigned q[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    unsigned b = (f >> (8 * i)) & 0xFFu;
    b = (b | (b << 12)) & 0x000F000Fu;
    b = (b | (b << 6)) & 0x03030303u;
    b = (b | (b << 3)) & 0x11111111u;
    q[i] = b * x;
  }
  return make_uint4(q[0], q[1], q[2], q[3]);
}

// Called once per word by the level's owner of visited-bitmap word w (an
// all-word pass) with the word's vertices f found at depth D.
__device__ __forceinline__ void plane_store(const BfsParams& p, int64_t w, unsigned f, int D) {
  if (!BFS_IN(p, w, p.words)) return;
  uint4* p0 = reinterpret_cast<uint4*>(p.planes) + w;
  if (f && (D & 15)) {
    const uint4 a = spread_nibbles(f, (unsigned)(D & 15));
    uint4 o = *p0;
    o.x |= a.x;
    o.y |= a.y;
    o.z |= a.z;
    o.w |= a.w;
    *p0 = o;
  }
  if (D >= 16) {
    for (int k = 1; k < p.planes_n; ++k) {
      const unsigned x = (unsigned)(D >> (4 * k)) & 15u;
      uint4* pk = reinterpret_cast<uint4*>(p.planes + (int64_t)k * p.pstride) + w;
      if (D == (1 << (4 * k))) {
        *pk = spread_nibbles(f, x);
      } else if (f && x) {
        const uint4 a = spread_nibbles(f, x);
        uint4 o = *pk;
        o.x |= a.x;
        o.y |= a.y;
        o.z |= a.z;
        o.w |= a.w;
        *pk = o;
      }
    }
  }
}

// Depth nibbles of one vertex found at depth D outside an all-word pass (level 0
// from the source's row, deferred long rows): atomics, after the owners' stores.
__device__ __forceinline__ void plane_or(const BfsParams& p, int v, int D) {
  if (!BFS_IN(p, v, p.n_ni)) return;
  for (int k = 0; k < p.planes_n && (D >> (4 * k)); ++k) {
    const unsigned x = (unsigned)(D >> (4 * k)) & 15u;
    if (x) atomicOr(p.planes + (int64_t)k * p.pstride + (v >> 3), x << (4 * (v & 7)));
  }
}

// Visited-state probe for the pull scans, against the level's visited bitmap Vc
// (vertices at depth <= L; read-only during level L, whose discoveries go to the
// other buffer).  For an unvisited vertex (backward) or one found in level L
// (parent pick after a forward level) a neighbour in Vc is at depth L exactly.
// With kSub (per-subgraph directions), only neighbours of the classes in cls
// count: bit 0 delegates, bit 1 normal vertices.
template <bool kFix, bool kSub = false>
__device__ __forceinline__ bool probe(const BfsParams& p, int c, const uint32_t* __restrict__ Vc, unsigned cls = 3u) {
  if constexpr (kSub) {
    if (!((c < p.d) ? (cls & 1u) : (cls & 2u))) return false;
  }
  if (!BFS_IN(p, c, p.n_ni)) return false;
  return (Vc[c >> 5] >> (c & 31)) & 1u;
}

// Whole-warp scan of row entries [from, end) of a row starting at rbeg, 128
// entries (one 128-bit load per lane) per step; returns the first entry passing
// the probe (or -1) and kv = its position in the row + 1 (or end - rbeg).
template <bool kFix, bool kSub = false>
__device__ int warp_scan(const BfsParams& p, int64_t rbeg, int64_t from, int64_t end,
                         const uint32_t* __restrict__ Ncur, int64_t& kv, unsigned cls = 3u) {
  const int lane = lane_id();
  for (int64_t j0 = from & ~(int64_t)3; j0 < end; j0 += 128) {
    const int64_t j = j0 + lane * 4;
    unsigned best = 0xFFFFFFFFu;
    int bc = -1;
    if (j < end && BFS_IN(p, j + 3, p.nnz + kColPad)) {
      const int4 c4 = __ldg(reinterpret_cast<const int4*>(p.col + j));
      const int cs[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
      for (int t = 3; t >= 0; --t) {
        const int64_t idx = j + t;
        if (idx >= from && idx < end && probe<kFix, kSub>(p, cs[t], Ncur, cls)) {
          best = (unsigned)(idx - rbeg);
          bc = cs[t];
        }
      }
    }
    const unsigned wbest = __reduce_min_sync(kFull, best);
    if (wbest != 0xFFFFFFFFu) {
      const unsigned who = __ballot_sync(kFull, best == wbest);
      kv = (int64_t)wbest + 1;
      return __shfl_sync(kFull, bc, __ffs(who) - 1);
    }
  }
  kv = end - rbeg;
  return -1;
}

// Phases B and C of a pull scan: lanes with `more` have scanned the first
// kHead entries of their row [beg,end) without a hit.
//  B: rows with at most kShort entries left go to groups of kTailLanes (4)
//     lanes, eight rows at a time; each lane loads kTailPerLane (4) entries with
//     one 128-bit load, so a group reads 16 entries (64 bytes) per step, from a
//     4-entry boundary with the entries before the tail masked;
//  C: longer rows are finished by the whole warp, one row at a time, 128 entries
//     per step.
// On a hit, hit/k are set (k = first-hit position + 1); otherwise k = end - beg.
// With `defer` (backward levels), long rows are not scanned here: the lane's
// vertex and row start go to the level's long-row list and hit becomes kDeferred.
constexpr int kDeferred = -2;

template <bool kFix, bool kSub = false>
__device__ void pull_rest(const BfsParams& p, bool more, int64_t beg, int64_t end, const uint32_t* __restrict__ Ncur,
                          int& hit, int64_t& k, int defer_v = -1, LevelSlot* defer_slot = nullptr, unsigned cls = 3u) {
  constexpr int G = kTailLanes, P = kTailPerLane, R = 32 / G, S = G * P;
  static_assert(G == 2 || G == 4 || G == 8 || G == 16, "group scan: 2, 4, 8 or 16 lanes per row");
  static_assert(P == 1 || P == 2 || P == 4, "group scan: 1 entry, or one 64- or 128-bit load per lane");
  constexpr unsigned kGroupMask = (1u << G) - 1u;
  const int lane = lane_id();
  if (more) k = end - beg;
  const bool longrow = more && (end - beg - kHead) > kShort;
  unsigned rem = __ballot_sync(kFull, more && !longrow);
  const int g = lane / G, sub = lane % G;
  while (rem) {
    const int take = min(__popc(rem), R);
    unsigned r = rem;
    for (int q = 0; q < g && q < R - 1; ++q) r &= r - 1;
    const int srcl = (g < take) ? (__ffs(r) - 1) : 0;
    const int64_t rbeg = __shfl_sync(kFull, beg, srcl);
    const int64_t rend = __shfl_sync(kFull, end, srcl);
    // the group probes with the row owner's classes (kSub), not its own
    const unsigned gcls = kSub ? __shfl_sync(kFull, cls, srcl) : cls;
    const int64_t from = rbeg + kHead;
    bool gdone = g >= take;
    int ghit = -1;
    int64_t gk = 0;
    // with 128-bit loads a step starts on a 4-entry boundary; entries before
    // `from` are masked
    int64_t pos = from & ~(int64_t)(P - 1);
    while (__any_sync(kFull, !gdone)) {
      const int64_t j = pos + sub * P;
      int c = -1, t0 = 0;  // this lane's first passing entry and its offset in the lane's P entries
      if (!gdone && j < rend && BFS_IN(p, j + P - 1, p.nnz + kColPad)) {
        if constexpr (P == 1) {
          const int c1 = p.col[j];
          if (probe<kFix, kSub>(p, c1, Ncur, gcls)) c = c1;
        } else {
          int cs[P];
          if constexpr (P == 4) {
            const int4 c4 = __ldg(reinterpret_cast<const int4*>(p.col + j));
            cs[0] = c4.x;
            cs[1] = c4.y;
            cs[2] = c4.z;
            cs[3] = c4.w;
          } else {
            const int2 c2 = __ldg(reinterpret_cast<const int2*>(p.col + j));
            cs[0] = c2.x;
            cs[1] = c2.y;
          }
          bool hh[P];
#pragma unroll
          for (int t = 0; t < P; ++t) hh[t] = j + t >= from && j + t < rend && probe<kFix, kSub>(p, cs[t], Ncur, gcls);
#pragma unroll
          for (int t = P - 1; t >= 0; --t)
            if (hh[t]) {
              c = cs[t];
              t0 = t;
            }
        }
      }
      const unsigned gb = (__ballot_sync(kFull, c >= 0) >> (g * G)) & kGroupMask;
      const int first = gb ? __ffs(gb) - 1 : 0;
      const int hc = __shfl_sync(kFull, c, g * G + first);
      const int ht = P == 1 ? 0 : __shfl_sync(kFull, t0, g * G + first);
      if (!gdone) {
        if (gb) {
          ghit = hc;
          gk = pos + first * P + ht - rbeg + 1;
          gdone = true;
        } else {
          pos += S;
          if (pos >= rend) {
            gdone = true;
            gk = rend - rbeg;
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const int h2 = __shfl_sync(kFull, ghit, q * G);
      const int64_t k2 = __shfl_sync(kFull, gk, q * G);
      const int owner = __shfl_sync(kFull, srcl, q * G);
      if (q < take && lane == owner) {
        hit = h2;
        k = k2;
      }
    }
    for (int q = 0; q < take; ++q) rem &= rem - 1;
  }
  unsigned lrem = __ballot_sync(kFull, longrow);
  if (defer_slot && lrem) {
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(&defer_slot->nlong, (unsigned long long)__popc(lrem));
    base = __shfl_sync(kFull, base, 0);
    if (longrow) {
      const unsigned long long at = base + __popc(lrem & ((1u << lane) - 1u));
      if (BFS_IN(p, at, p.long_cap)) p.longq[at] = defer_v;
      hit = kDeferred;
    }
    lrem = 0;
  }
  while (lrem) {
    const int owner = __ffs(lrem) - 1;
    lrem &= lrem - 1;
    const int64_t rbeg = __shfl_sync(kFull, beg, owner);
    const int64_t rend = __shfl_sync(kFull, end, owner);
    const unsigned ocls = kSub ? __shfl_sync(kFull, cls, owner) : cls;
    int64_t k2;
    const int h2 = warp_scan<kFix, kSub>(p, rbeg, rbeg + kHead, rend, Ncur, k2, ocls);
    if (lane == owner) {
      hit = h2;
      k = k2;
    }
  }
}

// Phase A of a pull scan, one vertex per lane: loads the head record of v (its
// first kHead neighbours and their caller ids, one coalesced sector) and its
// degree.  Split from the probes so a caller can put several vertices' loads in
// flight before the first probe.
struct HeadRec {
  int nb[kHead], cid[kHead];
  int deg;
};

__device__ __forceinline__ HeadRec head_load(const BfsParams& p, bool act, int v) {
  HeadRec h;
#pragma unroll
  for (int t = 0; t < kHead; ++t) h.nb[t] = h.cid[t] = -1;
  h.deg = 0;
  if (act && BFS_IN(p, v, p.n_ni)) {
    if constexpr (kHead >= 4) {
#pragma unroll
      for (int t = 0; t < kHead; t += 4) {
        const int4 a = __ldg(p.head + kHeadVecs * (int64_t)v + t / 4);
        const int4 b = __ldg(p.head + kHeadVecs * (int64_t)v + kHead / 4 + t / 4);
        h.nb[t] = a.x;
        h.nb[t + 1] = a.y;
        h.nb[t + 2] = a.z;
        h.nb[t + 3] = a.w;
        h.cid[t] = b.x;
        h.cid[t + 1] = b.y;
        h.cid[t + 2] = b.z;
        h.cid[t + 3] = b.w;
      }
    } else {
      const int4 a = __ldg(p.head + (int64_t)v);
      h.nb[0] = a.x;
      h.nb[1] = a.y;
      h.cid[0] = a.z;
      h.cid[1] = a.w;
    }
    h.deg = __ldg(p.deg + v);
  }
  return h;
}

// Probes the head entries of a loaded record: first hit (internal id, caller
// id) and k = its position + 1, or k = min(degree, kHead) and hit = -1.
template <bool kFix, bool kSub = false>
__device__ __forceinline__ void head_probe(const BfsParams& p, const HeadRec& h, const uint32_t* __restrict__ Ncur,
                                           int& hit, int& cid, int64_t& k, unsigned cls = 3u) {
  const int* nb = h.nb;
  const int* cs = h.cid;
  bool hh[kHead];
#pragma unroll
  for (int t = 0; t < kHead; ++t) hh[t] = nb[t] >= 0 && probe<kFix, kSub>(p, nb[t], Ncur, cls);
  hit = -1;
  cid = -1;
  k = h.deg < kHead ? h.deg : kHead;
#pragma unroll
  for (int t = kHead - 1; t >= 0; --t)
    if (hh[t]) {
      hit = nb[t];
      cid = cs[t];
      k = t + 1;
    }
}

// Phases B/C for the lanes whose row continues past the head entries without a
// hit: loads the row offset and finishes the scan (warp-collective).
template <bool kFix, bool kSub = false>
__device__ __forceinline__ void pull_tail(const BfsParams& p, bool act, int v, int deg,
                                          const uint32_t* __restrict__ Ncur, int& hit, int& cid, int64_t& k,
                                          LevelSlot* defer_slot = nullptr, unsigned cls = 3u) {
  const bool more = act && hit < 0 && deg > kHead;
  int64_t beg = 0, end = 0;
  if (more) {
    beg = p.off[v];
    end = beg + deg;
  }
  pull_rest<kFix, kSub>(p, more, beg, end, Ncur, hit, k, v, defer_slot, cls);
  if (more && hit >= 0) cid = p.caller_of[hit];
}

// Pull scan, one vertex per lane: lanes with `act` scan the row of v in order
// and stop at the first neighbour passing the probe.  Returns the neighbour's
// internal id or -1, its caller id in hit_cid, kv = entries examined (first-hit
// position + 1, or the degree), and the degree.
template <bool kFix>
__device__ int pull_head(const BfsParams& p, bool act, int v, const uint32_t* __restrict__ Ncur, int64_t& kv,
                         int& hit_cid, int& degree) {
  const HeadRec h = head_load(p, act, v);
  int hit = -1, cid = -1;
  int64_t k = 0;
  if (act) head_probe<kFix>(p, h, Ncur, hit, cid, k);
  pull_tail<kFix>(p, act, v, h.deg, Ncur, hit, cid, k);
  kv = k;
  hit_cid = cid;
  degree = h.deg;
  return hit;
}

// ---- forward level ------------------------------------------------------------------------

// Four row entries of one lane: the four visited-bit probes are issued before
// any reduction, so they are in flight together.
template <bool kSub = false>
__device__ __forceinline__ void td_edge4(const BfsParams& p, const uint32_t* __restrict__ Vc, const int (&v)[4],
                                         int pcaller, uint32_t* __restrict__ N, bool& found, unsigned allow = 3u) {
  unsigned vw[4];
#pragma unroll
  for (int t = 0; t < 4; ++t) vw[t] = (v[t] >= 0 && BFS_IN(p, v[t], p.n_ni)) ? Vc[(unsigned)v[t] >> 5] : kFull;
  // consecutive row entries often fall in one bitmap word (delegates are numbered in
  // caller order, and rows are sorted by caller id): their discovered bits are
  // OR-ed together and set with one atomic per run of equal words
  unsigned rw = 0xFFFFFFFFu, rb = 0u;
  // the targets' parent slots are read first and only a smaller offer is sent:
  // a hub frontier offers each delegate target several parents, and the L2's
  // atomic rate bounds such a level; a stale read only costs an extra atomic
  // (parents only decrease)
  int pcur[4];
#pragma unroll
  for (int t = 0; t < 4; ++t)
    pcur[t] = (v[t] >= 0 && !((vw[t] >> (v[t] & 31)) & 1u) && p.td_parent == BFS_TD_PARENT_ATOMICMIN) ? __ldcg(p.parent_i + v[t]) : INT_MIN;
#pragma unroll
  for (int t = 0; t < 4; ++t) {
    if (v[t] < 0 || ((vw[t] >> (v[t] & 31)) & 1u)) continue;
    if constexpr (kSub) {
      if (!((v[t] < p.d) ? (allow & 1u) : (allow & 2u))) continue;
    }
    found = true;
    if (pcur[t] > pcaller) atomicMin(p.parent_i + v[t], pcaller);
    // a parent slot already offered at this level: its first offerer sets the bit
    if (!kSub && pcur[t] != INT_MAX && pcur[t] != INT_MIN) continue;
    const unsigned w = (unsigned)v[t] >> 5, bit = 1u << (v[t] & 31);
    if (w != rw) {
      if (rb) atomicOr(N + rw, rb);
      rw = w;
      rb = 0u;
    }
    if (!(p.tuning & 1) || !(__ldcg(N + w) & bit)) rb |= bit;
  }
  if (rb) atomicOr(N + rw, rb);
}

// 32 normal-queue entries: lane i owns vertex Qc[b*32+i]; the warp walks the
// concatenation of the 32 rows 128 entries at a time, four per lane (entry e
// belongs to the lane whose inclusive degree prefix first exceeds e).
template <bool kSub = false>
__device__ void td_batch(const BfsParams& p, const uint32_t* __restrict__ Vc, const int32_t* __restrict__ Qc,
                         int64_t qn, int64_t b, uint32_t* __restrict__ N, bool& found, unsigned allow = 3u) {
  const int lane = lane_id();
  const int64_t i = b * 32 + lane;
  const int u = i < qn ? Qc[i] : -1;
  int64_t beg = 0, deg = 0;
  int cu = INT_MAX;  // the frontier vertex's caller id, loaded with its row bounds
  if (u >= 0 && BFS_IN(p, u, p.n_ni)) {
    beg = p.off[u];
    deg = p.deg[u];
    if (p.td_parent == BFS_TD_PARENT_ATOMICMIN) cu = p.caller_of[u];
  }
  const int64_t incl = warp_incl_scan(deg);
  const int64_t total = __shfl_sync(kFull, incl, 31);
  const int64_t excl = incl - deg;
  // up to four entries per lane per step (entries base + lane + 32 t), their
  // column loads and visited probes in flight together
  for (int64_t base = 0; base < total; base += 128) {
    int v[4], ou[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int64_t e = base + lane + 32 * t;
      int pos = 0;
#pragma unroll
      for (int s = 16; s >= 1; s >>= 1) {
        const int64_t x = __shfl_sync(kFull, incl, pos + s - 1);
        if (x <= e) pos += s;
      }
      const int64_t ob = __shfl_sync(kFull, beg, pos);
      const int64_t ox = __shfl_sync(kFull, excl, pos);
      ou[t] = __shfl_sync(kFull, cu, pos);
      v[t] = (e < total && BFS_IN(p, ob + (e - ox), p.nnz)) ? p.col[ob + (e - ox)] : -1;
    }
    unsigned un = 0;  // bit t: entry t meets an unvisited target
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (v[t] >= 0 && !BFS_IN(p, v[t], p.n_ni)) v[t] = -1;
      if constexpr (kSub) {  // per-subgraph directions: only targets of the classes in allow
        if (v[t] >= 0 && !((v[t] < p.d) ? (allow & 1u) : (allow & 2u))) v[t] = -1;
      }
      if (v[t] >= 0 && !((Vc[(unsigned)v[t] >> 5] >> (v[t] & 31)) & 1u)) un |= 1u << t;
    }
    if (!un) continue;
    found = true;
    // offers go out without reading the slot first (fire-and-forget reductions)
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (!((un >> t) & 1u)) continue;
      if (p.td_parent == BFS_TD_PARENT_ATOMICMIN) atomicMin(p.parent_i + v[t], ou[t]);
      const unsigned bit = 1u << (v[t] & 31);
      uint32_t* nw = N + ((unsigned)v[t] >> 5);
      if (!(p.tuning & 1) || !(__ldcg(nw) & bit)) atomicOr(nw, bit);
    }
  }
}

// One kChunk-entry piece of a delegate's row, 128-bit loads.
template <bool kSub = false>
__device__ void td_chunk(const BfsParams& p, const uint32_t* __restrict__ Vc, int2 ck, uint32_t* __restrict__ N,
                         bool& found, unsigned allow = 3u) {
  const int lane = lane_id();
  const int u = ck.x;
  if (!BFS_IN(p, u, p.n_ni)) return;
  const int64_t rb = p.off[u], re = p.off[u + 1];
  const int64_t beg = rb + (int64_t)ck.y * kChunk;
  const int64_t end = min(beg + kChunk, re);
  const int pc = (p.td_parent == BFS_TD_PARENT_ATOMICMIN) ? p.caller_of[u] : 0;
  // two 128-bit column loads per lane per step (256 entries per warp)
  for (int64_t j0 = beg & ~(int64_t)3; j0 < end; j0 += 256) {
    const int64_t ja = j0 + lane * 4, jb = ja + 128;
    int4 ca = make_int4(-1, -1, -1, -1), cb = ca;
    if (ja < end) ca = __ldg(reinterpret_cast<const int4*>(p.col + ja));
    if (jb < end) cb = __ldg(reinterpret_cast<const int4*>(p.col + jb));
    if (ja < end) {
      const int v[4] = {ja >= beg ? ca.x : -1, (ja + 1 >= beg && ja + 1 < end) ? ca.y : -1,
                        (ja + 2 >= beg && ja + 2 < end) ? ca.z : -1, (ja + 3 >= beg && ja + 3 < end) ? ca.w : -1};
      td_edge4<kSub>(p, Vc, v, pc, N, found, allow);
    }
    if (jb < end) {
      const int v[4] = {cb.x, jb + 1 < end ? cb.y : -1, jb + 2 < end ? cb.z : -1, jb + 3 < end ? cb.w : -1};
      td_edge4<kSub>(p, Vc, v, pc, N, found, allow);
    }
  }
}

// Work split: warp w first takes item w; items beyond the first `warps` are
// handed out from a shared counter in runs of g (about four runs per warp), so
// warps that drew light items take over the rest without one atomic per item.
// With no more items than warps the counter is never touched.
struct WorkCursor {
  long long it, lim, total, nwarps, g;
  unsigned long long* ctr;
  __device__ WorkCursor(long long total_, long long gwarp, long long nwarps_, unsigned long long* ctr_)
      : it(gwarp), lim(gwarp + 1), total(total_), nwarps(nwarps_), ctr(ctr_) {
    const long long rest = total_ - nwarps_;
    g = rest > 0 ? (rest + 4 * nwarps_ - 1) / (4 * nwarps_) : 1;
  }
  // next item of this warp, or a value >= total when there is none (warp-uniform)
  __device__ long long next() {
    if (it < lim) return it++;
    if (total <= nwarps) return total;
    unsigned long long x = 0;
    if (lane_id() == 0) x = atomicAdd(ctr, (unsigned long long)g);
    it = nwarps + (long long)__shfl_sync(kFull, x, 0);
    lim = it + g;
    return it++;
  }
};

// Work items of a forward level: the delegate chunks of F_L, then the normal
// queue in batches of 32; warp w takes items w, w + warps, ... (a shared counter
// measured slower here: the chunks are uniform).
// With kSub, allow_n / allow_d are the target classes that normal / delegate
// frontier vertices push to (bit 0 delegates, bit 1 normal vertices).
template <bool kSub = false>
__device__ void expand_td(const BfsParams& p, const uint32_t* __restrict__ Vc, int L, bool& found,
                          unsigned allow_n = 3u, unsigned allow_d = 3u) {
  const LevelSlot* sc = p.slot + (L & (kSlots - 1));
  const int64_t qn = (int64_t)__ldcg(&sc->qn);
  const int64_t nch = (int64_t)__ldcg(&sc->nch);
  const int64_t total = nch + (qn + 31) / 32;
  const int32_t* Qc = (L & 1) ? p.Q1 : p.Q0;
  const int2* CLc = (L & 1) ? p.CL1 : p.CL0;
  uint32_t* N = (L & 1) ? p.N1 : p.N0;
  const int64_t gwarp = spread_warp();
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t it = gwarp; it < total; it += nwarps) {
    if (it < nch) {
      if (!kSub || allow_d) td_chunk<kSub>(p, Vc, CLc[it], N, found, allow_d);
    } else {
      td_batch<kSub>(p, Vc, Qc, qn, it - nch, N, found, allow_n);
    }
  }
}

// ---- backward level -----------------------------------------------------------------------

// Position of the r-th (0-based) set bit of m; r < popc(m).
__device__ __forceinline__ int nth_set_bit(unsigned m, int r) {
  int pos = 0;
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const int c = __popc(m & ((1u << s) - 1u));
    if (r >= c) {
      r -= c;
      m >>= s;
      pos += s;
    }
  }
  return pos;
}

// Appends the vertices of this lane's word bits f (vertices v0 .. v0+31) to the
// next forward level's lists: normal vertices to the queue Q, delegates as their
// kChunk-entry row chunks to CL, with one reservation per list and warp
// (warp-collective).  Backward levels with few unvisited vertices left call it,
// so that a switch back to forward finds its frontier lists ready.
__device__ void append_next(const BfsParams& p, int64_t v0, unsigned f, int32_t* __restrict__ Q,
                            int2* __restrict__ CL, LevelSlot* slot) {
  const int lane = lane_id();
  unsigned dmask = 0;  // delegate bits of this lane's word
  if (v0 < p.d) dmask = (p.d - v0 >= 32) ? kFull : ((1u << (p.d - v0)) - 1u);
  const unsigned fn = f & ~dmask, fd = f & dmask;
  if (__any_sync(kFull, fn != 0)) {
    const int c = __popc(fn);
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += t;
    }
    unsigned long long base = 0;
    if (lane == 31) base = atomicAdd(&slot->qn, (unsigned long long)incl);
    base = __shfl_sync(kFull, base, 31) + (unsigned long long)(incl - c);
    for (unsigned m = fn; m; m &= m - 1, ++base)
      if (BFS_IN(p, base, p.n_ni)) Q[base] = (int32_t)(v0 + __ffs(m) - 1);
  }
  if (__any_sync(kFull, fd != 0)) {
    long long c = 0;
    for (unsigned m = fd; m; m &= m - 1) c += ((long long)p.deg[v0 + __ffs(m) - 1] + kChunk - 1) / kChunk;
    long long incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long t = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += t;
    }
    unsigned long long base = 0;
    if (lane == 31) base = atomicAdd(&slot->nch, (unsigned long long)incl);
    base = __shfl_sync(kFull, base, 31) + (unsigned long long)(incl - c);
    for (unsigned m = fd; m; m &= m - 1) {
      const int v = (int)(v0 + __ffs(m) - 1);
      const int nc = (int)(((long long)p.deg[v] + kChunk - 1) / kChunk);
      for (int k = 0; k < nc; ++k, ++base)
        if (BFS_IN(p, base, p.cl_cap)) CL[base] = make_int2(v, k);
    }
  }
}

// One backward item: bitmap words [w0, w0+iw) (iw <= 32) of this warp.  Its
// unvisited vertices are gathered 32 at a time (lane i takes the i-th one), so a
// sparse item costs one batch, not one pass per word; two batches are in flight
// per step.  A vertex that finds its parent gets depth and parent; its bit is
// collected in the warp's shared copy of the item's words (the warp owns them)
// and each word is written to N once.
__device__ bool bu_item(const BfsParams& p, const uint32_t* __restrict__ Vc, uint32_t* __restrict__ Vn,
                        uint32_t* __restrict__ Nclr, int L, int64_t w0, int iw, unsigned* found,
                        uint32_t* __restrict__ N, LevelSlot* sc, Acc& acc, LevelSlot* qslot) {
  bool deferred = false;
  const int lane = lane_id();
  const int64_t W = p.words;
  const int tail = p.n_ni & 31;
  const int64_t w = w0 + lane;
  unsigned vis = kFull, vraw = 0;
  if (lane < iw && w < W) {
    vraw = Vc[w];
    vis = vraw;
    if (w == W - 1 && tail) vis |= ~((1u << tail) - 1u);
  }
  const unsigned unv = ~vis;
  const int cnt = __popc(unv);
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += t;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  const int excl = incl - cnt;
  // the k-th unvisited vertex of the item: word = first lane whose prefix exceeds k
  auto locate = [&](int k, int& j, int& bit) {
    j = 0;
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
      const int t = __shfl_sync(kFull, incl, j + s - 1);
      if (t <= k) j += s;
    }
    const unsigned m = __shfl_sync(kFull, unv, j);
    const int ex = __shfl_sync(kFull, excl, j);
    bit = k < total ? nth_set_bit(m, k - ex) : 0;
  };
  for (int b = 0; b < total; b += 64) {
    int jA, jB, bA, bB;
    locate(b + lane, jA, bA);
    locate(b + 32 + lane, jB, bB);
    const bool aA = b + lane < total, aB = b + 32 + lane < total;
    const int vA = (int)((w0 + jA) * 32 + bA), vB = (int)((w0 + jB) * 32 + bB);
    const HeadRec hA = head_load(p, aA, vA);
    const HeadRec hB = head_load(p, aB, vB);
    int hitA = -1, cidA = -1, hitB = -1, cidB = -1;
    int64_t kA = 0, kB = 0;
    if (aA) head_probe<false>(p, hA, Vc, hitA, cidA, kA);
    if (aB) head_probe<false>(p, hB, Vc, hitB, cidB, kB);
    pull_tail<false>(p, aA, vA, hA.deg, Vc, hitA, cidA, kA, sc);
    pull_tail<false>(p, aB, vB, hB.deg, Vc, hitB, cidB, kB, sc);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      deferred |= (q ? aB : aA) && (q ? hitB : hitA) == kDeferred;
      const bool act = (q ? aB : aA) && (q ? hitB : hitA) != kDeferred;
      const int hit = q ? hitB : hitA;
      const int v = q ? vB : vA;
      const int j = q ? jB : jA;
      // lanes of one batch that share a word are adjacent: OR their bits
      const unsigned fbit = (act && hit >= 0) ? (1u << (q ? bB : bA)) : 0u;
      const unsigned grp = __match_any_sync(kFull, (unsigned)j);
      const unsigned orb = __reduce_or_sync(grp, fbit);
      if (orb && lane == __ffs(grp) - 1) found[j] |= orb;
      if (!act) continue;
      acc.scanned += 1;
      acc.edges += (unsigned long long)(q ? kB : kA);
      if (hit >= 0 && BFS_IN(p, v, p.n_ni)) {
        p.parent_i[v] = q ? cidB : cidA;
        acc.nf += 1;
        acc.mf += (unsigned long long)(q ? hB.deg : hA.deg);
      }
    }
    __syncwarp();
  }
  // the warp owns its words: found bits, the next visited bitmap, and the other
  // discovered bitmap cleared for the level after (deferred rows add their bits
  // after the next grid barrier)
  unsigned f = 0u;
  if (lane < iw && w < W) {
    f = found[lane];
    N[w] = f;
    Vn[w] = vraw | f;
    Nclr[w] = 0u;
    found[lane] = 0u;
    plane_store(p, w, f, L + 1);
  }
  if (qslot) append_next(p, w * 32, f, (L & 1) ? p.Q0 : p.Q1, (L & 1) ? p.CL0 : p.CL1, qslot);
  __syncwarp();
  return deferred;
}

// Words of a dense backward item handled per step (their lead records are in
// flight together).
constexpr int kDenseStep = 4;

// Settles the pending vertices pend[0..cnt) (cnt <= 32, one per lane) of a dense
// backward item: their first entry missed, so they scan on from the full head
// record and the row tail, exactly as the sparse items do; found vertices get
// depth and parent and their bit in the warp's found words (item-relative).
__device__ bool bu_settle(const BfsParams& p, const uint32_t* __restrict__ Vc, int L, int64_t w0, const int* pend,
                          int cnt, unsigned* found, LevelSlot* sc, Acc& acc) {
  const int lane = lane_id();
  const bool act = lane < cnt;
  const int v = act ? pend[lane] : 0;
  const HeadRec h = head_load(p, act && BFS_IN(p, v, p.n_ni), v);
  int hit = -1, cid = -1;
  int64_t k = 0;
  if (act) head_probe<false>(p, h, Vc, hit, cid, k);
  pull_tail<false>(p, act, v, h.deg, Vc, hit, cid, k, sc);
  bool deferred = false;
  if (act) {
    if (hit == kDeferred) {
      deferred = true;
    } else {
      acc.scanned += 1;
      acc.edges += (unsigned long long)k;
      if (hit >= 0 && BFS_IN(p, (v >> 5) - w0, 32)) {
        p.parent_i[v] = cid;
        acc.nf += 1;
        acc.mf += (unsigned long long)h.deg;
        atomicOr(found + ((v >> 5) - w0), 1u << (v & 31));
      }
    }
  }
  __syncwarp();
  return __any_sync(kFull, deferred);
}

// A dense backward item (most vertices unvisited): bitmap words [w0, w0+iw),
// iw a multiple of kDenseStep up to 32.
// The 32 vertices of a word go to the 32 lanes (lane = bit), kDenseStep words
// per step: every unvisited vertex loads its lead record (first entry and its
// caller id; a warp reads 256 contiguous bytes per word) and degree, and probes
// the first entry.  A hit settles the vertex (canonical parent: the first entry
// in caller order); a miss with more entries joins the warp's pending list,
// settled 32 at a time by bu_settle.  No compaction, no per-vertex search.
__device__ bool bu_dense_item(const BfsParams& p, const uint32_t* __restrict__ Vc, uint32_t* __restrict__ Vn,
                              uint32_t* __restrict__ Nclr, int L, int64_t w0, int iw, unsigned* found, int* pend,
                              uint32_t* __restrict__ N, LevelSlot* sc, Acc& acc, LevelSlot* qslot) {
  bool deferred = false;
  const int lane = lane_id();
  const int64_t W = p.words;
  const int tail = p.n_ni & 31;
  const int64_t wl = w0 + lane;
  const bool own = lane < iw && wl < W;  // this lane's word belongs to the item
  unsigned vraw = 0, vis = kFull;
  if (own) {
    vraw = Vc[wl];
    vis = vraw;
    if (wl == W - 1 && tail) vis |= ~((1u << tail) - 1u);
  }
  unsigned fword = 0;  // first-entry hits of word w0 + lane
  int npend = 0;       // warp-uniform
  for (int s0 = 0; s0 < iw; s0 += kDenseStep) {
    int2 a[kDenseStep];
    int dg[kDenseStep];
    bool un[kDenseStep];
#pragma unroll
    for (int u = 0; u < kDenseStep; ++u) {
      un[u] = !((__shfl_sync(kFull, vis, s0 + u) >> lane) & 1u);
      const int v = (int)((w0 + s0 + u) * 32 + lane);
      un[u] = un[u] && BFS_IN(p, v, p.n_ni);
      a[u] = un[u] ? __ldg(p.lead + v) : make_int2(-1, -1);
      dg[u] = un[u] ? __ldg(p.deg + v) : 0;
    }
    unsigned pw[kDenseStep];
#pragma unroll
    for (int u = 0; u < kDenseStep; ++u) pw[u] = (a[u].x >= 0 && BFS_IN(p, a[u].x, p.n_ni)) ? Vc[a[u].x >> 5] : 0u;
#pragma unroll
    for (int u = 0; u < kDenseStep; ++u) {
      const int v = (int)((w0 + s0 + u) * 32 + lane);
      const bool h0 = un[u] && a[u].x >= 0 && ((pw[u] >> (a[u].x & 31)) & 1u);
      const bool more = un[u] && !h0 && dg[u] > 1;
      if (h0) {
        p.parent_i[v] = a[u].y;
        acc.nf += 1;
        acc.mf += (unsigned long long)dg[u];
      }
      if (un[u] && !more) {  // settled here: a first-entry hit, or a one-entry row that missed
        acc.scanned += 1;
        acc.edges += 1;
      }
      const unsigned hb = __ballot_sync(kFull, h0);
      if (lane == s0 + u) fword = hb;
      const unsigned mb = __ballot_sync(kFull, more);
      if (more) pend[npend + __popc(mb & ((1u << lane) - 1u))] = v;
      npend += __popc(mb);
    }
    // settle full batches once the step's records are dead (pend holds < 32 before the step)
    int done = 0;
    for (; npend - done >= 32; done += 32) {
      __syncwarp();
      deferred |= bu_settle(p, Vc, L, w0, pend + done, 32, found, sc, acc);
    }
    if (done) {
      const int rest = npend - done;
      const int x = lane < rest ? pend[done + lane] : 0;
      __syncwarp();
      if (lane < rest) pend[lane] = x;
      __syncwarp();
      npend = rest;
    }
  }
  if (npend > 0) {
    __syncwarp();
    deferred |= bu_settle(p, Vc, L, w0, pend, npend, found, sc, acc);
  }
  __syncwarp();
  unsigned f = 0u;
  if (own) {
    f = fword | found[lane];
    N[wl] = f;
    Vn[wl] = vraw | f;
    Nclr[wl] = 0u;
    plane_store(p, wl, f, L + 1);
  }
  found[lane] = 0u;
  if (qslot) append_next(p, wl * 32, f, (L & 1) ? p.Q0 : p.Q1, (L & 1) ? p.CL0 : p.CL1, qslot);
  __syncwarp();
  return deferred;
}

// A backward level: items of iw bitmap words (iw = 4..32, larger when few
// vertices are left), split statically; rows still unsettled after kHead +
// kShort entries are deferred to the level's long-row list, which all warps then
// drain with dynamic hand-out, one row per warp and 128-bit loads, so that long
// scans spread over the grid instead of stalling the warp that met them.
__device__ bool expand_bu(const BfsParams& p, const uint32_t* __restrict__ Vc, uint32_t* __restrict__ Vn,
                          uint32_t* __restrict__ Nclr, int L, int iw, Acc& acc, bool build_next, bool dense) {
  __shared__ unsigned s_found[kMaxWarpsPerBlock][32];
  __shared__ int s_pend[kMaxWarpsPerBlock][32 * (kDenseStep + 1)];
  uint32_t* N = (L & 1) ? p.N1 : p.N0;
  const int lane = lane_id();
  unsigned* found = s_found[threadIdx.x >> 5];
  found[lane] = 0u;
  __syncwarp();
  const int64_t W = p.words;
  const int64_t gwarp = spread_warp();
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  LevelSlot* sc = p.slot + (L & (kSlots - 1));
  const int64_t nitems = (W + iw - 1) / iw;
  bool deferred = false;
  LevelSlot* qslot = build_next ? p.slot + ((L + 1) & (kSlots - 1)) : nullptr;
  if (dense) {
    // items of 32 words, narrower (down to kDenseStep) until every warp has two
    int iwd = 32;
    while (iwd > kDenseStep && (W + iwd - 1) / iwd < 2 * nwarps) iwd >>= 1;
    int* pend = s_pend[threadIdx.x >> 5];
    for (int64_t it = gwarp; it * iwd < W; it += nwarps)
      deferred |= bu_dense_item(p, Vc, Vn, Nclr, L, it * iwd, iwd, found, pend, N, sc, acc, qslot);
    return deferred;
  }
  for (int64_t it = gwarp; it < nitems; it += nwarps)
    deferred |= bu_item(p, Vc, Vn, Nclr, L, it * iw, iw, found, N, sc, acc, qslot);
  return deferred;
}

// Backward pulls under per-subgraph directions (Sec. IV-B): an unvisited
// delegate pulls from the classes whose subgraph into the delegates is backward
// (cls_del: bit 0 dd, from delegates; bit 1 nd, from normal vertices), an
// unvisited normal vertex from the delegates when dn is backward (cls_norm bit
// 0).  The scan stops at the first neighbour of an allowed class in the
// visited bitmap; that neighbour is the smallest-id parent among those classes.
// A forward push of the same level may offer other parents, so the hit is
// offered by atomicMin and marked in N by atomicOr; the level end writes the
// depth.  Items of 32 bitmap words, 32 unvisited vertices per step.
__device__ void expand_bu_sub(const BfsParams& p, const uint32_t* __restrict__ Vc, int L, unsigned cls_del,
                              unsigned cls_norm, Acc& acc, bool& found) {
  uint32_t* N = (L & 1) ? p.N1 : p.N0;
  const int lane = lane_id();
  const int64_t W = cls_norm ? p.words : min(p.words, ((int64_t)p.d + 31) / 32);
  const int tail = p.n_ni & 31;
  const int64_t gwarp = spread_warp();
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w0 = gwarp * 32; w0 < W; w0 += nwarps * 32) {
    const int64_t w = w0 + lane;
    unsigned unv = 0;
    if (w < W) {
      unsigned vis = Vc[w];
      if (w == p.words - 1 && tail) vis |= ~((1u << tail) - 1u);
      const int64_t v0 = w * 32;
      unsigned dmask = 0;  // delegate bits of this word
      if (v0 < p.d) dmask = (p.d - v0 >= 32) ? kFull : ((1u << (p.d - v0)) - 1u);
      unv = ~vis & ((cls_del ? dmask : 0u) | (cls_norm ? ~dmask : 0u));
    }
    const int cnt = __popc(unv);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(kFull, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    const int excl = incl - cnt;
    for (int b = 0; b < total; b += 32) {
      const int k = b + lane;
      int j = 0;
#pragma unroll
      for (int sh = 16; sh >= 1; sh >>= 1) {
        const int t = __shfl_sync(kFull, incl, j + sh - 1);
        if (t <= k) j += sh;
      }
      const unsigned m = __shfl_sync(kFull, unv, j);
      const int ex = __shfl_sync(kFull, excl, j);
      const bool act = k < total;
      const int bit = act ? nth_set_bit(m, k - ex) : 0;
      const int v = (int)((w0 + j) * 32 + bit);
      const unsigned cls = v < p.d ? cls_del : (cls_norm ? 1u : 0u);
      const HeadRec h = head_load(p, act, v);
      int hit = -1, cid = -1;
      int64_t kv = 0;
      if (act) head_probe<false, true>(p, h, Vc, hit, cid, kv, cls);
      pull_tail<false, true>(p, act, v, h.deg, Vc, hit, cid, kv, nullptr, cls);
      if (act) {
        acc.scanned += 1;
        acc.edges += (unsigned long long)kv;
        if (hit >= 0) {
          atomicMin(p.parent_i + v, cid);
          atomicOr(N + (v >> 5), 1u << (v & 31));
          found = true;
        }
      }
    }
  }
}

// Second half of a backward level, between two grid barriers (so the long-row
// list is complete and V is still read-only): all warps take deferred rows from
// a shared counter in runs and scan them with 128-bit loads; a vertex found here
// sets its bit in N with an atomic.
__device__ void drain_long_rows(const BfsParams& p, const uint32_t* __restrict__ Vc, uint32_t* __restrict__ Vn, int L,
                                Acc& acc, bool build_next) {
  LevelSlot* sc = p.slot + (L & (kSlots - 1));
  uint32_t* Ncur = (L & 1) ? p.N1 : p.N0;
  const long long nl = (long long)__ldcg(&sc->nlong);
  if (nl == 0) return;
  const int64_t gwarp = spread_warp();
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  WorkCursor wc(nl, gwarp, nwarps, &sc->work2);
  for (long long e = wc.next(); e < nl; e = wc.next()) {
    const int v = p.longq[e];
    if (!BFS_IN(p, v, p.n_ni)) continue;  // warp-uniform
    const int64_t rb = p.off[v], re = rb + p.deg[v];
    int64_t kv;
    const int hit = warp_scan<false>(p, rb, rb + kHead, re, Vc, kv);
    if (lane_id() == 0) {
      acc.scanned += 1;
      acc.edges += (unsigned long long)kv;
      if (hit >= 0) {
        p.parent_i[v] = p.caller_of[hit];
        plane_or(p, v, L + 1);
        atomicOr(Ncur + (v >> 5), 1u << (v & 31));
        atomicOr(Vn + (v >> 5), 1u << (v & 31));
        acc.nf += 1;
        acc.mf += (unsigned long long)(re - rb);
        if (build_next) {  // the next forward level's lists (see append_next)
          LevelSlot* sq = p.slot + ((L + 1) & (kSlots - 1));
          if (v >= p.d) {
            const unsigned long long at = atomicAdd(&sq->qn, 1ull);
            if (BFS_IN(p, at, p.n_ni)) ((L & 1) ? p.Q0 : p.Q1)[at] = v;
          } else {
            const long long nc = ((long long)(re - rb) + kChunk - 1) / kChunk;
            const unsigned long long b = atomicAdd(&sq->nch, (unsigned long long)nc);
            for (long long k = 0; k < nc; ++k)
              if (BFS_IN(p, b + k, p.cl_cap)) ((L & 1) ? p.CL0 : p.CL1)[b + k] = make_int2(v, (int)k);
          }
        }
      }
    }
  }
}

// ---- bitmap -> frontier queues --------------------------------------------------------------

// Reads the discovered bitmap Nsrc of a level and writes the next frontier as a
// normal-vertex queue Q and a delegate chunk list CL.  Each warp takes items of
// 32 bitmap words (1024 vertices; 2 words in the delegate prefix, which is dense
// in new vertices), so no item is long: lane i loads word i, a warp scan of the bit counts gives every set bit a
// rank, the warp reserves its queue and chunk ranges with one atomic each, and
// then handles the item's new vertices 32 at a time (rank -> word by a binary
// search over the lanes' prefixes, bit by rank within the word).  With `merge`,
// also writes the next visited bitmap Vn = Vc | Nsrc and clears Nclr.  With `count` (after a forward level),
// also writes depth `depth` for every new vertex and adds n_f and m_f.  With Q
// null, no lists are written (a later conversion pass builds them).
// Counters of the per-subgraph schedule over a set of vertices (LevelSlot::sub).
struct SubAcc {
  unsigned long long c[6] = {0, 0, 0, 0, 0, 0};
};

__device__ __forceinline__ void sub_count(const BfsParams& p, int v, int deg, SubAcc& a) {
  const int dd = p.deg_del[v], dn = deg - dd;
  if (v < p.d) {
    a.c[0] += dd > 0;
    a.c[2] += dn > 0;
    a.c[3] += (unsigned long long)dd;
    a.c[4] += (unsigned long long)dn;
  } else {
    a.c[1] += dd > 0;
    a.c[5] += (unsigned long long)dd;
  }
}

// Adds every thread's SubAcc into slot->sub with one atomic per CTA and counter.
__device__ void flush_sub(SubAcc& a, LevelSlot* slot) {
  __shared__ unsigned long long s_sub[6];
  if (threadIdx.x < 6) s_sub[threadIdx.x] = 0;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const unsigned long long x = warp_sum(a.c[i]);
    if (lane_id() == 0 && x) atomicAdd(&s_sub[i], x);
  }
  __syncthreads();
  if (threadIdx.x < 6 && s_sub[threadIdx.x]) atomicAdd(&slot->sub[threadIdx.x], s_sub[threadIdx.x]);
  a = SubAcc();
}

template <bool kSub = false>
__device__ void frontier_from_bitmap(const BfsParams& p, const uint32_t* __restrict__ Vc, uint32_t* __restrict__ Vn,
                                     const uint32_t* __restrict__ Nsrc, uint32_t* __restrict__ Nclr,
                                     int32_t* __restrict__ Q, int2* __restrict__ CL, LevelSlot* slot, bool merge,
                                     bool count, int depth, Acc& acc, SubAcc* sacc = nullptr) {
  const int64_t W = p.words;
  const int lane = lane_id();
  const int64_t gwarp = spread_warp();
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  // the delegate prefix is dense in new vertices after a forward level: items of
  // two words there, 32 words elsewhere
  constexpr int kDelWords = 2;
  const int64_t Wd = min(W, ((int64_t)p.d + 31) / 32);
  const int64_t nd_items = (Wd + kDelWords - 1) / kDelWords;
  const int64_t Wd2 = min(W, nd_items * kDelWords);
  const int64_t nitems = nd_items + (W - Wd2 + 31) / 32;
  for (int64_t it = gwarp; it < nitems; it += nwarps) {
    const bool del_item = it < nd_items;
    const int64_t wb = del_item ? it * kDelWords : Wd2 + (it - nd_items) * 32;
    const int nw = del_item ? kDelWords : 32;
    const int64_t w = wb + lane;
    unsigned nb = 0;
    if (lane < nw && w < W) {
      nb = __ldcg(Nsrc + w);
      if (merge) {
        Vn[w] = Vc[w] | nb;
        Nclr[w] = 0u;
      }
      if (count) plane_store(p, w, nb, depth);
    }
    if (!__any_sync(kFull, nb != 0)) continue;
    const int64_t v0 = w * 32;
    unsigned dmask = 0;  // delegate bits of this lane's word
    if (v0 < p.d) dmask = (p.d - v0 >= 32) ? kFull : ((1u << (p.d - v0)) - 1u);
    const int cnt = __popc(nb), ncnt = __popc(nb & ~dmask);
    int incl = cnt, nincl = ncnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int a = __shfl_up_sync(kFull, incl, o), b = __shfl_up_sync(kFull, nincl, o);
      if (lane >= o) {
        incl += a;
        nincl += b;
      }
    }
    const int T = __shfl_sync(kFull, incl, 31), Tn = __shfl_sync(kFull, nincl, 31);
    const int excl = incl - cnt, nexcl = nincl - ncnt;
    unsigned long long qbase = 0;
    if (Q && lane == 0 && Tn) qbase = atomicAdd(&slot->qn, (unsigned long long)Tn);
    qbase = __shfl_sync(kFull, qbase, 0);
    for (int k0 = 0; k0 < T; k0 += 32) {
      const int k = k0 + lane;
      const bool act = k < T;
      int j = 0;
#pragma unroll
      for (int sh = 16; sh >= 1; sh >>= 1) {
        const int t = __shfl_sync(kFull, incl, j + sh - 1);
        if (t <= k) j += sh;
      }
      const unsigned m = __shfl_sync(kFull, nb, j);
      const unsigned dm = __shfl_sync(kFull, dmask, j);
      const int ex = __shfl_sync(kFull, excl, j), nex = __shfl_sync(kFull, nexcl, j);
      const int bit = act ? nth_set_bit(m, k - ex) : 0;
      const int v = (int)((wb + j) * 32 + bit);
      const int dg = act ? p.deg[v] : 0;
      unsigned long long nc = 0;
      if (act) {
        if (count) {
          acc.nf += 1;
          acc.mf += (unsigned long long)dg;
          if constexpr (kSub) sub_count(p, v, dg, *sacc);
        }
        if (!Q) {  // counts only
        } else if (v >= p.d) {
          const unsigned long long at = qbase + nex + __popc(m & ~dm & ((1u << bit) - 1u));
          if (BFS_IN(p, at, p.n_ni)) Q[at] = v;
        } else
          nc = ((unsigned long long)dg + kChunk - 1) / kChunk;
      }
      if (__any_sync(kFull, nc != 0)) {  // delegates: their row chunks, 32 entries per step
        long long ci = (long long)nc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const long long t = __shfl_up_sync(kFull, ci, o);
          if (lane >= o) ci += t;
        }
        const long long C = __shfl_sync(kFull, ci, 31);
        unsigned long long cbase = 0;
        if (lane == 0) cbase = atomicAdd(&slot->nch, (unsigned long long)C);
        cbase = __shfl_sync(kFull, cbase, 0);
        for (long long e0 = 0; e0 < C; e0 += 32) {
          const long long e = e0 + lane;
          int o = 0;
#pragma unroll
          for (int sh = 16; sh >= 1; sh >>= 1) {
            const long long t = __shfl_sync(kFull, ci, o + sh - 1);
            if (t <= e) o += sh;
          }
          const int ov = __shfl_sync(kFull, v, o);
          const long long oex = __shfl_sync(kFull, ci, o) - (long long)__shfl_sync(kFull, nc, o);
          if (e < C && BFS_IN(p, cbase + e, p.cl_cap)) CL[cbase + e] = make_int2(ov, (int)(e - oex));
        }
      }
    }
  }
}

// Level 0 forward, directly from the source's row: F_0 = {s}, so every row
// entry u is new at depth 1 with parent s (the row holds no loop and no
// duplicate).  All warps take 32-entry pieces of the row; each writes depth and
// parent, sets u's bits in N and in the next visited bitmap (which the set-up
// seeded with {s}), appends u to the next queue (normal) or its row chunks to
// the next chunk list (delegate), and counts n_f and m_f.  This replaces the
// expansion, its barrier and the bitmap sweep of a general forward level (with
// atomicMin parents; the PULL option keeps the general level and its pass).
__device__ void first_level(const BfsParams& p, int s, uint32_t* __restrict__ Vn, uint32_t* __restrict__ N,
                            int32_t* __restrict__ Q, int2* __restrict__ CL, LevelSlot* sn, Acc& acc) {
  const int lane = lane_id();
  const int64_t gwarp = spread_warp();
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t rb = p.off[s], re = p.off[s + 1];
  for (int64_t e0 = rb + gwarp * 32; e0 < re; e0 += nwarps * 32) {
    const int64_t e = e0 + lane;
    const int u0 = e < re ? p.col[e] : 0;
    const bool act = e < re && BFS_IN(p, u0, p.n_ni);
    const int u = act ? u0 : 0;
    const int dg = act ? p.deg[u] : 0;
    if (act) {
      plane_or(p, u, 1);
      p.parent_i[u] = p.src_c;
      atomicOr(N + (u >> 5), 1u << (u & 31));
      atomicOr(Vn + (u >> 5), 1u << (u & 31));
      acc.nf += 1;
      acc.mf += (unsigned long long)dg;
    }
    const unsigned nm = __ballot_sync(kFull, act && u >= p.d);
    if (nm) {
      unsigned long long qb = 0;
      if (lane == 0) qb = atomicAdd(&sn->qn, (unsigned long long)__popc(nm));
      qb = __shfl_sync(kFull, qb, 0);
      const unsigned long long at = qb + __popc(nm & ((1u << lane) - 1u));
      if (((nm >> lane) & 1u) && BFS_IN(p, at, p.n_ni)) Q[at] = u;
    }
    const long long nc = (act && u < p.d) ? ((long long)dg + kChunk - 1) / kChunk : 0;
    if (__any_sync(kFull, nc != 0)) {  // delegates: their row chunks, 32 entries per step
      long long ci = nc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(kFull, ci, o);
        if (lane >= o) ci += t;
      }
      const long long C = __shfl_sync(kFull, ci, 31);
      unsigned long long cbase = 0;
      if (lane == 0) cbase = atomicAdd(&sn->nch, (unsigned long long)C);
      cbase = __shfl_sync(kFull, cbase, 0);
      for (long long c0 = 0; c0 < C; c0 += 32) {
        const long long c = c0 + lane;
        int o = 0;
#pragma unroll
        for (int sh = 16; sh >= 1; sh >>= 1) {
          const long long t = __shfl_sync(kFull, ci, o + sh - 1);
          if (t <= c) o += sh;
        }
        const int ov = __shfl_sync(kFull, u, o);
        const long long oex = __shfl_sync(kFull, ci, o) - __shfl_sync(kFull, nc, o);
        if (c < C && BFS_IN(p, cbase + c, p.cl_cap)) CL[cbase + c] = make_int2(ov, (int)(c - oex));
      }
    }
  }
}

// Canonical parents of the vertices found by a forward level, by a first-hit
// scan of their sorted rows (the PULL option).
__device__ void pull_parents(const BfsParams& p, const uint32_t* __restrict__ Vc, int L, Acc& acc) {
  const LevelSlot* sn = p.slot + ((L + 1) & (kSlots - 1));
  const int64_t qn = (int64_t)__ldcg(&sn->qn);
  const int64_t nch = (int64_t)__ldcg(&sn->nch);
  const int32_t* Qn = (L & 1) ? p.Q0 : p.Q1;
  const int2* CLn = (L & 1) ? p.CL0 : p.CL1;
  const int lane = lane_id();
  const int64_t gwarp = spread_warp();
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t b = gwarp; b * 32 < qn; b += nwarps) {
    const int64_t i = b * 32 + lane;
    const bool act = i < qn;
    const int v = act ? Qn[i] : 0;
    int64_t kv = 0;
    int cid = -1, deg = 0;
    const int hit = pull_head<true>(p, act, v, Vc, kv, cid, deg);
    if (act) {
      acc.fix += (unsigned long long)kv;
      if (hit >= 0) p.parent_i[v] = cid;
    }
  }
  for (int64_t e = gwarp; e < nch; e += nwarps) {
    const int2 ck = CLn[e];
    if (ck.y != 0) continue;
    const int64_t rb = p.off[ck.x], re = p.off[ck.x + 1];
    int64_t kv;
    const int hit = warp_scan<true>(p, rb, rb, re, Vc, kv);
    if (lane == 0) {
      acc.fix += (unsigned long long)kv;
      if (hit >= 0) p.parent_i[ck.x] = p.caller_of[hit];
    }
  }
}

// Direction of level L+1 from its frontier (Sec. IV-B), computed alike by every CTA.
__device__ int decide(const BfsParams& p, int L1, int cur, unsigned long long nf, unsigned long long mf,
                      unsigned long long prev_nf, long long m_u, long long unvisited) {
  switch (p.schedule) {
    case BFS_SCHED_TOPDOWN:
      return 0;
    case BFS_SCHED_BOTTOMUP:
      return L1 >= 1 ? 1 : 0;
    case BFS_SCHED_ALTERNATE:
      return L1 & 1;
    case BFS_SCHED_MASK:
      return (int)((p.schedule_mask >> (L1 < 63 ? L1 : 63)) & 1ull);
    case BFS_SCHED_PAPER: {
      // FV = frontier degree sum; BV = |U| (q + s) / q with q = |frontier| and
      // U = s = unvisited vertices (one symmetric graph on one GPU).
      const double q = (double)nf, s = (double)(unvisited > 0 ? unvisited : 0);
      const double fv = (double)mf, bv = s * (q + s) / q;
      if (cur == 0) return fv > p.factor0 * bv ? 1 : 0;
      return fv < p.factor1 * bv ? 0 : 1;
    }
    default: {  // Beamer alpha/beta; BFS_SCHED_BEAMER_STAY: BU->TD also needs the TD->BU test to fail
      const bool td_bu = (long long)(mf * (unsigned long long)p.alpha) > m_u;
      if (cur == 0) return td_bu ? 1 : 0;
      const bool small = nf * (unsigned long long)p.beta < (unsigned long long)p.n;
      const bool stay = p.schedule == BFS_SCHED_BEAMER_STAY && td_bu;
      return (small && nf < prev_nf && !stay) ? 0 : 1;
    }
  }
}

// One subgraph's direction for the next level under the per-subgraph schedule
// (Sec. IV-B): q frontier vertices of its source class with an entry in it, fv
// those entries, U unvisited vertices of its destination class with an entry
// of the reversed subgraph, su unvisited vertices of its source class with an
// entry; BV = U (q + su) / q in double.  With q = 0 there is nothing to visit
// and the direction is kept.
__device__ __forceinline__ int sub_rule(int cur, unsigned long long q, unsigned long long fv, long long U, long long su,
                                        double f0, double f1) {
  if (q == 0) return cur;
  const double qd = (double)q, sd = (double)(su > 0 ? su : 0), fvd = (double)fv;
  const double bv = (double)(U > 0 ? U : 0) * (qd + sd) / qd;
  return cur == 0 ? (fvd > f0 * bv ? 1 : 0) : (fvd < f1 * bv ? 0 : 1);
}

// Spread of the CTAs' finishing times of an expansion (the tracing option).
__device__ void trace_done(LevelSlot* sc) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long t = gtimer();
    atomicMin(&sc->t_first, t);
    atomicMax(&sc->t_last, t);
  }
}

template <bool kSub>
__device__ void run_body(const BfsParams& p);


// Builds of the same kernel: 2 CTAs of 512 threads per SM (64 registers) or
// 3 (40 registers, some spilled to local memory), one of 1024; kSub: the
// per-subgraph direction schedule (BFS_SCHED_PAPER_SUBGRAPH).
template <int kMinBlocks, int kThr, bool kSub = false>
__global__ void __launch_bounds__(kThr, kMinBlocks) bfs_level_loop(BfsParams p) {
  run_body<kSub>(p);
}

// Bits a barrier's master hands to every CTA.
constexpr int kBitBackward = 1, kBitDone = 2, kBitConvert = 4, kBitDrain = 8;
// a backward level that also builds the next forward level's lists (bits 4-5: item width)
constexpr int kBitLists = 64;
// arrival flag of a forward expansion's barrier: the CTA met an unvisited target
constexpr int kFlagFound = 16;
// a backward level with at least half of the non-isolated vertices unvisited
// takes the dense items (bu_dense_item)
constexpr int kBitDense = 128;
__device__ __forceinline__ int dense_bit(long long unvisited, const BfsParams& p) {
  return (!(p.tuning & 4) && unvisited * 2 >= (long long)p.n_ni) ? kBitDense : 0;
}
// Item width 4 << c words of a backward level: about 64 unvisited vertices per
// item, or 128 when under 1/64 of the vertices are delegates (a graph of
// near-uniform degree, whose rows cost alike, so wider items lose no balance).
__device__ __forceinline__ int iw_code(long long unvisited, const BfsParams& p) {
  const long long per = (long long)p.d * 64 < (long long)p.n_ni ? 4 : 2;
  int c = 0;
  while (c < 3 && (long long)(4 << c) * unvisited < per * p.n_ni) ++c;
  return c << 4;
}

// Bits of the per-subgraph schedule's directions in the barrier word (the
// single-direction bits they reuse have no meaning in that schedule).
constexpr int kBitSubDD = kBitBackward, kBitSubDN = kBitDrain, kBitSubND = kBitLists;

__device__ __forceinline__ unsigned sub_dirs(int bits) {
  return ((bits & kBitSubDD) ? 1u : 0u) | ((bits & kBitSubDN) ? 2u : 0u) | ((bits & kBitSubND) ? 4u : 0u);
}

template <bool kSub>
__device__ void run_body(const BfsParams& p) {
  // state of the direction decision, kept by CTA 0 (the barriers' master)
  __shared__ long long s_mu, s_unv;
  // per-subgraph schedule: unvisited vertices of the three categories of LevelSlot::sub
  __shared__ long long s_su[3];
  __shared__ unsigned long long s_prev_nf, s_reach_e, s_reach_v, s_tb, s_te, s_tnf, s_log[5];
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  const bool leader = blockIdx.x == 0 && threadIdx.x == 0;
  const bool trace = (p.tuning & 2) != 0;
  unsigned seq = 0;
  Acc acc;

  // ---- init: clear bitmaps, seed the source ----
  const int src_i = p.internal_of[p.src_c];
  const bool src_in = src_i < p.n_ni;
  const int64_t sw = src_in ? (src_i >> 5) : -1;
  const unsigned sbit = 1u << (src_i & 31);
  const int64_t W4 = (p.words + 3) / 4;
  for (int64_t q = gtid; q < W4; q += gthreads) {
    uint4 v4 = make_uint4(0, 0, 0, 0);
    if (q == (sw >> 2)) {
      const int t = (int)(sw & 3);
      v4.x = t == 0 ? sbit : 0u;
      v4.y = t == 1 ? sbit : 0u;
      v4.z = t == 2 ? sbit : 0u;
      v4.w = t == 3 ? sbit : 0u;
    }
    reinterpret_cast<uint4*>(p.V)[q] = v4;
    reinterpret_cast<uint4*>(p.V1)[q] = v4;  // level 0 adds the source's row to this copy
    reinterpret_cast<uint4*>(p.N0)[q] = make_uint4(0, 0, 0, 0);
    reinterpret_cast<uint4*>(p.N1)[q] = make_uint4(0, 0, 0, 0);
  }
  // depth nibble plane 0: one 16-byte word per visited-bitmap word
  for (int64_t q = gtid; q < p.words; q += gthreads) reinterpret_cast<uint4*>(p.planes)[q] = make_uint4(0, 0, 0, 0);
  if (kSub || p.td_parent == BFS_TD_PARENT_ATOMICMIN) {
    const int64_t P4 = ((int64_t)p.n_ni + 3) / 4;
    for (int64_t q = gtid; q < P4; q += gthreads) {
      int4 x = make_int4(INT_MAX, INT_MAX, INT_MAX, INT_MAX);
      if (q == ((int64_t)src_i >> 2) && src_in) {
        const int t = src_i & 3;
        if (t == 0) x.x = p.src_c;
        if (t == 1) x.y = p.src_c;
        if (t == 2) x.z = p.src_c;
        if (t == 3) x.w = p.src_c;
      }
      reinterpret_cast<int4*>(p.parent_i)[q] = x;
    }
  }
  unsigned long long src_deg = 0;
  if (src_in) src_deg = (unsigned long long)(p.off[src_i + 1] - p.off[src_i]);
  if (leader) {
    for (int k = 0; k < kSlots; ++k) {
      p.slot[k] = LevelSlot();
      p.slot[k].t_first = ~0ull;
    }
    p.hdr->t0 = gtimer();
    if (src_in) {
      p.parent_i[src_i] = p.src_c;
      p.slot[0].n_f = 1;
      p.slot[0].m_f = src_deg;
      if (src_i >= p.d) {
        p.Q0[0] = src_i;
        p.slot[0].qn = 1;
      } else {
        const int64_t nch = ((int64_t)src_deg + kChunk - 1) / kChunk;
        for (int64_t k = 0; k < nch; ++k) p.CL0[k] = make_int2(src_i, (int)k);
        p.slot[0].nch = (unsigned long long)nch;
      }
    }
    s_mu = (long long)p.nnz - (long long)src_deg;
    s_unv = (long long)p.n_ni - (src_in ? 1 : 0);
    s_prev_nf = 1;
    s_reach_e = src_deg;
    s_reach_v = 1;
  }
  if (p.test_skip_barrier && blockIdx.x == 0) return;  // the others' bounded wait must expire
  int bits;
  if constexpr (kSub) {
    // level 0 from F_0 = {s}, every subgraph forward before it
    bits = grid_sync(p, seq, [&](int) {
      if (!src_in) return kBitDone;
      SubAcc a;
      sub_count(p, src_i, (int)src_deg, a);
      for (int i = 0; i < 3; ++i) s_su[i] = (long long)p.sub_tot[i] - (long long)a.c[i];
      const int dd = sub_rule(0, a.c[0], a.c[3], s_su[0], s_su[0], p.sf0[0], p.sf1[0]);
      const int dn = sub_rule(0, a.c[2], a.c[4], s_su[1], s_su[2], p.sf0[1], p.sf1[1]);
      const int nd = sub_rule(0, a.c[1], a.c[5], s_su[2], s_su[1], p.sf0[2], p.sf1[2]);
      return (dd ? kBitSubDD : 0) | (dn ? kBitSubDN : 0) | (nd ? kBitSubND : 0) | iw_code(s_unv, p);
    });
  } else {
    bits = grid_sync(p, seq, [&](int) {
      return (src_in ? 0 : kBitDone) | (decide(p, 0, 0, 1, src_deg, 1, s_mu, s_unv) ? kBitBackward : 0) |
             iw_code(s_unv, p) | dense_bit(s_unv, p);
    });
  }
  if (bits < 0) return;

  const unsigned long long t_start = gtimer();
  if (leader) p.hdr->t_init = t_start;
  int L = 0;
  int vpar = 0;  // visited bitmap of the current level: V (0) or V1 (1)
  bool lists_ready = false;  // the previous (backward) level built this level's forward lists
  bool ended = false;        // a forward level found nothing and ended the run before its sweep
  while (!(bits & kBitDone)) {
    // Bounds against a run that does not end: at most n_ni+1 levels, and the
    // run's deadline.  A failure set here ends every CTA at its next barrier.
    if (threadIdx.x == 0 && (L > p.n_ni + 1 || gtimer() - t_start > p.run_timeout_ns))
      set_failed(p, BFS_ERR_TIMEOUT);
    if constexpr (kSub) {
      // Per-subgraph directions (Sec. IV-B): nn forward always; dd, dn, nd as decided.
      // One phase pushes from the frontier lists to the allowed target classes and
      // pulls for the unvisited vertices of the backward subgraphs; the level end
      // builds the next lists, depths and counters.
      const unsigned sd = sub_dirs(bits);
      LevelSlot* sc = p.slot + (L & (kSlots - 1));
      LevelSlot* sn = p.slot + ((L + 1) & (kSlots - 1));
      uint32_t* Ncur = (L & 1) ? p.N1 : p.N0;
      uint32_t* Noth = (L & 1) ? p.N0 : p.N1;
      const uint32_t* Vc = vpar ? p.V1 : p.V;
      uint32_t* Vn = vpar ? p.V : p.V1;
      if (leader) s_tb = gtimer();
      auto master_sub = [&](int) {
        const unsigned long long nf = __ldcg(&sn->n_f), mf = __ldcg(&sn->m_f);
        s_log[0] = __ldcg(&sc->n_f);
        s_log[1] = __ldcg(&sc->m_f);
        s_log[2] = __ldcg(&sc->scanned);
        s_log[3] = __ldcg(&sc->edges);
        s_log[4] = __ldcg(&sc->qn);
        s_tnf = nf;
        s_unv -= (long long)nf;
        s_reach_e += mf;
        s_reach_v += nf;
        if (nf == 0) return kBitDone;
        unsigned long long c[6];
        for (int i = 0; i < 6; ++i) c[i] = __ldcg(&sn->sub[i]);
        for (int i = 0; i < 3; ++i) s_su[i] -= (long long)c[i];
        const int dd = sub_rule((sd & 1u) ? 1 : 0, c[0], c[3], s_su[0], s_su[0], p.sf0[0], p.sf1[0]);
        const int dn = sub_rule((sd & 2u) ? 1 : 0, c[2], c[4], s_su[1], s_su[2], p.sf0[1], p.sf1[1]);
        const int nd = sub_rule((sd & 4u) ? 1 : 0, c[1], c[5], s_su[2], s_su[1], p.sf0[2], p.sf1[2]);
        return (dd ? kBitSubDD : 0) | (dn ? kBitSubDN : 0) | (nd ? kBitSubND : 0) | iw_code(s_unv, p);
      };
      bool found = false;
      // normal sources push to normal targets (nn) and, unless nd is backward, to delegates;
      // delegate sources to delegates unless dd, to normal vertices unless dn is backward
      const unsigned allow_n = 2u | ((sd & 4u) ? 0u : 1u);
      const unsigned allow_d = ((sd & 1u) ? 0u : 1u) | ((sd & 2u) ? 0u : 2u);
      expand_td<true>(p, Vc, L, found, allow_n, allow_d);
      const unsigned cls_del = ((sd & 1u) ? 1u : 0u) | ((sd & 4u) ? 2u : 0u);
      const unsigned cls_norm = (sd & 2u) ? 1u : 0u;
      if (cls_del | cls_norm) expand_bu_sub(p, Vc, L, cls_del, cls_norm, acc, found);
      flush_block(acc, nullptr, nullptr, &sc->edges, &sc->scanned, nullptr);
      if (trace) trace_done(sc);
      const int eb = grid_sync(p, seq, [&](int fl) { return (fl & kFlagFound) ? 0 : master_sub(fl); },
                               found ? kFlagFound : 0);
      if (eb < 0) return;
      if (leader) s_te = gtimer();
      if (eb & kBitDone) {
        bits = eb;
        ended = true;
      } else {
        SubAcc sacc;
        frontier_from_bitmap<true>(p, Vc, Vn, Ncur, Noth, (L & 1) ? p.Q0 : p.Q1, (L & 1) ? p.CL0 : p.CL1, sn, true,
                                   true, L + 1, acc, &sacc);
        flush_block(acc, &sn->n_f, &sn->m_f, nullptr, nullptr, nullptr);
        flush_sub(sacc, sn);
        if (leader) {
          p.slot[(L + 2) & (kSlots - 1)] = LevelSlot();
          p.slot[(L + 2) & (kSlots - 1)].t_first = ~0ull;
        }
        bits = grid_sync(p, seq, master_sub);
      }
      if (bits < 0) return;
      if (leader && L < BFS_LOG_LEVELS) {
        LevelLogDev& lg = p.log[L];
        lg.t_end = gtimer();
        lg.dir = sd ? 1 : 0;
        lg.subdirs = (int)sd;
        lg.converted = 0;
        lg.n_f = s_log[0];
        lg.m_f = s_log[1];
        lg.scanned = s_log[2];
        lg.edges = s_log[3];
        lg.fix_edges = 0ull;
        lg.found = s_tnf;
        lg.qn = s_log[4];
        lg.t_begin = s_tb;
        lg.t_expand = s_te;
        lg.t_first = trace ? __ldcg(&sc->t_first) : 0ull;
        lg.t_last = trace ? __ldcg(&sc->t_last) : 0ull;
      }
      if (!ended) vpar ^= 1;
      ++L;
      continue;
    }
    const int dir = (bits & kBitBackward) ? 1 : 0;
    const bool conv = (bits & kBitConvert) != 0 && !lists_ready;
    const bool build_lists = dir == 1 && (bits & kBitLists) != 0;
    const int iw = 4 << ((bits >> 4) & 3);
    LevelSlot* sc = p.slot + (L & (kSlots - 1));
    LevelSlot* sn = p.slot + ((L + 1) & (kSlots - 1));
    uint32_t* Ncur = (L & 1) ? p.N1 : p.N0;
    uint32_t* Noth = (L & 1) ? p.N0 : p.N1;
    const uint32_t* Vc = vpar ? p.V1 : p.V;  // depth <= L, read-only during the level
    uint32_t* Vn = vpar ? p.V : p.V1;        // depth <= L+1, written during the level
    if (conv) {
      // F_L is the bitmap of the previous (backward) level's discoveries.
      frontier_from_bitmap(p, Vc, Vn, Noth, nullptr, (L & 1) ? p.Q1 : p.Q0, (L & 1) ? p.CL1 : p.CL0, sc, false, false,
                           0, acc);
      if (grid_sync(p, seq, no_master) < 0) return;
    }
    if (leader) s_tb = gtimer();
    // A big forward level (more frontier entries than bitmap words) usually
    // hands over to a backward level: its sweep leaves the next lists to a
    // conversion pass at the start of the next level, run only if that level
    // is forward too.
    bool defer_lists = false;
    // The barrier master's step once the level's counters are complete: the
    // direction of level L+1, and this level's log counters (loaded together).
    auto master = [&](int) {
      const unsigned long long nf = __ldcg(&sn->n_f), mf = __ldcg(&sn->m_f);
      s_log[0] = __ldcg(&sc->n_f);
      s_log[1] = __ldcg(&sc->m_f);
      s_log[2] = __ldcg(&sc->scanned);
      s_log[3] = __ldcg(&sc->edges);
      s_log[4] = __ldcg(&sc->qn);
      s_tnf = nf;
      s_mu -= (long long)mf;
      s_unv -= (long long)nf;
      s_reach_e += mf;
      s_reach_v += nf;
      if (nf == 0) return kBitDone;
      const int nd = decide(p, L + 1, dir, nf, mf, s_prev_nf, s_mu, s_unv);
      s_prev_nf = nf;
      // a backward level with few unvisited vertices left builds the next
      // forward level's lists as it goes, so a switch back needs no conversion
      const int lists = (nd && s_unv * kListsFraction < (long long)p.n_ni) ? kBitLists : 0;
      return (nd ? kBitBackward : 0) | ((nd == 0 && (dir == 1 || defer_lists)) ? kBitConvert : 0) |
             iw_code(s_unv, p) | lists | (nd ? dense_bit(s_unv, p) : 0);
    };
    if (dir == 0 && L == 0 && p.td_parent == BFS_TD_PARENT_ATOMICMIN) {
      first_level(p, src_i, Vn, Ncur, p.Q1, p.CL1, sn, acc);
      if (trace) trace_done(sc);
      if (leader) s_te = gtimer();
      flush_block(acc, &sn->n_f, &sn->m_f, nullptr, nullptr, nullptr);
      if (leader) {
        p.slot[2] = LevelSlot();
        p.slot[2].t_first = ~0ull;
      }
      bits = grid_sync(p, seq, master);
    } else if (dir == 0) {
      bool found = false;  // this thread met an unvisited target
      expand_td(p, Vc, L, found);
      if (trace) trace_done(sc);
      // a level that met no unvisited target found nothing: its barrier's master
      // ends the run at once (no sweep, no second barrier; V stays depth <= L)
      const int eb = grid_sync(p, seq, [&](int fl) { return (fl & kFlagFound) ? 0 : master(fl); },
                               found ? kFlagFound : 0);
      if (eb < 0) return;
      if (leader) s_te = gtimer();
      if (eb & kBitDone) {
        bits = eb;
        ended = true;
      } else {
        // the next frontier's depths and counts (and its lists, when parents are
        // pulled); Vn = Vc | N
        defer_lists = p.td_parent != BFS_TD_PARENT_PULL && __ldcg(&sc->m_f) > (unsigned long long)p.words;
        frontier_from_bitmap(p, Vc, Vn, Ncur, Noth, defer_lists ? nullptr : ((L & 1) ? p.Q0 : p.Q1),
                             (L & 1) ? p.CL0 : p.CL1, sn, true, true, L + 1, acc);
        flush_block(acc, &sn->n_f, &sn->m_f, nullptr, nullptr, nullptr);
        if (p.td_parent == BFS_TD_PARENT_PULL) {
          if (grid_sync(p, seq, no_master) < 0) return;  // the queues of F_{L+1} are complete
          pull_parents(p, Vc, L, acc);
          flush_block(acc, nullptr, nullptr, nullptr, nullptr, &sc->fix_edges);
        }
        if (leader) {
          p.slot[(L + 2) & (kSlots - 1)] = LevelSlot();
          p.slot[(L + 2) & (kSlots - 1)].t_first = ~0ull;
        }
        bits = grid_sync(p, seq, master);
      }
    } else {
      // backward: the items write N, Vn and the cleared other bitmap themselves,
      // so one barrier ends the level unless long rows were deferred
      const bool deferred = expand_bu(p, Vc, Vn, Noth, L, iw, acc, build_lists, (bits & kBitDense) != 0);
      flush_block(acc, &sn->n_f, &sn->m_f, &sc->edges, &sc->scanned, nullptr);
      if (trace) trace_done(sc);
      if (leader) {
        s_te = gtimer();
        p.slot[(L + 2) & (kSlots - 1)] = LevelSlot();
        p.slot[(L + 2) & (kSlots - 1)].t_first = ~0ull;
      }
      bits = grid_sync(p, seq, [&](int fl) { return (fl & kBitDrain) ? kBitDrain : master(fl); },
                       deferred ? kBitDrain : 0);
      if (bits >= 0 && (bits & kBitDrain)) {
        drain_long_rows(p, Vc, Vn, L, acc, build_lists);
        flush_block(acc, &sn->n_f, &sn->m_f, &sc->edges, &sc->scanned, nullptr);
        bits = grid_sync(p, seq, master);
      }
    }
    if (bits < 0) return;
    if (leader && L < BFS_LOG_LEVELS) {  // the level's log (slot L stays intact until L+2)
      LevelLogDev& lg = p.log[L];
      lg.t_end = gtimer();
      lg.dir = dir;
      lg.converted = conv ? 1 : 0;
      lg.n_f = s_log[0];
      lg.m_f = s_log[1];
      lg.scanned = s_log[2];
      lg.edges = dir == 0 ? s_log[1] : s_log[3];
      lg.fix_edges = p.td_parent == BFS_TD_PARENT_PULL ? __ldcg(&sc->fix_edges) : 0ull;
      lg.found = s_tnf;
      lg.qn = s_log[4];
      lg.t_begin = s_tb;
      lg.t_expand = s_te;
      lg.t_first = trace ? __ldcg(&sc->t_first) : 0ull;
      lg.t_last = trace ? __ldcg(&sc->t_last) : 0ull;
      lg.subdirs = 0;
    }
    lists_ready = build_lists;
    if (!ended) vpar ^= 1;
    ++L;
  }

  // ---- the results in caller ids are written by bfs_results, launched next ----
  if (leader) p.hdr->t_loop = gtimer();
  if (leader) {
    p.hdr->levels = src_in ? L : 1;
    p.hdr->levels_run = L;
    p.hdr->t1 = p.hdr->t_loop;
    p.hdr->reached_edges = src_in ? s_reach_e : 0;
    p.hdr->reached = src_in ? s_reach_v : 1;
  }
}

// Delegate neighbours of every non-isolated vertex (one warp per row) and the
// totals of the per-subgraph schedule's three vertex categories: delegates with
// a delegate neighbour, normal vertices with a delegate neighbour, delegates
// with a normal neighbour.
__global__ void k_deg_del(const int64_t* __restrict__ off, const int32_t* __restrict__ col, int32_t n_ni, int32_t d,
                          int32_t* __restrict__ deg_del, unsigned long long* __restrict__ tot) {
  __shared__ unsigned long long s_t[3];
  if (threadIdx.x < 3) s_t[threadIdx.x] = 0;
  __syncthreads();
  const int lane = lane_id();
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long t[3] = {0, 0, 0};
  for (int64_t v = gwarp; v < n_ni; v += nwarps) {
    const int64_t b = off[v], e = off[v + 1];
    int c = 0;
    for (int64_t j = b + lane; j < e; j += 32) c += col[j] < d;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if (lane == 0) {
      deg_del[v] = c;
      const int64_t dn = (e - b) - c;
      if (v < d) {
        t[0] += c > 0;
        t[2] += dn > 0;
      } else {
        t[1] += c > 0;
      }
    }
  }
  for (int i = 0; i < 3; ++i)
    if (t[i]) atomicAdd(&s_t[i], t[i]);
  __syncthreads();
  if (threadIdx.x < 3 && s_t[threadIdx.x]) atomicAdd(&tot[threadIdx.x], s_t[threadIdx.x]);
}

// One quad of results (caller ids 4q .. 4q+3) in the output form of the run.
__device__ __forceinline__ void write_quad(const BfsParams& p, int64_t q, const int (&dv)[4], const int (&pv)[4]) {
  const int64_t c = q * 4;
  if (p.out_depth8) {  // uint8 form: 255 = unreached
    unsigned d8 = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      if (dv[t] > 254) set_failed(p, BFS_ERR_OVERFLOW);
      d8 |= (unsigned)(dv[t] < 0 ? 255 : (dv[t] & 0xFF)) << (8 * t);
    }
    if (p.out_vec4 && c + 3 < p.n) {
      reinterpret_cast<unsigned*>(p.out_depth8)[q] = d8;
      if (p.out_parent) reinterpret_cast<int4*>(p.out_parent)[q] = make_int4(pv[0], pv[1], pv[2], pv[3]);
    } else {
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (c + t < p.n) {
          p.out_depth8[c + t] = (uint8_t)(d8 >> (8 * t));
          if (p.out_parent) p.out_parent[c + t] = pv[t];
        }
    }
  } else if (p.out_vec4 && c + 3 < p.n) {
    reinterpret_cast<int4*>(p.out_depth)[q] = make_int4(dv[0], dv[1], dv[2], dv[3]);
    reinterpret_cast<int4*>(p.out_parent)[q] = make_int4(pv[0], pv[1], pv[2], pv[3]);
  } else {
#pragma unroll
    for (int t = 0; t < 4; ++t)
      if (c + t < p.n) {
        p.out_depth[c + t] = dv[t];
        p.out_parent[c + t] = pv[t];
      }
  }
}

// Results in caller ids: a kernel of its own, launched after the level loop on
// the same stream.  A caller id's internal id comes from its word of the
// caller-rank table (which of the word's callers are delegates / non-isolated
// normal vertices, and how many of each precede the word: both classes are
// numbered in caller order); isolated vertices are never reached but the
// source.  The depth is the vertex's nibbles, zero meaning unreached (the source
// is set apart).  A thread takes kResultQuads quads of 4 consecutive caller ids
// per step, their loads all in flight before the first is used; at 32
// registers four 512-thread CTAs fit an SM (RMAT-26: 162 us against 177 us with
// two quads per thread at two CTAs per SM).
constexpr int kResultQuads = 1;

__global__ void __launch_bounds__(kThreads, 4) bfs_results(BfsParams p) {
  if (run_failed(p)) return;  // outputs are unspecified after a failed run
  const int L = *(volatile int*)&p.hdr->levels_run;
  const int64_t gtid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x;
  // nibble planes that hold a depth of this run: the last level run found
  // nothing, so the deepest vertex is at depth L - 1
  int nib_used = 1;
  while (nib_used < p.planes_n && ((L - 1) >> (4 * nib_used)) > 0) ++nib_used;
  const int64_t C4 = ((int64_t)p.n + 3) / 4;
  constexpr int U = kResultQuads;
  for (int64_t q0 = gtid; q0 < C4; q0 += gthreads * U) {
    int vs[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t q = q0 + (int64_t)u * gthreads;
      const int4 rk = q < C4 ? p.crank[q >> 3] : make_int4(0, 0, 0, 0);
      const int b0 = (int)((q & 7) * 4);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int b = b0 + t;
        const unsigned lo = (1u << b) - 1u;
        int v = -1;
        if (((unsigned)rk.x >> b) & 1u)
          v = rk.z + __popc((unsigned)rk.x & lo);
        else if (((unsigned)rk.y >> b) & 1u)
          v = p.d + rk.w + __popc((unsigned)rk.y & lo);
        vs[u][t] = v;
      }
    }
    // the depth word and the parent slot of every non-isolated vertex are loaded
    // together (almost all of them are reached)
    unsigned nw[U][4];
    int pp[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        nw[u][t] = vs[u][t] >= 0 ? p.planes[vs[u][t] >> 3] : 0u;
        pp[u][t] = vs[u][t] >= 0 ? p.parent_i[vs[u][t]] : -1;
      }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t q = q0 + (int64_t)u * gthreads;
      if (q >= C4) break;
      int dv[4], pv[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int v = vs[u][t];
        int dd = v >= 0 ? (int)((nw[u][t] >> (4 * (v & 7))) & 15u) : 0;
        for (int k = 1; k < nib_used && v >= 0; ++k)
          dd |= (int)((p.planes[(int64_t)k * p.pstride + (v >> 3)] >> (4 * (v & 7))) & 15u) << (4 * k);
        const bool r = dd > 0;
        dv[t] = r ? dd : -1;
        pv[t] = r ? pp[u][t] : -1;
        if (q * 4 + t == p.src_c) {
          dv[t] = 0;
          pv[t] = p.src_c;
        }
      }
      write_quad(p, q, dv, pv);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) atomicMax(&p.hdr->t1, gtimer());
}

}  // namespace

int configure_run(bfs_graph* g) {
  int sms = 0, per_sm = 0;
  cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
  if (e != cudaSuccess) return cuda_fail(e, "device attributes");
  int coop = 0;
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, g->device);
  if (!coop) return fail(BFS_ERR_CUDA, "device does not support cooperative launch");
  // 0 = by size: one 1024-thread CTA per SM once the non-isolated vertices pass
  // 2^24 (measured faster there: RMAT-26 -1.8 %, ER-2^26 -1.1 %), else two of 512
  const int bps = g->opt.blocks_per_sm != 0 ? g->opt.blocks_per_sm : (g->n_ni > (1 << 24) ? 1 : 2);
  const int variant = bps == 3 ? 3 : (bps == 1 ? 1 : 2);
  if (variant == 3) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bfs_level_loop<3, kThreads>, kThreads, 0);
  else if (variant == 1) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bfs_level_loop<1, 2 * kThreads>, 2 * kThreads, 0);
  else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bfs_level_loop<2, kThreads>, kThreads, 0);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy");
  if (per_sm < 1) return fail(BFS_ERR_CUDA, "level-loop kernel does not fit on an SM");
  const int want = per_sm < variant ? per_sm : variant;
  g->variant = variant;
  g->grid_blocks = sms * want;
  if (g->grid_blocks > kMaxBlocks) g->grid_blocks = kMaxBlocks;
  int per_sm_sub = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_sub, bfs_level_loop<2, kThreads, true>, kThreads, 0);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy");
  if (per_sm_sub < 1) return fail(BFS_ERR_CUDA, "per-subgraph level-loop kernel does not fit on an SM");
  g->grid_blocks_sub = sms * (per_sm_sub < 2 ? per_sm_sub : 2);
  if (g->grid_blocks_sub > kMaxBlocks) g->grid_blocks_sub = kMaxBlocks;
  return BFS_OK;
}

// The per-subgraph schedule's per-vertex delegate-neighbour counts and category
// totals, made on its first run (asynchronous on s).
static int prepare_subgraph(bfs_graph* g, cudaStream_t s) {
  if (g->deg_del) return BFS_OK;
  cudaError_t e = cudaMalloc((void**)&g->deg_del, sizeof(int32_t) * ((size_t)g->n_ni + 1));
  if (e == cudaSuccess) e = cudaMalloc((void**)&g->sub_tot, sizeof(unsigned long long) * 4);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->sub_tot, 0, sizeof(unsigned long long) * 4, s);
  if (e != cudaSuccess) {
    if (g->deg_del) cudaFree(g->deg_del);
    g->deg_del = nullptr;
    g->sub_tot = nullptr;
    return cuda_fail(e, "per-subgraph schedule state");
  }
  g->device_bytes += (int64_t)sizeof(int32_t) * ((int64_t)g->n_ni + 1) + 32;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device);
  if (g->n_ni > 0) k_deg_del<<<sms * 4, 256, 0, s>>>(g->off, g->col, g->n_ni, g->d, g->deg_del, g->sub_tot);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "per-subgraph degree pass");
  return BFS_OK;
}

int launch_run(bfs_graph* g, int32_t source, int32_t* out_depth, int32_t* out_parent, cudaStream_t s, int grid,
               uint8_t* out_depth8) {
  BfsParams p;
  p.off = g->off;
  p.col = g->col;
  p.caller_of = g->caller_of;
  p.internal_of = g->internal_of;
  p.head = g->head;
  p.deg = g->deg;
  p.lead = g->lead;
  p.longq = g->longq;
  p.V = g->V;
  p.V1 = g->V1;
  p.N0 = g->N0;
  p.N1 = g->N1;
  p.planes = g->planes;
  p.planes_n = g->planes_n;
  p.pstride = g->pstride;
  p.cl_cap = g->cl_cap;
  p.long_cap = g->long_cap;
  p.crank = g->crank;
  p.parent_i = g->parent_i;
  p.Q0 = g->Q0;
  p.Q1 = g->Q1;
  p.CL0 = g->CL0;
  p.CL1 = g->CL1;
  p.slot = g->slot;
  p.log = g->log;
  p.hdr = g->hdr;
  p.arrive = g->arrive;
  p.out_depth = out_depth;
  p.out_parent = out_parent;
  p.out_depth8 = out_depth8;
  p.nnz = g->nnz;
  p.words = g->words;
  p.n = g->n;
  p.n_ni = g->n_ni;
  p.d = g->d;
  p.src_c = source;
  p.schedule = g->opt.schedule;
  p.alpha = g->opt.alpha;
  p.beta = g->opt.beta;
  p.td_parent = g->opt.td_parent;
  p.schedule_mask = g->opt.schedule_mask;
  p.factor0 = g->opt.factor0;
  p.factor1 = g->opt.factor1;
  p.timeout_ns = (unsigned long long)g->opt.barrier_timeout_ms * 1000000ull;
  p.test_skip_barrier = g->opt.test_skip_barrier;
  p.run_timeout_ns = (unsigned long long)g->opt.run_timeout_ms * 1000000ull;
  p.out_vec4 = out_depth8 ? ((((uintptr_t)out_depth8) & 3) == 0 && (((uintptr_t)out_parent) & 15) == 0)
                         : ((((uintptr_t)out_depth) | ((uintptr_t)out_parent)) & 15) == 0;
  p.tuning = g->opt.tuning;
  const bool sub = g->opt.schedule == BFS_SCHED_PAPER_SUBGRAPH;
  if (sub) {
    const int rc = prepare_subgraph(g, s);
    if (rc) return rc;
  }
  p.deg_del = g->deg_del;
  p.sub_tot = g->sub_tot;
  for (int i = 0; i < 3; ++i) {
    p.sf0[i] = g->opt.subgraph_factor0[i];
    p.sf1[i] = g->opt.subgraph_factor1[i];
  }
  p.epoch = ++g->epoch & 0x0FFFFFFFu;
  if (p.epoch == 0) p.epoch = ++g->epoch & 0x0FFFFFFFu;
  if (p.epoch == 1) {  // first run, or the run counter wrapped: barrier words must restart below any tag
    cudaError_t e0 = cudaMemsetAsync(g->arrive, 0, sizeof(unsigned long long) * kMaxBlocks * 4, s);
    if (e0 == cudaSuccess) e0 = cudaMemsetAsync(&g->hdr->release, 0, sizeof(unsigned long long), s);
    if (e0 != cudaSuccess) return cuda_fail(e0, "reset barrier words");
  }
  void* args[] = {&p};
  const void* fn = sub                ? (const void*)bfs_level_loop<2, kThreads, true>
                   : g->variant == 3 ? (const void*)bfs_level_loop<3, kThreads>
                   : g->variant == 1 ? (const void*)bfs_level_loop<1, 2 * kThreads>
                                     : (const void*)bfs_level_loop<2, kThreads>;
  // grid is counted in 512-thread CTAs (the serving slices); a 1024-thread CTA takes two
  const int want = (!sub && g->variant == 1) ? (grid + 1) / 2 : grid;
  const int full = sub ? g->grid_blocks_sub : g->grid_blocks;
  const int blocks = want > 0 && want < full ? want : full;
  const int threads = (!sub && g->variant == 1) ? 2 * kThreads : kThreads;
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(blocks), dim3(threads), args, 0, s);
  if (e != cudaSuccess) return cuda_fail(e, "level-loop launch");
  // the results, on the same SMs (a serving slice stays a slice): four result
  // CTAs per SM where the loop has two
  const int rblocks = blocks * threads / kThreads * 2;
  bfs_results<<<rblocks, kThreads, 0, s>>>(p);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "result-pass launch");
  return BFS_OK;
}

}  // namespace bfsgb
