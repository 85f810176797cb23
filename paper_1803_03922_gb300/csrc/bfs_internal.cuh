// Internal layout shared by the builder, the level-loop kernel and the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "bfs_gb300.h"

namespace bfsgb {

constexpr int kThreads = 512;         // level-loop CTA size (16 warps)
constexpr int kWarpsPerBlock = kThreads / 32;
constexpr int kMaxWarpsPerBlock = 32;  // shared arrays indexed by warp fit 1024-thread CTAs
constexpr int64_t kChunk = 512;       // row entries per delegate work item in a forward level
constexpr int kColPad = 32;           // int32 slack after the last column (128-bit over-reads)
constexpr int kHead = 4;              // row entries kept in the per-vertex head record
constexpr int kHeadVecs = kHead / 2;  // int4 words per head record: kHead ids, then kHead caller ids
static_assert(kHead == 2 || kHead == 4 || kHead == 8, "head records hold 2, 4 or 8 entries");
constexpr int64_t kShort = 4096;      // rows with more entries left after the head go to the long-row path
constexpr int kTailLanes = 4;         // lanes per row in the short-row group scan of a pull (2, 4, 8 or 16)
constexpr int kTailPerLane = 4;       // row entries per lane and step there (1, or 2 / 4 as one 64- / 128-bit load)
constexpr long long kListsFraction = 4;  // backward levels with under n_ni/4 unvisited build the next queue
constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kMaxBlocks = 2048;      // upper bound of the level-loop grid (arrival words)

// Per-level counters; a ring of kSlots indexed by level.
struct __align__(64) LevelSlot {
  unsigned long long qn;        // normal-queue entries holding this level's frontier
  unsigned long long nch;       // delegate chunk entries holding this level's frontier
  unsigned long long n_f;       // frontier vertices
  unsigned long long m_f;       // frontier degree sum
  unsigned long long work;      // dynamic work counter of this level's expansion
  unsigned long long edges;     // backward: sum of k_v
  unsigned long long scanned;   // backward: unvisited vertices scanned
  unsigned long long fix_edges; // forward: row entries read to pick parents
  unsigned long long t_first;   // %globaltimer when the first / last CTA finished the expansion
  unsigned long long t_last;
  unsigned long long work2;     // hand-out counter of the deferred long rows
  unsigned long long nlong;     // deferred long rows (backward)
  unsigned long long pad[4];
  // per-subgraph schedule, over this level's frontier: vertices that are delegates with a
  // delegate neighbour, normal with a delegate neighbour, delegates with a normal neighbour;
  // then the delegate neighbours of its delegates, their normal neighbours, and the delegate
  // neighbours of its normal vertices (FV of dd, dn and nd)
  unsigned long long sub[6];
};
constexpr int kSlots = 4;

struct LevelLogDev {
  int32_t dir, converted, subdirs, pad;
  unsigned long long n_f, m_f, scanned, edges, fix_edges, found, qn;
  unsigned long long t_begin, t_expand, t_end, t_first, t_last;
};

struct RunHeader {
  unsigned long long release;  // last released grid barrier: (epoch << 36) | (seq << 8) | decision bits
  unsigned int err;    // (epoch << 4) | -BFS_ERR_*, written by the device on failure
  unsigned int exited; // unused
  int levels;          // max depth + 1
  int levels_run;      // levels executed by the loop (0 for an isolated source)
  unsigned long long t0, t1;
  unsigned long long t_init, t_loop;  // end of the set-up, end of the level loop
  unsigned long long reached_edges;  // sum of m_f over all levels (= 2 x component edges)
  unsigned long long reached;        // sum of n_f over all levels
};

// Everything the level-loop kernel reads, by value.
struct BfsParams {
  const int64_t* off;        // [n_ni+1]
  const int32_t* col;        // [nnz + kColPad]
  const int32_t* caller_of;  // [n]
  const int32_t* internal_of;// [n]
  const int4* head;          // [kHeadVecs n_ni]: first kHead neighbours (internal ids, -1 pad), then their caller ids
  const int32_t* deg;        // [n_ni] degree
  const int2* lead;          // [n_ni] first row entry (internal id, -1 if none) and its caller id
  uint32_t* V;               // visited bitmaps, [words] each: level L reads one and writes
  uint32_t* V1;              // the other (depth <= L and depth <= L+1)
  uint32_t* N0;              // discovered-this-level bitmaps, [words] each
  uint32_t* N1;
  uint32_t* planes;          // depth nibble planes: plane k (< planes_n) at planes + k * pstride,
                             // 8 vertices per word (4 words per visited-bitmap word)
  int32_t* parent_i;         // [n_ni], caller ids
  int32_t* longq;            // vertices whose backward scan is deferred to the end of the level, [long_cap]
  int32_t* Q0;               // normal-vertex frontier queues, [n_ni] each
  int32_t* Q1;
  int2* CL0;                 // delegate chunk lists (vertex, chunk), [cl_cap] each
  int2* CL1;
  LevelSlot* slot;           // [kSlots]
  LevelLogDev* log;          // [BFS_LOG_LEVELS]
  RunHeader* hdr;
  unsigned long long* arrive;// grid-barrier arrival words, one per CTA, 32 bytes apart
  int32_t* out_depth;        // [n] caller-indexed (unused when out_depth8 is set)
  int32_t* out_parent;       // [n] or null
  uint8_t* out_depth8;       // [n] uint8 depth (255 unreached) instead of out_depth, or null
  const int4* crank;         // [ceil(n/32)] per caller word: delegate bits, non-isolated normal bits,
                             // delegates and non-isolated normal vertices before the word
  int64_t nnz;
  int64_t words;             // ceil(n_ni / 32)
  int64_t pstride;           // words of a nibble plane: 4 (words + 1), a multiple of 4
  int64_t cl_cap, long_cap;  // entries of the chunk lists and of the long-row list
  int32_t planes_n;          // nibble planes: enough for any depth below n_ni
  int32_t n, n_ni, d;
  int32_t src_c;             // source, caller id
  int32_t schedule;
  int32_t alpha, beta;
  int32_t td_parent;
  uint64_t schedule_mask;
  double factor0, factor1;
  unsigned long long timeout_ns;
  unsigned int epoch;        // run number; tags the status word
  int32_t test_skip_barrier; // testing only: CTA 0 skips the first barrier
  unsigned long long run_timeout_ns;
  int32_t out_vec4;          // out_depth/out_parent are 16-byte aligned
  int32_t tuning;            // bfs_options.tuning
  // per-subgraph schedule: delegate neighbours per vertex [n_ni]; totals of the three vertex
  // categories of LevelSlot::sub over the whole graph [3]; factors of dd, dn, nd
  const int32_t* deg_del;
  const unsigned long long* sub_tot;
  double sf0[3], sf1[3];
};

}  // namespace bfsgb

struct bfs_graph {
  int device = 0;
  int32_t n = 0, n_ni = 0, d = 0;
  int64_t th = 0, nnz = 0, max_deg = 0;
  int64_t sub[4] = {0, 0, 0, 0};
  int64_t cl_cap = 0;
  int64_t words = 0;
  int64_t device_bytes = 0;
  bfs_options opt{};
  // graph
  int64_t* off = nullptr;
  int32_t* col = nullptr;
  int32_t* caller_of = nullptr;
  int32_t* internal_of = nullptr;
  int4* head = nullptr;
  int32_t* deg = nullptr;
  int2* lead = nullptr;
  // run state
  uint32_t* V = nullptr;
  uint32_t* V1 = nullptr;
  uint32_t* N0 = nullptr;
  uint32_t* N1 = nullptr;
  uint32_t* planes = nullptr;      // depth nibble planes
  int32_t planes_n = 0;
  int64_t pstride = 0;
  int4* crank = nullptr;           // caller-rank words (built with the graph)
  int32_t* parent_i = nullptr;
  int32_t* Q0 = nullptr;
  int32_t* Q1 = nullptr;
  int2* CL0 = nullptr;
  int2* CL1 = nullptr;
  int32_t* longq = nullptr;
  int64_t long_cap = 0;            // vertices whose row is longer than kHead + kShort
  bfsgb::LevelSlot* slot = nullptr;
  bfsgb::LevelLogDev* log = nullptr;
  bfsgb::RunHeader* hdr = nullptr;
  unsigned long long* arrive = nullptr;  // [kMaxBlocks * 4]
  int32_t* out_scratch = nullptr;  // [2n], for runs with host output buffers
  // bfs_run_many: two staging pairs of results and the stream and events that
  // overlap one run's copy to the host with the next run (made on first use)
  int32_t* stage = nullptr;        // [4 n4]: depth/parent of slot 0, then of slot 1
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t ev_run[2] = {nullptr, nullptr}, ev_copy[2] = {nullptr, nullptr}, ev_join = nullptr;
  bfsgb::RunHeader* hdr_many = nullptr;  // pinned host copies of the run headers
  int64_t hdr_many_cap = 0;
  int32_t* deg_del = nullptr;       // per-subgraph schedule (made on first use): delegate neighbours
  unsigned long long* sub_tot = nullptr;  // and the three category totals
  int grid_blocks = 0;
  int grid_blocks_sub = 0;         // CTAs of the per-subgraph build
  int variant = 2;                 // CTAs per SM of the level-loop build in use
  unsigned int epoch = 0;          // runs launched
};

namespace bfsgb {
// Thread-local error text (bfs_last_error).
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);
void* pinned_device_ptr(void* p);
// Level-loop set-up and launch (bfs_run.cu).
int configure_run(bfs_graph* g);
// grid: CTAs of the cooperative launch (0 = the graph's full grid); out_depth8:
// uint8 depths (255 unreached, BFS_ERR_OVERFLOW past 254) instead of out_depth.
int launch_run(bfs_graph* g, int32_t source, int32_t* out_depth, int32_t* out_parent, cudaStream_t s, int grid = 0,
               uint8_t* out_depth8 = nullptr);
int64_t model_bytes_from_log(const bfs_graph* g, const bfs_stats* st);

// Multi-source batches (msbfs.cu).  ms_batch_bytes: device bytes of a batch
// context.  ms_launch: one asynchronous launch on s with per-lane output rows
// (parent == nullptr: depths only), then a copy of the run header to hdr_out
// (pinned host, may be null); *epoch_out gets the run's epoch for
// ms_header_status, which turns a header into BFS_OK or the run's error code.
int64_t ms_batch_bytes(const bfs_graph* g, int with_parents);
int ms_header_status(const RunHeader& h, unsigned epoch);
int ms_launch(bfs_batch* b, const int32_t* sources, int k, uint8_t* const* depth, int32_t* const* parent,
              cudaStream_t s, RunHeader* hdr_out, unsigned* epoch_out);
}  // namespace bfsgb
