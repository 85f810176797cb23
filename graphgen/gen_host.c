/* Host twin of the seeded graph generator (input generation only; see gg_core.h). */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>

#include "gg_core.h"

typedef struct {
  int kind; /* 0 rmat, 1 er, 2 rmat without the id permutation */
  int scale;
  uint32_t n;
  uint64_t seed;
  int64_t begin, end;
  int32_t* src;
  int32_t* dst;
} gg_job;

static void* gg_worker(void* arg) {
  gg_job* j = (gg_job*)arg;
  if (j->kind == 0 || j->kind == 2) {
    uint64_t stream = gg_stream(j->seed, GG_TAG_RMAT);
    gg_perm p = gg_perm_make(j->seed, j->scale);
    for (int64_t e = j->begin; e < j->end; ++e) {
      uint32_t u, v;
      gg_rmat_edge(stream, j->scale, (uint64_t)e, &u, &v);
      j->src[e] = (int32_t)(j->kind == 0 ? gg_perm_apply(&p, u) : u);
      j->dst[e] = (int32_t)(j->kind == 0 ? gg_perm_apply(&p, v) : v);
    }
  } else {
    uint64_t stream = gg_stream(j->seed, GG_TAG_ER);
    for (int64_t e = j->begin; e < j->end; ++e) {
      uint32_t u, v;
      gg_er_edge(stream, j->n, (uint64_t)e, &u, &v);
      j->src[e] = (int32_t)u;
      j->dst[e] = (int32_t)v;
    }
  }
  return NULL;
}

static int gg_run(int kind, int scale, uint32_t n, int64_t m, uint64_t seed, int32_t* src,
                  int32_t* dst, int nthreads) {
  if (m < 0 || !src || !dst) return -1;
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if (m < 65536) nthreads = 1;
  gg_job jobs[256];
  pthread_t th[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t].kind = kind;
    jobs[t].scale = scale;
    jobs[t].n = n;
    jobs[t].seed = seed;
    jobs[t].begin = m * t / nthreads;
    jobs[t].end = m * (t + 1) / nthreads;
    jobs[t].src = src;
    jobs[t].dst = dst;
  }
  for (int t = 1; t < nthreads; ++t) pthread_create(&th[t], NULL, gg_worker, &jobs[t]);
  gg_worker(&jobs[0]);
  for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
  return 0;
}

/* RMAT edges at the given scale: m = edge_factor * 2^scale pairs, ids permuted
 * (permute = 0 returns the raw quadrant-recursion ids, for statistical tests). */
int gg_rmat_host(int scale, int edge_factor, uint64_t seed, int32_t* src, int32_t* dst,
                 int nthreads, int permute) {
  if (scale < 0 || scale > 30 || edge_factor < 0) return -1;
  int64_t m = (int64_t)edge_factor << scale;
  return gg_run(permute ? 0 : 2, scale, 1u << scale, m, seed, src, dst, nthreads);
}

/* Erdos-Renyi: m uniform pairs on n vertices. */
int gg_er_host(int32_t n, int64_t m, uint64_t seed, int32_t* src, int32_t* dst, int nthreads) {
  if (n <= 0) return -1;
  return gg_run(1, 0, (uint32_t)n, m, seed, src, dst, nthreads);
}

uint32_t gg_perm_host(int scale, uint64_t seed, uint32_t x) {
  gg_perm p = gg_perm_make(seed, scale);
  return gg_perm_apply(&p, x);
}

/* mask[v] = 1 iff v is an endpoint of some pair with distinct endpoints. */
void gg_mark_nonisolated_host(int32_t n, int64_t m, const int32_t* src, const int32_t* dst,
                              uint8_t* mask) {
  for (int32_t v = 0; v < n; ++v) mask[v] = 0;
  for (int64_t e = 0; e < m; ++e)
    if (src[e] != dst[e]) {
      mask[src[e]] = 1;
      mask[dst[e]] = 1;
    }
}

/* Seeded BFS sources: uniform draws over [0,n), rejecting masked-out vertices
 * and repeats, first k kept.  Returns how many were found (< k only when fewer
 * than k vertices qualify). */
int32_t gg_sample_sources(int32_t n, const uint8_t* mask, int32_t k, uint64_t seed, int32_t* out) {
  int64_t avail = 0;
  for (int32_t v = 0; v < n; ++v) avail += mask[v] ? 1 : 0;
  int32_t want = (int64_t)k < avail ? k : (int32_t)avail;
  uint64_t s = gg_stream(seed, GG_TAG_SRC);
  int32_t got = 0;
  for (uint64_t i = 0; got < want; ++i) {
    int32_t v = (int32_t)gg_scale(gg_draw(s, i), (uint32_t)n);
    if (!mask[v]) continue;
    int dup = 0;
    for (int32_t j = 0; j < got; ++j)
      if (out[j] == v) dup = 1;
    if (!dup) out[got++] = v;
  }
  return got;
}
