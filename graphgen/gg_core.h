/*
 * Seeded synthetic graph inputs (shared by the CPU oracle's tests and the GPU path).
 *
 * This header holds input generation only: no step of the BFS method.  It is
 * compiled as plain C for the host twin and as CUDA for the device generator,
 * so both produce the same edge lists bit for bit.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014; the 64-bit finalizer constants are Vigna's
 * public-domain reference), used as a counter-based stream: output i of the
 * stream with seed s is mix(s + (i+1) * gamma).
 *
 * RMAT: the recursive quadrant choice of the Graph500 generator with
 * a,b,c,d = 0.57, 0.19, 0.19, 0.05 and 16 * 2^N edges (Sec. VI-A.3 of
 * Pan, Pearce, Owens, arXiv 1803.03922), one 32-bit draw per level, compared
 * against integer thresholds, and no noise.  Vertex ids are then randomized by
 * a seeded bijection of [0, 2^N) ("deterministic hashing" in the same section).
 * Erdos-Renyi: independent uniform endpoint pairs.
 */
#ifndef GG_CORE_H
#define GG_CORE_H

#include <stdint.h>

#ifdef __CUDACC__
#define GG_HD __host__ __device__ __forceinline__
#else
#define GG_HD static inline
#endif

#define GG_GAMMA 0x9E3779B97F4A7C15ull

GG_HD uint64_t gg_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Output i (0-based) of the SplitMix64 stream seeded with s. */
GG_HD uint64_t gg_draw(uint64_t s, uint64_t i) { return gg_mix64(s + (i + 1) * GG_GAMMA); }

/* floor(x * n / 2^64) without 128-bit types: uniform in [0, n) for n < 2^32. */
GG_HD uint32_t gg_scale(uint64_t x, uint32_t n) {
  uint64_t hi = x >> 32, lo = x & 0xFFFFFFFFull;
  uint64_t t = lo * (uint64_t)n;
  return (uint32_t)((hi * (uint64_t)n + (t >> 32)) >> 32);
}

/* Stream seeds derived from the user seed, one per use. */
GG_HD uint64_t gg_stream(uint64_t seed, uint64_t tag) { return gg_mix64(seed * GG_GAMMA + tag); }
#define GG_TAG_RMAT 0x524D4154ull  /* edge draws */
#define GG_TAG_PERM 0x5045524Dull  /* permutation constants */
#define GG_TAG_ER 0x45522020ull    /* Erdos-Renyi endpoints */
#define GG_TAG_SRC 0x53524353ull   /* BFS sources */

/* Cumulative quadrant thresholds of a,b,c = .57,.19,.19 on 32-bit draws. */
#define GG_TA ((uint64_t)57 * 4294967296ull / 100)
#define GG_TAB ((uint64_t)76 * 4294967296ull / 100)
#define GG_TABC ((uint64_t)95 * 4294967296ull / 100)

/* RMAT edge e at scale N (N <= 31), before the id permutation. */
GG_HD void gg_rmat_edge(uint64_t stream, int scale, uint64_t e, uint32_t* u, uint32_t* v) {
  uint32_t a = 0, b = 0;
  int words = (scale + 1) / 2;
  for (int j = 0; j < words; ++j) {
    uint64_t x = gg_draw(stream, e * (uint64_t)words + (uint64_t)j);
    for (int h = 0; h < 2; ++h) {
      int level = 2 * j + h;
      if (level >= scale) break;
      uint64_t r = h ? (x >> 32) : (x & 0xFFFFFFFFull);
      uint32_t bu = 0, bv = 0;
      if (r < GG_TA) {
      } else if (r < GG_TAB) {
        bv = 1;
      } else if (r < GG_TABC) {
        bu = 1;
      } else {
        bu = 1;
        bv = 1;
      }
      a = (a << 1) | bu;
      b = (b << 1) | bv;
    }
  }
  *u = a;
  *v = b;
}

/* Seeded bijection of [0, 2^N): four rounds of an odd multiply-add followed by
 * an xorshift, each invertible modulo 2^N. */
typedef struct {
  uint32_t mul[4], add[4], mask;
  int shift;
} gg_perm;

GG_HD gg_perm gg_perm_make(uint64_t seed, int scale) {
  gg_perm p;
  uint64_t s = gg_stream(seed, GG_TAG_PERM);
  p.mask = (scale >= 32) ? 0xFFFFFFFFu : ((1u << scale) - 1u);
  p.shift = scale / 2 > 0 ? scale / 2 : 1;
  for (int i = 0; i < 4; ++i) {
    p.mul[i] = ((uint32_t)gg_draw(s, 2 * i) | 1u) & p.mask;
    p.add[i] = (uint32_t)gg_draw(s, 2 * i + 1) & p.mask;
    if (p.mul[i] == 0) p.mul[i] = 1; /* scale 0 */
  }
  return p;
}

GG_HD uint32_t gg_perm_apply(const gg_perm* p, uint32_t x) {
  for (int i = 0; i < 4; ++i) {
    x = (uint32_t)(((uint64_t)x * p->mul[i] + p->add[i]) & p->mask);
    x ^= x >> p->shift;
  }
  return x;
}

/* Erdos-Renyi edge e on n vertices. */
GG_HD void gg_er_edge(uint64_t stream, uint32_t n, uint64_t e, uint32_t* u, uint32_t* v) {
  *u = gg_scale(gg_draw(stream, 2 * e), n);
  *v = gg_scale(gg_draw(stream, 2 * e + 1), n);
}

#endif
