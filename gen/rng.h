/* Counter-based random numbers for the seeded synthetic inputs.
 *
 * This header belongs to the input-generator module.  It is the one piece of
 * code that both the CPU oracle's tests and the GPU path's tests use, and it
 * holds none of the graph method's arithmetic: it only turns (seed, stream,
 * counter) into bits, and bits into edge endpoints.
 *
 * Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014).  Its state advances by the golden-ratio
 * increment 0x9E3779B97F4A7C15 and each output is the state passed through
 * the variant-13 64-bit finaliser.  Because the k-th output depends only on
 * the start state and k, value k can be computed directly, which is what
 * makes the host generator and its CUDA twin produce identical bits in any
 * order or thread layout.
 *
 * Every function here is integer-only, so x86 and Arm hosts and the GPU agree
 * bit for bit.
 */
#ifndef GPR_GEN_RNG_H
#define GPR_GEN_RNG_H

#include <stdint.h>

#if defined(__CUDACC__)
#define GEN_FN static __host__ __device__ __forceinline__
#else
#define GEN_FN static inline
#endif

#define GEN_GAMMA 0x9E3779B97F4A7C15ULL

/* Stream identifiers: independent sequences drawn from one user seed. */
#define GEN_STREAM_UNIFORM 1u  /* uniform (u, v) draws, Erdos-Renyi */
#define GEN_STREAM_RMAT 2u     /* R-MAT quadrant draws */
#define GEN_STREAM_PERM 3u     /* Fisher-Yates id permutation */
#define GEN_STREAM_SEEDS 4u    /* personalised-PageRank seed nodes */

/* R-MAT: one 64-bit word gives two 32-bit level draws; at most 64 attempts
 * per edge slot before the documented fallback. */
#define GEN_RMAT_MAX_ATTEMPTS 64

GEN_FN uint64_t gen_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Start state of stream `stream` under user seed `seed`. */
GEN_FN uint64_t gen_stream_key(uint64_t seed, uint64_t stream) {
  return gen_mix64(seed ^ gen_mix64(stream * GEN_GAMMA + 0x632BE59BD9B4E019ULL));
}

/* Output number `ctr` (0-based) of the SplitMix64 sequence that starts at
 * state `key`. */
GEN_FN uint64_t gen_at(uint64_t key, uint64_t ctr) {
  return gen_mix64(key + (ctr + 1u) * GEN_GAMMA);
}

/* Map 32 random bits to [0, n) by a 32x32->64 multiply (Lemire's method
 * without the rejection step; the bias is below n / 2^32). */
GEN_FN uint32_t gen_below(uint32_t r, uint32_t n) {
  return (uint32_t)(((uint64_t)r * (uint64_t)n) >> 32);
}

/* Edge slot i of a uniform COO stream over [0, n)^2. */
GEN_FN void gen_uniform_edge(uint64_t key, uint64_t i, uint32_t n, int32_t* s, int32_t* d) {
  uint64_t r = gen_at(key, i);
  *s = (int32_t)gen_below((uint32_t)(r & 0xFFFFFFFFu), n);
  *d = (int32_t)gen_below((uint32_t)(r >> 32), n);
}

/* Edge slot i of an R-MAT stream (Chakrabarti, Zhan and Faloutsos, SDM 2004).
 * At each of `scale` levels (most significant bit first) one 32-bit draw r
 * picks the quadrant: r < ta -> (0,0); r < tab -> (0,1); r < tabc -> (1,0);
 * else (1,1), where the first bit goes to the source and the second to the
 * destination.  No per-level noise.  An endpoint >= n rejects the attempt and
 * the slot draws again with the next attempt counter; after
 * GEN_RMAT_MAX_ATTEMPTS rejections the last draw is reduced modulo n.
 * Counter layout: (i << 10) | (attempt << 4) | (level >> 1). */
GEN_FN void gen_rmat_edge(uint64_t key, uint64_t i, int scale, uint32_t n, uint32_t ta,
                          uint32_t tab, uint32_t tabc, int32_t* s, int32_t* d) {
  uint32_t u = 0, v = 0;
  for (int a = 0; a < GEN_RMAT_MAX_ATTEMPTS; ++a) {
    u = 0;
    v = 0;
    uint64_t w = 0;
    for (int l = 0; l < scale; ++l) {
      if ((l & 1) == 0) w = gen_at(key, (i << 10) | ((uint64_t)a << 4) | (uint64_t)(l >> 1));
      uint32_t r = (l & 1) ? (uint32_t)(w >> 32) : (uint32_t)(w & 0xFFFFFFFFu);
      uint32_t sb = (r >= tab) ? 1u : 0u;
      uint32_t db = (r < ta) ? 0u : (r < tab) ? 1u : (r < tabc) ? 0u : 1u;
      u = (u << 1) | sb;
      v = (v << 1) | db;
    }
    if (u < n && v < n) {
      *s = (int32_t)u;
      *d = (int32_t)v;
      return;
    }
  }
  *s = (int32_t)(u % n);
  *d = (int32_t)(v % n);
}

#endif /* GPR_GEN_RNG_H */
