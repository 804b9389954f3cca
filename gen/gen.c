/* Host side of the seeded input generators (see gen.h). Plain C, no method
 * arithmetic: endpoints only. */
#include "gen.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "rng.h"

int gen_rmat_thresholds(double a, double b, double c, uint32_t* ta, uint32_t* tab,
                        uint32_t* tabc) {
  if (!(a >= 0 && b >= 0 && c >= 0 && a + b + c <= 1.0)) return -1;
  const double two32 = 4294967296.0;
  double fa = floor(a * two32), fab = floor((a + b) * two32), fabc = floor((a + b + c) * two32);
  if (fa > 4294967295.0) fa = 4294967295.0;
  if (fab > 4294967295.0) fab = 4294967295.0;
  if (fabc > 4294967295.0) fabc = 4294967295.0;
  *ta = (uint32_t)fa;
  *tab = (uint32_t)fab;
  *tabc = (uint32_t)fabc;
  return 0;
}

int gen_uniform_coo(int32_t n, int64_t m_raw, uint64_t seed, int32_t* src, int32_t* dst) {
  if (n <= 0 || m_raw < 0) return -1;
  uint64_t key = gen_stream_key(seed, GEN_STREAM_UNIFORM);
  for (int64_t i = 0; i < m_raw; ++i) gen_uniform_edge(key, (uint64_t)i, (uint32_t)n, &src[i], &dst[i]);
  return 0;
}

/* Open-addressing set of 64-bit pair codes, used only to know when G(n, m)
 * has m distinct pairs. */
typedef struct {
  uint64_t* slot;
  uint64_t mask;
} pairset;

static int pairset_insert(pairset* ps, uint64_t code) {
  uint64_t h = gen_mix64(code) & ps->mask;
  for (;;) {
    uint64_t cur = ps->slot[h];
    if (cur == 0) {
      ps->slot[h] = code;
      return 1;
    }
    if (cur == code) return 0;
    h = (h + 1) & ps->mask;
  }
}

int gen_er_gnm(int32_t n, int64_t m, uint64_t seed, int32_t* src, int32_t* dst, int64_t cap,
               int64_t* m_raw) {
  if (n <= 0 || m < 0 || !m_raw) return -1;
  if ((double)m > (double)n * ((double)n - 1.0) / 2.0) return -1;
  uint64_t size = 16;
  while (size < (uint64_t)m * 2 + 2) size <<= 1;
  pairset ps;
  ps.slot = (uint64_t*)calloc(size, sizeof(uint64_t));
  if (!ps.slot) return -3;
  ps.mask = size - 1;
  uint64_t key = gen_stream_key(seed, GEN_STREAM_UNIFORM);
  int64_t distinct = 0, i = 0;
  while (distinct < m) {
    if (i >= cap) {
      free(ps.slot);
      return -2;
    }
    int32_t u, v;
    gen_uniform_edge(key, (uint64_t)i, (uint32_t)n, &u, &v);
    src[i] = u;
    dst[i] = v;
    ++i;
    /* code + 1 keeps the empty-slot marker 0 free */
    if (u != v && pairset_insert(&ps, (((uint64_t)(uint32_t)u << 32) | (uint32_t)v) + 1u)) ++distinct;
  }
  free(ps.slot);
  *m_raw = i;
  return 0;
}

int gen_permutation(int32_t n, uint64_t seed, int32_t* perm) {
  if (n <= 0) return -1;
  uint64_t key = gen_stream_key(seed, GEN_STREAM_PERM);
  for (int32_t i = 0; i < n; ++i) perm[i] = i;
  for (int32_t i = n - 1; i >= 1; --i) {
    uint32_t j = gen_below((uint32_t)(gen_at(key, (uint64_t)i) >> 32), (uint32_t)i + 1u);
    int32_t t = perm[i];
    perm[i] = perm[j];
    perm[j] = t;
  }
  return 0;
}

int gen_rmat_coo(int scale, int32_t n, int64_t m_raw, double a, double b, double c, uint64_t seed,
                 const int32_t* perm, int32_t* src, int32_t* dst) {
  if (scale < 1 || scale > 31 || n <= 0 || m_raw < 0) return -1;
  if ((int64_t)n > ((int64_t)1 << scale)) return -1;
  uint32_t ta, tab, tabc;
  if (gen_rmat_thresholds(a, b, c, &ta, &tab, &tabc)) return -1;
  uint64_t key = gen_stream_key(seed, GEN_STREAM_RMAT);
  for (int64_t i = 0; i < m_raw; ++i) {
    int32_t u, v;
    gen_rmat_edge(key, (uint64_t)i, scale, (uint32_t)n, ta, tab, tabc, &u, &v);
    if (perm) {
      u = perm[u];
      v = perm[v];
    }
    src[i] = u;
    dst[i] = v;
  }
  return 0;
}

int gen_seed_nodes(int32_t n, int64_t count, uint64_t seed, int32_t* out) {
  if (n <= 0 || count < 0) return -1;
  uint64_t key = gen_stream_key(seed, GEN_STREAM_SEEDS);
  for (int64_t i = 0; i < count; ++i) out[i] = (int32_t)gen_below((uint32_t)(gen_at(key, (uint64_t)i) >> 32), (uint32_t)n);
  return 0;
}

int gen_unit_draws(uint64_t seed, uint32_t stream, int64_t count, double* out) {
  if (count < 0) return -1;
  uint64_t key = gen_stream_key(seed, stream);
  for (int64_t i = 0; i < count; ++i) out[i] = (double)(gen_at(key, (uint64_t)i) >> 11) * 0x1.0p-53;
  return 0;
}
