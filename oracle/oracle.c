/* CPU oracle: TEST INFRASTRUCTURE ONLY (see oracle.h for the definitions and
 * the passages they follow).  Plain single-threaded C, FP64, written for a
 * reader to check against the definitions by eye, not for speed. */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---- graph build: E = distinct (u, v) with u != v, CSC grouped by v,
 * sources ascending within a group (section 3 TNGraph; section 5 sorted
 * adjacency). ---- */

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return (x > y) - (x < y);
}

int64_t oracle_build_csc(int32_t n, int64_t m_raw, const int32_t* src, const int32_t* dst,
                         int32_t* col_ptr, int32_t* row_idx, int32_t* outdeg) {
  if (n <= 0 || m_raw < 0) return -1;
  for (int64_t i = 0; i < m_raw; ++i)
    if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return -1;

  /* 1. the pairs (v, u) of non-loop edges, as (v << 32) | u so that numeric
   * order is (destination, source) order */
  uint64_t* pairs = (uint64_t*)malloc((size_t)(m_raw > 0 ? m_raw : 1) * sizeof(uint64_t));
  if (!pairs) return -2;
  int64_t cnt = 0;
  for (int64_t i = 0; i < m_raw; ++i) {
    if (src[i] == dst[i]) continue;
    pairs[cnt++] = ((uint64_t)(uint32_t)dst[i] << 32) | (uint32_t)src[i];
  }

  /* 2. sort and keep one copy of each pair */
  qsort(pairs, (size_t)cnt, sizeof(uint64_t), cmp_u64);
  int64_t m = 0;
  for (int64_t i = 0; i < cnt; ++i)
    if (i == 0 || pairs[i] != pairs[i - 1]) pairs[m++] = pairs[i];

  /* 3. CSC arrays */
  for (int32_t v = 0; v <= n; ++v) col_ptr[v] = 0;
  for (int32_t u = 0; u < n; ++u) outdeg[u] = 0;
  for (int64_t e = 0; e < m; ++e) {
    int32_t v = (int32_t)(pairs[e] >> 32);
    int32_t u = (int32_t)(pairs[e] & 0xFFFFFFFFu);
    col_ptr[v + 1] += 1; /* in-degree of v, turned into offsets below */
    row_idx[e] = u;
    outdeg[u] += 1;
  }
  for (int32_t v = 0; v < n; ++v) col_ptr[v + 1] += col_ptr[v];
  free(pairs);
  return m;
}

/* ---- PageRank power iteration (section 4 Table "snap_methods": PageRank and
 * personalised PageRank; the update is written out in oracle.h). ---- */

int32_t oracle_pagerank(int32_t n, const int32_t* col_ptr, const int32_t* row_idx,
                        const int32_t* outdeg, double d, const double* t, const double* x0,
                        int32_t max_iters, double tol, double* x_out, double* resid) {
  if (n <= 0 || max_iters < 0 || !(d > 0.0 && d < 1.0)) return -1;
  double* x = (double*)malloc((size_t)n * sizeof(double));
  double* xn = (double*)malloc((size_t)n * sizeof(double));
  if (!x || !xn) {
    free(x);
    free(xn);
    return -1;
  }
  memcpy(x, x0, (size_t)n * sizeof(double));
  int32_t k = 0;
  while (k < max_iters) {
    /* dangling mass D_k */
    double dangling = 0.0;
    for (int32_t u = 0; u < n; ++u)
      if (outdeg[u] == 0) dangling += x[u];
    /* x_{k+1}[v] = (1 - d) t[v] + d (sum_{u -> v} x_k[u] / outdeg(u) + D_k t[v]) */
    double delta = 0.0;
    for (int32_t v = 0; v < n; ++v) {
      double pulled = 0.0;
      for (int32_t e = col_ptr[v]; e < col_ptr[v + 1]; ++e) {
        int32_t u = row_idx[e];
        pulled += x[u] / (double)outdeg[u];
      }
      xn[v] = (1.0 - d) * t[v] + d * (pulled + dangling * t[v]);
      double diff = xn[v] - x[v];
      delta += diff < 0 ? -diff : diff;
    }
    if (resid) resid[k] = delta;
    double* sw = x;
    x = xn;
    xn = sw;
    ++k;
    if (tol > 0.0 && (d / (1.0 - d)) * delta <= tol) break;
  }
  memcpy(x_out, x, (size_t)n * sizeof(double));
  free(x);
  free(xn);
  return k;
}

int32_t oracle_pagerank_uniform(int32_t n, const int32_t* col_ptr, const int32_t* row_idx,
                                const int32_t* outdeg, double d, int32_t iters, double* x_out,
                                double* resid) {
  if (n <= 0) return -1;
  double* t = (double*)malloc((size_t)n * sizeof(double));
  if (!t) return -1;
  for (int32_t v = 0; v < n; ++v) t[v] = 1.0 / (double)n;
  int32_t k = oracle_pagerank(n, col_ptr, row_idx, outdeg, d, t, t, iters, 0.0, x_out, resid);
  free(t);
  return k;
}

int32_t oracle_ppr(int32_t n, const int32_t* col_ptr, const int32_t* row_idx, const int32_t* outdeg,
                   double d, int32_t seed, int32_t max_iters, double tol, double* x_out) {
  if (n <= 0 || seed < 0 || seed >= n) return -1;
  double* t = (double*)calloc((size_t)n, sizeof(double));
  if (!t) return -1;
  t[seed] = 1.0;
  int32_t k = oracle_pagerank(n, col_ptr, row_idx, outdeg, d, t, t, max_iters, tol, x_out, NULL);
  free(t);
  return k;
}

/* ---- sampled rows and degrees straight from the raw COO ---- */

static int32_t find_sorted(const int32_t* keys, const int32_t* order, int32_t k, int32_t x) {
  /* keys[order[...]] ascending; returns the position in `order` or -1 */
  int32_t lo = 0, hi = k - 1;
  while (lo <= hi) {
    int32_t mid = lo + (hi - lo) / 2;
    int32_t y = keys[order[mid]];
    if (y == x) return mid;
    if (y < x)
      lo = mid + 1;
    else
      hi = mid - 1;
  }
  return -1;
}

static const int32_t* g_keys_for_sort;
static int cmp_by_key(const void* a, const void* b) {
  int32_t x = g_keys_for_sort[*(const int32_t*)a], y = g_keys_for_sort[*(const int32_t*)b];
  return (x > y) - (x < y);
}

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}

static int32_t* order_of(const int32_t* keys, int32_t k) {
  int32_t* order = (int32_t*)malloc((size_t)(k > 0 ? k : 1) * sizeof(int32_t));
  if (!order) return NULL;
  for (int32_t i = 0; i < k; ++i) order[i] = i;
  g_keys_for_sort = keys;
  qsort(order, (size_t)k, sizeof(int32_t), cmp_by_key);
  return order;
}

/* Collect, for each listed key node, the partner endpoint of every non-loop
 * raw edge whose `side` endpoint equals it; then sort and de-duplicate each
 * list.  side_is_dst = 1: lists of sources of edges into the node. */
static int64_t collect_lists(int32_t n, int64_t m_raw, const int32_t* src, const int32_t* dst,
                             int32_t k, const int32_t* nodes, int side_is_dst, int64_t* off,
                             int32_t** out_list) {
  int32_t* order = order_of(nodes, k);
  if (!order) return -2;
  int64_t* cnt = (int64_t*)calloc((size_t)k + 1, sizeof(int64_t));
  if (!cnt) {
    free(order);
    return -2;
  }
  for (int64_t i = 0; i < m_raw; ++i) {
    if (src[i] == dst[i]) continue;
    int32_t key = side_is_dst ? dst[i] : src[i];
    int32_t pos = find_sorted(nodes, order, k, key);
    if (pos >= 0) cnt[order[pos] + 1] += 1;
  }
  for (int32_t j = 0; j < k; ++j) cnt[j + 1] += cnt[j];
  int32_t* list = (int32_t*)malloc((size_t)(cnt[k] > 0 ? cnt[k] : 1) * sizeof(int32_t));
  int64_t* fill = (int64_t*)malloc((size_t)(k > 0 ? k : 1) * sizeof(int64_t));
  if (!list || !fill) {
    free(order);
    free(cnt);
    free(list);
    free(fill);
    return -2;
  }
  for (int32_t j = 0; j < k; ++j) fill[j] = cnt[j];
  for (int64_t i = 0; i < m_raw; ++i) {
    if (src[i] == dst[i]) continue;
    int32_t key = side_is_dst ? dst[i] : src[i];
    int32_t pos = find_sorted(nodes, order, k, key);
    if (pos >= 0) list[fill[order[pos]]++] = side_is_dst ? src[i] : dst[i];
  }
  /* sort + unique each list, compacting in place */
  int64_t w = 0;
  off[0] = 0;
  for (int32_t j = 0; j < k; ++j) {
    int64_t a = cnt[j], b = cnt[j + 1];
    qsort(list + a, (size_t)(b - a), sizeof(int32_t), cmp_i32);
    for (int64_t e = a; e < b; ++e)
      if (e == a || list[e] != list[e - 1]) list[w++] = list[e];
    off[j + 1] = w;
  }
  (void)n;
  free(order);
  free(cnt);
  free(fill);
  *out_list = list;
  return w;
}

int64_t oracle_sample_in_rows(int32_t n, int64_t m_raw, const int32_t* src, const int32_t* dst,
                              int32_t k, const int32_t* rows, int64_t* row_off, int32_t* row_src,
                              int64_t cap) {
  if (n <= 0 || m_raw < 0 || k < 0) return -1;
  for (int32_t j = 0; j < k; ++j)
    if (rows[j] < 0 || rows[j] >= n) return -1;
  int32_t* list = NULL;
  int64_t total = collect_lists(n, m_raw, src, dst, k, rows, 1, row_off, &list);
  if (total < 0) return total;
  if (total > cap) {
    free(list);
    return -2;
  }
  memcpy(row_src, list, (size_t)total * sizeof(int32_t));
  free(list);
  return total;
}

int32_t oracle_sample_outdeg(int32_t n, int64_t m_raw, const int32_t* src, const int32_t* dst,
                             int32_t k, const int32_t* nodes, int32_t* outdeg_out) {
  if (n <= 0 || m_raw < 0 || k < 0) return -1;
  for (int32_t j = 0; j < k; ++j)
    if (nodes[j] < 0 || nodes[j] >= n) return -1;
  int64_t* off = (int64_t*)malloc(((size_t)k + 1) * sizeof(int64_t));
  if (!off) return -2;
  int32_t* list = NULL;
  int64_t total = collect_lists(n, m_raw, src, dst, k, nodes, 0, off, &list);
  if (total < 0) {
    free(off);
    return (int32_t)total;
  }
  for (int32_t j = 0; j < k; ++j) outdeg_out[j] = (int32_t)(off[j + 1] - off[j]);
  free(list);
  free(off);
  return 0;
}

/* ---- HITS and eigenvector centrality -------------------------------------
 * Both are power iterations with an L2 normalisation after every product
 * (readings stated in oracle.h).  A^T x pulls over in-neighbours (the CSC
 * rows); A x sums each node's out-neighbours, written here as a scatter over
 * the same CSC rows. */

static double l2_norm(int32_t n, const double* x) {
  double s = 0.0;
  for (int32_t i = 0; i < n; ++i) s += x[i] * x[i];
  return sqrt(s);
}

static void scale_unit(int32_t n, double* x) {
  const double nrm = l2_norm(n, x);
  if (nrm > 0.0)
    for (int32_t i = 0; i < n; ++i) x[i] /= nrm;
}

/* y = A^T x: y[v] = sum of x[u] over the in-neighbours u of v */
static void pull_in(int32_t n, const int32_t* col_ptr, const int32_t* row_idx, const double* x, double* y) {
  for (int32_t v = 0; v < n; ++v) {
    double s = 0.0;
    for (int32_t e = col_ptr[v]; e < col_ptr[v + 1]; ++e) s += x[row_idx[e]];
    y[v] = s;
  }
}

/* y = A x: y[u] = sum of x[v] over the out-neighbours v of u */
static void push_out(int32_t n, const int32_t* col_ptr, const int32_t* row_idx, const double* x, double* y) {
  for (int32_t u = 0; u < n; ++u) y[u] = 0.0;
  for (int32_t v = 0; v < n; ++v)
    for (int32_t e = col_ptr[v]; e < col_ptr[v + 1]; ++e) y[row_idx[e]] += x[v];
}

int32_t oracle_hits(int32_t n, const int32_t* col_ptr, const int32_t* row_idx, int32_t iters, double* hub,
                    double* auth) {
  if (n <= 0 || iters < 0 || !col_ptr || !row_idx || !hub || !auth) return -1;
  const double h0 = 1.0 / sqrt((double)n);
  for (int32_t i = 0; i < n; ++i) hub[i] = auth[i] = h0;
  for (int32_t t = 0; t < iters; ++t) {
    pull_in(n, col_ptr, row_idx, hub, auth);
    scale_unit(n, auth);
    push_out(n, col_ptr, row_idx, auth, hub);
    scale_unit(n, hub);
  }
  return 0;
}

int32_t oracle_eigen_centrality(int32_t n, const int32_t* col_ptr, const int32_t* row_idx, int32_t iters,
                                double* x) {
  if (n <= 0 || iters < 0 || !col_ptr || !row_idx || !x) return -1;
  double* y = (double*)malloc((size_t)n * sizeof(double));
  if (!y) return -1;
  for (int32_t i = 0; i < n; ++i) x[i] = 1.0 / sqrt((double)n);
  for (int32_t t = 0; t < iters; ++t) {
    pull_in(n, col_ptr, row_idx, x, y);
    scale_unit(n, y);
    for (int32_t i = 0; i < n; ++i) x[i] = y[i];
  }
  free(y);
  return 0;
}

/* ---- weakly connected components -----------------------------------------
 * Union-find with path halving; each union keeps the smaller root, so a
 * root is the smallest id of its set and labels are the roots. */

static int32_t uf_find(int32_t* parent, int32_t v) {
  while (parent[v] != v) {
    parent[v] = parent[parent[v]];
    v = parent[v];
  }
  return v;
}

int32_t oracle_wcc(int32_t n, const int32_t* col_ptr, const int32_t* row_idx, int32_t* labels) {
  if (n <= 0 || !col_ptr || !row_idx || !labels) return -1;
  int32_t* parent = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  if (!parent) return -1;
  for (int32_t v = 0; v < n; ++v) parent[v] = v;
  for (int32_t v = 0; v < n; ++v) {
    for (int32_t e = col_ptr[v]; e < col_ptr[v + 1]; ++e) {
      const int32_t a = uf_find(parent, row_idx[e]), b = uf_find(parent, v);
      if (a < b)
        parent[b] = a;
      else if (b < a)
        parent[a] = b;
    }
  }
  int32_t count = 0;
  for (int32_t v = 0; v < n; ++v) {
    labels[v] = uf_find(parent, v);
    if (labels[v] == v) ++count;
  }
  free(parent);
  return count;
}

/* ---- single-target personalised PageRank (bidirectional) ------------------ */

int64_t oracle_reverse_push(int32_t n, const int32_t* col_ptr, const int32_t* row_idx, const int32_t* outdeg,
                            int32_t target, double d, double r_max, double* p, double* r) {
  if (n <= 0 || target < 0 || target >= n || !(d > 0.0 && d < 1.0) || !(r_max > 0.0) || !col_ptr || !row_idx ||
      !outdeg || !p || !r)
    return -1;
  const double a = 1.0 - d;
  int32_t* queue = (int32_t*)malloc((size_t)n * sizeof(int32_t));
  char* queued = (char*)calloc((size_t)n, 1);
  if (!queue || !queued) {
    free(queue);
    free(queued);
    return -1;
  }
  for (int32_t v = 0; v < n; ++v) p[v] = r[v] = 0.0;
  r[target] = 1.0;
  int64_t head = 0, size = 0, pushes = 0; /* ring buffer of n entries: each node at most once */
  queue[0] = target;
  queued[target] = 1;
  size = 1;
  while (size > 0) {
    const int32_t v = queue[head];
    head = (head + 1) % n;
    --size;
    queued[v] = 0;
    if (!(r[v] > r_max)) continue;
    const double amt = r[v];
    r[v] = 0.0;
    p[v] += a * amt;
    ++pushes;
    for (int32_t e = col_ptr[v]; e < col_ptr[v + 1]; ++e) {
      const int32_t u = row_idx[e];
      r[u] += (1.0 - a) * amt / outdeg[u];
      if (r[u] > r_max && !queued[u]) {
        queue[(head + size) % n] = u;
        ++size;
        queued[u] = 1;
      }
    }
  }
  free(queue);
  free(queued);
  return pushes;
}

int32_t oracle_ppr_contrib(int32_t n, const int32_t* col_ptr, const int32_t* row_idx, const int32_t* outdeg,
                           int32_t target, double d, int32_t iters, double* q) {
  if (n <= 0 || target < 0 || target >= n || !(d > 0.0 && d < 1.0) || iters < 0 || !q) return -1;
  const double a = 1.0 - d;
  double* acc = (double*)malloc((size_t)n * sizeof(double));
  if (!acc) return -1;
  for (int32_t v = 0; v < n; ++v) q[v] = 0.0;
  for (int32_t k = 0; k < iters; ++k) {
    for (int32_t u = 0; u < n; ++u) acc[u] = 0.0;
    for (int32_t v = 0; v < n; ++v) /* edge u -> v: u's mean includes q(v) */
      for (int32_t e = col_ptr[v]; e < col_ptr[v + 1]; ++e) acc[row_idx[e]] += q[v];
    for (int32_t u = 0; u < n; ++u) q[u] = (u == target ? a : 0.0) + (outdeg[u] > 0 ? d * acc[u] / outdeg[u] : 0.0);
  }
  free(acc);
  return 0;
}

/* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", 2014): state += golden gamma, then the mix. */
static uint64_t sm64_next(uint64_t* state) {
  uint64_t z = (*state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static double sm64_unit(uint64_t* state) { return (double)(sm64_next(state) >> 11) * 0x1p-53; }

int32_t oracle_ppr_target(int32_t n, const int32_t* col_ptr, const int32_t* row_idx, const int32_t* outdeg,
                          int32_t target, double d, double r_max, const int32_t* sources, int32_t k,
                          int32_t walks, uint64_t seed, double* out) {
  if (k < 0 || walks < 1 || (k > 0 && (!sources || !out))) return -1;
  double* p = (double*)malloc((size_t)n * sizeof(double));
  double* r = (double*)malloc((size_t)n * sizeof(double));
  int64_t* optr = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  const int64_t m = n > 0 ? col_ptr[n] : 0;
  int32_t* olist = (int32_t*)malloc((size_t)(m > 0 ? m : 1) * sizeof(int32_t));
  int64_t* fill = (int64_t*)malloc((size_t)n * sizeof(int64_t));
  if (!p || !r || !optr || !olist || !fill || oracle_reverse_push(n, col_ptr, row_idx, outdeg, target, d, r_max, p, r) < 0) {
    free(p); free(r); free(optr); free(olist); free(fill);
    return -1;
  }
  /* out-adjacency, each list ascending: destinations v visited in order */
  for (int32_t u = 0; u < n; ++u) optr[u + 1] = optr[u] + outdeg[u];
  for (int32_t u = 0; u < n; ++u) fill[u] = optr[u];
  for (int32_t v = 0; v < n; ++v)
    for (int32_t e = col_ptr[v]; e < col_ptr[v + 1]; ++e) olist[fill[row_idx[e]]++] = v;
  const double a = 1.0 - d;
  for (int32_t i = 0; i < k; ++i) {
    const int32_t s = sources[i];
    if (s < 0 || s >= n) {
      free(p); free(r); free(optr); free(olist); free(fill);
      return -1;
    }
    double sum_r = 0.0;
    int64_t at_dangling = 0;
    for (int32_t w = 0; w < walks; ++w) {
      uint64_t st = seed ^ (((uint64_t)(uint32_t)i << 32) | (uint32_t)w) * 0xD6E8FEB86659FD93ull;
      int32_t u = s;
      for (int32_t step = 0; step < (1 << 20); ++step) {
        if (sm64_unit(&st) < a) break;
        if (outdeg[u] == 0) {
          u = s; /* dangling: the walk's mass goes back to the seed */
          continue;
        }
        /* uniform index: floor(X k / 2^53) for the draw's top 53 bits X (exact) */
        const uint64_t x53 = sm64_next(&st) >> 11;
        const int64_t j = (int64_t)(((unsigned __int128)x53 * (uint64_t)outdeg[u]) >> 53);
        u = olist[optr[u] + j];
      }
      sum_r += r[u];
      at_dangling += outdeg[u] == 0;
    }
    out[i] = p[s] * (1.0 + (d / a) * ((double)at_dangling / walks)) + sum_r / walks;
  }
  free(p); free(r); free(optr); free(olist); free(fill);
  return 0;
}
