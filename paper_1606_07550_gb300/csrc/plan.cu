// PageRank execution layout, derived from the relabelled CSC at build time.
//
// graph_build numbers the nodes by descending out-degree before it sorts the
// edges (build.cu), so on a power-law graph the contributions that the pull
// step reads most often sit in one compact address range at the front of the
// contribution vector, and within every in-adjacency list the sources are
// ascending, densest first: the lanes of a warp that walk a long list hit the
// same 32-byte sectors and the same L1 lines.  This file adds, per graph:
//   - inverse out-degrees (0 for dangling nodes);
//   - the rows of each in-degree bucket as an ascending row list, so each
//     bucket runs with a fixed number of lanes per row (1, 4, 8 or 32);
//   - the hot/cold split of every row: sources below hot_H, the contributions
//     a block can keep in shared memory, form a prefix of each sorted row;
//   - for rows above the last lane bucket, lists of edge chunks of at most
//     chunk_edges edges over their hot prefixes and their cold suffixes, one
//     warp per chunk; such rows are finished from their chunk sums in a
//     fixed order.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <string>

#include "gpr_internal.cuh"

namespace gpr {

constexpr int kPThreads = 256;

// Default buckets: inclusive upper in-degree bound and lanes per row (0 =
// warp chunks).  Overridable with GPR_BUCKETS="2:1,8:4,...,*:0" and
// GPR_CHUNK_EDGES.
struct BucketSpec {
  int32_t max_deg;
  int lanes;
};
static const BucketSpec kDefaultBuckets[] = {{2, 1}, {8, 4}, {32, 8}, {1024, 32}, {INT_MAX, 0}};
constexpr int32_t kDefaultChunkEdges = 2048;

static int parse_buckets(BucketSpec* out, int32_t* chunk_edges) {
  *chunk_edges = kDefaultChunkEdges;
  const char* ce = getenv("GPR_CHUNK_EDGES");
  if (ce && atoi(ce) >= 128) *chunk_edges = atoi(ce) & ~127;
  const char* env = getenv("GPR_BUCKETS");
  if (!env || !*env) {
    int nb = (int)(sizeof kDefaultBuckets / sizeof kDefaultBuckets[0]);
    for (int i = 0; i < nb; ++i) out[i] = kDefaultBuckets[i];
    return nb;
  }
  std::string s(env);
  int nb = 0;
  size_t pos = 0;
  while (pos < s.size() && nb < kMaxBuckets) {
    size_t comma = s.find(',', pos);
    std::string item = s.substr(pos, comma == std::string::npos ? std::string::npos : comma - pos);
    size_t colon = item.find(':');
    if (colon == std::string::npos) break;
    std::string a = item.substr(0, colon), b = item.substr(colon + 1);
    BucketSpec bs;
    bs.max_deg = (a == "*") ? INT_MAX : atoi(a.c_str());
    bs.lanes = atoi(b.c_str());
    if (bs.lanes != 0 && bs.lanes != 1 && bs.lanes != 2 && bs.lanes != 4 && bs.lanes != 8 && bs.lanes != 16 &&
        bs.lanes != 32)
      bs.lanes = 32;
    out[nb++] = bs;
    if (comma == std::string::npos) break;
    pos = comma + 1;
  }
  if (nb == 0 || out[nb - 1].max_deg != INT_MAX) {
    if (nb == kMaxBuckets) nb = kMaxBuckets - 1;
    out[nb++] = BucketSpec{INT_MAX, 0};
  }
  return nb;
}

struct Thresholds {
  int32_t v[kMaxBuckets];
};

struct PlanDev {
  int32_t n_dangling, max_in, max_out;
  int32_t bstart[kMaxBuckets + 1];
};

// Per row: inverse out-degree, statistics, and the bucket key
// (bucket << b | row) whose sort yields the per-bucket row lists.
__global__ void row_keys_kernel(const int32_t* __restrict__ col_ptr, const int32_t* __restrict__ outdeg,
                                int32_t n, int b, int nb, Thresholds th, float* __restrict__ inv_deg,
                                uint64_t* __restrict__ keys, PlanDev* __restrict__ pd) {
  int32_t dang = 0, mi = 0, mo = 0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t indeg = col_ptr[p + 1] - col_ptr[p];
    const int32_t od = outdeg[p];
    inv_deg[p] = od > 0 ? 1.0f / (float)od : 0.0f;
    int bk = 0;
    while (bk < nb - 1 && indeg > th.v[bk]) ++bk;
    keys[p] = ((uint64_t)bk << b) | (uint64_t)p;
    dang += (od == 0);
    mi = max(mi, indeg);
    mo = max(mo, od);
  }
  for (int o = 16; o > 0; o >>= 1) {
    dang += __shfl_xor_sync(0xffffffffu, dang, o);
    mi = max(mi, __shfl_xor_sync(0xffffffffu, mi, o));
    mo = max(mo, __shfl_xor_sync(0xffffffffu, mo, o));
  }
  if ((threadIdx.x & 31) == 0) {
    if (dang) atomicAdd(&pd->n_dangling, dang);
    atomicMax(&pd->max_in, mi);
    atomicMax(&pd->max_out, mo);
  }
}

__global__ void row_lists_kernel(const uint64_t* __restrict__ sorted, int32_t n, int b, int32_t* __restrict__ rows,
                                 PlanDev* __restrict__ pd) {
  const uint64_t mask = (1ull << b) - 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = sorted[i];
    rows[i] = (int32_t)(key & mask);
    const int bk = (int)(key >> b);
    const int pb = i > 0 ? (int)(sorted[i - 1] >> b) : -1;
    for (int q = pb + 1; q <= bk; ++q) pd->bstart[q] = (int32_t)i;
  }
}

// First edge of each row whose source is >= H (rows are sorted ascending).
__global__ void split_kernel(const int32_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx, int32_t n,
                             int32_t H, int32_t* __restrict__ split) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    int32_t lo = col_ptr[p], hi = col_ptr[p + 1];
    while (lo < hi) {
      const int32_t mid = lo + (hi - lo) / 2;
      if (row_idx[mid] < H)
        lo = mid + 1;
      else
        hi = mid;
    }
    split[p] = lo;
  }
}

// Hot and cold chunk counts of the long rows rows[i0, i1): ceil(hot prefix /
// C) and ceil(cold suffix / C).
__global__ void chunk_counts_kernel(const int32_t* __restrict__ rows, int32_t i0, int32_t i1,
                                    const int32_t* __restrict__ col_ptr, const int32_t* __restrict__ split, int32_t C,
                                    int32_t* __restrict__ hc, int32_t* __restrict__ cc) {
  for (int64_t i = i0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < i1; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = rows[i];
    const int64_t e0 = col_ptr[r], sp = split[r], e1 = col_ptr[r + 1];
    hc[i - i0] = (int32_t)((sp - e0 + C - 1) / C);
    cc[i - i0] = (int32_t)((e1 - sp + C - 1) / C);
  }
}

// The chunk entries and split records of the long rows rows[i0, i1), one warp
// per row: its hot chunks at hot_base + hoff, its cold chunks at cold_base +
// coff, its record at split_base + (i - i0).
struct ChunkLists {
  int32_t *chunk_row, *chunk_begin, *chunk_end;
  int32_t *split_row, *split_hbeg, *split_hend, *split_cbeg, *split_cend;
};
__global__ void chunk_lists_kernel(const int32_t* __restrict__ rows, int32_t i0, int32_t i1,
                                   const int32_t* __restrict__ col_ptr, const int32_t* __restrict__ split, int32_t C,
                                   const int32_t* __restrict__ hoff, const int32_t* __restrict__ coff,
                                   int32_t split_base, int32_t hot_base, int32_t cold_base, ChunkLists L) {
  const int lane = threadIdx.x & 31;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t wi = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; wi < i1 - i0; wi += nwarps) {
    const int32_t r = rows[i0 + wi];
    const int64_t e0 = col_ptr[r], sp = split[r], e1 = col_ptr[r + 1];
    const int32_t nh = (int32_t)((sp - e0 + C - 1) / C), nc = (int32_t)((e1 - sp + C - 1) / C);
    const int32_t h0 = hot_base + hoff[wi], c0 = cold_base + coff[wi];
    if (lane == 0) {
      const int32_t k = split_base + (int32_t)wi;
      L.split_row[k] = r;
      L.split_hbeg[k] = h0;
      L.split_hend[k] = h0 + nh;
      L.split_cbeg[k] = c0;
      L.split_cend[k] = c0 + nc;
    }
    for (int32_t j = lane; j < nh; j += 32) {
      L.chunk_row[h0 + j] = r;
      L.chunk_begin[h0 + j] = (int32_t)(e0 + (int64_t)j * C);
      L.chunk_end[h0 + j] = (int32_t)min(sp, e0 + (int64_t)(j + 1) * C);
    }
    for (int32_t j = lane; j < nc; j += 32) {
      L.chunk_row[c0 + j] = r;
      L.chunk_begin[c0 + j] = (int32_t)(sp + (int64_t)j * C);
      L.chunk_end[c0 + j] = (int32_t)min(e1, sp + (int64_t)(j + 1) * C);
    }
  }
}

void plan_free(Plan& p, cudaStream_t s) {
  dfree(p.new2old, s);
  dfree(p.old2new, s);
  dfree(p.inv_deg, s);
  dfree(p.rows, s);
  dfree(p.split, s);
  dfree(p.chunk_row, s);
  dfree(p.chunk_begin, s);
  dfree(p.chunk_end, s);
  dfree(p.split_row, s);
  dfree(p.split_hbeg, s);
  dfree(p.split_hend, s);
  dfree(p.split_cbeg, s);
  dfree(p.split_cend, s);
  p = Plan();
}

static int grid_for(int64_t items) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((items + kPThreads - 1) / kPThreads, (int64_t)num_sms() * 8));
}

void plan_build(gpr_graph* g, cudaStream_t s, int* derr) {
  Plan& P = g->plan;
  const int32_t n = g->n;
  const int b = g->id_bits;
  BucketSpec bs[kMaxBuckets];
  const int nb = parse_buckets(bs, &P.chunk_edges);
  Thresholds th{};
  for (int i = 0; i < nb; ++i) th.v[i] = bs[i].max_deg;

  std::vector<void*> tmp;
  auto T = [&](size_t bytes) {
    void* p = dalloc(bytes, s);
    tmp.push_back(p);
    return p;
  };
  try {
    PlanDev* pd = (PlanDev*)T(sizeof(PlanDev));
    PlanDev init{};
    for (int i = 0; i <= kMaxBuckets; ++i) init.bstart[i] = n;
    GPR_CUDA(cudaMemcpyAsync(pd, &init, sizeof init, cudaMemcpyHostToDevice, s));
    P.inv_deg = (float*)dalloc((size_t)n * 4, s);
    P.rows = (int32_t*)dalloc((size_t)n * 4, s);
    uint64_t* keys = (uint64_t*)T((size_t)n * 8);
    uint64_t* alt = (uint64_t*)T((size_t)n * 8);
    row_keys_kernel<<<grid_for(n), kPThreads, 0, s>>>(g->col_ptr, g->outdeg, n, b, nb, th, P.inv_deg, keys, pd);
    GPR_CUDA(cudaGetLastError());
    count_launches(1);
    int bb = 1;
    while ((1 << bb) < nb) ++bb;
    uint64_t* sorted = radix_sort_u64(keys, alt, n, b + bb, s, derr, nullptr);
    trace_phase("plan: bucket keys + sort", s);
    row_lists_kernel<<<grid_for(n), kPThreads, 0, s>>>(sorted, n, b, P.rows, pd);
    GPR_CUDA(cudaGetLastError());
    count_launches(1);
    PlanDev h{};
    GPR_CUDA(cudaMemcpyAsync(&h, pd, sizeof h, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    g->n_dangling = h.n_dangling;
    g->max_in = h.max_in;
    g->max_out = h.max_out;
    P.nbuckets = nb;
    for (int k = 0; k < nb; ++k) {
      P.bucket[k].row_begin = h.bstart[k];
      P.bucket[k].row_end = (k + 1 < nb) ? h.bstart[k + 1] : n;
      P.bucket[k].lanes = bs[k].lanes;
      P.deg_threshold[k] = bs[k].max_deg;
    }

    // hot/cold split of every row.  Off unless GPR_HOT asks for it: on the
    // billion-edge R-MAT graph the extra pass cost more than the shared-memory
    // gathers saved (3.66 ms per step without, 4.2-5.2 ms with H = 8K-56K).
    P.hot_H = 0;
    const char* hot_env = getenv("GPR_HOT");
    if (hot_env) P.hot_H = std::max<int32_t>(0, std::min<int32_t>(std::min(hot_capacity(), n), atoi(hot_env))) & ~7;
    trace_phase("plan: bucket lists", s);
    P.split = (int32_t*)dalloc((size_t)n * 4, s);
    split_kernel<<<grid_for(n), kPThreads, 0, s>>>(g->col_ptr, g->row_idx, n, P.hot_H, P.split);
    GPR_CUDA(cudaGetLastError());
    count_launches(1);

    // chunk lists of the long-row bucket(s): hot prefixes first, then cold
    // suffixes; counts per row, their prefix sums, then the entries
    struct LongRange {
      int32_t i0, i1;
      int32_t *hoff, *coff;
      int64_t hot, cold;
    };
    std::vector<LongRange> lr;
    int64_t n_hot = 0, n_cold = 0, n_long = 0;
    for (int k = 0; k < nb; ++k) {
      if (P.bucket[k].lanes != 0) continue;
      LongRange R{P.bucket[k].row_begin, P.bucket[k].row_end, nullptr, nullptr, 0, 0};
      const int32_t len = R.i1 - R.i0;
      if (len <= 0) continue;
      int32_t* hc = (int32_t*)T((size_t)len * 4);
      int32_t* cc = (int32_t*)T((size_t)len * 4);
      R.hoff = (int32_t*)T((size_t)len * 4);
      R.coff = (int32_t*)T((size_t)len * 4);
      chunk_counts_kernel<<<grid_for(len), kPThreads, 0, s>>>(P.rows, R.i0, R.i1, g->col_ptr, P.split, P.chunk_edges,
                                                             hc, cc);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
      R.hot = exclusive_scan_i32(hc, len, R.hoff, s);
      R.cold = exclusive_scan_i32(cc, len, R.coff, s);
      n_hot += R.hot;
      n_cold += R.cold;
      n_long += len;
      lr.push_back(R);
    }
    if (n_hot + n_cold > INT32_MAX) throw StatusFail{GPR_EINVAL, "too many long-row chunks"};
    P.n_hot_chunks = (int32_t)n_hot;
    P.nchunks = (int32_t)(n_hot + n_cold);
    P.nsplit = (int32_t)n_long;
    auto arr = [&](int64_t k) { return (int32_t*)dalloc((size_t)std::max<int64_t>(k, 1) * 4, s); };
    P.chunk_row = arr(P.nchunks);
    P.chunk_begin = arr(P.nchunks);
    P.chunk_end = arr(P.nchunks);
    P.split_row = arr(P.nsplit);
    P.split_hbeg = arr(P.nsplit);
    P.split_hend = arr(P.nsplit);
    P.split_cbeg = arr(P.nsplit);
    P.split_cend = arr(P.nsplit);
    const ChunkLists L{P.chunk_row,  P.chunk_begin, P.chunk_end,  P.split_row,
                       P.split_hbeg, P.split_hend,  P.split_cbeg, P.split_cend};
    int64_t sb = 0, hb = 0, cb = n_hot;
    for (const LongRange& R : lr) {
      const int32_t len = R.i1 - R.i0;
      chunk_lists_kernel<<<grid_for((int64_t)len * 32), kPThreads, 0, s>>>(
          P.rows, R.i0, R.i1, g->col_ptr, P.split, P.chunk_edges, R.hoff, R.coff, (int32_t)sb, (int32_t)hb,
          (int32_t)cb, L);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
      sb += len;
      hb += R.hot;
      cb += R.cold;
    }
    trace_phase("plan: split + long-row chunks", s);
    for (void* p : tmp) dfree(p, s);
  } catch (...) {
    for (void* p : tmp) dfree(p, s);
    throw;
  }
}

}  // namespace gpr
