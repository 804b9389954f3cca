// PageRank execution layout, derived from the canonical CSC at build time.
//
// The pull step reads, for every edge, the contribution of its source.  On a
// power-law graph a few sources carry most edges; once ids are relabelled so
// that rows are grouped by in-degree bucket and, inside a bucket, ordered by
// descending out-degree, the heavily read contributions sit in a few compact
// address ranges that stay resident in L2 / L1, and each degree bucket is a
// contiguous row range (no row lists to read per iteration).  Relabelling is
// a bijection: results are mapped back to the caller's ids on output, and
// the canonical CSC (the build's bit-exact product) is kept unchanged.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <climits>
#include <string>

#include "gpr_internal.cuh"

namespace gpr {

constexpr int kPThreads = 256;
constexpr uint64_t kOutMax = (1ull << 29) - 1;

// Default buckets: inclusive upper in-degree bound and lanes per row (0 =
// chunked block-per-row).  Overridable with GPR_BUCKETS="2:1,8:4,...,*:0".
struct BucketSpec {
  int32_t max_deg;
  int lanes;
};
static const BucketSpec kDefaultBuckets[] = {{2, 1}, {8, 4}, {32, 8}, {1024, 32}, {INT_MAX, 0}};
constexpr int32_t kDefaultChunkEdges = 8192;

static int parse_buckets(BucketSpec* out, int32_t* chunk_edges) {
  *chunk_edges = kDefaultChunkEdges;
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
    out[nb++] = bs;
    if (comma == std::string::npos) break;
    pos = comma + 1;
  }
  if (nb == 0 || out[nb - 1].max_deg != INT_MAX) {
    if (nb == kMaxBuckets) nb = kMaxBuckets - 1;
    out[nb++] = BucketSpec{INT_MAX, 0};
  }
  const char* ce = getenv("GPR_CHUNK_EDGES");
  if (ce && atoi(ce) >= 1024) *chunk_edges = atoi(ce) & ~1023;
  return nb;
}

struct PlanDev {
  int32_t n_dangling, max_in, max_out;
  int32_t bstart[kMaxBuckets + 1];
};

struct Thresholds {
  int32_t v[kMaxBuckets];
};

__global__ void node_keys_kernel(const int32_t* __restrict__ col_ptr, const int32_t* __restrict__ outdeg,
                                 int32_t n, int nb, Thresholds th, uint64_t* __restrict__ keys,
                                 PlanDev* __restrict__ pd) {
  int32_t dang = 0, mi = 0, mo = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t indeg = col_ptr[v + 1] - col_ptr[v];
    const int32_t od = outdeg[v];
    int b = 0;
    while (b < nb - 1 && indeg > th.v[b]) ++b;
    const uint64_t odc = (uint64_t)(od < 0 ? 0 : od);
    keys[v] = ((uint64_t)b << 60) | ((kOutMax - (odc < kOutMax ? odc : kOutMax)) << 31) | (uint64_t)v;
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

__global__ void perm_kernel(const uint64_t* __restrict__ sorted, const int32_t* __restrict__ col_ptr,
                            const int32_t* __restrict__ outdeg, int32_t n, int32_t* __restrict__ new2old,
                            int32_t* __restrict__ old2new, int32_t* __restrict__ pdeg, float* __restrict__ inv_deg,
                            PlanDev* __restrict__ pd) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t key = sorted[p];
    const int32_t v = (int32_t)(key & 0x7FFFFFFFull);
    new2old[p] = v;
    old2new[v] = (int32_t)p;
    pdeg[p] = col_ptr[v + 1] - col_ptr[v];
    const int32_t od = outdeg[v];
    inv_deg[p] = od > 0 ? 1.0f / (float)od : 0.0f;
    const int b = (int)(key >> 60);
    const int pb = p > 0 ? (int)(sorted[p - 1] >> 60) : -1;
    for (int q = pb + 1; q <= b; ++q) pd->bstart[q] = (int32_t)p;
  }
}

// Exclusive scan of n int32 counts into out[0..n] (out[n] = total), one
// pass, tiles chained by decoupled look-back.  Item j of warp w is tile
// position w*512 + j*32 + lane.
constexpr int kScanItems = 16;
constexpr int kScanTile = kPThreads * kScanItems;
__global__ void __launch_bounds__(kPThreads) scan_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                                        int64_t n, uint64_t* __restrict__ status,
                                                        uint32_t* __restrict__ tile_ctr, int* __restrict__ derr) {
  __shared__ uint32_t s_wsum[kPThreads / 32];
  __shared__ uint64_t s_excl;
  __shared__ uint32_t s_tile;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (t == 0) s_tile = atomicAdd(tile_ctr, 1u);
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t base = tile * kScanTile + (int64_t)w * (kScanItems * 32) + lane;
  uint32_t loc[kScanItems];
  uint32_t run = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t i = base + j * 32;
    const uint32_t v = i < n ? (uint32_t)in[i] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    loc[j] = run + x - v;
    run += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) s_wsum[w] = run;
  __syncthreads();
  if (t == 0) {
    uint64_t tot = 0;
    for (int ww = 0; ww < kPThreads / 32; ++ww) tot += s_wsum[ww];
    uint64_t excl = 0;
    if (tile == 0) {
      st_relaxed_u64(status, lb_word(1, kFlagInc, tot));
    } else {
      st_relaxed_u64(status + tile, lb_word(1, kFlagAgg, tot));
      excl = lookback(status, tile, 1, 1, derr);
      st_relaxed_u64(status + tile, lb_word(1, kFlagInc, excl + tot));
    }
    s_excl = excl;
  }
  __syncthreads();
  uint64_t off = s_excl;
  for (int ww = 0; ww < w; ++ww) off += s_wsum[ww];
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t i = base + j * 32;
    if (i < n) {
      out[i] = (int32_t)(off + loc[j]);
      if (i == n - 1) out[n] = (int32_t)(off + loc[j] + (uint32_t)in[i]);
    }
  }
}

// Relabelled edges: the edge at canonical position e (destination v, source
// u) goes to row old2new[v] at the same offset within the row, as source
// old2new[u].
__global__ void edge_map_kernel(const int32_t* __restrict__ row_idx, const int32_t* __restrict__ edge_dst,
                                const int32_t* __restrict__ col_ptr, const int32_t* __restrict__ old2new,
                                const int32_t* __restrict__ pcol_ptr, int64_t m, int32_t* __restrict__ prow_idx) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = edge_dst[e];
    const int32_t u = __ldcs(row_idx + e);
    const int32_t p = old2new[v];
    const int64_t pos = (int64_t)pcol_ptr[p] + (e - col_ptr[v]);
    prow_idx[pos] = old2new[u];
  }
}

void plan_free(Plan& p, cudaStream_t s) {
  dfree(p.new2old, s);
  dfree(p.old2new, s);
  dfree(p.col_ptr, s);
  dfree(p.row_idx, s);
  dfree(p.inv_deg, s);
  dfree(p.chunk_row, s);
  dfree(p.chunk_begin, s);
  dfree(p.chunk_end, s);
  dfree(p.chunk_whole, s);
  dfree(p.split_row, s);
  dfree(p.split_cbeg, s);
  dfree(p.split_cend, s);
  p = Plan();
}

static int grid_for(int64_t items) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((items + kPThreads - 1) / kPThreads, (int64_t)num_sms() * 8));
}

void plan_build_from(gpr_graph* g, const int32_t* edge_dst, cudaStream_t s, int* derr) {
  Plan& P = g->plan;
  const int32_t n = g->n;
  const int64_t m = g->m;
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
    uint64_t* keys = (uint64_t*)T((size_t)n * 8);
    uint64_t* alt = (uint64_t*)T((size_t)n * 8);
    node_keys_kernel<<<grid_for(n), kPThreads, 0, s>>>(g->col_ptr, g->outdeg, n, nb, th, keys, pd);
    GPR_CUDA(cudaGetLastError());
    count_launches(1);
    uint64_t* sorted = radix_sort_u64(keys, alt, n, 64, s, derr, nullptr);

    P.new2old = (int32_t*)dalloc((size_t)n * 4, s);
    P.old2new = (int32_t*)dalloc((size_t)n * 4, s);
    P.col_ptr = (int32_t*)dalloc(((size_t)n + 1) * 4, s);
    P.inv_deg = (float*)dalloc((size_t)n * 4, s);
    P.row_idx = (int32_t*)dalloc((size_t)std::max<int64_t>(m, 1) * 4, s);
    int32_t* pdeg = (int32_t*)T((size_t)n * 4);
    perm_kernel<<<grid_for(n), kPThreads, 0, s>>>(sorted, g->col_ptr, g->outdeg, n, P.new2old, P.old2new, pdeg,
                                                  P.inv_deg, pd);
    GPR_CUDA(cudaGetLastError());
    count_launches(1);
    const int64_t tiles = ((int64_t)n + kScanTile - 1) / kScanTile;
    uint64_t* status = (uint64_t*)T((size_t)tiles * 8);
    uint32_t* ctr = (uint32_t*)T(8);
    GPR_CUDA(cudaMemsetAsync(status, 0, (size_t)tiles * 8, s));
    GPR_CUDA(cudaMemsetAsync(ctr, 0, 8, s));
    scan_kernel<<<(unsigned)tiles, kPThreads, 0, s>>>(pdeg, P.col_ptr, n, status, ctr, derr);
    GPR_CUDA(cudaGetLastError());
    count_launches(1);
    if (m > 0) {
      edge_map_kernel<<<grid_for(m), kPThreads, 0, s>>>(g->row_idx, edge_dst, g->col_ptr, P.old2new, P.col_ptr, m,
                                                        P.row_idx);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
    }
    PlanDev h{};
    GPR_CUDA(cudaMemcpyAsync(&h, pd, sizeof h, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    g->n_dangling = h.n_dangling;
    g->max_in = h.max_in;
    g->max_out = h.max_out;

    P.nbuckets = nb;
    for (int b = 0; b < nb; ++b) {
      P.bucket[b].row_begin = h.bstart[b];
      P.bucket[b].row_end = (b + 1 < nb) ? h.bstart[b + 1] : n;
      P.bucket[b].lanes = bs[b].lanes;
      P.deg_threshold[b] = bs[b].max_deg;
    }

    // chunk list of the block bucket (the one with lanes == 0)
    std::vector<int32_t> crow, cbeg, cend, cwhole, srow, sbeg, send;
    for (int b = 0; b < nb; ++b) {
      if (P.bucket[b].lanes != 0) continue;
      const int32_t r0 = P.bucket[b].row_begin, r1 = P.bucket[b].row_end;
      if (r1 <= r0) continue;
      std::vector<int32_t> cp((size_t)(r1 - r0) + 1);
      GPR_CUDA(cudaMemcpyAsync(cp.data(), P.col_ptr + r0, cp.size() * 4, cudaMemcpyDeviceToHost, s));
      GPR_CUDA(cudaStreamSynchronize(s));
      for (int32_t r = r0; r < r1; ++r) {
        const int32_t e0 = cp[r - r0], e1 = cp[r - r0 + 1];
        if (e1 - e0 <= P.chunk_edges) {
          crow.push_back(r);
          cbeg.push_back(e0);
          cend.push_back(e1);
          cwhole.push_back(1);
        } else {
          srow.push_back(r);
          sbeg.push_back((int32_t)crow.size());
          for (int64_t e = e0; e < e1; e += P.chunk_edges) {
            crow.push_back(r);
            cbeg.push_back((int32_t)e);
            cend.push_back((int32_t)std::min<int64_t>(e1, e + P.chunk_edges));
            cwhole.push_back(0);
          }
          send.push_back((int32_t)crow.size());
        }
      }
    }
    P.nchunks = (int32_t)crow.size();
    P.nsplit = (int32_t)srow.size();
    auto up = [&](const std::vector<int32_t>& v) {
      int32_t* d = (int32_t*)dalloc(std::max<size_t>(v.size(), 1) * 4, s);
      if (!v.empty()) GPR_CUDA(cudaMemcpyAsync(d, v.data(), v.size() * 4, cudaMemcpyHostToDevice, s));
      return d;
    };
    P.chunk_row = up(crow);
    P.chunk_begin = up(cbeg);
    P.chunk_end = up(cend);
    P.chunk_whole = up(cwhole);
    P.split_row = up(srow);
    P.split_cbeg = up(sbeg);
    P.split_cend = up(send);
    GPR_CUDA(cudaStreamSynchronize(s));  // host vectors above must outlive the copies
    for (void* p : tmp) dfree(p, s);
  } catch (...) {
    for (void* p : tmp) dfree(p, s);
    throw;
  }
}

}  // namespace gpr
