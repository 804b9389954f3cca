// COO -> CSC graph build on the GPU.
//
// Computes the simple directed graph of section 3 (the TNGraph container: no
// multi-edges) with the sorted in-adjacency vectors of section 5
// ("Representation of Graphs and Networks": adjacency values are kept
// sorted), as one CSC:
//   pack     key = dst << b | src  (b = id bits); self-loops and invalid ids
//            become the sentinel ~0, which sorts last; the per-pass digit
//            histograms of the radix sort are counted in the same pass
//   sort     LSD radix sort, 8-bit digits, one read + one write of the keys
//            per pass (onesweep: Adinets and Merrill, 2022), tile prefixes by
//            decoupled look-back
//   dedupe   keep the first of each run of equal keys, drop sentinels;
//            compaction by decoupled look-back; writes row_idx, the CSC
//            offsets (row starts plus gap fill) and out-degrees in one pass
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <atomic>

#include "gpr_internal.cuh"

namespace gpr {

constexpr int kThreads = 256;
constexpr int kItems = 16;
constexpr int kTile = kThreads * kItems;  // 4096 keys per tile
constexpr int kWarps = kThreads / 32;
constexpr uint64_t kSentinel = ~0ull;
constexpr int kGapInline = 64;  // gaps of at most this many rows are filled by the finding thread

// ---------------------------------------------------------------- errors --
static thread_local std::string tl_error;
void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  tl_error = buf;
}
void clear_error() { tl_error.clear(); }
const char* last_error_cstr() { return tl_error.c_str(); }

// ------------------------------------------------------------ device info --
int device_ordinal() {
  int d = 0;
  cudaGetDevice(&d);
  return d;
}
int num_sms() {
  static int cached[64] = {0};
  int d = device_ordinal();
  if (d < 0 || d >= 64) d = 0;
  if (!cached[d]) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, d);
    cached[d] = v > 0 ? v : 1;
  }
  return cached[d];
}

static std::atomic<int64_t> g_launches{0};
void count_launches(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launches_so_far() { return g_launches.load(std::memory_order_relaxed); }

void* dalloc(size_t bytes, cudaStream_t s) {
  void* p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMallocAsync(&p, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw StatusFail{GPR_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed"};
  }
  return p;
}
void dfree(void* p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
}

// ------------------------------------------------------------ histograms --
__global__ void hist_kernel(const uint64_t* __restrict__ keys, int64_t n, int passes,
                            uint32_t* __restrict__ hist) {
  extern __shared__ uint32_t sh[];
  for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t k = keys[i];
    for (int p = 0; p < passes; ++p) atomicAdd(&sh[p * 256 + ((k >> (8 * p)) & 255)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * 256; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// Exclusive scan of each pass's 256 digit counts (block p = pass p).
__global__ void digit_starts_kernel(const uint32_t* __restrict__ hist, uint32_t* __restrict__ starts) {
  __shared__ uint32_t s[256];
  const int p = blockIdx.x, t = threadIdx.x;
  const uint32_t v = hist[p * 256 + t];
  s[t] = v;
  __syncthreads();
  for (int o = 1; o < 256; o <<= 1) {
    uint32_t a = t >= o ? s[t - o] : 0;
    __syncthreads();
    s[t] += a;
    __syncthreads();
  }
  starts[p * 256 + t] = s[t] - v;
}

// One stable counting pass on digit (key >> shift) & 255.  Keys of a tile are
// held warp-striped (item j of warp w is tile position w*512 + j*32 + lane),
// so (warp, item, lane) order is input order and the per-warp match-based
// ranking keeps the sort stable.
__global__ void __launch_bounds__(kThreads) onesweep_kernel(
    const uint64_t* __restrict__ in, uint64_t* __restrict__ out, int64_t n, int shift,
    const uint32_t* __restrict__ dstart, uint64_t* __restrict__ status, uint32_t* __restrict__ tile_ctr,
    uint32_t epoch, int* __restrict__ derr) {
  __shared__ uint64_t s_keys[kTile];
  __shared__ uint32_t s_wcnt[kWarps][256];
  __shared__ uint32_t s_tstart[256];
  __shared__ uint64_t s_gbase[256];
  __shared__ uint32_t s_wsum[kWarps];
  __shared__ uint32_t s_tile;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (t == 0) s_tile = atomicAdd(tile_ctr, 1u);
  for (int i = t; i < kWarps * 256; i += kThreads) (&s_wcnt[0][0])[i] = 0;
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t base = tile * kTile + (int64_t)w * (kItems * 32) + lane;

  uint64_t k[kItems];
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    int64_t i = base + j * 32;
    k[j] = i < n ? __ldcs(in + i) : kSentinel;
  }
  uint32_t rk[kItems];
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const uint32_t d = (uint32_t)(k[j] >> shift) & 255u;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t c = s_wcnt[w][d];
    rk[j] = c + __popc(peers & lt);
    __syncwarp();
    if ((peers & lt) == 0) s_wcnt[w][d] = c + __popc(peers);
    __syncwarp();
  }
  __syncthreads();

  // thread t owns digit t: per-warp exclusive offsets and the tile count
  uint32_t cnt = 0;
#pragma unroll
  for (int ww = 0; ww < kWarps; ++ww) {
    uint32_t v = s_wcnt[ww][t];
    s_wcnt[ww][t] = cnt;
    cnt += v;
  }
  if (tile == 0)
    st_relaxed_u64(status + t, lb_word(epoch, kFlagInc, cnt));
  else
    st_relaxed_u64(status + tile * 256 + t, lb_word(epoch, kFlagAgg, cnt));

  // tile-local exclusive scan over digits
  uint32_t v = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) s_wsum[w] = v;

  uint64_t excl = 0;
  if (tile != 0) {
    excl = lookback(status + t, tile, 256, epoch, derr);
    st_relaxed_u64(status + tile * 256 + t, lb_word(epoch, kFlagInc, excl + cnt));
  }
  s_gbase[t] = (uint64_t)dstart[t] + excl;
  __syncthreads();
  uint32_t woff = 0;
  for (int ww = 0; ww < w; ++ww) woff += s_wsum[ww];
  s_tstart[t] = woff + v - cnt;
  __syncthreads();

#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const uint32_t d = (uint32_t)(k[j] >> shift) & 255u;
    s_keys[s_tstart[d] + s_wcnt[w][d] + rk[j]] = k[j];
  }
  __syncthreads();
  for (int i = t; i < kTile; i += kThreads) {
    const uint64_t key = s_keys[i];
    const uint32_t d = (uint32_t)(key >> shift) & 255u;
    const uint64_t dst = s_gbase[d] + (uint64_t)(i - (int)s_tstart[d]);
    if (dst < (uint64_t)n) out[dst] = key;
  }
}

uint64_t* radix_sort_u64(uint64_t* keys, uint64_t* alt, int64_t n, int bits, cudaStream_t s,
                         int* derr, uint32_t* hist_in) {
  const int passes = (bits + 7) / 8;
  if (n <= 1 || passes == 0) return keys;
  const int64_t tiles = (n + kTile - 1) / kTile;
  uint32_t* hist = hist_in;
  uint32_t* own_hist = nullptr;
  uint32_t* starts = nullptr;
  uint64_t* status = nullptr;
  uint32_t* ctr = nullptr;
  try {
    if (!hist) {
      own_hist = (uint32_t*)dalloc(passes * 256 * sizeof(uint32_t), s);
      hist = own_hist;
      GPR_CUDA(cudaMemsetAsync(hist, 0, passes * 256 * sizeof(uint32_t), s));
      int grid = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)num_sms() * 8);
      hist_kernel<<<grid, kThreads, passes * 256 * sizeof(uint32_t), s>>>(keys, n, passes, hist);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
    }
    starts = (uint32_t*)dalloc(passes * 256 * sizeof(uint32_t), s);
    status = (uint64_t*)dalloc((size_t)tiles * 256 * sizeof(uint64_t), s);
    ctr = (uint32_t*)dalloc(passes * sizeof(uint32_t), s);
    GPR_CUDA(cudaMemsetAsync(status, 0, (size_t)tiles * 256 * sizeof(uint64_t), s));
    GPR_CUDA(cudaMemsetAsync(ctr, 0, passes * sizeof(uint32_t), s));
    digit_starts_kernel<<<passes, 256, 0, s>>>(hist, starts);
    GPR_CUDA(cudaGetLastError());
    count_launches(1);
    uint64_t* a = keys;
    uint64_t* b = alt;
    for (int p = 0; p < passes; ++p) {
      onesweep_kernel<<<(unsigned)tiles, kThreads, 0, s>>>(a, b, n, 8 * p, starts + 256 * p, status,
                                                          ctr + p, (uint32_t)(p + 1), derr);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
      std::swap(a, b);
    }
    dfree(own_hist, s);
    dfree(starts, s);
    dfree(status, s);
    dfree(ctr, s);
    return a;
  } catch (...) {
    dfree(own_hist, s);
    dfree(starts, s);
    dfree(status, s);
    dfree(ctr, s);
    throw;
  }
}

// -------------------------------------------------------------- packing --
// key = dst << b | src; a self-loop or an id outside [0, n) becomes the
// sentinel (the latter also raises DERR_BAD_ID).  Counts the digit
// histograms of all radix passes on the way.
__global__ void pack_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                            int64_t m, int32_t n, int b, int passes, uint64_t* __restrict__ keys,
                            uint32_t* __restrict__ hist, int* __restrict__ derr) {
  extern __shared__ uint32_t sh[];
  for (int i = threadIdx.x; i < passes * 256; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = __ldcs(src + i), v = __ldcs(dst + i);
    uint64_t key;
    if ((uint32_t)u >= (uint32_t)n || (uint32_t)v >= (uint32_t)n) {
      bad = true;
      key = kSentinel;
    } else if (u == v) {
      key = kSentinel;
    } else {
      key = ((uint64_t)(uint32_t)v << b) | (uint32_t)u;
    }
    keys[i] = key;
    for (int p = 0; p < passes; ++p) atomicAdd(&sh[p * 256 + ((key >> (8 * p)) & 255)], 1u);
  }
  if (bad) atomicOr(derr, DERR_BAD_ID);
  __syncthreads();
  for (int i = threadIdx.x; i < passes * 256; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// ------------------------------------------------------------- dedupe ----
struct Gap {
  int32_t first, last, value;
};

__device__ __forceinline__ void fill_rows(int32_t* col_ptr, int32_t first, int32_t last, int32_t value,
                                          Gap* gaps, uint32_t* ngaps) {
  if (first > last) return;
  if (last - first < kGapInline) {
    for (int32_t r = first; r <= last; ++r) col_ptr[r] = value;
  } else {
    uint32_t slot = atomicAdd(ngaps, 1u);
    gaps[slot] = Gap{first, last, value};
  }
}

// Neighbours of item j in input order, for warp-striped tiles.  All lanes
// take part in the shuffles; only lane 0 / lane 31 at a warp's first / last
// item read global memory.  kSentinel stands for "no neighbour".
__device__ __forceinline__ uint64_t prev_key(const uint64_t (&k)[kItems], int j, int lane, int64_t i,
                                             const uint64_t* __restrict__ keys, int64_t m_raw) {
  const uint64_t up = __shfl_up_sync(0xffffffffu, k[j], 1);
  const uint64_t row_last = __shfl_sync(0xffffffffu, k[j > 0 ? j - 1 : 0], 31);
  if (lane > 0) return up;
  if (j > 0) return row_last;
  return (i > 0 && i - 1 < m_raw) ? keys[i - 1] : kSentinel;
}
__device__ __forceinline__ uint64_t next_key(const uint64_t (&k)[kItems], int j, int lane, int64_t i,
                                             const uint64_t* __restrict__ keys, int64_t m_raw) {
  const uint64_t down = __shfl_down_sync(0xffffffffu, k[j], 1);
  const uint64_t row_first = __shfl_sync(0xffffffffu, k[j + 1 < kItems ? j + 1 : j], 0);
  if (lane < 31) return down;
  if (j + 1 < kItems) return row_first;
  return i + 1 < m_raw ? keys[i + 1] : kSentinel;
}

// Sorted keys -> CSC.  Item j of warp w is tile position w*512 + j*32 + lane
// (input order), so the ballot counts give each kept key its output index.
__global__ void __launch_bounds__(kThreads) dedupe_kernel(
    const uint64_t* __restrict__ keys, int64_t m_raw, int b, int32_t n, int32_t* __restrict__ row_idx,
    int32_t* __restrict__ edge_dst, int32_t* __restrict__ col_ptr, int32_t* __restrict__ outdeg,
    uint64_t* __restrict__ status, uint32_t* __restrict__ tile_ctr, int64_t* __restrict__ m_out,
    Gap* __restrict__ gaps, uint32_t* __restrict__ ngaps, int* __restrict__ derr) {
  __shared__ uint32_t s_wsum[kWarps];
  __shared__ uint64_t s_excl;
  __shared__ uint32_t s_tile;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (t == 0) s_tile = atomicAdd(tile_ctr, 1u);
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t base = tile * kTile + (int64_t)w * (kItems * 32) + lane;
  const uint64_t src_mask = (1ull << b) - 1;
  const uint32_t lt = lanemask_lt();

  uint64_t k[kItems];
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    int64_t i = base + j * 32;
    k[j] = i < m_raw ? __ldcs(keys + i) : kSentinel;
  }
  // keep flags in input order
  uint32_t ballot[kItems];
  uint32_t wtotal = 0;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int64_t i = base + j * 32;
    const uint64_t prev = prev_key(k, j, lane, i, keys, m_raw);
    const bool keep = (k[j] != kSentinel) && (i == 0 || k[j] != prev);
    ballot[j] = __ballot_sync(0xffffffffu, keep);
    wtotal += __popc(ballot[j]);
  }
  if (lane == 0) s_wsum[w] = wtotal;
  __syncthreads();
  if (t == 0) {
    uint32_t tot = 0;
    for (int ww = 0; ww < kWarps; ++ww) tot += s_wsum[ww];
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
  uint64_t o = s_excl;
  for (int ww = 0; ww < w; ++ww) o += s_wsum[ww];

#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const int64_t i = base + j * 32;
    const bool keep = (ballot[j] >> lane) & 1u;
    const uint64_t my_o = o + __popc(ballot[j] & lt);
    const uint64_t prev = prev_key(k, j, lane, i, keys, m_raw);
    const uint64_t next = next_key(k, j, lane, i, keys, m_raw);
    if (i < m_raw && k[j] != kSentinel) {
      const int32_t v = (int32_t)(k[j] >> b);
      if (keep) {
        const int32_t u = (int32_t)(k[j] & src_mask);
        row_idx[my_o] = u;
        edge_dst[my_o] = v;
        atomicAdd(&outdeg[u], 1);
        // rows (pv, v] start at my_o; the previous key is valid because
        // sentinels sort last
        const int32_t pv = (i > 0) ? (int32_t)(prev >> b) : -1;
        if (v != pv) fill_rows(col_ptr, pv + 1, v, (int32_t)my_o, gaps, ngaps);
      }
      if (next == kSentinel) {  // last valid key: rows (v, n] end at the total
        const int64_t total = (int64_t)my_o + (keep ? 1 : 0);
        *m_out = total;
        fill_rows(col_ptr, v + 1, n, (int32_t)total, gaps, ngaps);
      }
    }
    o += __popc(ballot[j]);
  }
}

__global__ void gap_fill_kernel(int32_t* __restrict__ col_ptr, const Gap* __restrict__ gaps,
                                const uint32_t* __restrict__ ngaps) {
  const uint32_t ng = *ngaps;
  for (uint32_t gi = blockIdx.x; gi < ng; gi += gridDim.x) {
    const Gap gp = gaps[gi];
    for (int64_t r = (int64_t)gp.first + threadIdx.x; r <= gp.last; r += blockDim.x) col_ptr[r] = gp.value;
  }
}

// ------------------------------------------------------------- driver ----
static int id_bits_for(int32_t n) {
  int b = 1;
  while (b < 31 && ((int64_t)1 << b) < (int64_t)n) ++b;
  return b;
}

struct BuildTemps {
  cudaStream_t s;
  std::vector<void*> ptrs;
  void* get(size_t bytes) {
    void* p = dalloc(bytes, s);
    ptrs.push_back(p);
    return p;
  }
  void release() {
    for (void* p : ptrs) dfree(p, s);
    ptrs.clear();
  }
};

void graph_free_device(gpr_graph* g, cudaStream_t s);
void plan_build_from(gpr_graph* g, const int32_t* edge_dst, cudaStream_t s, int* derr);

gpr_status build_graph(const int32_t* src_in, const int32_t* dst_in, int64_t m_raw, int32_t n, int flags,
                       cudaStream_t s, gpr_graph** out) {
  gpr_graph* g = new gpr_graph();
  g->n = n;
  g->m_raw = m_raw;
  g->id_bits = id_bits_for(n);
  g->device = device_ordinal();
  BuildTemps tmp{s, {}};
  try {
    int* derr = (int*)tmp.get(sizeof(int) * 2);
    int64_t* m_dev = (int64_t*)tmp.get(sizeof(int64_t));
    GPR_CUDA(cudaMemsetAsync(derr, 0, sizeof(int) * 2, s));
    GPR_CUDA(cudaMemsetAsync(m_dev, 0, sizeof(int64_t), s));

    const int32_t* src = src_in;
    const int32_t* dst = dst_in;
    if ((flags & GPR_PTR_HOST) && m_raw > 0) {
      int32_t* s_dev = (int32_t*)tmp.get((size_t)m_raw * 4);
      int32_t* d_dev = (int32_t*)tmp.get((size_t)m_raw * 4);
      GPR_CUDA(cudaMemcpyAsync(s_dev, src_in, (size_t)m_raw * 4, cudaMemcpyHostToDevice, s));
      GPR_CUDA(cudaMemcpyAsync(d_dev, dst_in, (size_t)m_raw * 4, cudaMemcpyHostToDevice, s));
      src = s_dev;
      dst = d_dev;
    }

    g->col_ptr = (int32_t*)dalloc(((size_t)n + 1) * 4, s);
    g->outdeg = (int32_t*)dalloc((size_t)n * 4, s);
    GPR_CUDA(cudaMemsetAsync(g->col_ptr, 0, ((size_t)n + 1) * 4, s));
    GPR_CUDA(cudaMemsetAsync(g->outdeg, 0, (size_t)n * 4, s));
    int32_t* row_idx_full = nullptr;
    int32_t* edge_dst = nullptr;
    if (m_raw > 0) {
      const int bits = 2 * g->id_bits;
      const int passes = (bits + 7) / 8;
      uint64_t* keys = (uint64_t*)tmp.get((size_t)m_raw * 8);
      uint64_t* alt = (uint64_t*)tmp.get((size_t)m_raw * 8);
      uint32_t* hist = (uint32_t*)tmp.get(passes * 256 * 4);
      GPR_CUDA(cudaMemsetAsync(hist, 0, passes * 256 * 4, s));
      const int grid = (int)std::min<int64_t>((m_raw + kThreads - 1) / kThreads, (int64_t)num_sms() * 8);
      pack_kernel<<<grid, kThreads, passes * 256 * 4, s>>>(src, dst, m_raw, n, g->id_bits, passes, keys, hist,
                                                           derr);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
      uint64_t* sorted = radix_sort_u64(keys, alt, m_raw, bits, s, derr, hist);

      const int64_t tiles = (m_raw + kTile - 1) / kTile;
      uint64_t* status = (uint64_t*)tmp.get((size_t)tiles * 8);
      uint32_t* ctr = (uint32_t*)tmp.get(8);
      const int64_t gap_cap = (int64_t)n / kGapInline + 4;
      Gap* gaps = (Gap*)tmp.get((size_t)gap_cap * sizeof(Gap));
      uint32_t* ngaps = (uint32_t*)tmp.get(8);
      GPR_CUDA(cudaMemsetAsync(status, 0, (size_t)tiles * 8, s));
      GPR_CUDA(cudaMemsetAsync(ctr, 0, 8, s));
      GPR_CUDA(cudaMemsetAsync(ngaps, 0, 8, s));
      row_idx_full = (int32_t*)tmp.get((size_t)m_raw * 4);
      edge_dst = (int32_t*)tmp.get((size_t)m_raw * 4);
      dedupe_kernel<<<(unsigned)tiles, kThreads, 0, s>>>(sorted, m_raw, g->id_bits, n, row_idx_full, edge_dst,
                                                         g->col_ptr, g->outdeg, status, ctr, m_dev, gaps, ngaps,
                                                         derr);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
      gap_fill_kernel<<<num_sms() * 2, kThreads, 0, s>>>(g->col_ptr, gaps, ngaps);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
    }
    int64_t m = 0;
    int herr = 0;
    GPR_CUDA(cudaMemcpyAsync(&m, m_dev, sizeof m, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaMemcpyAsync(&herr, derr, sizeof herr, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    if (herr & DERR_BAD_ID) throw StatusFail{GPR_EINVAL, "graph_build: an edge id is outside [0, n)"};
    if (herr & DERR_TIMEOUT) throw StatusFail{GPR_ETIMEOUT, "graph_build: a device-side wait timed out"};
    g->m = m;
    g->row_idx = (int32_t*)dalloc((size_t)std::max<int64_t>(m, 1) * 4, s);
    if (m > 0)
      GPR_CUDA(cudaMemcpyAsync(g->row_idx, row_idx_full, (size_t)m * 4, cudaMemcpyDeviceToDevice, s));
    plan_build_from(g, edge_dst, s, derr);
    GPR_CUDA(cudaMemcpyAsync(&herr, derr, sizeof herr, cudaMemcpyDeviceToHost, s));
    tmp.release();
    GPR_CUDA(cudaStreamSynchronize(s));
    if (herr & DERR_TIMEOUT) throw StatusFail{GPR_ETIMEOUT, "graph_build: a device-side wait timed out"};
    *out = g;
    return GPR_OK;
  } catch (const StatusFail& f) {
    tmp.release();
    graph_free_device(g, s);
    cudaStreamSynchronize(s);
    delete g;
    set_error("%s", f.msg.c_str());
    return f.st;
  } catch (const CudaFail& f) {
    cudaGetLastError();
    tmp.release();
    graph_free_device(g, s);
    cudaStreamSynchronize(s);
    delete g;
    set_error("graph_build: %s failed: %s", f.what, cudaGetErrorString(f.err));
    return GPR_ECUDA;
  }
}

}  // namespace gpr
