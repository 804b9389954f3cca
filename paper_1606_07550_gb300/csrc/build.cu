// COO -> CSC graph build on the GPU.
//
// Computes the simple directed graph of section 3 (the TNGraph container: no
// multi-edges) with the sorted in-adjacency vectors of section 5
// ("Representation of Graphs and Networks": adjacency values are kept
// sorted), as one CSC:
//   pack     key = dst << b | src  (b = id bits); self-loops and invalid ids
//            become the sentinel ~0, which sorts last; the per-pass digit
//            histograms of the radix sort are counted in the same pass
//   sort     LSD radix sort, 8-bit digits (the last ones 9 bits wide where
//            that saves a pass: 50-bit keys in 6 passes), one read + one write
//            of the keys per pass (onesweep: Adinets and Merrill, 2022), tile
//            prefixes by decoupled look-back
//   dedupe   keep the first of each run of equal keys, drop sentinels;
//            compaction by decoupled look-back; writes row_idx, the CSC
//            offsets (row starts plus gap fill) and out-degrees in one pass
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <mutex>

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

// ------------------------------------------------------------ phase trace --
// With GPR_TRACE=1 in the environment, trace_phase synchronises the stream and
// prints the host wall time since the previous mark of this thread to stderr
// (a timeline of a call's phases); otherwise it does nothing.
static bool trace_on() {
  static const bool on = [] {
    const char* e = getenv("GPR_TRACE");
    return e && atoi(e) != 0;
  }();
  return on;
}
void trace_phase(const char* what, cudaStream_t s) {
  if (!trace_on()) return;
  static thread_local std::chrono::steady_clock::time_point last;
  cudaStreamSynchronize(s);
  const auto now = std::chrono::steady_clock::now();
  if (what) fprintf(stderr, "[gpr trace] %-28s %9.3f ms\n", what, std::chrono::duration<double, std::milli>(now - last).count());
  last = now;
}

// The library allocates with the device's default stream-ordered pool.  The
// pool is told to keep freed memory mapped (a setting of this process only),
// so that repeated builds reuse it instead of mapping it again; set
// GPR_POOL_RELEASE=1 to return freed memory to the system at each sync.
static void keep_pool_memory() {
  static bool done[64] = {false};
  const int d = device_ordinal();
  if (d < 0 || d >= 64 || done[d]) return;
  done[d] = true;
  const char* env = getenv("GPR_POOL_RELEASE");
  if (env && atoi(env) != 0) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, d) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
}

void* dalloc(size_t bytes, cudaStream_t s) {
  void* p = nullptr;
  keep_pool_memory();
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

// ------------------------------------------------------------ sort scratch --
struct Slot {
  std::mutex mu;
  uint64_t* a = nullptr;
  uint64_t* b = nullptr;
  size_t cap = 0;  // keys per buffer
};
static Slot g_scratch[64];

SortScratch::SortScratch(size_t keys, cudaStream_t s) : s_(s) {
  int d = device_ordinal();
  if (d < 0 || d >= 64) d = 0;
  Slot& sl = g_scratch[d];
  if (!sl.mu.try_lock()) {  // lent: a pair of this call's own
    a = (uint64_t*)dalloc(keys * 8, s);
    try {
      b = (uint64_t*)dalloc(keys * 8, s);
    } catch (...) {
      dfree(a, s);
      throw;
    }
    return;
  }
  try {
    if (sl.cap < keys) {  // the last borrower synchronised its stream: the old pair is idle
      dfree(sl.a, s);
      dfree(sl.b, s);
      sl.a = sl.b = nullptr;
      sl.cap = 0;
      sl.a = (uint64_t*)dalloc(keys * 8, s);
      sl.b = (uint64_t*)dalloc(keys * 8, s);
      sl.cap = keys;
    }
  } catch (...) {
    sl.mu.unlock();
    throw;
  }
  slot_ = &sl;
  a = sl.a;
  b = sl.b;
}

SortScratch::~SortScratch() {
  if (slot_) {
    cudaStreamSynchronize(s_);
    slot_->mu.unlock();
  } else {
    dfree(a, s_);
    dfree(b, s_);
  }
}

// ------------------------------------------------------------ histograms --
// Digits of an LSD sort of `bits`-bit keys: 8-bit digits, or, where that takes
// a pass fewer, the last (bits - 8 * passes) digits 9 bits wide; with 9-bit
// digits the passes cover exactly `bits` bits, with 8-bit ones whole bytes.
DigitPlan digit_plan(int bits) {
  DigitPlan d{};
  bits = std::max(0, std::min(bits, 64));
  const int p8 = (bits + 7) / 8, p9 = (bits + 8) / 9;
  d.passes = p9 < p8 ? p9 : p8;
  const int nine = p9 < p8 ? bits - 8 * p9 : 0;  // the last `nine` passes are 9 bits wide
  int sh = 0;
  for (int p = 0; p < d.passes; ++p) {
    d.shift[p] = sh;
    d.width[p] = p >= d.passes - nine ? 9 : 8;
    sh += d.width[p];
  }
  return d;
}

__device__ __forceinline__ uint32_t digit_of(uint64_t k, const DigitPlan& dp, int p) {
  return (uint32_t)(k >> dp.shift[p]) & ((1u << dp.width[p]) - 1u);
}

// Digit counts of every pass: hist[p * kMaxRadix + digit].
__global__ void hist_kernel(const uint64_t* __restrict__ keys, int64_t n, DigitPlan dp,
                            uint32_t* __restrict__ hist) {
  extern __shared__ uint32_t sh[];
  for (int i = threadIdx.x; i < dp.passes * kMaxRadix; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t k = keys[i];
#pragma unroll
    for (int p = 0; p < kMaxPasses; ++p)
      if (p < dp.passes) atomicAdd(&sh[p * kMaxRadix + digit_of(k, dp, p)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < dp.passes * kMaxRadix; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// Exclusive scan of each pass's digit counts (block p = pass p, kMaxRadix
// threads).
__global__ void digit_starts_kernel(const uint32_t* __restrict__ hist, DigitPlan dp, uint32_t* __restrict__ starts) {
  __shared__ uint32_t s[kMaxRadix];
  const int p = blockIdx.x, t = threadIdx.x;
  const uint32_t v = t < (1 << dp.width[p]) ? hist[p * kMaxRadix + t] : 0u;
  s[t] = v;
  __syncthreads();
  for (int o = 1; o < kMaxRadix; o <<= 1) {
    uint32_t a = t >= o ? s[t - o] : 0;
    __syncthreads();
    s[t] += a;
    __syncthreads();
  }
  starts[p * kMaxRadix + t] = s[t] - v;
}

// One stable counting pass on the kBits-bit digit (key >> shift); the shift
// is kShift, or the argument where kShift is -1.  Keys of a tile are held
// warp-striped (item j of warp w is tile position w*512 + j*32 + lane), so
// (warp, item, lane) order is input order and the per-warp match-based
// ranking keeps the sort stable.  Thread t owns digits kDPT*t .. kDPT*t +
// kDPT - 1 for the tile's scans and look-backs.
template <int kBits, int kShift>
__global__ void __launch_bounds__(kThreads, 4) onesweep_kernel(
    const uint64_t* __restrict__ in, uint64_t* __restrict__ out, int64_t n, int shift_arg,
    const uint32_t* __restrict__ dstart, uint64_t* __restrict__ status, uint32_t* __restrict__ tile_ctr,
    uint32_t epoch, int* __restrict__ derr) {
  const int shift = kShift >= 0 ? kShift : shift_arg;
  constexpr int kRadix = 1 << kBits;
  constexpr uint32_t kMask = kRadix - 1;
  constexpr int kDPT = kRadix / kThreads;
  static_assert(kDPT >= 1 && kDPT * kThreads == kRadix, "whole digits per thread");
  __shared__ uint64_t s_keys[kTile];
  __shared__ uint32_t s_wcnt[kWarps][kRadix];
  __shared__ uint64_t s_goff[kRadix];
  __shared__ uint32_t s_wsum[kWarps];
  __shared__ uint32_t s_tile;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  if (t == 0) s_tile = atomicAdd(tile_ctr, 1u);
  for (int i = t; i < kWarps * kRadix; i += kThreads) (&s_wcnt[0][0])[i] = 0;
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t base = tile * kTile + (int64_t)w * (kItems * 32) + lane;

  uint64_t k[kItems];
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    int64_t i = base + j * 32;
    k[j] = i < n ? __ldcs(in + i) : kSentinel;
  }
  uint32_t rk[kItems / 2] = {};  // ranks in the warp (< 512), two 16-bit halves per word
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const uint32_t d = (uint32_t)(k[j] >> shift) & kMask;
    // the lanes holding the same digit: one vote per digit bit
    uint32_t peers = 0xffffffffu;
#pragma unroll
    for (int bb = 0; bb < kBits; ++bb) {
      const uint32_t bit = (d >> bb) & 1u;
      const uint32_t vote = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? vote : ~vote;
    }
    const uint32_t c = s_wcnt[w][d];
    rk[j >> 1] |= (c + __popc(peers & lt)) << (16 * (j & 1));
    __syncwarp();
    if ((peers & lt) == 0) s_wcnt[w][d] = c + __popc(peers);
    __syncwarp();
  }
  __syncthreads();

  // per owned digit: per-warp exclusive offsets and the tile count
  uint32_t cnt[kDPT];
  uint32_t tsum = 0;
#pragma unroll
  for (int q = 0; q < kDPT; ++q) {
    const int d = kDPT * t + q;
    uint32_t c = 0;
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) {
      const uint32_t v = s_wcnt[ww][d];
      s_wcnt[ww][d] = c;
      c += v;
    }
    cnt[q] = c;
    tsum += c;
    if (tile == 0)
      st_relaxed_u64(status + d, lb_word(epoch, kFlagInc, c));
    else
      st_relaxed_u64(status + tile * kRadix + d, lb_word(epoch, kFlagAgg, c));
  }

  // tile-local exclusive scan over digits (thread order is digit order)
  uint32_t v = tsum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += y;
  }
  if (lane == 31) s_wsum[w] = v;
  __syncthreads();
  uint32_t woff = 0;
  for (int ww = 0; ww < w; ++ww) woff += s_wsum[ww];
  uint32_t tstart[kDPT];
  tstart[0] = woff + v - tsum;
#pragma unroll
  for (int q = 1; q < kDPT; ++q) tstart[q] = tstart[q - 1] + cnt[q - 1];
  // s_wcnt[w][d]: where warp w's first key of digit d goes in the tile
#pragma unroll
  for (int q = 0; q < kDPT; ++q)
#pragma unroll
    for (int ww = 0; ww < kWarps; ++ww) s_wcnt[ww][kDPT * t + q] += tstart[q];
  __syncthreads();

  // the tile in digit order in shared memory, before the look-back, so that
  // no key is held in registers while the predecessors are waited for
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const uint32_t d = (uint32_t)(k[j] >> shift) & kMask;
    s_keys[s_wcnt[w][d] + ((rk[j >> 1] >> (16 * (j & 1))) & 0xFFFFu)] = k[j];
  }

#pragma unroll
  for (int q = 0; q < kDPT; ++q) {
    const int d = kDPT * t + q;
    uint64_t excl = 0;
    if (tile != 0) {
      excl = lookback(status + d, tile, kRadix, epoch, derr);
      st_relaxed_u64(status + tile * kRadix + d, lb_word(epoch, kFlagInc, excl + cnt[q]));
    }
    // output index of tile position i with digit d: s_goff[d] + i (the digit's
    // global start is at least its tile-local start, so no wrap)
    s_goff[d] = (uint64_t)dstart[d] + excl - tstart[q];
  }
  __syncthreads();
  if ((tile + 1) * kTile <= n) {  // a full tile: every index is below n
#pragma unroll 4
    for (int i = t; i < kTile; i += kThreads) {
      const uint64_t key = s_keys[i];
      out[s_goff[(uint32_t)(key >> shift) & kMask] + (uint64_t)i] = key;
    }
  } else {
    for (int i = t; i < kTile; i += kThreads) {
      const uint64_t key = s_keys[i];
      const uint64_t dst = s_goff[(uint32_t)(key >> shift) & kMask] + (uint64_t)i;
      if (dst < (uint64_t)n) out[dst] = key;
    }
  }
}

using SweepKernel = void (*)(const uint64_t*, uint64_t*, int64_t, int, const uint32_t*, uint64_t*, uint32_t*,
                            uint32_t, int*);
// 8-bit passes at whole bytes (shift fixed at compile time), 9-bit passes
static const SweepKernel kSweep8[8] = {onesweep_kernel<8, 0>,  onesweep_kernel<8, 8>,  onesweep_kernel<8, 16>,
                                       onesweep_kernel<8, 24>, onesweep_kernel<8, 32>, onesweep_kernel<8, 40>,
                                       onesweep_kernel<8, 48>, onesweep_kernel<8, 56>};
static const SweepKernel kSweep9 = onesweep_kernel<9, -1>;

uint64_t* radix_sort_u64(uint64_t* keys, uint64_t* alt, int64_t n, int bits, cudaStream_t s,
                         int* derr, uint32_t* hist_in) {
  const DigitPlan dp = digit_plan(bits);
  const int passes = dp.passes;
  if (n <= 1 || passes == 0) return keys;
  const int64_t tiles = (n + kTile - 1) / kTile;
  int radix = 0;
  for (int p = 0; p < passes; ++p) radix = std::max(radix, 1 << dp.width[p]);
  uint32_t* hist = hist_in;
  uint32_t* own_hist = nullptr;
  uint32_t* starts = nullptr;
  uint64_t* status = nullptr;
  uint32_t* ctr = nullptr;
  try {
    if (!hist) {
      own_hist = (uint32_t*)dalloc(passes * kMaxRadix * sizeof(uint32_t), s);
      hist = own_hist;
      GPR_CUDA(cudaMemsetAsync(hist, 0, passes * kMaxRadix * sizeof(uint32_t), s));
      int grid = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, (int64_t)num_sms() * 8);
      hist_kernel<<<grid, kThreads, passes * kMaxRadix * sizeof(uint32_t), s>>>(keys, n, dp, hist);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
    }
    starts = (uint32_t*)dalloc(passes * kMaxRadix * sizeof(uint32_t), s);
    status = (uint64_t*)dalloc((size_t)tiles * radix * sizeof(uint64_t), s);
    ctr = (uint32_t*)dalloc(passes * sizeof(uint32_t), s);
    GPR_CUDA(cudaMemsetAsync(status, 0, (size_t)tiles * radix * sizeof(uint64_t), s));
    GPR_CUDA(cudaMemsetAsync(ctr, 0, passes * sizeof(uint32_t), s));
    digit_starts_kernel<<<passes, kMaxRadix, 0, s>>>(hist, dp, starts);
    GPR_CUDA(cudaGetLastError());
    count_launches(1);
    static std::once_flag carveout;  // four blocks per SM need the largest shared-memory carve-out
    std::call_once(carveout, [] {
      for (SweepKernel f : kSweep8)
        cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
      cudaFuncSetAttribute(kSweep9, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared);
    });
    uint64_t* a = keys;
    uint64_t* b = alt;
    for (int p = 0; p < passes; ++p) {
      // 8-bit digits start at whole bytes until the first 9-bit one
      const SweepKernel f = dp.width[p] == 9 ? kSweep9 : kSweep8[dp.shift[p] / 8];
      f<<<(unsigned)tiles, kThreads, 0, s>>>(a, b, n, dp.shift[p], starts + kMaxRadix * p, status, ctr + p,
                                             (uint32_t)(p + 1), derr);
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

// ------------------------------------------------- relabelling (pi) --
// L2 eviction priority "last" for the node-sized arrays that random accesses
// hit (the counters, the relabelling map), so that the streamed edge arrays
// do not push them out.
__device__ __forceinline__ uint64_t l2_keep_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ int32_t ld_keep(const int32_t* a, uint64_t pol) {
  int32_t v;
  asm volatile("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ void red_add_keep(int32_t* a, int32_t v, uint64_t pol) {
  asm volatile("red.relaxed.gpu.global.add.L2::cache_hint.s32 [%0], %1, %2;" ::"l"(a), "r"(v), "l"(pol) : "memory");
}

// Raw out-degree counts (duplicates included) of the COO stream, and the
// id check: an id outside [0, n) raises DERR_BAD_ID.
__global__ void degree_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                              int32_t n, int32_t* __restrict__ odeg, int* __restrict__ derr) {
  bool bad = false;
  const uint64_t keep = l2_keep_policy();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t u = __ldcs(src + i), v = __ldcs(dst + i);
    if ((uint32_t)u >= (uint32_t)n || (uint32_t)v >= (uint32_t)n) {
      bad = true;
    } else if (u != v) {
      red_add_keep(odeg + u, 1, keep);
    }
  }
  if (bad) atomicOr(derr, DERR_BAD_ID);
}

// out[old2new[v]] = a[v]
__global__ void permute_kernel(const int32_t* __restrict__ a, const int32_t* __restrict__ old2new, int32_t n,
                               int32_t* __restrict__ out) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    out[old2new[v]] = a[v];
}

__global__ void max_kernel(const int32_t* __restrict__ a, int32_t n, int32_t* __restrict__ out) {
  int32_t mx = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    mx = max(mx, a[i]);
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, mx);
}

// Node order key: descending raw out-degree, then ascending id.
__global__ void node_order_keys_kernel(const int32_t* __restrict__ odeg, int32_t n, int b, int32_t maxdeg,
                                       uint64_t* __restrict__ keys) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    keys[v] = ((uint64_t)(uint32_t)(maxdeg - odeg[v]) << b) | (uint64_t)v;
}

__global__ void perm_from_sorted_kernel(const uint64_t* __restrict__ sorted, int32_t n, uint64_t id_mask,
                                        int32_t* __restrict__ new2old, int32_t* __restrict__ old2new) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = (int32_t)(sorted[p] & id_mask);
    new2old[p] = v;
    old2new[v] = (int32_t)p;
  }
}

// -------------------------------------------------------------- packing --
// key = map(dst) << b | map(src) (map = identity if null); a self-loop or an
// id outside [0, n) becomes the sentinel, which sorts last.  Counts the digit
// histograms of all radix passes on the way (hist[p * kMaxRadix + digit];
// none when dp.passes is 0).
__global__ void pack_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                            int32_t n, int b, const int32_t* __restrict__ map, DigitPlan dp,
                            uint64_t* __restrict__ keys, uint32_t* __restrict__ hist) {
  extern __shared__ uint32_t sh[];
  for (int i = threadIdx.x; i < dp.passes * kMaxRadix; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const uint64_t keep = l2_keep_policy();
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = __ldcs(src + i), v = __ldcs(dst + i);
    uint64_t key;
    if ((uint32_t)u >= (uint32_t)n || (uint32_t)v >= (uint32_t)n || u == v) {
      key = kSentinel;
    } else {
      if (map) {
        u = ld_keep(map + u, keep);
        v = ld_keep(map + v, keep);
      }
      key = ((uint64_t)(uint32_t)v << b) | (uint32_t)u;
    }
    __stcs(keys + i, key);
#pragma unroll
    for (int p = 0; p < kMaxPasses; ++p)
      if (p < dp.passes) atomicAdd(&sh[p * kMaxRadix + digit_of(key, dp, p)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < dp.passes * kMaxRadix; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// Keys of the edges of a CSC under a node map: key = map(row) << b | map(src).
__global__ void csc_keys_kernel(const int32_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                                int32_t n, int64_t m, int b, const int32_t* __restrict__ map,
                                uint64_t* __restrict__ keys) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t lo = 0, hi = n;  // row p: col_ptr[p] <= e < col_ptr[p + 1]
    while (hi - lo > 1) {
      const int32_t mid = lo + (hi - lo) / 2;
      if ((int64_t)col_ptr[mid] <= e)
        lo = mid;
      else
        hi = mid;
    }
    keys[e] = ((uint64_t)(uint32_t)map[lo] << b) | (uint32_t)map[row_idx[e]];
  }
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
// Keeps the first of each run of equal keys and drops sentinels; writes
// row_idx, the row starts (gaps of empty rows filled) and out-degrees.
__global__ void __launch_bounds__(kThreads) dedupe_kernel(
    const uint64_t* __restrict__ keys, int64_t m_raw, int b, int32_t n, int32_t* __restrict__ row_idx,
    int32_t* __restrict__ col_ptr, int32_t* __restrict__ outdeg, uint64_t* __restrict__ status,
    uint32_t* __restrict__ tile_ctr, int64_t* __restrict__ m_out, Gap* __restrict__ gaps,
    uint32_t* __restrict__ ngaps, int* __restrict__ derr, int withhold_tile0, int degree_from_raw) {
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
      // withhold_tile0: fault-injection hook for tests; the first tile never
      // publishes, so every later tile's bounded wait runs out
      if (!withhold_tile0) st_relaxed_u64(status, lb_word(1, kFlagInc, tot));
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
      const int32_t u = (int32_t)(k[j] & src_mask);
      if (!keep && degree_from_raw) atomicSub(&outdeg[u], 1);  // a duplicate: counted in the raw degree
      if (keep) {
        row_idx[my_o] = u;
        if (!degree_from_raw) atomicAdd(&outdeg[u], 1);
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
static int bits_for(uint32_t v) {
  int b = 0;
  while (b < 32 && (v >> b) != 0) ++b;
  return b;
}

struct Temps {
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

static int grid_for(int64_t items, int per_sm = 8) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((items + kThreads - 1) / kThreads, (int64_t)num_sms() * per_sm));
}

// The blocks of a kThreads-thread kernel that fit on the device at once (for
// kernels that deal their work out statically over the whole grid).
template <typename K>
static int resident_grid(K kernel) {
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, kThreads, 0);
  return num_sms() * std::max(b, 1);
}

// Sorted unique-or-not keys (length m_keys) -> CSC arrays; returns m.
// degree_from_raw: outdeg already holds each source's count of non-loop keys
// (duplicates included), and the de-duplication subtracts the duplicates;
// otherwise outdeg is counted from the kept keys.
static int64_t keys_to_csc(uint64_t* keys, uint64_t* alt, int64_t m_keys, int b, int32_t n, uint32_t* hist,
                           int32_t* col_ptr, int32_t* row_idx, int32_t* outdeg, int* derr, Temps& tmp,
                           cudaStream_t s, bool presorted = false, bool degree_from_raw = false) {
  GPR_CUDA(cudaMemsetAsync(col_ptr, 0, ((size_t)n + 1) * 4, s));
  if (!degree_from_raw) GPR_CUDA(cudaMemsetAsync(outdeg, 0, (size_t)n * 4, s));
  if (m_keys == 0) return 0;
  uint64_t* sorted = presorted ? keys : radix_sort_u64(keys, alt, m_keys, 2 * b, s, derr, hist);
  trace_phase("build: sort", s);
  const int64_t tiles = (m_keys + kTile - 1) / kTile;
  uint64_t* status = (uint64_t*)tmp.get((size_t)tiles * 8);
  uint32_t* ctr = (uint32_t*)tmp.get(8);
  const int64_t gap_cap = (int64_t)n / kGapInline + 4;
  Gap* gaps = (Gap*)tmp.get((size_t)gap_cap * sizeof(Gap));
  uint32_t* ngaps = (uint32_t*)tmp.get(8);
  int64_t* m_dev = (int64_t*)tmp.get(8);
  GPR_CUDA(cudaMemsetAsync(status, 0, (size_t)tiles * 8, s));
  GPR_CUDA(cudaMemsetAsync(ctr, 0, 8, s));
  GPR_CUDA(cudaMemsetAsync(ngaps, 0, 8, s));
  GPR_CUDA(cudaMemsetAsync(m_dev, 0, 8, s));
  const char* inj = getenv("GPR_INJECT_LOOKBACK_STALL");
  const int withhold = (inj && atoi(inj) != 0 && tiles > 1) ? 1 : 0;
  dedupe_kernel<<<(unsigned)tiles, kThreads, 0, s>>>(sorted, m_keys, b, n, row_idx, col_ptr, outdeg, status, ctr,
                                                     m_dev, gaps, ngaps, derr, withhold, degree_from_raw ? 1 : 0);
  GPR_CUDA(cudaGetLastError());
  count_launches(1);
  gap_fill_kernel<<<num_sms() * 2, kThreads, 0, s>>>(col_ptr, gaps, ngaps);
  GPR_CUDA(cudaGetLastError());
  count_launches(1);
  int64_t m = 0;
  GPR_CUDA(cudaMemcpyAsync(&m, m_dev, sizeof m, cudaMemcpyDeviceToHost, s));
  GPR_CUDA(cudaStreamSynchronize(s));
  return m;
}

// Keys (src << b | dst) of every edge of a CSC, in CSC order.
__global__ void __launch_bounds__(kThreads) transpose_keys_kernel(const int32_t* __restrict__ col_ptr,
                                                                  const int32_t* __restrict__ row_idx, int32_t n,
                                                                  int b, uint64_t* __restrict__ keys) {
  __shared__ int32_t s_rows[kWarps][kMarkStride];
  for_each_edge_with_row_marked(col_ptr, n, s_rows[threadIdx.x >> 5], [&](int64_t e, int32_t p) {
    keys[e] = ((uint64_t)(uint32_t)row_idx[e] << b) | (uint64_t)p;
  });
}

void graph_free_device(gpr_graph* g, cudaStream_t s);
void plan_build(gpr_graph* g, cudaStream_t s, int* derr);

// The copy stream and events of a chunked host-to-device COO copy, one set
// per device, made on first use and kept for the process.  Builds that take
// host input on one device are serialised by its mutex.  GPR_COPY_CHUNKS
// (1..8) sets the number of chunks.
constexpr int kCopyChunks = 8;
static int copy_chunks() {
  static const int c = [] {
    const char* e = getenv("GPR_COPY_CHUNKS");
    const int v = e ? atoi(e) : kCopyChunks;
    return v < 1 ? 1 : (v > kCopyChunks ? kCopyChunks : v);
  }();
  return c;
}
struct CopyLane {
  cudaStream_t stream = nullptr;
  cudaEvent_t start = nullptr;
  cudaEvent_t done[kCopyChunks] = {};
  std::mutex mu;
};
static CopyLane& copy_lane() {
  static CopyLane lanes[64];
  static std::once_flag made[64];
  int d = device_ordinal();
  if (d < 0 || d >= 64) d = 0;
  CopyLane& l = lanes[d];
  std::call_once(made[d], [&l] {
    cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking);
    cudaEventCreateWithFlags(&l.start, cudaEventDisableTiming);
    for (int c = 0; c < kCopyChunks; ++c) cudaEventCreateWithFlags(&l.done[c], cudaEventDisableTiming);
  });
  if (!l.stream || !l.start) throw CudaFail{cudaErrorUnknown, "creating the copy stream of a host COO"};
  return l;
}

gpr_status build_graph(const int32_t* src_in, const int32_t* dst_in, int64_t m_raw, int32_t n, int flags,
                       cudaStream_t s, gpr_graph** out) {
  gpr_graph* g = new gpr_graph();
  g->n = n;
  g->m_raw = m_raw;
  g->id_bits = id_bits_for(n);
  g->device = device_ordinal();
  Temps tmp{s, {}};
  const int b = g->id_bits;
  try {
    trace_phase(nullptr, s);
    int* derr = (int*)tmp.get(sizeof(int) * 2);
    GPR_CUDA(cudaMemsetAsync(derr, 0, sizeof(int) * 2, s));
    const int32_t* src = src_in;
    const int32_t* dst = dst_in;
    // 1. relabelling pi: nodes by descending raw out-degree (ties: ascending id)
    int32_t* odeg = (int32_t*)tmp.get((size_t)n * 4);
    int32_t* maxd = (int32_t*)tmp.get(8);
    GPR_CUDA(cudaMemsetAsync(odeg, 0, (size_t)n * 4, s));
    GPR_CUDA(cudaMemsetAsync(maxd, 0, 8, s));
    if ((flags & GPR_PTR_HOST) && m_raw > 0) {
      // a host COO goes up in chunks on a copy stream; each chunk's raw
      // out-degrees are counted on `s` while the next chunk is in flight
      int32_t* s_dev = (int32_t*)tmp.get((size_t)m_raw * 4);
      int32_t* d_dev = (int32_t*)tmp.get((size_t)m_raw * 4);
      CopyLane& cp = copy_lane();
      std::lock_guard<std::mutex> lk(cp.mu);
      GPR_CUDA(cudaEventRecord(cp.start, s));  // the copy stream waits for the allocations and memsets
      GPR_CUDA(cudaStreamWaitEvent(cp.stream, cp.start, 0));
      const int nch = copy_chunks();
      const int64_t chunk = (m_raw + nch - 1) / nch;
      for (int c = 0; c < nch; ++c) {
        const int64_t off = c * chunk, len = std::min<int64_t>(chunk, m_raw - off);
        if (len <= 0) break;
        GPR_CUDA(cudaMemcpyAsync(s_dev + off, src_in + off, (size_t)len * 4, cudaMemcpyHostToDevice, cp.stream));
        GPR_CUDA(cudaMemcpyAsync(d_dev + off, dst_in + off, (size_t)len * 4, cudaMemcpyHostToDevice, cp.stream));
        GPR_CUDA(cudaEventRecord(cp.done[c], cp.stream));
        GPR_CUDA(cudaStreamWaitEvent(s, cp.done[c], 0));
        degree_kernel<<<grid_for(len), kThreads, 0, s>>>(s_dev + off, d_dev + off, len, n, odeg, derr);
        GPR_CUDA(cudaGetLastError());
        count_launches(1);
      }
      src = s_dev;
      dst = d_dev;
      trace_phase("build: copy of the COO + raw out-degrees", s);
    } else if (m_raw > 0) {
      degree_kernel<<<grid_for(m_raw), kThreads, 0, s>>>(src, dst, m_raw, n, odeg, derr);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
    }
    max_kernel<<<grid_for(n), kThreads, 0, s>>>(odeg, n, maxd);
    GPR_CUDA(cudaGetLastError());
    count_launches(1);
    int32_t hmax = 0;
    int herr = 0;
    GPR_CUDA(cudaMemcpyAsync(&hmax, maxd, 4, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaMemcpyAsync(&herr, derr, 4, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    if (herr & DERR_BAD_ID) throw StatusFail{GPR_EINVAL, "graph_build: an edge id is outside [0, n)"};
    trace_phase("build: raw out-degrees", s);
    {
      uint64_t* nk = (uint64_t*)tmp.get((size_t)n * 8);
      uint64_t* na = (uint64_t*)tmp.get((size_t)n * 8);
      node_order_keys_kernel<<<grid_for(n), kThreads, 0, s>>>(odeg, n, b, hmax, nk);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
      uint64_t* ns = radix_sort_u64(nk, na, n, b + bits_for((uint32_t)hmax), s, derr, nullptr);
      g->plan.new2old = (int32_t*)dalloc((size_t)n * 4, s);
      g->plan.old2new = (int32_t*)dalloc((size_t)n * 4, s);
      perm_from_sorted_kernel<<<grid_for(n), kThreads, 0, s>>>(ns, n, (1ull << b) - 1, g->plan.new2old,
                                                               g->plan.old2new);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
    }
    trace_phase("build: relabelling", s);
    // 2. keys (pi(dst), pi(src)), sort, de-duplicate: the CSC in relabelled ids
    g->col_ptr = (int32_t*)dalloc(((size_t)n + 1) * 4, s);
    g->outdeg = (int32_t*)dalloc((size_t)n * 4, s);
    int64_t m = 0;
    int32_t* row_idx_full = nullptr;
    if (m_raw > 0) {
      const DigitPlan dp = digit_plan(2 * b);  // the plan radix_sort_u64 follows for these keys
      SortScratch sc((size_t)m_raw, s);
      uint64_t* keys = sc.a;
      uint64_t* alt = sc.b;
      uint32_t* hist = (uint32_t*)tmp.get(dp.passes * kMaxRadix * 4);
      GPR_CUDA(cudaMemsetAsync(hist, 0, dp.passes * kMaxRadix * 4, s));
      pack_kernel<<<grid_for(m_raw), kThreads, dp.passes * kMaxRadix * 4, s>>>(src, dst, m_raw, n, b,
                                                                              g->plan.old2new, dp, keys, hist);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
      // the row ids go straight into the graph (capacity m_raw: the kept edges
      // are not known yet); a build that drops many duplicates copies them
      // into an array of their own size below
      g->row_idx = (int32_t*)dalloc((size_t)m_raw * 4, s);
      row_idx_full = g->row_idx;
      permute_kernel<<<grid_for(n), kThreads, 0, s>>>(odeg, g->plan.old2new, n, g->outdeg);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
      trace_phase("build: pack", s);
      m = keys_to_csc(keys, alt, m_raw, b, n, hist, g->col_ptr, row_idx_full, g->outdeg, derr, tmp, s,
                      /*presorted=*/false, /*degree_from_raw=*/true);
      GPR_CUDA(cudaMemcpyAsync(&herr, derr, 4, cudaMemcpyDeviceToHost, s));
      GPR_CUDA(cudaStreamSynchronize(s));
      if (herr & DERR_TIMEOUT) throw StatusFail{GPR_ETIMEOUT, "graph_build: a device-side wait timed out"};
    } else {
      GPR_CUDA(cudaMemsetAsync(g->col_ptr, 0, ((size_t)n + 1) * 4, s));
      GPR_CUDA(cudaMemsetAsync(g->outdeg, 0, (size_t)n * 4, s));
    }
    g->m = m;
    if (!row_idx_full || m < m_raw - m_raw / 8) {
      int32_t* exact = (int32_t*)dalloc((size_t)std::max<int64_t>(m, 1) * 4, s);
      if (m > 0) GPR_CUDA(cudaMemcpyAsync(exact, row_idx_full, (size_t)m * 4, cudaMemcpyDeviceToDevice, s));
      dfree(row_idx_full, s);
      g->row_idx = exact;
    }
    tmp.release();
    trace_phase("build: dedupe", s);
    // 3. execution layout (degree buckets, chunks, inverse degrees)
    int* derr2 = (int*)dalloc(8, s);
    GPR_CUDA(cudaMemsetAsync(derr2, 0, 8, s));
    try {
      plan_build(g, s, derr2);
    } catch (...) {
      dfree(derr2, s);
      throw;
    }
    GPR_CUDA(cudaMemcpyAsync(&herr, derr2, 4, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    dfree(derr2, s);
    if (herr & DERR_TIMEOUT) throw StatusFail{GPR_ETIMEOUT, "graph_build: a device-side wait timed out"};
    trace_phase("build: plan", s);
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

// The out-adjacency of g as a CSC over the same relabelled ids: the keys
// (src, dst) of g's edges sorted and laid out like a build's, with its own
// execution plan.  Its `outdeg` counts in-degrees of g.
gpr_graph* build_transposed(const gpr_graph* g, cudaStream_t s) {
  gpr_graph* t = new gpr_graph();
  t->n = g->n;
  t->m_raw = g->m;
  t->id_bits = g->id_bits;
  t->device = g->device;
  Temps tmp{s, {}};
  const int32_t n = g->n;
  const int b = g->id_bits;
  try {
    int* derr = (int*)tmp.get(sizeof(int) * 2);
    GPR_CUDA(cudaMemsetAsync(derr, 0, sizeof(int) * 2, s));
    t->col_ptr = (int32_t*)dalloc(((size_t)n + 1) * 4, s);
    t->outdeg = (int32_t*)dalloc((size_t)n * 4, s);
    t->row_idx = (int32_t*)dalloc((size_t)std::max<int64_t>(g->m, 1) * 4, s);
    int64_t m = 0;
    if (g->m > 0) {
      uint64_t* keys = (uint64_t*)tmp.get((size_t)g->m * 8);
      uint64_t* alt = (uint64_t*)tmp.get((size_t)g->m * 8);
      transpose_keys_kernel<<<resident_grid(transpose_keys_kernel), kThreads, 0, s>>>(g->col_ptr, g->row_idx, n,
                                                                                     b, keys);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
      m = keys_to_csc(keys, alt, g->m, b, n, nullptr, t->col_ptr, t->row_idx, t->outdeg, derr, tmp, s);
    } else {
      GPR_CUDA(cudaMemsetAsync(t->col_ptr, 0, ((size_t)n + 1) * 4, s));
      GPR_CUDA(cudaMemsetAsync(t->outdeg, 0, (size_t)n * 4, s));
    }
    t->m = m;
    plan_build(t, s, derr);
    int herr = 0;
    GPR_CUDA(cudaMemcpyAsync(&herr, derr, 4, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    tmp.release();
    if (herr & DERR_TIMEOUT) throw StatusFail{GPR_ETIMEOUT, "transposed graph: a device-side wait timed out"};
    if (m != g->m) throw StatusFail{GPR_ECUDA, "transposed graph: edge count differs from the graph's"};
    return t;
  } catch (...) {
    tmp.release();
    graph_free_device(t, s);
    cudaStreamSynchronize(s);
    delete t;
    throw;
  }
}

// Keys (caller src << b | caller dst) of every edge.
__global__ void __launch_bounds__(kThreads) caller_keys_kernel(const int32_t* __restrict__ col_ptr,
                                                               const int32_t* __restrict__ row_idx,
                                                               const int32_t* __restrict__ new2old, int32_t n, int b,
                                                               uint64_t* __restrict__ keys) {
  __shared__ int32_t s_rows[kWarps][kMarkStride];
  for_each_edge_with_row_marked(col_ptr, n, s_rows[threadIdx.x >> 5], [&](int64_t e, int32_t p) {
    keys[e] = ((uint64_t)(uint32_t)new2old[row_idx[e]] << b) | (uint64_t)(uint32_t)new2old[p];
  });
}

// The out-adjacency in the caller's ids: out_ptr[u] .. out_ptr[u + 1] indexes
// out_adj, the destinations of u in ascending order.
void build_caller_out_adjacency(const gpr_graph* g, cudaStream_t s, int32_t** out_ptr, int32_t** out_adj) {
  Temps tmp{s, {}};
  const int32_t n = g->n;
  const int b = g->id_bits;
  int32_t* ptr = nullptr;
  int32_t* adj = nullptr;
  try {
    int* derr = (int*)tmp.get(sizeof(int) * 2);
    GPR_CUDA(cudaMemsetAsync(derr, 0, sizeof(int) * 2, s));
    ptr = (int32_t*)dalloc(((size_t)n + 1) * 4, s);
    adj = (int32_t*)dalloc((size_t)std::max<int64_t>(g->m, 1) * 4, s);
    int32_t* indeg = (int32_t*)tmp.get((size_t)n * 4);
    int64_t m = 0;
    if (g->m > 0) {
      uint64_t* keys = (uint64_t*)tmp.get((size_t)g->m * 8);
      uint64_t* alt = (uint64_t*)tmp.get((size_t)g->m * 8);
      caller_keys_kernel<<<resident_grid(caller_keys_kernel), kThreads, 0, s>>>(g->col_ptr, g->row_idx,
                                                                               g->plan.new2old, n, b, keys);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
      m = keys_to_csc(keys, alt, g->m, b, n, nullptr, ptr, adj, indeg, derr, tmp, s);
    } else {
      GPR_CUDA(cudaMemsetAsync(ptr, 0, ((size_t)n + 1) * 4, s));
    }
    int herr = 0;
    GPR_CUDA(cudaMemcpyAsync(&herr, derr, 4, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    tmp.release();
    if (herr & DERR_TIMEOUT) throw StatusFail{GPR_ETIMEOUT, "out-adjacency: a device-side wait timed out"};
    if (m != g->m) throw StatusFail{GPR_ECUDA, "out-adjacency: edge count differs from the graph's"};
    *out_ptr = ptr;
    *out_adj = adj;
  } catch (...) {
    tmp.release();
    dfree(ptr, s);
    dfree(adj, s);
    throw;
  }
}

// ---- in-place edge updates ---------------------------------------------------
// E' = (E \ D) u I for a batch of deletions D and insertions I (caller ids;
// self-loops in I are dropped, deleting a missing edge does nothing).  The
// graph's keys (row << b | source, relabelled ids) are already sorted: the
// kept ones are compacted by a prefix scan and the sorted insert keys are
// placed among them by rank (an insert goes before an equal kept key, so the
// de-duplication keeps one copy), and the merged keys go through the build's
// de-duplication and offset pass without a sort.  The node numbering stays.

__global__ void check_ids_kernel(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                                 int32_t n, int* __restrict__ derr) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    bad |= (uint32_t)src[i] >= (uint32_t)n || (uint32_t)dst[i] >= (uint32_t)n;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(derr, DERR_BAD_ID);
}

// key = row << b | source for every edge of a CSC, in CSC (= key) order.
__global__ void __launch_bounds__(kThreads) own_keys_kernel(const int32_t* __restrict__ col_ptr,
                                                            const int32_t* __restrict__ row_idx, int32_t n, int b,
                                                            uint64_t* __restrict__ keys) {
  __shared__ int32_t s_rows[kWarps][kMarkStride];
  for_each_edge_with_row_marked(col_ptr, n, s_rows[threadIdx.x >> 5], [&](int64_t e, int32_t p) {
    keys[e] = ((uint64_t)p << b) | (uint64_t)(uint32_t)row_idx[e];
  });
}

__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t* a, int64_t n, uint64_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (a[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}
__device__ __forceinline__ int64_t upper_bound_u64(const uint64_t* a, int64_t n, uint64_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (a[mid] <= key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// keep[i] = 1 unless keys[i] is among the sorted deletion keys
__global__ void keep_kernel(const uint64_t* __restrict__ keys, int64_t m, const uint64_t* __restrict__ del,
                            int64_t nd, int32_t* __restrict__ keep) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = lower_bound_u64(del, nd, keys[i]);
    keep[i] = (j < nd && del[j] == keys[i]) ? 0 : 1;
  }
}

// Exclusive scan of int32 flags in tiles of kScanTile: tile sums, one block
// scanning the tile sums, then each tile's own scan.
constexpr int kScanTile = 4096;
__global__ void tile_sums_kernel(const int32_t* __restrict__ v, int64_t m, int64_t* __restrict__ sums) {
  __shared__ int64_t s[kThreads / 32];
  const int64_t t0 = blockIdx.x * (int64_t)kScanTile;
  int64_t a = 0;
  for (int64_t i = t0 + threadIdx.x; i < min(m, t0 + kScanTile); i += blockDim.x) a += v[i];
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s[w];
    sums[blockIdx.x] = t;
  }
}
__global__ void scan_sums_kernel(int64_t* __restrict__ sums, int64_t nt, int64_t* __restrict__ total) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t run = 0;
  for (int64_t i = 0; i < nt; ++i) {
    const int64_t v = sums[i];
    sums[i] = run;
    run += v;
  }
  *total = run;
}
__global__ void tile_scan_kernel(const int32_t* __restrict__ v, int64_t m, const int64_t* __restrict__ offs,
                                 int32_t* __restrict__ out) {
  __shared__ int32_t s_w[kThreads / 32];
  const int64_t t0 = blockIdx.x * (int64_t)kScanTile;
  constexpr int kPer = kScanTile / kThreads;  // consecutive items per thread
  const int64_t i0 = t0 + (int64_t)threadIdx.x * kPer;
  int32_t loc[kPer];
  int32_t sum = 0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    loc[j] = i0 + j < m ? v[i0 + j] : 0;
    sum += loc[j];
  }
  int32_t inc = sum;  // inclusive scan of the per-thread sums across the block
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_w[w] = inc;
  __syncthreads();
  int32_t wo = 0;
  for (int ww = 0; ww < w; ++ww) wo += s_w[ww];
  int64_t run = offs[blockIdx.x] + wo + inc - sum;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    if (i0 + j < m) out[i0 + j] = (int32_t)run;
    run += loc[j];
  }
}

// Exclusive prefix sums of v[0, m) into out (the total must fit in int32 for
// out's entries) and their total, read back to the host (synchronises s).
int64_t exclusive_scan_i32(const int32_t* v, int64_t m, int32_t* out, cudaStream_t s) {
  if (m <= 0) return 0;
  const int64_t nt = (m + kScanTile - 1) / kScanTile;
  int64_t* sums = (int64_t*)dalloc((size_t)(nt + 1) * sizeof(int64_t), s);
  int64_t total = 0;
  try {
    tile_sums_kernel<<<(unsigned)nt, kThreads, 0, s>>>(v, m, sums);
    scan_sums_kernel<<<1, 32, 0, s>>>(sums, nt, sums + nt);
    tile_scan_kernel<<<(unsigned)nt, kThreads, 0, s>>>(v, m, sums, out);
    GPR_CUDA(cudaGetLastError());
    count_launches(3);
    GPR_CUDA(cudaMemcpyAsync(&total, sums + nt, sizeof total, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
  } catch (...) {
    dfree(sums, s);
    throw;
  }
  dfree(sums, s);
  return total;
}

// merged[kpos[i] + #(inserts <= key)] = key for every kept old key
__global__ void place_kept_kernel(const uint64_t* __restrict__ keys, int64_t m, const int32_t* __restrict__ keep,
                                  const int32_t* __restrict__ kpos, const uint64_t* __restrict__ ins, int64_t ni,
                                  uint64_t* __restrict__ merged) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    if (keep[i]) merged[(int64_t)kpos[i] + upper_bound_u64(ins, ni, keys[i])] = keys[i];
}

// merged[j + #(kept old keys < ins[j])] = ins[j]
__global__ void place_ins_kernel(const uint64_t* __restrict__ ins, int64_t ni, const uint64_t* __restrict__ keys,
                                 int64_t m, const int32_t* __restrict__ kpos, const int32_t* __restrict__ keep,
                                 uint64_t* __restrict__ merged) {
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ni; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lb = lower_bound_u64(keys, m, ins[j]);
    const int64_t before = lb < m ? (int64_t)kpos[lb] : (m > 0 ? (int64_t)kpos[m - 1] + keep[m - 1] : 0);
    merged[j + before] = ins[j];
  }
}

// Index of the first sentinel in sorted keys (the count of real keys).
__global__ void count_real_kernel(const uint64_t* __restrict__ keys, int64_t n, int64_t* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = lower_bound_u64(keys, n, kSentinel);
}

// Sorted keys of a batch of caller-id pairs (self-loops sort last as
// sentinels); returns the number of real keys.  Ids already checked.
static int64_t batch_keys(const gpr_graph* g, const int32_t* src, const int32_t* dst, int64_t k, Temps& tmp,
                          int* derr, uint64_t** out, cudaStream_t s) {
  *out = nullptr;
  if (k <= 0) return 0;
  uint64_t* keys = (uint64_t*)tmp.get((size_t)k * 8);
  uint64_t* alt = (uint64_t*)tmp.get((size_t)k * 8);
  pack_kernel<<<grid_for(k), kThreads, 0, s>>>(src, dst, k, g->n, g->id_bits, g->plan.old2new, DigitPlan{}, keys,
                                                nullptr);
  GPR_CUDA(cudaGetLastError());
  count_launches(1);
  uint64_t* sorted = radix_sort_u64(keys, alt, k, 64, s, derr, nullptr);  // sentinels need every bit
  int64_t* cnt = (int64_t*)tmp.get(8);
  count_real_kernel<<<1, 32, 0, s>>>(sorted, k, cnt);
  count_launches(1);
  int64_t real = 0;
  GPR_CUDA(cudaMemcpyAsync(&real, cnt, 8, cudaMemcpyDeviceToHost, s));
  GPR_CUDA(cudaStreamSynchronize(s));
  *out = sorted;
  return real;
}

gpr_status update_graph(gpr_graph* g, const int32_t* ins_src, const int32_t* ins_dst, int64_t n_ins,
                        const int32_t* del_src, const int32_t* del_dst, int64_t n_del, int flags, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g->mu);
  Temps tmp{s, {}};
  const int32_t n = g->n;
  const int b = g->id_bits;
  int32_t* new_col_ptr = nullptr;
  int32_t* new_row_idx = nullptr;
  int32_t* new_outdeg = nullptr;
  try {
    int* derr = (int*)tmp.get(sizeof(int) * 2);
    GPR_CUDA(cudaMemsetAsync(derr, 0, sizeof(int) * 2, s));
    // the batches on the device, ids checked before anything changes
    auto to_dev = [&](const int32_t* p, int64_t k) -> const int32_t* {
      if (!(flags & GPR_PTR_HOST) || k <= 0) return p;
      int32_t* d = (int32_t*)tmp.get((size_t)k * 4);
      GPR_CUDA(cudaMemcpyAsync(d, p, (size_t)k * 4, cudaMemcpyHostToDevice, s));
      return d;
    };
    const int32_t* is = to_dev(ins_src, n_ins);
    const int32_t* id = to_dev(ins_dst, n_ins);
    const int32_t* ds = to_dev(del_src, n_del);
    const int32_t* dd = to_dev(del_dst, n_del);
    if (n_ins > 0) check_ids_kernel<<<grid_for(n_ins), kThreads, 0, s>>>(is, id, n_ins, n, derr);
    if (n_del > 0) check_ids_kernel<<<grid_for(n_del), kThreads, 0, s>>>(ds, dd, n_del, n, derr);
    GPR_CUDA(cudaGetLastError());
    int herr = 0;
    GPR_CUDA(cudaMemcpyAsync(&herr, derr, 4, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    if (herr & DERR_BAD_ID) throw StatusFail{GPR_EINVAL, "graph_update: an edge id is outside [0, n)"};
    uint64_t* ins = nullptr;
    uint64_t* del = nullptr;
    const int64_t ni = batch_keys(g, is, id, n_ins, tmp, derr, &ins, s);
    const int64_t nd = batch_keys(g, ds, dd, n_del, tmp, derr, &del, s);
    const int64_t m = g->m;
    // kept old keys and their compacted positions
    uint64_t* keys = (uint64_t*)tmp.get((size_t)std::max<int64_t>(m, 1) * 8);
    int32_t* keep = (int32_t*)tmp.get((size_t)std::max<int64_t>(m, 1) * 4);
    int32_t* kpos = (int32_t*)tmp.get((size_t)std::max<int64_t>(m, 1) * 4);
    int64_t kept = 0;
    if (m > 0) {
      own_keys_kernel<<<resident_grid(own_keys_kernel), kThreads, 0, s>>>(g->col_ptr, g->row_idx, n, b, keys);
      keep_kernel<<<grid_for(m), kThreads, 0, s>>>(keys, m, del, nd, keep);
      const int64_t nt = (m + kScanTile - 1) / kScanTile;
      int64_t* sums = (int64_t*)tmp.get((size_t)nt * 8 + 8);
      tile_sums_kernel<<<(unsigned)nt, kThreads, 0, s>>>(keep, m, sums);
      scan_sums_kernel<<<1, 32, 0, s>>>(sums, nt, sums + nt);
      tile_scan_kernel<<<(unsigned)nt, kThreads, 0, s>>>(keep, m, sums, kpos);
      GPR_CUDA(cudaGetLastError());
      count_launches(5);
      GPR_CUDA(cudaMemcpyAsync(&kept, sums + nt, 8, cudaMemcpyDeviceToHost, s));
      GPR_CUDA(cudaStreamSynchronize(s));
    }
    const int64_t total = kept + ni;
    if (total >= ((int64_t)1 << 31)) throw StatusFail{GPR_EINVAL, "graph_update: more than 2^31 - 1 edges"};
    uint64_t* merged = (uint64_t*)tmp.get((size_t)std::max<int64_t>(total, 1) * 8);
    if (m > 0) {
      place_kept_kernel<<<grid_for(m), kThreads, 0, s>>>(keys, m, keep, kpos, ins, ni, merged);
      count_launches(1);
    }
    if (ni > 0) {
      place_ins_kernel<<<grid_for(ni), kThreads, 0, s>>>(ins, ni, keys, m, kpos, keep, merged);
      count_launches(1);
    }
    GPR_CUDA(cudaGetLastError());
    new_col_ptr = (int32_t*)dalloc(((size_t)n + 1) * 4, s);
    new_outdeg = (int32_t*)dalloc((size_t)n * 4, s);
    int32_t* row_full = (int32_t*)tmp.get((size_t)std::max<int64_t>(total, 1) * 4);
    const int64_t m2 = keys_to_csc(merged, nullptr, total, b, n, nullptr, new_col_ptr, row_full, new_outdeg, derr, tmp,
                                   s, /*presorted=*/true);
    GPR_CUDA(cudaMemcpyAsync(&herr, derr, 4, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    if (herr & DERR_TIMEOUT) throw StatusFail{GPR_ETIMEOUT, "graph_update: a device-side wait timed out"};
    new_row_idx = (int32_t*)dalloc((size_t)std::max<int64_t>(m2, 1) * 4, s);
    if (m2 > 0) GPR_CUDA(cudaMemcpyAsync(new_row_idx, row_full, (size_t)m2 * 4, cudaMemcpyDeviceToDevice, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    tmp.release();
    // swap in the new CSC; everything derived from the old one goes
    GPR_CUDA(cudaDeviceSynchronize());  // work queued on other streams may still read the graph
    if (g->work) {
      pagerank_work_free(g->work);
      g->work = nullptr;
    }
    if (g->transposed) {
      graph_free_device(g->transposed, s);
      delete g->transposed;
      g->transposed = nullptr;
    }
    dfree(g->walk_ptr, s);
    dfree(g->walk_adj, s);
    dfree(g->walk_nbr, s);
    g->walk_ptr = g->walk_adj = nullptr;
    g->walk_nbr = nullptr;
    int32_t* n2o = g->plan.new2old;
    int32_t* o2n = g->plan.old2new;
    g->plan.new2old = g->plan.old2new = nullptr;
    plan_free(g->plan, s);
    g->plan.new2old = n2o;
    g->plan.old2new = o2n;
    dfree(g->col_ptr, s);
    dfree(g->row_idx, s);
    dfree(g->outdeg, s);
    g->col_ptr = new_col_ptr;
    g->row_idx = new_row_idx;
    g->outdeg = new_outdeg;
    new_col_ptr = new_row_idx = new_outdeg = nullptr;
    g->m = m2;
    g->m_raw = m2;
    int* derr2 = (int*)dalloc(8, s);
    GPR_CUDA(cudaMemsetAsync(derr2, 0, 8, s));
    try {
      plan_build(g, s, derr2);
    } catch (...) {
      dfree(derr2, s);
      throw;
    }
    GPR_CUDA(cudaMemcpyAsync(&herr, derr2, 4, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    dfree(derr2, s);
    if (herr & DERR_TIMEOUT) throw StatusFail{GPR_ETIMEOUT, "graph_update: a device-side wait timed out"};
    return GPR_OK;
  } catch (const StatusFail& f) {
    tmp.release();
    dfree(new_col_ptr, s);
    dfree(new_row_idx, s);
    dfree(new_outdeg, s);
    set_error("%s", f.msg.c_str());
    return f.st;
  } catch (const CudaFail& f) {
    cudaGetLastError();
    tmp.release();
    dfree(new_col_ptr, s);
    dfree(new_row_idx, s);
    dfree(new_outdeg, s);
    set_error("graph_update: %s failed: %s", f.what, cudaGetErrorString(f.err));
    return GPR_ECUDA;
  }
}

// The CSC in the caller's ids: the relabelled edges mapped back through
// new2old, sorted, and laid out by keys_to_csc (no duplicates remain).
gpr_status export_graph(const gpr_graph* g, int32_t* col_ptr_h, int32_t* row_idx_h, int32_t* outdeg_h) {
  cudaStream_t s = nullptr;
  Temps tmp{s, {}};
  try {
    const int32_t n = g->n;
    const int64_t m = g->m;
    const int b = g->id_bits;
    int* derr = (int*)tmp.get(8);
    GPR_CUDA(cudaMemsetAsync(derr, 0, 8, s));
    int32_t* cp = (int32_t*)tmp.get(((size_t)n + 1) * 4);
    int32_t* ri = (int32_t*)tmp.get((size_t)std::max<int64_t>(m, 1) * 4);
    int32_t* od = (int32_t*)tmp.get((size_t)n * 4);
    if (m > 0) {
      uint64_t* keys = (uint64_t*)tmp.get((size_t)m * 8);
      uint64_t* alt = (uint64_t*)tmp.get((size_t)m * 8);
      csc_keys_kernel<<<grid_for(m), kThreads, 0, s>>>(g->col_ptr, g->row_idx, n, m, b, g->plan.new2old, keys);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
      const int64_t m2 = keys_to_csc(keys, alt, m, b, n, nullptr, cp, ri, od, derr, tmp, s);
      if (m2 != m) throw StatusFail{GPR_ECUDA, "graph_export: edge count changed under relabelling"};
    } else {
      GPR_CUDA(cudaMemsetAsync(cp, 0, ((size_t)n + 1) * 4, s));
      GPR_CUDA(cudaMemsetAsync(od, 0, (size_t)n * 4, s));
    }
    if (col_ptr_h) GPR_CUDA(cudaMemcpy(col_ptr_h, cp, ((size_t)n + 1) * 4, cudaMemcpyDeviceToHost));
    if (row_idx_h && m > 0) GPR_CUDA(cudaMemcpy(row_idx_h, ri, (size_t)m * 4, cudaMemcpyDeviceToHost));
    if (outdeg_h) GPR_CUDA(cudaMemcpy(outdeg_h, od, (size_t)n * 4, cudaMemcpyDeviceToHost));
    int herr = 0;
    GPR_CUDA(cudaMemcpy(&herr, derr, 4, cudaMemcpyDeviceToHost));
    tmp.release();
    GPR_CUDA(cudaStreamSynchronize(s));
    if (herr & DERR_TIMEOUT) throw StatusFail{GPR_ETIMEOUT, "graph_export: a device-side wait timed out"};
    return GPR_OK;
  } catch (const StatusFail& f) {
    tmp.release();
    cudaStreamSynchronize(s);
    set_error("%s", f.msg.c_str());
    return f.st;
  } catch (const CudaFail& f) {
    cudaGetLastError();
    tmp.release();
    cudaStreamSynchronize(s);
    set_error("graph_export: %s failed: %s", f.what, cudaGetErrorString(f.err));
    return GPR_ECUDA;
  }
}

}  // namespace gpr
