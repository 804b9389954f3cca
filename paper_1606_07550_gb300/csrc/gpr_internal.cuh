// Internal declarations of the gpr library (not part of the C-ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gpr.h"

namespace gpr {

// ---- errors ---------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

// Device-side error bits (an int in device memory, OR-ed by kernels).
enum : int {
  DERR_BAD_ID = 1,   // an edge endpoint outside [0, n)
  DERR_TIMEOUT = 2,  // a bounded spin-wait gave up
};

// Bounded spin: after this many polls a wait reports DERR_TIMEOUT and returns.
constexpr uint32_t kSpinLimit = 1u << 20;

struct CudaFail {
  cudaError_t err;
  const char* what;
};

#define GPR_CUDA(call)                                   \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) throw ::gpr::CudaFail{e_, #call}; \
  } while (0)

struct StatusFail {
  gpr_status st;
  std::string msg;
};

// ---- device memory: stream-ordered allocations ----------------------------
void* dalloc(size_t bytes, cudaStream_t s);  // throws StatusFail(GPR_ENOMEM)
void dfree(void* p, cudaStream_t s);

int num_sms();
int device_ordinal();

// With GPR_TRACE=1: synchronise s and print the wall time since the previous
// mark on this thread, labelled `what` (null: just set the mark).
void trace_phase(const char* what, cudaStream_t s);
// Exclusive prefix sums of v[0, m) into out; returns their total (read back to
// the host: synchronises s).
int64_t exclusive_scan_i32(const int32_t* v, int64_t m, int32_t* out, cudaStream_t s);

// Host-side count of kernels this library has launched (a CUDA graph launch
// counts its kernel nodes).
void count_launches(int64_t k);
int64_t launches_so_far();

// Entries of the contribution vector that one block can hold in shared
// memory (FP32), a multiple of 8.
int32_t hot_capacity();

// ---- sort scratch (build.cu) -----------------------------------------------
// Two buffers of `keys` 64-bit keys for a large sort.  One pair per device is
// kept for the process and lent to one call at a time (stream-ordered
// allocations of tens of GB cost milliseconds per call even when the pool
// holds the memory); a call that finds it lent allocates its own pair.  The
// destructor synchronises the stream before the pair is lent again, so the
// caller's work on it is complete.  Throws like dalloc.
class SortScratch {
 public:
  SortScratch(size_t keys, cudaStream_t s);
  ~SortScratch();
  SortScratch(const SortScratch&) = delete;
  SortScratch& operator=(const SortScratch&) = delete;
  uint64_t* a = nullptr;
  uint64_t* b = nullptr;

 private:
  cudaStream_t s_;
  struct Slot* slot_ = nullptr;
};

// ---- radix sort of 64-bit keys (onesweep-style, build.cu) -----------------
// The digits of a sort of `bits`-bit keys: 8 bits wide, or, where that saves
// a pass, the last ones 9 bits wide (then exactly `bits` bits are sorted).
constexpr int kMaxRadix = 512;
constexpr int kMaxPasses = 8;
struct DigitPlan {
  int passes;
  int shift[kMaxPasses];
  int width[kMaxPasses];
};
DigitPlan digit_plan(int bits);

// Sorts keys[0..n) ascending on the low `bits` bits (stable LSD, the digits of
// digit_plan(bits)), using `alt` (n entries) as the second buffer.  Returns
// the buffer holding the result (keys or alt).  hist: the caller already
// filled it (passes x kMaxRadix digit counts, device, digit_plan(bits)'s
// digits); if null it is computed.
uint64_t* radix_sort_u64(uint64_t* keys, uint64_t* alt, int64_t n, int bits, cudaStream_t s,
                         int* derr, uint32_t* hist = nullptr);

// ---- PageRank execution layout -------------------------------------------
// The CSC is stored in relabelled ids (descending out-degree).  Rows are run
// by in-degree bucket from ascending row lists; each bucket has a fixed
// number of lanes per row (1..32), or, for the last bucket, warp-sized edge
// chunks (plan.cu).
constexpr int kMaxBuckets = 6;

struct Bucket {
  int32_t row_begin, row_end;  // range in Plan::rows
  int lanes;                   // 1, 2, 4, 8, 16, 32 lanes per row; 0 = warp chunks
};

struct Plan {
  int32_t* new2old = nullptr;  // n: relabelled node p is the caller's node new2old[p]
  int32_t* old2new = nullptr;  // n
  float* inv_deg = nullptr;    // n, 1/outdeg (0 for dangling)
  int32_t* rows = nullptr;     // n: rows grouped by bucket, ascending within a bucket
  int nbuckets = 0;
  Bucket bucket[kMaxBuckets];
  int32_t deg_threshold[kMaxBuckets];  // upper in-degree bound of each bucket (last: INT_MAX)
  // Hot/cold split: sources below hot_H (the most-read contributions) are
  // gathered by a pass that keeps c[0, hot_H) in shared memory.  Rows are
  // sorted, so the hot sources of row p are the prefix [col_ptr[p], split[p]).
  int32_t hot_H = 0;
  int32_t* split = nullptr;  // n
  // edge chunks of the long-row bucket: (row, edge_begin, edge_end); chunks
  // [0, n_hot_chunks) cover hot prefixes, the rest cold suffixes.  Every long
  // row is finished from its chunk sums: hot chunks [hbeg, hend), cold chunks
  // [cbeg, cend).
  int32_t* chunk_row = nullptr;
  int32_t* chunk_begin = nullptr;
  int32_t* chunk_end = nullptr;
  int32_t nchunks = 0;
  int32_t n_hot_chunks = 0;
  int32_t* split_row = nullptr;  // the long rows
  int32_t* split_hbeg = nullptr;
  int32_t* split_hend = nullptr;
  int32_t* split_cbeg = nullptr;
  int32_t* split_cend = nullptr;
  int32_t nsplit = 0;
  int32_t chunk_edges = 0;
};

struct PagerankWork;  // pagerank.cu

}  // namespace gpr

struct gpr_graph {
  int32_t n = 0;
  int64_t m_raw = 0;
  int64_t m = 0;
  int id_bits = 0;
  int32_t n_dangling = 0;
  int32_t max_in = 0, max_out = 0;
  int device = 0;
  // the CSC in relabelled ids (plan.new2old / plan.old2new): in-adjacency of
  // row p is row_idx[col_ptr[p] .. col_ptr[p+1]), ascending
  int32_t* col_ptr = nullptr;  // n + 1
  int32_t* row_idx = nullptr;  // m
  int32_t* outdeg = nullptr;   // n
  gpr::Plan plan;
  int64_t device_bytes = 0;
  std::mutex mu;                    // guards `work`, `transposed` and the walk arrays
  gpr::PagerankWork* work = nullptr;  // lazily made by pagerank()
  // the out-adjacency as a CSC over the same relabelled ids (row u lists the
  // destinations of u, ascending), made by the first call that needs it
  gpr_graph* transposed = nullptr;
  // the out-adjacency for random walks, made by the first call that walks:
  // node u (caller id) lists its destinations in walk_ptr[u] ..
  // walk_ptr[u + 1), by ascending caller id; walk_adj holds each
  // destination's relabelled id and walk_nbr its (walk_ptr, out-degree)
  int32_t* walk_ptr = nullptr;  // n + 1
  int32_t* walk_adj = nullptr;  // m
  int2* walk_nbr = nullptr;     // m
};

namespace gpr {
void plan_build(gpr_graph* g, cudaStream_t s, int* derr);
// The transposed graph of g (throws StatusFail / CudaFail).
gpr_graph* build_transposed(const gpr_graph* g, cudaStream_t s);
// The caller-id out-adjacency of g into two new device arrays (throws).
void build_caller_out_adjacency(const gpr_graph* g, cudaStream_t s, int32_t** out_ptr, int32_t** out_adj);
void graph_free_device(gpr_graph* g, cudaStream_t s);
gpr_status export_graph(const gpr_graph* g, int32_t* col_ptr, int32_t* row_idx, int32_t* outdeg);
void plan_free(Plan& p, cudaStream_t s);
void pagerank_work_free(PagerankWork* w);

// ---- device helpers -----------------------------------------------------

// f(e, p) for every edge e of the CSC with its row p, through row marks in
// shared memory: a warp takes kMarkChunk consecutive edges (the warps of the
// grid take consecutive chunks, so the streams stay close together), marks
// the first edge of each row that starts among them (the largest row where
// empty rows share a start), and a running maximum gives each edge its row;
// edges are then visited lane-strided (coalesced).  s_rows: kMarkStride ints
// per warp.
constexpr int kMarkChunk = 1024;
constexpr int kMarkStride = kMarkChunk + kMarkChunk / 32;  // lane l's 32 positions start in bank l
__device__ __forceinline__ int mark_slot(int i) { return i + (i >> 5); }
template <typename F>
__device__ __forceinline__ void for_each_edge_with_row_marked(const int32_t* __restrict__ col_ptr, int32_t n,
                                                              int32_t* s_row, F f) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t m = col_ptr[n];
  for (int64_t cb = warp * kMarkChunk; cb < m; cb += nwarps * kMarkChunk) {
    const int len = (int)(m - cb < kMarkChunk ? m - cb : kMarkChunk);
    int32_t p0 = 0, hi = n;  // the row of edge cb: the last p with col_ptr[p] <= cb
    while (hi - p0 > 1) {
      const int32_t mid = p0 + (hi - p0) / 2;
      if (col_ptr[mid] <= cb)
        p0 = mid;
      else
        hi = mid;
    }
    for (int i = lane; i < kMarkChunk; i += 32) s_row[mark_slot(i)] = -1;
    __syncwarp();
    if (lane == 0) s_row[0] = p0;  // rows after p0 start after cb
    __syncwarp();
    for (int32_t r0 = p0 + 1; r0 < n; r0 += 32) {  // starts do not decrease: stop at the first batch past the chunk
      const int32_t r = r0 + lane;
      const int64_t st = r < n ? (int64_t)col_ptr[r] : m;
      const bool in = r < n && st < cb + len;
      if (in) atomicMax(&s_row[mark_slot((int)(st - cb))], r);
      if (!__shfl_sync(0xffffffffu, in, 31)) break;
    }
    __syncwarp();
    // running maximum: lane l owns positions 32l .. 32l + 31
    int32_t mx = -1;
#pragma unroll 8
    for (int i = 0; i < 32; ++i) mx = max(mx, s_row[mark_slot(32 * lane + i)]);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, mx, o);
      if (lane >= o) mx = max(mx, y);
    }
    int32_t run = __shfl_up_sync(0xffffffffu, mx, 1);
    if (lane == 0) run = -1;
#pragma unroll 8
    for (int i = 0; i < 32; ++i) {
      const int k = mark_slot(32 * lane + i);
      run = max(run, s_row[k]);
      s_row[k] = run;
    }
    __syncwarp();
    if (len == kMarkChunk) {
#pragma unroll 8
      for (int i = lane; i < kMarkChunk; i += 32) f(cb + i, s_row[mark_slot(i)]);
    } else {
      for (int i = lane; i < len; i += 32) f(cb + i, s_row[mark_slot(i)]);
    }
    __syncwarp();
  }
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Look-back status words: [63:60] epoch, [59:58] flag, [57:0] value.
constexpr uint64_t kFlagAgg = 1, kFlagInc = 2;
constexpr uint64_t kValMask = (1ull << 58) - 1;
__device__ __forceinline__ uint64_t lb_word(uint32_t epoch, uint64_t flag, uint64_t v) {
  return ((uint64_t)epoch << 60) | (flag << 58) | (v & kValMask);
}

// Decoupled look-back (Merrill and Garland, "Single-pass parallel prefix scan
// with decoupled look-back", 2016): the exclusive prefix of tile `tile` from
// the status words of tiles tile-1, tile-2, ... (stride `stride` words apart).
// The words of kLookBatch predecessors are read at once, so one round trip to
// L2 walks past up to kLookBatch aggregates.  Every wait is bounded; on
// timeout it sets DERR_TIMEOUT and returns what it has.
constexpr int kLookBatch = 4;
__device__ __forceinline__ uint64_t lookback(const uint64_t* status, int64_t tile, int64_t stride,
                                             uint32_t epoch, int* derr) {
  uint64_t excl = 0;
  int64_t k = tile - 1;
  uint32_t spins = 0;
  while (k >= 0) {
    uint64_t w[kLookBatch];
#pragma unroll
    for (int j = 0; j < kLookBatch; ++j) w[j] = k - j >= 0 ? ld_relaxed_u64(status + (k - j) * stride) : 0ull;
    // take the published words in order, up to the first inclusive one
    int took = 0;
    bool inc = false;
#pragma unroll
    for (int j = 0; j < kLookBatch; ++j) {
      const uint64_t fl = (w[j] >> 58) & 3;
      const bool ok = (uint32_t)(w[j] >> 60) == epoch && fl != 0;
      if (took == j && !inc && ok) {
        excl += w[j] & kValMask;
        took = j + 1;
        inc = fl == kFlagInc;
      }
    }
    if (inc) break;
    k -= took;
    if (took == 0) {
      if (++spins > kSpinLimit) {
        atomicOr(derr, DERR_TIMEOUT);
        return excl;
      }
      if (spins > 64) {
        __nanosleep(64);
        // once any waiter has given up, the rest of the grid stops waiting too
        if ((spins & 255) == 0 && (*(volatile int*)derr & DERR_TIMEOUT)) return excl;
      }
    }
  }
  return excl;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

}  // namespace gpr
