// PageRank power iteration on the relabelled CSC (section 4 Table
// "snap_methods"; section 6 Tables "exp_algs" and "exp_parallel" time it as a
// fixed number of iterations).
//
// Per step, for every row v of the relabelled graph:
//   y[v]  = sum over in-neighbours u of c[u],   c = x * inv_outdeg   (pull)
//   x'[v] = coefB + coefA * y[v]
//   c'[v] = x'[v] * inv_outdeg[v]
// with coefA = d / S and coefB = (1 - d)/N + d D / (N S), where S = sum(x)
// and D = the dangling mass of x, both FP64.  This is the step
//   x'[v] = (1 - d)/N + d (sum_{u->v} x[u]/outdeg(u) + D/N)
// applied to x / S (mass normalisation).  Every kernel also leaves per-block
// partials of S', D' and ||x' - x||_1 (FP32 per thread and per warp, FP64
// across warps); the last block of the step's final kernel folds all of them
// in a fixed order, so repeated runs are bitwise identical, and writes the
// next step's coefficients.
//
// Rows run by in-degree bucket from ascending row lists: 1, 4, 8 or 32 lanes
// per row, and rows above the last lane bucket as warp-sized edge chunks
// (128-bit index loads, 16 gathers in flight per lane).  A row longer than
// one chunk is finished from its chunk sums, in chunk order, by the finish
// kernel.  The bucket kernels of a step are independent and run as parallel
// branches of one CUDA graph that holds the whole iteration loop.
#include <algorithm>
#include <map>
#include <tuple>
#include <vector>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "blocked.cuh"
#include "pr_step.cuh"

namespace gpr {

// Warp-cooperative sum of c over edges [e0, e1): 128-bit index loads on the
// 16-byte-aligned body, up to 16 gathers in flight per lane.  Every lane
// returns its own partial; the caller reduces.
template <typename T>
__device__ __forceinline__ float warp_gather(const int32_t* __restrict__ row_idx, const T* __restrict__ c_in,
                                             int32_t e0, int32_t e1, int lane) {
  float y = 0.f;
  const int32_t h = min(e1, (e0 + 3) & ~3);
  if (e0 + lane < h) y += ld_rank(c_in, __ldcs(row_idx + e0 + lane));
  const int32_t body_end = h + ((e1 - h) & ~3);
  int32_t e = h + 4 * lane;
  for (; e + 3 * 128 < body_end; e += 4 * 128) {
    const int4 q0 = __ldcs(reinterpret_cast<const int4*>(row_idx + e));
    const int4 q1 = __ldcs(reinterpret_cast<const int4*>(row_idx + e + 128));
    const int4 q2 = __ldcs(reinterpret_cast<const int4*>(row_idx + e + 256));
    const int4 q3 = __ldcs(reinterpret_cast<const int4*>(row_idx + e + 384));
    const float a0 = ld_rank(c_in, q0.x), a1 = ld_rank(c_in, q0.y), a2 = ld_rank(c_in, q0.z), a3 = ld_rank(c_in, q0.w);
    const float b0 = ld_rank(c_in, q1.x), b1 = ld_rank(c_in, q1.y), b2 = ld_rank(c_in, q1.z), b3 = ld_rank(c_in, q1.w);
    const float c0 = ld_rank(c_in, q2.x), c1 = ld_rank(c_in, q2.y), c2 = ld_rank(c_in, q2.z), c3 = ld_rank(c_in, q2.w);
    const float d0 = ld_rank(c_in, q3.x), d1 = ld_rank(c_in, q3.y), d2 = ld_rank(c_in, q3.z), d3 = ld_rank(c_in, q3.w);
    y += ((a0 + a1) + (a2 + a3)) + ((b0 + b1) + (b2 + b3)) + ((c0 + c1) + (c2 + c3)) + ((d0 + d1) + (d2 + d3));
  }
  for (; e < body_end; e += 128) {
    const int4 q = __ldcs(reinterpret_cast<const int4*>(row_idx + e));
    const float a0 = ld_rank(c_in, q.x), a1 = ld_rank(c_in, q.y), a2 = ld_rank(c_in, q.z), a3 = ld_rank(c_in, q.w);
    y += (a0 + a1) + (a2 + a3);
  }
  if (body_end + lane < e1) y += ld_rank(c_in, __ldcs(row_idx + body_end + lane));
  return y;
}

// G lanes per row (G in {1, 2, 4, 8, 16, 32}) over rows[i0, i1).
// Cold pass: the part of each row from split[r] on (from col_ptr[r] when
// split is null), plus the hot-pass sum y_hot[r] (when not null).
template <int G, typename T>
__global__ void __launch_bounds__(256) rows_kernel(const int32_t* __restrict__ col_ptr,
                                                   const int32_t* __restrict__ row_idx, const int32_t* __restrict__ rows,
                                                   int32_t i0, int32_t i1, const int32_t* __restrict__ split,
                                                   const float* __restrict__ y_hot, const T* __restrict__ c_in,
                                                   const float* __restrict__ x_in, const float* __restrict__ inv_deg,
                                                   float* __restrict__ x_out, T* __restrict__ c_out,
                                                   const StepParams* __restrict__ prm, double* __restrict__ partials) {
  const float A = prm->coefA, B = prm->coefB;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (G - 1);
  constexpr int kRowsPerWarp = 32 / G;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float mass = 0.f, dang = 0.f, res = 0.f;
  for (int64_t wi = i0 + warp * kRowsPerWarp; wi < i1; wi += nwarps * kRowsPerWarp) {
    const int64_t i = wi + lane / G;
    const bool active = i < i1;
    int32_t r = 0, e0 = 0, e1 = 0;
    if (active) {
      r = rows[i];
      e0 = split ? split[r] : col_ptr[r];
      e1 = col_ptr[r + 1];
    }
    float y;
    if constexpr (G == 32) {
      y = warp_gather(row_idx, c_in, e0, e1, lane);
    } else {
      y = 0.f;
      for (int32_t e = e0 + sub; e < e1; e += G) y += ld_rank(c_in, __ldcs(row_idx + e));
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
    if (active && sub == 0) {
      if (y_hot) y += y_hot[r];
      finish_row(r, y, A, B, x_in, inv_deg, x_out, c_out, mass, dang, res);
    }
  }
  block_partials3(mass, dang, res, partials + 3 * (int64_t)blockIdx.x);
}

// Cold pass over long rows: one edge chunk per warp, chunks [c0, c1); each
// leaves its sum in chunk_sum (the finish kernel completes the rows).
template <typename T>
__global__ void __launch_bounds__(256) wchunks_kernel(const int32_t* __restrict__ row_idx, const T* __restrict__ c_in,
                                                      const int32_t* __restrict__ chunk_begin,
                                                      const int32_t* __restrict__ chunk_end, int32_t c0, int32_t c1,
                                                      float* __restrict__ chunk_sum) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t ch = c0 + warp; ch < c1; ch += nwarps) {
    const float y = warp_sum(warp_gather(row_idx, c_in, chunk_begin[ch], chunk_end[ch], lane));
    if (lane == 0) chunk_sum[ch] = y;
  }
}

// Hot pass.  Each block copies c[0, H) into shared memory, then sums, over
// the hot prefix [col_ptr[r], split[r]) of every row, contributions read from
// that copy only: rows of the lane buckets into y_hot[r], hot chunks of the
// long rows into chunk_sum.  Same lane layout per bucket as the cold pass.
struct HotLayout {
  int nb;
  int lanes[kMaxBuckets];
  int32_t begin[kMaxBuckets], end[kMaxBuckets];
};

template <typename T>
__device__ __forceinline__ float sm_f(const T* s, int32_t u);
template <>
__device__ __forceinline__ float sm_f<float>(const float* s, int32_t u) {
  return s[u];
}
template <>
__device__ __forceinline__ float sm_f<__nv_bfloat16>(const __nv_bfloat16* s, int32_t u) {
  return __bfloat162float(s[u]);
}

template <int G, typename T>
__device__ __forceinline__ void hot_rows(const int32_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                                         const int32_t* __restrict__ rows, int32_t i0, int32_t i1,
                                         const int32_t* __restrict__ split, const T* s_c, float* __restrict__ y_hot) {
  const int lane = threadIdx.x & 31;
  const int sub = lane & (G - 1);
  constexpr int kRowsPerWarp = 32 / G;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t wi = i0 + warp * kRowsPerWarp; wi < i1; wi += nwarps * kRowsPerWarp) {
    const int64_t i = wi + lane / G;
    const bool active = i < i1;
    int32_t r = 0, e0 = 0, e1 = 0;
    if (active) {
      r = rows[i];
      e0 = col_ptr[r];
      e1 = split[r];
    }
    float y = 0.f;
    for (int32_t e = e0 + sub; e < e1; e += G) y += sm_f(s_c, __ldcs(row_idx + e));
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
    if (active && sub == 0) y_hot[r] = y;
  }
}

template <typename T>
__global__ void __launch_bounds__(1024, 1) hot_kernel(const int32_t* __restrict__ col_ptr,
                                                      const int32_t* __restrict__ row_idx,
                                                      const int32_t* __restrict__ rows, HotLayout lay,
                                                      const int32_t* __restrict__ split, const T* __restrict__ c_in,
                                                      int32_t H, const int32_t* __restrict__ chunk_begin,
                                                      const int32_t* __restrict__ chunk_end, int32_t n_hot_chunks,
                                                      float* __restrict__ y_hot, float* __restrict__ chunk_sum) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* s_c = reinterpret_cast<T*>(smem_raw);
  {
    const int4* src = reinterpret_cast<const int4*>(c_in);
    int4* dst = reinterpret_cast<int4*>(s_c);
    const int32_t nvec = (int32_t)((int64_t)H * sizeof(T) / 16);  // H is a multiple of 8
    for (int32_t i = threadIdx.x; i < nvec; i += blockDim.x) dst[i] = __ldg(src + i);
  }
  __syncthreads();
  for (int k = 0; k < lay.nb; ++k) {
    const int32_t i0 = lay.begin[k], i1 = lay.end[k];
    switch (lay.lanes[k]) {
      case 1: hot_rows<1, T>(col_ptr, row_idx, rows, i0, i1, split, s_c, y_hot); break;
      case 2: hot_rows<2, T>(col_ptr, row_idx, rows, i0, i1, split, s_c, y_hot); break;
      case 4: hot_rows<4, T>(col_ptr, row_idx, rows, i0, i1, split, s_c, y_hot); break;
      case 8: hot_rows<8, T>(col_ptr, row_idx, rows, i0, i1, split, s_c, y_hot); break;
      case 16: hot_rows<16, T>(col_ptr, row_idx, rows, i0, i1, split, s_c, y_hot); break;
      case 32: hot_rows<32, T>(col_ptr, row_idx, rows, i0, i1, split, s_c, y_hot); break;
      default: break;
    }
  }
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t ch = warp; ch < n_hot_chunks; ch += nwarps) {
    const int32_t e0 = chunk_begin[ch], e1 = chunk_end[ch];
    float y = 0.f;
    for (int32_t e = e0 + lane; e < e1; e += 32) y += sm_f(s_c, __ldcs(row_idx + e));
    y = warp_sum(y);
    if (lane == 0) chunk_sum[ch] = y;
  }
}

// x_0 = 1/N (or the warm-start vector), c_0 = x_0 * inv_outdeg.
template <typename T>
__global__ void init_kernel(float* __restrict__ x, T* __restrict__ c, const float* __restrict__ inv_deg, int32_t n,
                            double* __restrict__ partials, const float* __restrict__ x_start) {
  float mass = 0.f, dang = 0.f;
  const float x0 = 1.0f / (float)n;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const float idg = inv_deg[v];
    const float xv = x_start ? x_start[v] : x0;  // a warm start, else uniform
    x[v] = xv;
    store_rank(c, v, xv * idg);
    mass += xv;
    if (idg == 0.0f) dang += xv;
  }
  block_partials3(mass, dang, 0.f, partials + 3 * (int64_t)blockIdx.x);
}

// Finishes the long rows (grid-stride; hot then cold chunk sums, in order),
// then the last block to arrive folds all `npartials` block partials of the
// step (this kernel's own are the last gridDim.x of them) in index order,
// logs (mass, dangling, residual) and writes the next coefficients.
template <typename T>
__global__ void __launch_bounds__(256) finish_kernel(
    const float* __restrict__ x_in, const float* __restrict__ inv_deg, float* __restrict__ x_out,
    T* __restrict__ c_out, const int32_t* __restrict__ split_row, const int32_t* __restrict__ split_hbeg,
    const int32_t* __restrict__ split_hend, const int32_t* __restrict__ split_cbeg,
    const int32_t* __restrict__ split_cend, int32_t nsplit, const float* __restrict__ chunk_sum,
    double* __restrict__ partials, int32_t npartials, StepParams* __restrict__ prm, double* __restrict__ log_row,
    unsigned int* __restrict__ arrive) {
  __shared__ bool s_last;
  const float A = prm->coefA, B = prm->coefB;
  float fm = 0.f, fd = 0.f, fr = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nsplit; i += (int64_t)gridDim.x * blockDim.x) {
    float y = 0.f;
    for (int32_t c = split_hbeg[i]; c < split_hend[i]; ++c) y += chunk_sum[c];
    for (int32_t c = split_cbeg[i]; c < split_cend[i]; ++c) y += chunk_sum[c];
    finish_row(split_row[i], y, A, B, x_in, inv_deg, x_out, c_out, fm, fd, fr);
  }
  block_partials3(fm, fd, fr, partials + 3 * (int64_t)(npartials - gridDim.x + blockIdx.x));
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(arrive, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  fold_step(partials, npartials, prm, log_row);
  if (threadIdx.x == 0) *arrive = 0;  // ready for the next step
}

// x_start[p] = x[new2old[p]]: a caller-ordered vector in relabelled order.
__global__ void start_kernel(const float* __restrict__ x, const int32_t* __restrict__ new2old, int32_t n,
                             float* __restrict__ x_start) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    x_start[p] = x[new2old[p]];
}

__global__ void output_kernel(const float* __restrict__ x, const int32_t* __restrict__ old2new, int32_t n,
                              float* __restrict__ out) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    out[v] = x[old2new[v]];
}

// ---- host side -------------------------------------------------------------

struct LaunchShape {
  int grid;
  int partial_off;
};

// A schedule with, for the blocked one, its shape.
struct Choice {
  int sched = kSchedPull;
  int sb = 15, wb = 14;   // source-block and bin bits
  int64_t unit = 1 << 16; // edges per work unit
  int32_t dense = -1;     // dense sources (-1: as many as the layout takes)
};

struct PagerankWork {
  int device = 0;
  float* x[2] = {nullptr, nullptr};  // n floats each: the rank vector, always FP32
  // n * 4 bytes each: contributions x / outdeg, FP32 or BF16 (pull), or
  // their 32-bit fixed-point codes (blocked)
  void* c[2] = {nullptr, nullptr};
  float* out_tmp = nullptr;          // n floats, for host-pointer output
  float* y_hot = nullptr;            // n floats: hot-pass row sums
  int hot_grid = 0;                  // 0: no hot pass
  size_t hot_smem32 = 0, hot_smem16 = 0;
  double* partials = nullptr;
  int32_t npartials = 0;  // per step: lane-bucket kernels' blocks + finish blocks
  float* chunk_sum = nullptr;
  StepParams* prm = nullptr;
  unsigned int* arrive = nullptr;
  double* log = nullptr;  // (iters + 1) x 3
  int32_t log_cap = 0;
  LaunchShape shape[kMaxBuckets];
  int finish_grid = 1;
  int init_grid = 1;
  cudaStream_t cap = nullptr;
  cudaEvent_t ev_t0 = nullptr, ev_t1 = nullptr;  // around the iteration graph, for gpr_stats
  cudaStream_t side[kMaxBuckets] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_join[kMaxBuckets] = {};
  Blocked* blk = nullptr;  // the blocked schedule's edge layout, made on first use
  float* ones = nullptr;   // n ones: unit weights for the centralities
  float* x_start = nullptr;  // n: a warm start's vector in relabelled order
  bool tuned = false;      // `choice` was measured on this graph
  Choice choice;
  cudaGraphExec_t exec = nullptr;
  int32_t exec_iters = -1;
  int exec_dt = -1;
  int exec_sched = -1;
  bool exec_warm = false;
  int64_t exec_kernels = 0;  // kernel nodes in `exec`
};

void pagerank_work_free(PagerankWork* w) {
  if (!w) return;
  if (w->exec) cudaGraphExecDestroy(w->exec);
  cudaStream_t s = w->cap;
  blocked_free(w->blk, s);
  for (int i = 0; i < 2; ++i) {
    dfree(w->x[i], s);
    dfree(w->c[i], s);
  }
  dfree(w->out_tmp, s);
  dfree(w->ones, s);
  dfree(w->x_start, s);
  dfree(w->y_hot, s);
  dfree(w->partials, s);
  dfree(w->chunk_sum, s);
  dfree(w->prm, s);
  dfree(w->arrive, s);
  dfree(w->log, s);
  if (w->ev_fork) cudaEventDestroy(w->ev_fork);
  if (w->ev_t0) cudaEventDestroy(w->ev_t0);
  if (w->ev_t1) cudaEventDestroy(w->ev_t1);
  for (int i = 0; i < kMaxBuckets; ++i) {
    if (w->ev_join[i]) cudaEventDestroy(w->ev_join[i]);
    if (w->side[i]) cudaStreamDestroy(w->side[i]);
  }
  if (s) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  delete w;
}

int32_t hot_capacity() {
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device_ordinal());
  const int64_t bytes = optin > 4096 ? (int64_t)optin - 4096 : 0;  // leave room for static shared memory
  return (int32_t)((bytes / 4) & ~(int64_t)7);
}

template <typename T>
static int hot_grid_for(size_t smem) {
  cudaFuncSetAttribute(hot_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)std::max<size_t>(smem, 1));
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hot_kernel<T>, 1024, smem);
  return num_sms() * std::max(per_sm, 1);
}

template <typename K>
static int resident_grid(K kernel, int64_t blocks_needed) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0);
  per_sm = std::max(per_sm, 1);
  return (int)std::max<int64_t>(1, std::min<int64_t>(blocks_needed, (int64_t)num_sms() * per_sm));
}

template <typename T>
static int grid_for_bucket(const Bucket& b, int32_t nchunks) {
  const int64_t rows = b.row_end - b.row_begin;
  auto blocks = [&](int G) { return (rows * G + 255) / 256; };
  switch (b.lanes) {
    case 1: return resident_grid(rows_kernel<1, T>, blocks(1));
    case 2: return resident_grid(rows_kernel<2, T>, blocks(2));
    case 4: return resident_grid(rows_kernel<4, T>, blocks(4));
    case 8: return resident_grid(rows_kernel<8, T>, blocks(8));
    case 16: return resident_grid(rows_kernel<16, T>, blocks(16));
    case 32: return resident_grid(rows_kernel<32, T>, blocks(32));
    default: return resident_grid(wchunks_kernel<T>, ((int64_t)nchunks + 7) / 8);
  }
}

template <typename T>
static void launch_bucket(const Bucket& b, int grid, cudaStream_t s, const gpr_graph* g, const float* y_hot,
                          const T* c_in, const float* x_in, float* x_out, T* c_out, float* chunk_sum,
                          const StepParams* prm, double* part, const float* inv_deg) {
  const Plan& P = g->plan;
  // only warp-per-row rows are split; narrower buckets read their whole rows
  const bool split_rows = P.hot_H > 0 && b.lanes == 32;
  const int32_t* split = split_rows ? P.split : nullptr;
  if (!split_rows) y_hot = nullptr;
#define GPR_ROWS(GL)                                                                                            \
  rows_kernel<GL, T><<<grid, 256, 0, s>>>(g->col_ptr, g->row_idx, P.rows, b.row_begin, b.row_end, split, y_hot, \
                                          c_in, x_in, inv_deg, x_out, c_out, prm, part)
  switch (b.lanes) {
    case 1: GPR_ROWS(1); break;
    case 2: GPR_ROWS(2); break;
    case 4: GPR_ROWS(4); break;
    case 8: GPR_ROWS(8); break;
    case 16: GPR_ROWS(16); break;
    case 32: GPR_ROWS(32); break;
    default:
      wchunks_kernel<T><<<grid, 256, 0, s>>>(g->row_idx, c_in, P.chunk_begin, P.chunk_end, P.n_hot_chunks,
                                             P.nchunks, chunk_sum);
      break;
  }
#undef GPR_ROWS
}

// Records init + `iters` steps on w->cap (which is capturing).  A step is the
// hot pass, then the cold-pass bucket kernels forked onto side streams, joined
// before the finish kernel.
template <typename T>
static void record_iterations(gpr_graph* g, PagerankWork* w, int32_t iters, int sched, bool warm) {
  const Plan& P = g->plan;
  cudaStream_t s = w->cap;
  float* x[2] = {w->x[0], w->x[1]};
  T* c[2] = {(T*)w->c[0], (T*)w->c[1]};
  const bool hot = w->hot_grid > 0;
  const size_t hot_smem = sizeof(T) == 2 ? w->hot_smem16 : w->hot_smem32;
  HotLayout hl{};
  hl.nb = P.nbuckets;
  for (int k = 0; k < P.nbuckets; ++k) {
    hl.lanes[k] = P.bucket[k].lanes == 32 ? 32 : 0;  // the hot pass takes warp-per-row rows and long rows only
    hl.begin[k] = P.bucket[k].row_begin;
    hl.end[k] = P.bucket[k].row_end;
  }
  init_kernel<T><<<w->init_grid, 256, 0, s>>>(x[0], c[0], P.inv_deg, g->n, w->partials, warm ? w->x_start : nullptr);
  finish_kernel<T><<<1, 256, 0, s>>>(x[0], P.inv_deg, x[0], c[0], P.split_row, P.split_hbeg, P.split_hend,
                                    P.split_cbeg, P.split_cend, 0, w->chunk_sum, w->partials, w->init_grid + 1,
                                    w->prm, w->log, w->arrive);
  if (sched == kSchedBlocked) {
    uint32_t* cc[2] = {(uint32_t*)w->c[0], (uint32_t*)w->c[1]};
    blocked_record_codes<T>(w->blk, g, x[0], P.inv_deg, cc[0], s);
    blocked_record_reset(w->blk, s);
    for (int32_t it = 0; it < iters; ++it) {
      const int a = it & 1, b = a ^ 1;
      blocked_record_step<T>(w->blk, g, cc[a], x[a], x[b], cc[b], P.inv_deg, w->prm, w->log + 3 * (int64_t)(it + 1),
                             it, s);
    }
    return;
  }
  for (int32_t it = 0; it < iters; ++it) {
    const int a = it & 1, b = a ^ 1;
    if (hot)
      hot_kernel<T><<<w->hot_grid, 1024, hot_smem, s>>>(g->col_ptr, g->row_idx, P.rows, hl, P.split, c[a], P.hot_H,
                                                        P.chunk_begin, P.chunk_end, P.n_hot_chunks, w->y_hot,
                                                        w->chunk_sum);
    GPR_CUDA(cudaEventRecord(w->ev_fork, s));
    for (int bi = 0; bi < P.nbuckets; ++bi) {
      GPR_CUDA(cudaStreamWaitEvent(w->side[bi], w->ev_fork, 0));
      launch_bucket<T>(P.bucket[bi], w->shape[bi].grid, w->side[bi], g, hot ? w->y_hot : nullptr, c[a], x[a], x[b],
                       c[b], w->chunk_sum, w->prm, w->partials + 3 * (int64_t)w->shape[bi].partial_off, P.inv_deg);
      GPR_CUDA(cudaEventRecord(w->ev_join[bi], w->side[bi]));
      GPR_CUDA(cudaStreamWaitEvent(s, w->ev_join[bi], 0));
    }
    finish_kernel<T><<<w->finish_grid, 256, 0, s>>>(x[a], P.inv_deg, x[b], c[b], P.split_row, P.split_hbeg,
                                                    P.split_hend, P.split_cbeg, P.split_cend, P.nsplit, w->chunk_sum,
                                                    w->partials, w->npartials, w->prm,
                                                    w->log + 3 * (int64_t)(it + 1), w->arrive);
  }
}

static PagerankWork* work_make(gpr_graph* g, cudaStream_t s) {
  PagerankWork* w = new PagerankWork();
  w->device = g->device;
  try {
    GPR_CUDA(cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking));
    for (int i = 0; i < kMaxBuckets; ++i) {
      GPR_CUDA(cudaStreamCreateWithFlags(&w->side[i], cudaStreamNonBlocking));
      GPR_CUDA(cudaEventCreateWithFlags(&w->ev_join[i], cudaEventDisableTiming));
    }
    GPR_CUDA(cudaEventCreateWithFlags(&w->ev_fork, cudaEventDisableTiming));
    GPR_CUDA(cudaEventCreate(&w->ev_t0));
    GPR_CUDA(cudaEventCreate(&w->ev_t1));
    const size_t vb = (size_t)g->n * 4;
    for (int i = 0; i < 2; ++i) {
      w->x[i] = (float*)dalloc(vb, s);
      w->c[i] = dalloc(vb, s);
    }
    const Plan& P = g->plan;
    const int32_t n_cold_chunks = P.nchunks - P.n_hot_chunks;
    int off = 0;
    for (int bi = 0; bi < P.nbuckets; ++bi) {
      const int g32 = grid_for_bucket<float>(P.bucket[bi], n_cold_chunks);
      const int g16 = grid_for_bucket<__nv_bfloat16>(P.bucket[bi], n_cold_chunks);
      w->shape[bi].grid = std::max(g32, g16);
      w->shape[bi].partial_off = off;
      if (P.bucket[bi].lanes != 0) off += w->shape[bi].grid;  // the chunk kernel finishes no rows
    }
    if (P.hot_H > 0) {
      w->hot_smem32 = (size_t)P.hot_H * 4;
      w->hot_smem16 = (size_t)P.hot_H * 2;
      w->hot_grid = std::max(hot_grid_for<float>(w->hot_smem32), hot_grid_for<__nv_bfloat16>(w->hot_smem16));
      w->y_hot = (float*)dalloc((size_t)g->n * 4, s);
    }
    w->finish_grid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)P.nsplit + 255) / 256, num_sms() * 2));
    w->npartials = off + w->finish_grid;
    w->init_grid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)g->n + 255) / 256, num_sms() * 4));
    const int32_t np = std::max(w->npartials, w->init_grid + 1);
    w->partials = (double*)dalloc((size_t)np * 3 * sizeof(double), s);
    GPR_CUDA(cudaMemsetAsync(w->partials, 0, (size_t)np * 3 * sizeof(double), s));
    w->chunk_sum = (float*)dalloc((size_t)std::max(P.nchunks, 1) * 4, s);
    w->prm = (StepParams*)dalloc(sizeof(StepParams), s);
    w->arrive = (unsigned int*)dalloc(16, s);
    GPR_CUDA(cudaMemsetAsync(w->arrive, 0, 16, s));
    return w;
  } catch (...) {
    pagerank_work_free(w);
    throw;
  }
}

// ---- schedule choice and the autotuner ----------------------------------------

// Units of about m / 1024 edges, between 2^16 and 2^21: every SM gets
// several, and few bins are cut into parts that meet in global memory.
static int64_t default_unit(const gpr_graph* g) {
  int64_t u = 1 << 16;
  while (u < (1 << 21) && u * 1024 < g->m) u <<= 1;
  return u;
}

// GPR_BLOCK_BITS="sb,w[,log2 unit[,dense sources]]" overrides the blocked
// shape (tests, experiments); returns false if unset.
static bool env_block_shape(Choice* c) {
  const char* e = getenv("GPR_BLOCK_BITS");
  if (!e) return false;
  int a = 0, b = 0, u = 0, dn = -1;
  const int k = sscanf(e, "%d,%d,%d,%d", &a, &b, &u, &dn);
  if (k < 2) return false;
  c->sb = a;
  c->wb = b;
  if (k >= 3 && u >= 12 && u <= 30) c->unit = (int64_t)1 << u;
  if (k == 4) c->dense = dn;
  return true;
}

// The dense-source count a choice asks of g's layout.
static int32_t dense_of(const gpr_graph* g, const Choice& c) {
  const int32_t cap = blocked_max_dense(g, c.sb, c.wb);
  return c.dense < 0 ? cap : std::min(c.dense, cap);
}

// Tuned choices by graph shape (ceil log2 n, ceil log2 m, storage type):
// graphs of one shape reuse the first one's measurement.
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int, int>, Choice> g_tuned;

static int ceil_log2(int64_t v) {
  int b = 0;
  while (((int64_t)1 << b) < v) ++b;
  return b;
}
static std::tuple<int, int, int> shape_key(const gpr_graph* g, gpr_dtype dt) {
  return std::make_tuple(ceil_log2(g->n), ceil_log2(std::max<int64_t>(g->m, 1)), (int)dt);
}

// Graphs below this many edges are launch- and latency-bound: the pull
// schedule, without tuning.
constexpr int64_t kTuneMinEdges = 1 << 22;

static void drop_exec(PagerankWork* w) {
  if (w->exec) {
    cudaGraphExecDestroy(w->exec);
    w->exec = nullptr;
  }
}

// The blocked layout of shape c (rebuilt if another shape is held).
static void ensure_layout(gpr_graph* g, PagerankWork* w, const Choice& c, cudaStream_t s) {
  const int32_t nd = (dense_of(g, c) >> c.sb) << c.sb;
  if (w->blk && (w->blk->sb_bits != c.sb || w->blk->w_bits != c.wb || w->blk->unit_edges != c.unit ||
                 w->blk->n_dense != nd)) {
    drop_exec(w);
    GPR_CUDA(cudaStreamSynchronize(s));
    blocked_free(w->blk, s);
    w->blk = nullptr;
  }
  if (!w->blk) w->blk = blocked_build(g, c.sb, c.wb, nd, c.unit, s);
}

// The iteration loop of `iters` steps with schedule `sched`, as a CUDA graph.
static void ensure_exec(gpr_graph* g, PagerankWork* w, int32_t iters, gpr_dtype dt, int sched, bool warm,
                        cudaStream_t s) {
  if (w->log_cap < iters + 1) {
    dfree(w->log, s);
    w->log = nullptr;
    w->log_cap = 0;
    const int32_t cap = std::max(iters + 1, 128);
    w->log = (double*)dalloc((size_t)cap * 3 * sizeof(double), s);
    w->log_cap = cap;
    drop_exec(w);
  }
  if (w->exec && w->exec_iters == iters && w->exec_dt == (int)dt && w->exec_sched == sched && w->exec_warm == warm)
    return;
  drop_exec(w);
  // the capture stream must see the allocations made on `s`
  GPR_CUDA(cudaStreamSynchronize(s));
  trace_phase(nullptr, s);
  cudaGraph_t graph = nullptr;
  GPR_CUDA(cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeThreadLocal));
  try {
    if (dt == GPR_BF16)
      record_iterations<__nv_bfloat16>(g, w, iters, sched, warm);
    else
      record_iterations<float>(g, w, iters, sched, warm);
  } catch (...) {
    cudaGraph_t junk = nullptr;
    cudaStreamEndCapture(w->cap, &junk);
    if (junk) cudaGraphDestroy(junk);
    throw;
  }
  cudaError_t e = cudaStreamEndCapture(w->cap, &graph);
  if (e != cudaSuccess) throw CudaFail{e, "cudaStreamEndCapture"};
  trace_phase("pagerank: capture", s);
  e = cudaGraphInstantiate(&w->exec, graph, 0);
  trace_phase("pagerank: instantiate", s);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    w->exec = nullptr;
    throw CudaFail{e, "cudaGraphInstantiate"};
  }
  w->exec_iters = iters;
  w->exec_dt = (int)dt;
  w->exec_sched = sched;
  w->exec_warm = warm;
  w->exec_kernels = sched == kSchedBlocked ? 3 + (int64_t)iters * 2
                                           : 2 + (int64_t)iters * (g->plan.nbuckets + 1 + (w->hot_grid > 0 ? 1 : 0));
}

// Device time of `iters` steps of schedule c, after one untimed run.
static double time_choice(gpr_graph* g, PagerankWork* w, const Choice& c, int32_t iters, gpr_dtype dt,
                          cudaStream_t s) {
  if (c.sched == kSchedBlocked) ensure_layout(g, w, c, s);
  ensure_exec(g, w, iters, dt, c.sched, false, s);
  const StepParams hp{0.f, 0.f, 0.85, (double)g->n};
  float best = 0.f;
  for (int rep = 0; rep < 2; ++rep) {
    GPR_CUDA(cudaMemcpyAsync(w->prm, &hp, sizeof hp, cudaMemcpyHostToDevice, s));
    GPR_CUDA(cudaEventRecord(w->ev_t0, s));
    GPR_CUDA(cudaGraphLaunch(w->exec, s));
    GPR_CUDA(cudaEventRecord(w->ev_t1, s));
    count_launches(w->exec_kernels);
    GPR_CUDA(cudaStreamSynchronize(s));
    GPR_CUDA(cudaEventElapsedTime(&best, w->ev_t0, w->ev_t1));
  }
  return best;
}

// Times the pull schedule and blocked shapes on g (trial_steps steps each),
// keeps the fastest for g and for its shape.  Lock held.
static Choice tune(gpr_graph* g, PagerankWork* w, gpr_dtype dt, int32_t trial_steps, cudaStream_t s,
                   gpr_tune_result* out) {
  std::vector<Choice> cands;
  cands.push_back(Choice{});  // pull
  const int64_t u = default_unit(g);
  // block shapes with the most dense sources; for the first shape also a
  // quarter of them, none, and halved and doubled units
  const int shapes[][2] = {{15, 14}, {14, 14}, {15, 13}};
  for (const auto& sh : shapes) {
    if (!blocked_eligible(g, sh[0], sh[1])) continue;
    const int32_t cap = blocked_max_dense(g, sh[0], sh[1]);
    cands.push_back(Choice{kSchedBlocked, sh[0], sh[1], u, cap});
    if (cands.size() > 2) continue;
    if (((cap / 4) >> sh[0]) > 0) cands.push_back(Choice{kSchedBlocked, sh[0], sh[1], u, (cap / 4) >> sh[0] << sh[0]});
    if (cap > 0) cands.push_back(Choice{kSchedBlocked, sh[0], sh[1], u, 0});
    cands.push_back(Choice{kSchedBlocked, sh[0], sh[1], std::max<int64_t>(u / 2, 1 << 14), cap});
    cands.push_back(Choice{kSchedBlocked, sh[0], sh[1], u * 2, cap});
  }
  Choice best;
  double best_ms = 0.0, pull_ms = 0.0;
  for (size_t i = 0; i < cands.size(); ++i) {
    const double ms = time_choice(g, w, cands[i], trial_steps, dt, s) / std::max(trial_steps, 1);
    if (i == 0) pull_ms = ms;
    if (i == 0 || ms < best_ms) {
      best = cands[i];
      best_ms = ms;
    }
  }
  w->tuned = true;
  w->choice = best;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[shape_key(g, dt)] = best;
  }
  if (out) {
    out->schedule = best.sched == kSchedBlocked ? GPR_SPMV_BLOCKED : GPR_SPMV_PULL;
    out->sb_bits = best.sched == kSchedBlocked ? best.sb : 0;
    out->w_bits = best.sched == kSchedBlocked ? best.wb : 0;
    out->unit_edges = best.sched == kSchedBlocked ? best.unit : 0;
    out->dense_sources = best.sched == kSchedBlocked ? dense_of(g, best) : 0;
    out->ms_per_step = best_ms;
    out->pull_ms_per_step = pull_ms;
    out->candidates = (int32_t)cands.size();
  }
  return best;
}

// The schedule of a call: forced by flags (blocked with the tuned or default
// shape), else GPR_SPMV=pull|blocked, else the graph's tuned choice, else
// the choice tuned for its shape, else (graphs of at least kTuneMinEdges
// edges) tuned now, else pull.
static Choice pick(gpr_graph* g, PagerankWork* w, int flags, gpr_dtype dt, cudaStream_t s) {
  Choice blocked{kSchedBlocked, 15, 14, default_unit(g)};
  if (w->tuned && w->choice.sched == kSchedBlocked) blocked = w->choice;
  const bool env_shape = env_block_shape(&blocked);
  if (flags & GPR_SPMV_PULL) return Choice{};
  if (flags & GPR_SPMV_BLOCKED) return blocked;
  if (const char* e = getenv("GPR_SPMV")) {
    if (!strcmp(e, "blocked") && blocked_eligible(g, blocked.sb, blocked.wb)) return blocked;
    if (!strcmp(e, "pull")) return Choice{};
  }
  if (env_shape && blocked_eligible(g, blocked.sb, blocked.wb)) return blocked;
  if (w->tuned) return w->choice;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(shape_key(g, dt));
    if (it != g_tuned.end()) return it->second;
  }
  if (g->m >= kTuneMinEdges) return tune(g, w, dt, 5, s, nullptr);
  return Choice{};
}

gpr_status run_pagerank(gpr_graph* g, double damping, int32_t iters, gpr_dtype dt, int flags, float* x_out,
                        gpr_stats* st, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g->mu);
  try {
    const auto t_setup0 = std::chrono::steady_clock::now();
    trace_phase(nullptr, s);
    if (!g->work) g->work = work_make(g, s);
    PagerankWork* w = g->work;
    trace_phase("pagerank: workspace", s);
    const Choice ch = pick(g, w, flags, dt, s);
    trace_phase("pagerank: schedule choice", s);
    const int sched = ch.sched;
    if (sched == kSchedBlocked) ensure_layout(g, w, ch, s);
    const bool warm = (flags & GPR_WARM_START) != 0;
    if (warm) {
      // the caller's start vector (x_out, caller ids) into relabelled order
      if (!w->x_start) w->x_start = (float*)dalloc((size_t)g->n * 4, s);
      const float* src = x_out;
      if (flags & GPR_PTR_HOST) {
        if (!w->out_tmp) w->out_tmp = (float*)dalloc((size_t)g->n * 4, s);
        GPR_CUDA(cudaMemcpyAsync(w->out_tmp, x_out, (size_t)g->n * 4, cudaMemcpyHostToDevice, s));
        src = w->out_tmp;
      }
      const int og = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)g->n + 255) / 256, num_sms() * 8));
      start_kernel<<<og, 256, 0, s>>>(src, g->plan.new2old, g->n, w->x_start);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
    }
    ensure_exec(g, w, iters, dt, sched, warm, s);
    StepParams hp{0.f, 0.f, damping, (double)g->n};
    GPR_CUDA(cudaMemcpyAsync(w->prm, &hp, sizeof hp, cudaMemcpyHostToDevice, s));
    const double t_setup =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_setup0).count();
    if (st) GPR_CUDA(cudaEventRecord(w->ev_t0, s));
    GPR_CUDA(cudaGraphLaunch(w->exec, s));
    if (st) GPR_CUDA(cudaEventRecord(w->ev_t1, s));
    count_launches(w->exec_kernels);
    const float* xf = w->x[iters & 1];
    float* dst = (flags & GPR_PTR_HOST) ? nullptr : x_out;
    if (!dst) {
      if (!w->out_tmp) w->out_tmp = (float*)dalloc((size_t)g->n * 4, s);
      dst = w->out_tmp;
    }
    const int og = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)g->n + 255) / 256, num_sms() * 8));
    output_kernel<<<og, 256, 0, s>>>(xf, g->plan.old2new, g->n, dst);
    GPR_CUDA(cudaGetLastError());
    count_launches(1);
    if (flags & GPR_PTR_HOST) {
      GPR_CUDA(cudaMemcpyAsync(x_out, dst, (size_t)g->n * 4, cudaMemcpyDeviceToHost, s));
    }
    if (st) {
      double row[3];
      GPR_CUDA(cudaMemcpyAsync(row, w->log + 3 * (int64_t)iters, sizeof row, cudaMemcpyDeviceToHost, s));
      GPR_CUDA(cudaStreamSynchronize(s));
      st->iters_run = iters;
      st->mass = row[0];
      st->dangling = row[1];
      st->residual_l1 = iters > 0 ? row[2] : 0.0;
      float ms = 0.f;
      GPR_CUDA(cudaEventElapsedTime(&ms, w->ev_t0, w->ev_t1));
      st->t_iter_ms = ms;
      st->t_setup_ms = t_setup;
      st->schedule = sched == kSchedBlocked ? GPR_SPMV_BLOCKED : GPR_SPMV_PULL;
    } else if (flags & GPR_PTR_HOST) {
      GPR_CUDA(cudaStreamSynchronize(s));
    }
    return GPR_OK;
  } catch (const StatusFail& f) {
    set_error("pagerank: %s", f.msg.c_str());
    return f.st;
  } catch (const CudaFail& f) {
    cudaGetLastError();
    set_error("pagerank: %s failed: %s", f.what, cudaGetErrorString(f.err));
    return GPR_ECUDA;
  }
}

gpr_status run_pagerank_tune(gpr_graph* g, gpr_dtype dt, int32_t trial_steps, gpr_tune_result* out,
                             cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g->mu);
  try {
    if (!g->work) g->work = work_make(g, s);
    tune(g, g->work, dt, trial_steps, s, out);
    return GPR_OK;
  } catch (const StatusFail& f) {
    set_error("pagerank_tune: %s", f.msg.c_str());
    return f.st;
  } catch (const CudaFail& f) {
    cudaGetLastError();
    set_error("pagerank_tune: %s failed: %s", f.what, cudaGetErrorString(f.err));
    return GPR_ECUDA;
  }
}

// ---- HITS and eigenvector centrality ------------------------------------------
// (section 4 Table "snap_methods" names both).  The power iterations
//   authorities a = A^T h,  hubs h = A a   (HITS)
//   x = A^T x                              (eigenvector centrality)
// run on the pull kernels of the PageRank step with unit weights (an
// inverse-degree vector of ones) and d = 1: each step's fold leaves
// coefA = 1 / ||previous vector||_1, so every product starts from the L1-
// normalised previous vector.  Scaling does not change a direction, so the
// vectors match the L2-normalised iteration; the output is scaled to unit L2
// norm once, at the end.  A^T x pulls over g's CSC; A x pulls over the CSC of
// the transposed graph (same relabelled ids), built on first use.

__global__ void fill_kernel(float* __restrict__ p, float v, int32_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// Block partials of sum x^2 (FP32 per thread, FP64 across warps).
__global__ void sumsq_kernel(const float* __restrict__ x, int32_t n, double* __restrict__ partials) {
  float a = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    a = fmaf(x[i], x[i], a);
  block_partials3(a, 0.f, 0.f, partials + 3 * (int64_t)blockIdx.x);
}

// out[v] = x[old2new[v]] / ||x||_2, the norm folded from the partials in
// index order by every block (0 stays 0).
__global__ void l2_output_kernel(const float* __restrict__ x, const int32_t* __restrict__ old2new, int32_t n,
                                 const double* __restrict__ partials, int32_t np, float* __restrict__ out) {
  __shared__ float s_inv;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int32_t i = 0; i < np; ++i) t += partials[3 * (int64_t)i];
    s_inv = t > 0.0 ? (float)(1.0 / sqrt(t)) : 0.f;
  }
  __syncthreads();
  const float inv = s_inv;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    out[v] = x[old2new[v]] * inv;
}

// One pull step of g's kernels on stream s: x_out = coefA * (A-pull of c_in),
// c_out = x_out * inv_deg, partials folded into prm and log_row.
static void launch_pull_step(gpr_graph* g, PagerankWork* w, cudaStream_t s, const float* c_in, const float* x_in,
                             float* x_out, float* c_out, const float* inv_deg, StepParams* prm, double* log_row) {
  const Plan& P = g->plan;
  if (w->hot_grid > 0) {
    HotLayout hl{};
    hl.nb = P.nbuckets;
    for (int k = 0; k < P.nbuckets; ++k) {
      hl.lanes[k] = P.bucket[k].lanes == 32 ? 32 : 0;
      hl.begin[k] = P.bucket[k].row_begin;
      hl.end[k] = P.bucket[k].row_end;
    }
    hot_kernel<float><<<w->hot_grid, 1024, w->hot_smem32, s>>>(g->col_ptr, g->row_idx, P.rows, hl, P.split, c_in,
                                                              P.hot_H, P.chunk_begin, P.chunk_end, P.n_hot_chunks,
                                                              w->y_hot, w->chunk_sum);
    count_launches(1);
  }
  GPR_CUDA(cudaEventRecord(w->ev_fork, s));
  for (int bi = 0; bi < P.nbuckets; ++bi) {
    GPR_CUDA(cudaStreamWaitEvent(w->side[bi], w->ev_fork, 0));
    launch_bucket<float>(P.bucket[bi], w->shape[bi].grid, w->side[bi], g, w->hot_grid > 0 ? w->y_hot : nullptr, c_in,
                         x_in, x_out, c_out, w->chunk_sum, prm, w->partials + 3 * (int64_t)w->shape[bi].partial_off,
                         inv_deg);
    GPR_CUDA(cudaEventRecord(w->ev_join[bi], w->side[bi]));
    GPR_CUDA(cudaStreamWaitEvent(s, w->ev_join[bi], 0));
  }
  finish_kernel<float><<<w->finish_grid, 256, 0, s>>>(x_in, inv_deg, x_out, c_out, P.split_row, P.split_hbeg,
                                                      P.split_hend, P.split_cbeg, P.split_cend, P.nsplit,
                                                      w->chunk_sum, w->partials, w->npartials, prm, log_row,
                                                      w->arrive);
  GPR_CUDA(cudaGetLastError());
  count_launches(P.nbuckets + 1);
}

static void ensure_log(PagerankWork* w, int32_t rows, cudaStream_t s) {
  if (w->log_cap >= rows) return;
  drop_exec(w);  // the captured PageRank loop writes into the old log
  dfree(w->log, s);
  w->log = nullptr;
  w->log_cap = 0;
  const int32_t cap = std::max(rows, 128);
  w->log = (double*)dalloc((size_t)cap * 3 * sizeof(double), s);
  w->log_cap = cap;
}

// out (device or, with GPR_PTR_HOST, host) = x / ||x||_2 by caller id.
static void write_l2_output(gpr_graph* g, PagerankWork* w, const float* x, float* out, int flags, cudaStream_t s) {
  const int32_t n = g->n;
  float* dst = out;
  if (flags & GPR_PTR_HOST) {
    if (!w->out_tmp) w->out_tmp = (float*)dalloc((size_t)n * 4, s);
    dst = w->out_tmp;
  }
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)n + 255) / 256, (int64_t)w->npartials));
  sumsq_kernel<<<grid, 256, 0, s>>>(x, n, w->partials);
  l2_output_kernel<<<grid, 256, 0, s>>>(x, g->plan.old2new, n, w->partials, grid, dst);
  GPR_CUDA(cudaGetLastError());
  count_launches(2);
  if (flags & GPR_PTR_HOST) {
    GPR_CUDA(cudaMemcpyAsync(out, dst, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
  }
}

// kind 0: eigenvector centrality into out_x; kind 1: HITS into out_hub and out_auth.
gpr_status run_centrality(gpr_graph* g, int kind, int32_t iters, float* out_x, float* out_hub, int flags,
                          cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g->mu);
  try {
    if (!g->work) g->work = work_make(g, s);
    PagerankWork* w = g->work;
    const int32_t n = g->n;
    if (!w->ones) {
      w->ones = (float*)dalloc((size_t)n * 4, s);
      fill_kernel<<<(int)std::min<int64_t>(((int64_t)n + 255) / 256, num_sms() * 8), 256, 0, s>>>(w->ones, 1.f, n);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
    }
    gpr_graph* t = nullptr;
    PagerankWork* wt = nullptr;
    if (kind == 1) {
      if (!g->transposed) g->transposed = build_transposed(g, s);
      t = g->transposed;
      if (!t->work) t->work = work_make(t, s);
      wt = t->work;
      // the authorities start uniform too (the output of 0 steps)
      fill_kernel<<<(int)std::min<int64_t>(((int64_t)n + 255) / 256, num_sms() * 8), 256, 0, s>>>(w->x[0],
                                                                                              1.f / (float)n, n);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
    }
    // the blocked schedule (unit weights: c = x) when asked for, or on a large
    // graph; vectors are L1-normalised between products, so every row sum is
    // at most 1, within the fixed-point range of the blocked sums
    // The layout's shape is the one PageRank uses on this graph: its
    // autotuner's choice (tuned now if this shape has not been), the products
    // being PageRank's step kernels with unit weights.
    Choice bc{kSchedBlocked, 15, 14, default_unit(g)};
    if (!(flags & GPR_SPMV_PULL) && g->m >= kTuneMinEdges) {
      const Choice ch = pick(g, w, 0, GPR_FP32, s);
      if (ch.sched == kSchedBlocked) bc = ch;
    }
    if (w->tuned && w->choice.sched == kSchedBlocked) bc = w->choice;
    env_block_shape(&bc);
    bool blocked = (flags & GPR_SPMV_BLOCKED) || (!(flags & GPR_SPMV_PULL) && g->m >= kTuneMinEdges);
    blocked = blocked && blocked_eligible(g, bc.sb, bc.wb) && (kind == 0 || blocked_eligible(t, bc.sb, bc.wb));
    if (blocked) {
      ensure_layout(g, w, bc, s);
      blocked_record_reset(w->blk, s);
      if (kind == 1) {
        ensure_layout(t, wt, bc, s);
        blocked_record_reset(wt->blk, s);
      }
    }
    int32_t it_g = 0, it_t = 0;  // steps since the reset, per layout
    auto product = [&](gpr_graph* gg, PagerankWork* ww, const float* c_in, const float* x_in, float* x_out,
                       float* c_out, double* log_row) {
      if (blocked)  // the contributions are held as codes
        blocked_record_step<float>(ww->blk, gg, (const uint32_t*)c_in, x_in, x_out, (uint32_t*)c_out, w->ones,
                                   w->prm, log_row, gg == g ? it_g++ : it_t++, s);
      else
        launch_pull_step(gg, ww, s, c_in, x_in, x_out, c_out, w->ones, w->prm, log_row);
    };
    ensure_log(w, 2 * iters + 2, s);
    const StepParams hp{0.f, 0.f, 1.0, (double)n};  // d = 1: no teleport, coefA = 1 / mass
    GPR_CUDA(cudaMemcpyAsync(w->prm, &hp, sizeof hp, cudaMemcpyHostToDevice, s));
    // the start vector: uniform (1/n; its direction is 1/sqrt(n)), its fold sets coefA = 1
    float* x0 = kind == 1 ? wt->x[0] : w->x[0];
    float* c0 = kind == 1 ? (float*)wt->c[0] : (float*)w->c[0];
    init_kernel<float><<<w->init_grid, 256, 0, s>>>(x0, c0, w->ones, n, w->partials, nullptr);
    finish_kernel<float><<<1, 256, 0, s>>>(x0, w->ones, x0, c0, g->plan.split_row, g->plan.split_hbeg,
                                          g->plan.split_hend, g->plan.split_cbeg, g->plan.split_cend, 0,
                                          w->chunk_sum, w->partials, w->init_grid + 1, w->prm, w->log, w->arrive);
    GPR_CUDA(cudaGetLastError());
    count_launches(2);
    if (blocked) {  // the first product reads c0 through g's layout
      blocked_record_codes<float>(w->blk, g, x0, w->ones, (uint32_t*)c0, s);
      count_launches(1);
    }
    if (kind == 0) {
      for (int32_t it = 0; it < iters; ++it) {
        const int a = it & 1, b = a ^ 1;
        product(g, w, (const float*)w->c[a], w->x[a], w->x[b], (float*)w->c[b], w->log + 3 * (int64_t)(it + 1));
      }
      write_l2_output(g, w, w->x[iters & 1], out_x, flags, s);
    } else {
      // hubs in wt->x / wt->c[0], authorities in w->x / w->c[0]; one coefficient
      // block, so each fold hands 1 / ||x||_1 to the other product
      for (int32_t it = 0; it < iters; ++it) {
        const int a = it & 1, b = a ^ 1;
        product(g, w, (const float*)wt->c[0], w->x[a], w->x[b], (float*)w->c[0], w->log + 3 * (int64_t)(2 * it + 1));
        product(t, wt, (const float*)w->c[0], wt->x[a], wt->x[b], (float*)wt->c[0],
                w->log + 3 * (int64_t)(2 * it + 2));
      }
      write_l2_output(g, w, wt->x[iters & 1], out_hub, flags, s);
      write_l2_output(g, w, w->x[iters & 1], out_x, flags, s);
    }
    return GPR_OK;
  } catch (const StatusFail& f) {
    set_error("%s: %s", kind == 1 ? "hits" : "eigen_centrality", f.msg.c_str());
    return f.st;
  } catch (const CudaFail& f) {
    cudaGetLastError();
    set_error("%s: %s failed: %s", kind == 1 ? "hits" : "eigen_centrality", f.what, cudaGetErrorString(f.err));
    return GPR_ECUDA;
  }
}

}  // namespace gpr
