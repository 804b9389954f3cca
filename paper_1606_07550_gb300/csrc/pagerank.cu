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
// applied to x / S (mass normalisation).  Each kernel also forms per-block
// FP64 partials of S', D' and ||x' - x||_1 from FP32 per-thread and per-warp
// sums; one single-block kernel folds the partials in a fixed order (so
// repeated runs are bitwise identical) and writes the next coefficients.
//
// Rows are processed by in-degree bucket: 1, 4, 8 or 32 lanes per row, and
// rows above the last lane bucket in chunks of edges per thread block (rows
// longer than a chunk are split and finished by the fold kernel).  The whole
// iteration loop is one CUDA graph.
#include <algorithm>
#include <cstring>

#include "gpr_internal.cuh"

namespace gpr {

struct StepParams {
  float coefA, coefB;
  double d;
  double n;
};

// ---- storage of the gathered contributions c = x / outdeg: FP32 or BF16.
// The rank vector x itself and all accumulation stay FP32. --------------
template <typename T>
__device__ __forceinline__ float ld_rank(const T* p, int64_t i);
template <>
__device__ __forceinline__ float ld_rank<float>(const float* p, int64_t i) {
  return __ldg(p + i);
}
template <>
__device__ __forceinline__ float ld_rank<__nv_bfloat16>(const __nv_bfloat16* p, int64_t i) {
  return __bfloat162float(__ldg(p + i));
}
template <typename T>
__device__ __forceinline__ float store_rank(T* p, int64_t i, float v);  // returns the stored value
template <>
__device__ __forceinline__ float store_rank<float>(float* p, int64_t i, float v) {
  p[i] = v;
  return v;
}
template <>
__device__ __forceinline__ float store_rank<__nv_bfloat16>(__nv_bfloat16* p, int64_t i, float v) {
  const __nv_bfloat16 b = __float2bfloat16_rn(v);
  p[i] = b;
  return __bfloat162float(b);
}

// ---- reductions ----------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block partial of three per-thread FP32 sums: FP32 within each warp, FP64
// across warps, written to out[0..2].  Call with all threads of the block.
__device__ __forceinline__ void block_partials3(float a, float b, float c, double* out) {
  __shared__ double s[3][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  a = warp_sum(a);
  b = warp_sum(b);
  c = warp_sum(c);
  if (lane == 0) {
    s[0][w] = a;
    s[1][w] = b;
    s[2][w] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0, tb = 0, tc = 0;
    for (int i = 0; i < nw; ++i) {
      ta += s[0][i];
      tb += s[1][i];
      tc += s[2][i];
    }
    out[0] = ta;
    out[1] = tb;
    out[2] = tc;
  }
}

// Finish one row: store x' and c', accumulate mass, dangling mass, residual.
template <typename T>
__device__ __forceinline__ void finish_row(int64_t r, float y, float A, float B, const float* __restrict__ x_in,
                                           const float* __restrict__ inv_deg, float* __restrict__ x_out,
                                           T* __restrict__ c_out, float& mass, float& dang, float& res) {
  const float idg = inv_deg[r];
  const float xs = fmaf(A, y, B);
  x_out[r] = xs;
  store_rank(c_out, r, xs * idg);
  mass += xs;
  res += fabsf(xs - x_in[r]);
  if (idg == 0.0f) dang += xs;
}

// G lanes per row, G in {1, 2, 4, 8, 16, 32}; warps stride over row groups.
template <int G, typename T>
__global__ void __launch_bounds__(256) rows_kernel(const int32_t* __restrict__ col_ptr,
                                                   const int32_t* __restrict__ row_idx, const T* __restrict__ c_in,
                                                   const float* __restrict__ x_in, const float* __restrict__ inv_deg,
                                                   float* __restrict__ x_out, T* __restrict__ c_out, int32_t r0,
                                                   int32_t r1, const StepParams* __restrict__ prm,
                                                   double* __restrict__ partials) {
  const float A = prm->coefA, B = prm->coefB;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (G - 1);
  constexpr int kRowsPerWarp = 32 / G;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  float mass = 0.f, dang = 0.f, res = 0.f;
  for (int64_t wr = r0 + warp * kRowsPerWarp; wr < r1; wr += nwarps * kRowsPerWarp) {
    const int64_t r = wr + lane / G;
    const bool active = r < r1;
    int32_t e0 = 0, e1 = 0;
    if (active) {
      e0 = col_ptr[r];
      e1 = col_ptr[r + 1];
    }
    float y = 0.f;
    if constexpr (G == 32) {
      // 128-bit index loads on the 16-byte-aligned body of the row
      const int32_t h = min(e1, (e0 + 3) & ~3);
      if (e0 + lane < h) y += ld_rank(c_in, __ldcs(row_idx + e0 + lane));
      const int32_t body_end = h + ((e1 - h) & ~3);
      for (int32_t e = h + 4 * lane; e < body_end; e += 128) {
        const int4 q = __ldcs(reinterpret_cast<const int4*>(row_idx + e));
        const float a0 = ld_rank(c_in, q.x), a1 = ld_rank(c_in, q.y);
        const float a2 = ld_rank(c_in, q.z), a3 = ld_rank(c_in, q.w);
        y += (a0 + a1) + (a2 + a3);
      }
      if (body_end + lane < e1) y += ld_rank(c_in, __ldcs(row_idx + body_end + lane));
    } else {
      for (int32_t e = e0 + sub; e < e1; e += G) y += ld_rank(c_in, __ldcs(row_idx + e));
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
    if (active && sub == 0) finish_row(r, y, A, B, x_in, inv_deg, x_out, c_out, mass, dang, res);
  }
  block_partials3(mass, dang, res, partials + 3 * (int64_t)blockIdx.x);
}

// One chunk of edges per block iteration.  A chunk that is a whole row is
// finished here; a piece of a split row leaves its sum in chunk_sum.
template <typename T>
__global__ void __launch_bounds__(256) chunks_kernel(
    const int32_t* __restrict__ row_idx, const T* __restrict__ c_in, const float* __restrict__ x_in,
    const float* __restrict__ inv_deg, float* __restrict__ x_out, T* __restrict__ c_out,
    const int32_t* __restrict__ chunk_row, const int32_t* __restrict__ chunk_begin,
    const int32_t* __restrict__ chunk_end, const int32_t* __restrict__ chunk_whole, int32_t nchunks,
    float* __restrict__ chunk_sum, const StepParams* __restrict__ prm, double* __restrict__ partials) {
  __shared__ float s_w[8];
  const float A = prm->coefA, B = prm->coefB;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  float mass = 0.f, dang = 0.f, res = 0.f;
  for (int32_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int32_t e0 = chunk_begin[ch], e1 = chunk_end[ch];
    float y = 0.f;
    const int32_t h = min(e1, (e0 + 3) & ~3);
    if (e0 + t < h) y += ld_rank(c_in, __ldcs(row_idx + e0 + t));
    const int32_t body_end = h + ((e1 - h) & ~3);
    for (int32_t e = h + 4 * t; e < body_end; e += 4 * 256) {
      const int4 q = __ldcs(reinterpret_cast<const int4*>(row_idx + e));
      const float a0 = ld_rank(c_in, q.x), a1 = ld_rank(c_in, q.y);
      const float a2 = ld_rank(c_in, q.z), a3 = ld_rank(c_in, q.w);
      y += (a0 + a1) + (a2 + a3);
    }
    if (body_end + t < e1) y += ld_rank(c_in, __ldcs(row_idx + body_end + t));
    y = warp_sum(y);
    if (lane == 0) s_w[w] = y;
    __syncthreads();
    if (t == 0) {
      float tot = 0.f;
      for (int i = 0; i < 8; ++i) tot += s_w[i];
      if (chunk_whole[ch])
        finish_row(chunk_row[ch], tot, A, B, x_in, inv_deg, x_out, c_out, mass, dang, res);
      else
        chunk_sum[ch] = tot;
    }
    __syncthreads();
  }
  block_partials3(mass, dang, res, partials + 3 * (int64_t)blockIdx.x);
}

// x_0 = 1/N, c_0 = x_0 * inv_outdeg.
template <typename T>
__global__ void init_kernel(float* __restrict__ x, T* __restrict__ c, const float* __restrict__ inv_deg, int32_t n,
                            double* __restrict__ partials) {
  float mass = 0.f, dang = 0.f;
  const float x0 = 1.0f / (float)n;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const float idg = inv_deg[v];
    const float xs = x0;
    x[v] = xs;
    store_rank(c, v, xs * idg);
    mass += xs;
    if (idg == 0.0f) dang += xs;
  }
  block_partials3(mass, dang, 0.f, partials + 3 * (int64_t)blockIdx.x);
}

// Single block: finish split rows, fold all block partials in a fixed order,
// log (mass, dangling, residual) for step `it` and write the next
// coefficients.
template <typename T>
__global__ void __launch_bounds__(1024) fold_kernel(
    const float* __restrict__ x_in, const float* __restrict__ inv_deg, float* __restrict__ x_out,
    T* __restrict__ c_out, const int32_t* __restrict__ split_row, const int32_t* __restrict__ split_cbeg,
    const int32_t* __restrict__ split_cend, int32_t nsplit, const float* __restrict__ chunk_sum,
    const double* __restrict__ partials, int32_t npartials, StepParams* __restrict__ prm,
    double* __restrict__ log_row) {
  __shared__ double s[3][32];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  const float A = prm->coefA, B = prm->coefB;
  float fm = 0.f, fd = 0.f, fr = 0.f;
  for (int32_t i = t; i < nsplit; i += blockDim.x) {
    float y = 0.f;
    for (int32_t c = split_cbeg[i]; c < split_cend[i]; ++c) y += chunk_sum[c];
    finish_row(split_row[i], y, A, B, x_in, inv_deg, x_out, c_out, fm, fd, fr);
  }
  double a = fm, b = fd, c = fr;
  for (int32_t i = t; i < npartials; i += blockDim.x) {
    a += partials[3 * (int64_t)i];
    b += partials[3 * (int64_t)i + 1];
    c += partials[3 * (int64_t)i + 2];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if (lane == 0) {
    s[0][w] = a;
    s[1][w] = b;
    s[2][w] = c;
  }
  __syncthreads();
  if (t == 0) {
    double mass = 0, dang = 0, res = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      mass += s[0][i];
      dang += s[1][i];
      res += s[2][i];
    }
    log_row[0] = mass;
    log_row[1] = dang;
    log_row[2] = res;
    const double d = prm->d, n = prm->n;
    prm->coefA = (float)(d / mass);
    prm->coefB = (float)((1.0 - d) / n + d * dang / (n * mass));
  }
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

struct PagerankWork {
  int device = 0;
  void* x[2] = {nullptr, nullptr};  // n floats each: the rank vector, always FP32
  void* c[2] = {nullptr, nullptr};  // n * 4 bytes each: contributions x / outdeg, FP32 or BF16
  float* out_tmp = nullptr;         // n floats, for host-pointer output
  double* partials = nullptr;
  int32_t npartials = 0;
  float* chunk_sum = nullptr;
  StepParams* prm = nullptr;
  double* log = nullptr;  // (iters + 1) x 3
  int32_t log_cap = 0;
  LaunchShape shape[kMaxBuckets];
  LaunchShape init_shape;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  int32_t exec_iters = -1;
  int exec_dt = -1;
  int64_t exec_kernels = 0;  // kernel nodes in `exec`
};

void pagerank_work_free(PagerankWork* w) {
  if (!w) return;
  if (w->exec) cudaGraphExecDestroy(w->exec);
  cudaStream_t s = w->cap;
  for (int i = 0; i < 2; ++i) {
    dfree(w->x[i], s);
    dfree(w->c[i], s);
  }
  dfree(w->out_tmp, s);
  dfree(w->partials, s);
  dfree(w->chunk_sum, s);
  dfree(w->prm, s);
  dfree(w->log, s);
  if (s) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  delete w;
}

template <int G, typename T>
static int rows_grid(int64_t rows) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rows_kernel<G, T>, 256, 0);
  per_sm = std::max(per_sm, 1);
  const int64_t warps = (rows + (32 / G) - 1) / (32 / G);
  const int64_t blocks = (warps + 7) / 8;
  return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)num_sms() * per_sm));
}

template <typename T>
static int grid_for_bucket(const Bucket& b, int32_t nchunks) {
  const int64_t rows = b.row_end - b.row_begin;
  switch (b.lanes) {
    case 1: return rows_grid<1, T>(rows);
    case 2: return rows_grid<2, T>(rows);
    case 4: return rows_grid<4, T>(rows);
    case 8: return rows_grid<8, T>(rows);
    case 16: return rows_grid<16, T>(rows);
    case 32: return rows_grid<32, T>(rows);
    default: {
      int per_sm = 0;
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, chunks_kernel<T>, 256, 0);
      per_sm = std::max(per_sm, 1);
      return (int)std::max<int64_t>(1, std::min<int64_t>(nchunks, (int64_t)num_sms() * per_sm));
    }
  }
}

template <typename T>
static void launch_rows(const Bucket& b, int grid, cudaStream_t s, const Plan& P, const T* c_in, const float* x_in,
                        float* x_out, T* c_out, const StepParams* prm, double* part) {
#define GPR_ROWS(GL)                                                                                       \
  rows_kernel<GL, T><<<grid, 256, 0, s>>>(P.col_ptr, P.row_idx, c_in, x_in, P.inv_deg, x_out, c_out, b.row_begin, \
                                          b.row_end, prm, part)
  switch (b.lanes) {
    case 1: GPR_ROWS(1); break;
    case 2: GPR_ROWS(2); break;
    case 4: GPR_ROWS(4); break;
    case 8: GPR_ROWS(8); break;
    case 16: GPR_ROWS(16); break;
    case 32: GPR_ROWS(32); break;
    default: break;
  }
#undef GPR_ROWS
}

template <typename T>
static void record_iterations(gpr_graph* g, PagerankWork* w, int32_t iters, cudaStream_t s) {
  const Plan& P = g->plan;
  float* x[2] = {(float*)w->x[0], (float*)w->x[1]};
  T* c[2] = {(T*)w->c[0], (T*)w->c[1]};
  init_kernel<T><<<w->init_shape.grid, 256, 0, s>>>(x[0], c[0], P.inv_deg, g->n, w->partials);
  fold_kernel<T><<<1, 1024, 0, s>>>(x[0], P.inv_deg, x[0], c[0], P.split_row, P.split_cbeg, P.split_cend, 0,
                                   w->chunk_sum, w->partials, w->init_shape.grid, w->prm, w->log);
  for (int32_t it = 0; it < iters; ++it) {
    const int a = it & 1, b = a ^ 1;
    for (int bi = 0; bi < P.nbuckets; ++bi) {
      const Bucket& bk = P.bucket[bi];
      double* part = w->partials + 3 * (int64_t)w->shape[bi].partial_off;
      if (bk.lanes == 0) {
        chunks_kernel<T><<<w->shape[bi].grid, 256, 0, s>>>(P.row_idx, c[a], x[a], P.inv_deg, x[b], c[b],
                                                           P.chunk_row, P.chunk_begin, P.chunk_end, P.chunk_whole,
                                                           P.nchunks, w->chunk_sum, w->prm, part);
      } else {
        launch_rows<T>(bk, w->shape[bi].grid, s, P, c[a], x[a], x[b], c[b], w->prm, part);
      }
    }
    fold_kernel<T><<<1, 1024, 0, s>>>(x[a], P.inv_deg, x[b], c[b], P.split_row, P.split_cbeg, P.split_cend,
                                     P.nsplit, w->chunk_sum, w->partials, w->npartials, w->prm,
                                     w->log + 3 * (int64_t)(it + 1));
  }
}

static PagerankWork* work_make(gpr_graph* g, cudaStream_t s) {
  PagerankWork* w = new PagerankWork();
  w->device = g->device;
  try {
    GPR_CUDA(cudaStreamCreateWithFlags(&w->cap, cudaStreamNonBlocking));
    const size_t vb = (size_t)g->n * 4;
    for (int i = 0; i < 2; ++i) {
      w->x[i] = dalloc(vb, s);
      w->c[i] = dalloc(vb, s);
    }
    const Plan& P = g->plan;
    int off = 0;
    for (int bi = 0; bi < P.nbuckets; ++bi) {
      // grid sizes of both storage types agree (same kernels' occupancy up to
      // register use); take the FP32 ones and the max with BF16
      int g32 = grid_for_bucket<float>(P.bucket[bi], P.nchunks);
      int g16 = grid_for_bucket<__nv_bfloat16>(P.bucket[bi], P.nchunks);
      w->shape[bi].grid = std::max(g32, g16);
      w->shape[bi].partial_off = off;
      off += w->shape[bi].grid;
    }
    w->npartials = off;
    w->init_shape.grid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)g->n + 255) / 256, num_sms() * 4));
    const int32_t np = std::max(w->npartials, w->init_shape.grid);
    w->partials = (double*)dalloc((size_t)np * 3 * sizeof(double), s);
    GPR_CUDA(cudaMemsetAsync(w->partials, 0, (size_t)np * 3 * sizeof(double), s));
    w->chunk_sum = (float*)dalloc((size_t)std::max(P.nchunks, 1) * 4, s);
    w->prm = (StepParams*)dalloc(sizeof(StepParams), s);
    return w;
  } catch (...) {
    pagerank_work_free(w);
    throw;
  }
}

gpr_status run_pagerank(gpr_graph* g, double damping, int32_t iters, gpr_dtype dt, int flags, float* x_out,
                        gpr_stats* st, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g->mu);
  try {
    if (!g->work) g->work = work_make(g, s);
    PagerankWork* w = g->work;
    if (w->log_cap < iters + 1) {
      dfree(w->log, s);
      w->log = nullptr;
      w->log_cap = 0;
      const int32_t cap = std::max(iters + 1, 128);
      w->log = (double*)dalloc((size_t)cap * 3 * sizeof(double), s);
      w->log_cap = cap;
      if (w->exec) {
        cudaGraphExecDestroy(w->exec);
        w->exec = nullptr;
      }
    }
    StepParams hp{0.f, 0.f, damping, (double)g->n};
    GPR_CUDA(cudaMemcpyAsync(w->prm, &hp, sizeof hp, cudaMemcpyHostToDevice, s));
    if (!w->exec || w->exec_iters != iters || w->exec_dt != (int)dt) {
      if (w->exec) {
        cudaGraphExecDestroy(w->exec);
        w->exec = nullptr;
      }
      // the capture stream must see the allocations made on `s`
      GPR_CUDA(cudaStreamSynchronize(s));
      cudaGraph_t graph = nullptr;
      GPR_CUDA(cudaStreamBeginCapture(w->cap, cudaStreamCaptureModeThreadLocal));
      if (dt == GPR_BF16)
        record_iterations<__nv_bfloat16>(g, w, iters, w->cap);
      else
        record_iterations<float>(g, w, iters, w->cap);
      cudaError_t e = cudaStreamEndCapture(w->cap, &graph);
      if (e != cudaSuccess) throw CudaFail{e, "cudaStreamEndCapture"};
      e = cudaGraphInstantiate(&w->exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        w->exec = nullptr;
        throw CudaFail{e, "cudaGraphInstantiate"};
      }
      w->exec_iters = iters;
      w->exec_dt = (int)dt;
      w->exec_kernels = 2 + (int64_t)iters * (g->plan.nbuckets + 1);
    }
    GPR_CUDA(cudaGraphLaunch(w->exec, s));
    count_launches(w->exec_kernels);
    const void* xf = w->x[iters & 1];
    float* dst = (flags & GPR_PTR_HOST) ? nullptr : x_out;
    if (!dst) {
      if (!w->out_tmp) w->out_tmp = (float*)dalloc((size_t)g->n * 4, s);
      dst = w->out_tmp;
    }
    const int og = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)g->n + 255) / 256, num_sms() * 8));
    output_kernel<<<og, 256, 0, s>>>((const float*)xf, g->plan.old2new, g->n, dst);
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

}  // namespace gpr
