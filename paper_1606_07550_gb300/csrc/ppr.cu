// Batched personalised PageRank (section 4 Table "snap_methods" and section
// 4.3, "Fast Random Walk Algorithms": personalised PageRank scores from the
// point of view of a given node).
//
// One column per seed s with teleport vector e_s, the dangling mass of each
// column returned to its own seed:
//   x_0 = e_s,  x_{k+1}[v] = (1 - d) e_s[v] + d (sum_{u->v} x_k[u]/outdeg(u) + D_k e_s[v])
// A job is one graph with up to 64 columns, stored node-major (row p holds
// the 64 columns of node p): the pull step gathers whole 256-byte rows
// (128 bytes with BF16 contributions), one warp per row, two columns per
// lane.  Rows longer than one warp's fair share are handled by the whole
// block with a fixed-order combine.
//
// ppr_batch: each job runs on one thread-block cluster for all of its steps,
// in a per-cluster workspace.  The
// cluster's blocks split the rows by edge count; after each step they meet at
// the hardware cluster barrier, then every block folds the per-column FP64
// partials of all blocks (read through distributed shared memory) in rank
// order, so every block holds identical D, residual and stop decisions.
// Clusters pull jobs from a global queue (largest first) until it is empty:
// one persistent launch covers the whole batch.
//
// Per-column arithmetic does not depend on the other columns of a job or on
// the batch around it: a column gives the same bits alone or in any mix.
//
// Storage of the gathered contributions c = x / outdeg: FP32; FP16 times
// 2^10; or BF16 as error-feedback deltas.  With BF16, a node keeps in FP32
// the sum s of every value it has sent so far and sends q = bf16(c - s) (round
// to nearest), then s += q; a row keeps in FP32 the running sum y of the
// q it has gathered, so that y is the sum of its in-neighbours' s.  Each s
// differs from the exact c by one rounding of the last difference c - s,
// which shrinks with the step-to-step change of x: the rounding of one step
// is corrected by the next instead of staying in the result.  The state per
// node and column is y and s (FP32); x is not stored: x = d y + b at the
// seed row (d y elsewhere), b the step's seed coefficient, kept per column;
// the gathers read 2 bytes.
#include <cooperative_groups.h>

#include <algorithm>
#include <climits>
#include <cstdlib>
#include <map>
#include <mutex>
#include <numeric>
#include <type_traits>
#include <vector>

#include <cuda_fp16.h>

#include "gpr_internal.cuh"
#include "ppr_internal.cuh"

namespace cg = cooperative_groups;

namespace gpr {

constexpr int kPprThreads = 1024;
constexpr int kPprWarps = kPprThreads / 32;

// FP16 contributions are stored times 2^10 (values of a personalised column
// lie in [0, 1], so they stay below 1024 and far above the subnormal range
// for any contribution that matters); the power-of-two scale adds no rounding.
constexpr float kHalfScale = 1024.0f;
constexpr float kHalfUnscale = 1.0f / 1024.0f;

__device__ __forceinline__ float2 ld_pair(const float* p) { return __ldcg(reinterpret_cast<const float2*>(p)); }
__device__ __forceinline__ float2 ld_pair(const __half* p) {
  const unsigned int u = __ldcg(reinterpret_cast<const unsigned int*>(p));
  const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&u));
  return make_float2(f.x * kHalfUnscale, f.y * kHalfUnscale);
}
__device__ __forceinline__ float2 ld_pair(const __nv_bfloat16* p) {
  const unsigned int u = __ldcg(reinterpret_cast<const unsigned int*>(p));
  __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&u);
  return __bfloat1622float2(b);
}
__device__ __forceinline__ void st_pair(float* p, float a, float b, uint32_t) {
  *reinterpret_cast<float2*>(p) = make_float2(a, b);
}
__device__ __forceinline__ void st_pair(__half* p, float a, float b, uint32_t) {
  *reinterpret_cast<__half2*>(p) = __floats2half2_rn(a * kHalfScale, b * kHalfScale);
}
template <typename T>
__device__ __forceinline__ void st_one(T* p, float a);
template <>
__device__ __forceinline__ void st_one<float>(float* p, float a) {
  *p = a;
}
template <>
__device__ __forceinline__ void st_one<__nv_bfloat16>(__nv_bfloat16* p, float a) {
  *p = __float2bfloat16_rn(a);
}
template <>
__device__ __forceinline__ void st_one<__half>(__half* p, float a) {
  *p = __float2half_rn(a * kHalfScale);
}

// Sum of the contribution rows of the sources of edges [e0, e1), two columns
// per lane.  Warp-cooperative: all lanes call it with the same range; each
// group of 32 indices is loaded once, coalesced, and broadcast by shuffles.
// A lane whose two columns are not running (on = false) loads nothing: the
// sectors of a row's dead columns are then not fetched at all.
template <typename T>
__device__ __forceinline__ float2 gather_row(const int32_t* __restrict__ row_idx, const T* __restrict__ C,
                                             int32_t e0, int32_t e1, int lane, bool on = true) {
  float ax = 0.f, ay = 0.f;
  for (int32_t e = e0; e < e1; e += 32) {
    const int32_t idx = (e + lane < e1) ? __ldcs(row_idx + e + lane) : 0;
    const int cnt = min(32, e1 - e);
    int j = 0;
    // eight 256-byte row gathers in flight per warp (128 bytes with 16-bit
    // storage); whole groups unmasked, then the tail in a group of eight or,
    // for at most four edges (most rows of a power-law graph), of four
    for (; j + 8 <= cnt; j += 8) {
      float2 v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int32_t u = __shfl_sync(0xffffffffu, idx, j + q);
        v[q] = on ? ld_pair(C + (int64_t)u * kPprCols + 2 * lane) : make_float2(0.f, 0.f);
      }
      ax += ((v[0].x + v[1].x) + (v[2].x + v[3].x)) + ((v[4].x + v[5].x) + (v[6].x + v[7].x));
      ay += ((v[0].y + v[1].y) + (v[2].y + v[3].y)) + ((v[4].y + v[5].y) + (v[6].y + v[7].y));
    }
    if (cnt - j > 4) {
      float2 v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int32_t u = __shfl_sync(0xffffffffu, idx, (j + q) & 31);
        v[q] = (on && j + q < cnt) ? ld_pair(C + (int64_t)u * kPprCols + 2 * lane) : make_float2(0.f, 0.f);
      }
      ax += ((v[0].x + v[1].x) + (v[2].x + v[3].x)) + ((v[4].x + v[5].x) + (v[6].x + v[7].x));
      ay += ((v[0].y + v[1].y) + (v[2].y + v[3].y)) + ((v[4].y + v[5].y) + (v[6].y + v[7].y));
    } else if (cnt - j > 0) {
      float2 v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int32_t u = __shfl_sync(0xffffffffu, idx, (j + q) & 31);
        v[q] = (on && j + q < cnt) ? ld_pair(C + (int64_t)u * kPprCols + 2 * lane) : make_float2(0.f, 0.f);
      }
      ax += (v[0].x + v[1].x) + (v[2].x + v[3].x);
      ay += (v[0].y + v[1].y) + (v[2].y + v[3].y);
    }
  }
  return make_float2(ax, ay);
}

struct ColRegs {
  float a0, a1;      // d of the two columns
  float b0, b1;      // seed coefficient (1 - d) + d D
  int32_t s0, s1;    // relabelled seed rows
  bool l0, l1;       // live
  float bp0, bp1;    // seed coefficient of the previous step (BF16 deltas: x of the previous step)
};

// The row's previous state: loaded before the gathers so its latency overlaps them.
__device__ __forceinline__ float2 ld_state(const float* X, int32_t p, int lane) {
  return *reinterpret_cast<const float2*>(X + (int64_t)p * kPprCols + 2 * lane);
}
// BF16 deltas: the row's running sums (y0, y1) and sent sums (s0, s1) of the
// lane's two columns, one 16-byte record per lane (null for other storage).
__device__ __forceinline__ float4 ld_ys(const float4* YS, int32_t p, int lane) {
  return YS ? YS[(int64_t)p * 32 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
}
__device__ __forceinline__ uint32_t bf16_bits_rn(float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  return (uint32_t)*reinterpret_cast<const uint16_t*>(&h);
}
__device__ __forceinline__ float bf16_bits_to_float(uint32_t b) { return __uint_as_float(b << 16); }

template <typename T>
__device__ __forceinline__ void finish_ppr_row(int32_t p, float2 y, float2 xo, float4 ys, const ColRegs& c,
                                               float* __restrict__ X, float4* __restrict__ YS,
                                               T* __restrict__ Cout, const float* __restrict__ inv_deg, int lane,
                                               float (&acc)[2][3]) {
  const float inv = inv_deg[p];
  constexpr bool kDelta = std::is_same<T, __nv_bfloat16>::value;
  float n0, n1;
  if constexpr (kDelta) {
    // y holds this step's gathered deltas: add the running sums; x of the
    // previous step from the previous running sums and seed coefficient
    const float y0 = ys.x + y.x, y1 = ys.y + y.y;
    xo.x = fmaf(c.a0, ys.x, p == c.s0 ? c.bp0 : 0.f);
    xo.y = fmaf(c.a1, ys.y, p == c.s1 ? c.bp1 : 0.f);
    n0 = fmaf(c.a0, y0, p == c.s0 ? c.b0 : 0.f);
    n1 = fmaf(c.a1, y1, p == c.s1 ? c.b1 : 0.f);
    // the new contributions as deltas against what was sent (0 for columns
    // that are not running)
    const uint32_t q0 = c.l0 ? bf16_bits_rn(n0 * inv - ys.z) : 0u;
    const uint32_t q1 = c.l1 ? bf16_bits_rn(n1 * inv - ys.w) : 0u;
    YS[(int64_t)p * 32 + lane] = make_float4(c.l0 ? y0 : ys.x, c.l1 ? y1 : ys.y, ys.z + bf16_bits_to_float(q0),
                                             ys.w + bf16_bits_to_float(q1));
    *reinterpret_cast<uint32_t*>(Cout + (int64_t)p * kPprCols + 2 * lane) = q0 | (q1 << 16);
  } else {
    n0 = c.l0 ? fmaf(c.a0, y.x, p == c.s0 ? c.b0 : 0.f) : xo.x;
    n1 = c.l1 ? fmaf(c.a1, y.y, p == c.s1 ? c.b1 : 0.f) : xo.y;
    *reinterpret_cast<float2*>(X + (int64_t)p * kPprCols + 2 * lane) = make_float2(n0, n1);
    st_pair(Cout + (int64_t)p * kPprCols + 2 * lane, n0 * inv, n1 * inv, 0u);
  }
  acc[0][0] += n0;
  acc[1][0] += n1;
  if (inv == 0.f) {
    acc[0][1] += n0;
    acc[1][1] += n1;
  }
  acc[0][2] += fabsf(n0 - xo.x);
  acc[1][2] += fabsf(n1 - xo.y);
}

// x of column k at row p from the BF16 delta state: d y + b at the seed row.
__device__ __forceinline__ float x_from_ys(const float4* YS, int32_t p, int k, float d, int32_t seed_row, float b) {
  const float* ysf = reinterpret_cast<const float*>(YS + (int64_t)p * 32 + (k >> 1));
  return fmaf(d, ysf[k & 1], p == seed_row ? b : 0.f);
}

// A row costs three 256-byte row accesses (its state read and written, its
// contributions written) besides one gather per edge: rows are split among
// CTAs and parts by edges + kRowWeight * rows.
constexpr int64_t kRowWeight = 3;

// The first row p in [0, n] with col_ptr[p] + kRowWeight * p >= key.
__device__ __forceinline__ int32_t lower_bound_work(const int32_t* col_ptr, int32_t n, int64_t key) {
  int32_t lo = 0, hi = n;
  while (lo < hi) {
    const int32_t mid = lo + (hi - lo) / 2;
    if ((int64_t)col_ptr[mid] + kRowWeight * mid < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

__device__ __forceinline__ int32_t lower_bound_i32(const int32_t* a, int32_t n, int64_t key) {
  int32_t lo = 0, hi = n;
  while (lo < hi) {
    const int32_t mid = lo + (hi - lo) / 2;
    if ((int64_t)a[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Rows [r0, r1) split into kPprWarps contiguous ranges of about equal
// (edges + rows): warp w takes [first, last).  Deterministic, and balanced so
// that no warp holds the block at its per-step barriers.
__device__ __forceinline__ void warp_rows(const int32_t* __restrict__ col_ptr, int32_t r0, int32_t r1, int w,
                                          int32_t& first, int32_t& last) {
  const int64_t k0 = (int64_t)col_ptr[r0] + r0, k1 = (int64_t)col_ptr[r1] + r1;
  auto at = [&](int ww) -> int32_t {
    if (ww <= 0) return r0;
    if (ww >= kPprWarps) return r1;
    const int64_t target = k0 + (k1 - k0) * ww / kPprWarps;
    int32_t lo = r0, hi = r1;  // first p in [r0, r1] with col_ptr[p] + p >= target
    while (lo < hi) {
      const int32_t mid = lo + (hi - lo) / 2;
      if ((int64_t)col_ptr[mid] + mid < target)
        lo = mid + 1;
      else
        hi = mid;
    }
    return lo;
  };
  first = at(w);
  last = at(w + 1);
}

template <typename T>
__global__ void __launch_bounds__(kPprThreads, 1) ppr_kernel(PprJob* __restrict__ jobs,
                                                            const int32_t* __restrict__ order, int32_t njobs,
                                                            uint32_t* __restrict__ queue, char* __restrict__ ws,
                                                            int64_t ws_stride, int32_t cluster_size) {
  cg::cluster_group cl = cg::this_cluster();
  const int crank = (int)cl.block_rank();
  const int64_t cid = blockIdx.x / cluster_size;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  __shared__ int s_job;
  __shared__ float s_wpart[kPprWarps][3][kPprCols];
  __shared__ double s_part[2][3][kPprCols];
  __shared__ float s_heavy[kPprWarps][kPprCols];
  __shared__ int32_t s_seed[kPprCols];
  __shared__ float s_d[kPprCols], s_tol[kPprCols];
  __shared__ double s_best[kPprCols];
  __shared__ int32_t s_stall[kPprCols];
  __shared__ double s_D[kPprCols], s_res[kPprCols];
  __shared__ float s_bused[kPprCols];  // seed coefficient of each column's latest step (1 before its first)
  __shared__ int32_t s_status[kPprCols], s_iters[kPprCols], s_maxit[kPprCols], s_newdone[kPprCols];

  for (;;) {
    if (crank == 0 && tid == 0) s_job = (int)atomicAdd(queue, 1u);
    cl.sync();
    const int jq = *cl.map_shared_rank(&s_job, 0);
    cl.sync();
    if (jq >= njobs) break;
    PprJob* J = &jobs[order[jq]];
    const int32_t n = J->n;
    const int32_t* __restrict__ col_ptr = J->col_ptr;
    const int32_t* __restrict__ row_idx = J->row_idx;
    const float* __restrict__ inv_deg = J->inv_deg;
    char* base = ws + cid * ws_stride;
    // workspace: x (FP32 and FP16 storage only), two contribution buffers,
    // and with BF16 deltas the running and sent sums
    constexpr bool kDelta = std::is_same<T, __nv_bfloat16>::value;
    float* X = kDelta ? nullptr : (float*)base;
    T* Cb[2];
    Cb[0] = (T*)(base + (kDelta ? 0 : (int64_t)J->n_cap * kPprCols * 4));
    Cb[1] = Cb[0] + (int64_t)J->n_cap * kPprCols;
    float4* YS = kDelta ? reinterpret_cast<float4*>(Cb[1] + (int64_t)J->n_cap * kPprCols) : nullptr;
    int parity = 0;

    // this block's rows: split by edges + kRowWeight * rows
    const int64_t work = (int64_t)col_ptr[n] + kRowWeight * n;
    auto split = [&](int r) -> int32_t {
      if (r <= 0) return 0;
      if (r >= cluster_size) return n;
      return lower_bound_work(col_ptr, n, (work * r + cluster_size - 1) / cluster_size);
    };
    const int32_t r0 = min(split(crank), n), r1 = max(r0, min(split(crank + 1), n));
    // long rows of this block: the part of the (ascending) long-row list in [r0, r1)
    const int32_t h0 = lower_bound_i32(J->heavy_rows, J->n_heavy, r0);
    const int32_t h1 = lower_bound_i32(J->heavy_rows, J->n_heavy, r1);
    const int32_t heavy_deg = J->heavy_deg;

    // column records
    if (tid < kPprCols) {
      const PprCol cr = J->cols[tid];
      s_status[tid] = cr.status;
      s_newdone[tid] = 0;
      if (cr.status == kColFresh) {
        s_seed[tid] = J->old2new[cr.seed];
        s_D[tid] = inv_deg[s_seed[tid]] == 0.f ? 1.0 : 0.0;
        s_iters[tid] = 0;
        s_res[tid] = 0.0;
        s_best[tid] = INFINITY;
        s_stall[tid] = 0;
        s_bused[tid] = 1.f;  // x_0 = e_seed
      } else {
        s_seed[tid] = cr.status == kColEmpty ? -1 : J->old2new[cr.seed];
        s_D[tid] = cr.dangling;
        s_iters[tid] = cr.iters;
        s_res[tid] = cr.residual;
        s_best[tid] = cr.best;
        s_stall[tid] = cr.stall;
        s_bused[tid] = cr.bused;
      }
      s_d[tid] = cr.damping;
      s_tol[tid] = cr.tol;
      s_maxit[tid] = cr.max_iters;
    }
    __syncthreads();
    // every column starts at e_seed in X and in the current contribution
    // buffer; the other buffer starts at 0 too (rows without in-edges are
    // never written again: their x stays 0 for every column not seeded there)
    {
      T* Cc = Cb[parity];
      T* Co = Cb[parity ^ 1];
      for (int64_t i = (int64_t)r0 * kPprCols + tid; i < (int64_t)r1 * kPprCols; i += kPprThreads) {
        if (X) X[i] = 0.f;
        st_one(Cc + i, 0.f);
        st_one(Co + i, 0.f);
      }
      if (YS)
        for (int64_t i = (int64_t)r0 * 32 + tid; i < (int64_t)r1 * 32; i += kPprThreads)
          YS[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      __syncthreads();
      if (tid < kPprCols && s_status[tid] == kColFresh) {
        const int32_t s = s_seed[tid];
        if (s >= r0 && s < r1) {
          if (X) X[(int64_t)s * kPprCols + tid] = 1.f;
          st_one(Cc + (int64_t)s * kPprCols + tid, inv_deg[s]);
          if (YS) {  // the first delta is the whole contribution: it is what has been sent
            float* ysf = reinterpret_cast<float*>(YS + (int64_t)s * 32 + (tid >> 1));
            ysf[2 + (tid & 1)] = bf16_bits_to_float(bf16_bits_rn(inv_deg[s]));
          }
        }
      }
      __syncthreads();
      if (tid < kPprCols && s_status[tid] == kColFresh) s_status[tid] = kColRunning;
      // a column with no steps to run is finished as it stands
      if (tid < kPprCols && s_status[tid] == kColRunning && s_iters[tid] >= s_maxit[tid]) {
        s_status[tid] = kColDone;
        s_newdone[tid] = 1;
      }
    }
    cl.sync();

    for (int32_t it = 0; it < J->iters; ++it) {
      // any live column left?
      const int live_any = __syncthreads_or(tid < kPprCols && s_status[tid] == kColRunning);
      if (!live_any) break;
      const T* __restrict__ Cin = Cb[parity];
      T* __restrict__ Cout = Cb[parity ^ 1];
      ColRegs c;
      {
        const int k0 = 2 * lane, k1 = 2 * lane + 1;
        c.l0 = s_status[k0] == kColRunning;
        c.l1 = s_status[k1] == kColRunning;
        c.a0 = s_d[k0];
        c.a1 = s_d[k1];
        c.b0 = (float)((1.0 - (double)s_d[k0]) + (double)s_d[k0] * s_D[k0]);
        c.b1 = (float)((1.0 - (double)s_d[k1]) + (double)s_d[k1] * s_D[k1]);
        c.s0 = s_seed[k0];
        c.s1 = s_seed[k1];
        c.bp0 = s_bused[k0];
        c.bp1 = s_bused[k1];
      }
      float acc[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
      // light rows: one warp per row, round-robin (neighbouring rows share
      // sources, so warps that walk them together share cache lines)
      // (a lane whose two columns are not running reads and writes nothing)
      const bool on = c.l0 || c.l1;
      for (int32_t p = r0 + warp; p < r1; p += kPprWarps) {
        const int32_t e0 = col_ptr[p], e1 = col_ptr[p + 1];
        if (e1 - e0 > heavy_deg) continue;
        // a row without in-edges keeps x = 0 (and contributions 0) unless it
        // is a running column's seed
        if (e0 == e1 && !__any_sync(0xffffffffu, (c.l0 && p == c.s0) || (c.l1 && p == c.s1))) continue;
        const float2 xo = on && X ? ld_state(X, p, lane) : make_float2(0.f, 0.f);
        const float4 ys = on ? ld_ys(YS, p, lane) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float2 y = gather_row(row_idx, Cin, e0, e1, lane, on);
        if (on) finish_ppr_row(p, y, xo, ys, c, X, YS, Cout, inv_deg, lane, acc);
      }
      // long rows: the whole block, fixed-order combine
      for (int32_t hi = h0; hi < h1; ++hi) {
        const int32_t p = J->heavy_rows[hi];
        const int32_t e0 = col_ptr[p], e1 = col_ptr[p + 1];
        const int32_t per = (((e1 - e0) + kPprWarps - 1) / kPprWarps + 31) & ~31;
        const int32_t a = min(e1, e0 + warp * per), b = min(e1, a + per);
        const float2 y = gather_row(row_idx, Cin, a, b, lane, on);
        s_heavy[warp][2 * lane] = y.x;
        s_heavy[warp][2 * lane + 1] = y.y;
        __syncthreads();
        if (warp == 0) {
          float yx = 0.f, yy = 0.f;
          for (int w = 0; w < kPprWarps; ++w) {
            yx += s_heavy[w][2 * lane];
            yy += s_heavy[w][2 * lane + 1];
          }
          if (on)
            finish_ppr_row(p, make_float2(yx, yy), X ? ld_state(X, p, lane) : make_float2(0.f, 0.f),
                           ld_ys(YS, p, lane), c, X, YS, Cout, inv_deg, lane, acc);
        }
        __syncthreads();
      }
      // per-column partials: FP32 per warp, FP64 across warps and blocks
      for (int v = 0; v < 3; ++v) {
        s_wpart[warp][v][2 * lane] = acc[0][v];
        s_wpart[warp][v][2 * lane + 1] = acc[1][v];
      }
      __syncthreads();
      if (tid < 3 * kPprCols) {
        const int v = tid / kPprCols, k = tid % kPprCols;
        double sum = 0.0;
        for (int w = 0; w < kPprWarps; ++w) sum += (double)s_wpart[w][v][k];
        s_part[it & 1][v][k] = sum;
      }
      cl.sync();
      if (tid < kPprCols && s_status[tid] == kColRunning) {
        double tot[3] = {0.0, 0.0, 0.0};
        for (int r = 0; r < cluster_size; ++r) {
          const double* pp = cl.map_shared_rank(&s_part[it & 1][0][0], r);
          tot[0] += pp[tid];
          tot[1] += pp[kPprCols + tid];
          tot[2] += pp[2 * kPprCols + tid];
        }
        // the seed coefficient this step used (as the step computed it), then the new D
        s_bused[tid] = (float)((1.0 - (double)s_d[tid]) + (double)s_d[tid] * s_D[tid]);
        s_D[tid] = tot[1];
        s_res[tid] = tot[2];
        const int32_t k_it = s_iters[tid] + 1;
        s_iters[tid] = k_it;
        const double d = s_d[tid];
        if (tot[2] < s_best[tid]) {
          s_best[tid] = tot[2];
          s_stall[tid] = 0;
        } else {
          ++s_stall[tid];
        }
        const bool converged =
            s_tol[tid] > 0.f && ((d / (1.0 - d)) * tot[2] <= (double)s_tol[tid] || s_stall[tid] >= kStallSteps);
        if (converged || k_it >= s_maxit[tid]) {
          s_status[tid] = kColDone;
          s_newdone[tid] = 1;
        }
      }
      parity ^= 1;
      __syncthreads();
    }

    // columns that finished in this launch: write them out by node id
    {
      const int32_t v0 = (int32_t)((int64_t)n * crank / cluster_size);
      const int32_t v1 = (int32_t)((int64_t)n * (crank + 1) / cluster_size);
      for (int k = 0; k < kPprCols; ++k) {
        if (!s_newdone[k]) continue;
        float* out = J->cols[k].out;
        const int32_t ldo = J->cols[k].ldo;
        for (int32_t v = v0 + tid; v < v1; v += kPprThreads) {
          const int32_t p = J->old2new[v];
          out[(int64_t)v * ldo] = kDelta ? x_from_ys(YS, p, k, s_d[k], s_seed[k], s_bused[k])
                                         : X[(int64_t)p * kPprCols + k];
        }
      }
    }
    if (crank == 0) {
      if (tid < kPprCols) {
        PprCol* cr = &J->cols[tid];
        cr->status = s_status[tid];
        cr->iters = s_iters[tid];
        cr->dangling = s_D[tid];
        cr->residual = s_res[tid];
        cr->best = s_best[tid];
        cr->stall = s_stall[tid];
        cr->bused = s_bused[tid];
      }
    }
    cl.sync();  // the workspace and s_job are reused by the next job
  }
}

// ---- step-major kernel (the server) ------------------------------------------
//
// One launch = one step of every (slot, part) item.  Launch sequence of a
// tick with T steps: kStepInit (fresh columns start at e_seed; state st[0]),
// kStepRun with step = 1..T (fold the previous step's part sums in part
// order, decide stops, then pull), kStepFinish (fold step T, write the
// records).  Run step s reads st[(s-1)&1] and psum[(s-1)&1] and writes
// st[s&1] and psum[s&1]; every part of a slot computes the same decisions and
// only part 0 writes them.  A finished column is written out, by node id,
// by every part for its own rows, at the launch that detects it.

template <typename T>
__global__ void __launch_bounds__(kPprThreads, 1) ppr_step_kernel(const SlotDesc* __restrict__ slots,
                                                                 const StepItem* __restrict__ items, int32_t nitems,
                                                                 int mode, int32_t step) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  __shared__ float s_wpart[kPprWarps][3][kPprCols];
  __shared__ int32_t s_seed[kPprCols], s_status[kPprCols], s_iters[kPprCols], s_newdone[kPprCols];
  __shared__ float s_d[kPprCols];
  __shared__ double s_D[kPprCols];
  __shared__ float s_bprev[kPprCols];  // seed coefficient of each column's previous step
  const int cur = step & 1, prev = cur ^ 1;
  for (int32_t ii = blockIdx.x; ii < nitems; ii += gridDim.x) {
    const StepItem item = items[ii];
    const SlotDesc* S = slots + item.slot;
    const int32_t r0 = S->part_rows[item.part], r1 = S->part_rows[item.part + 1];
    const float* __restrict__ inv_deg = S->inv_deg;
    constexpr bool kDelta = std::is_same<T, __nv_bfloat16>::value;
    float* X = kDelta ? nullptr : S->X;
    float4* YS = kDelta ? S->YS : nullptr;

    // ---- column state for this launch
    if (tid < kPprCols) {
      const PprCol cr = S->rec[tid];
      const int32_t seed_row = cr.status == kColEmpty ? -1 : S->old2new[cr.seed];
      s_seed[tid] = seed_row;
      s_d[tid] = cr.damping;
      int32_t status, iters, stall;
      double D, res, best;
      float bprev;  // seed coefficient of the column's latest executed step (1 before its first)
      int newdone = 0;
      if (mode == kStepInit) {
        status = cr.status;
        iters = cr.iters;
        D = cr.dangling;
        res = cr.residual;
        best = cr.best;
        stall = cr.stall;
        bprev = cr.bused;
        if (status == kColFresh) {
          bprev = 1.f;
          status = kColRunning;
          iters = 0;
          res = 0.0;
          best = INFINITY;
          stall = 0;
          D = inv_deg[seed_row] == 0.f ? 1.0 : 0.0;
          if (iters >= cr.max_iters) {
            status = kColDone;
            newdone = 1;
          }
        }
      } else {
        const ColState cs = S->st[prev][tid];
        status = cs.status;
        iters = cs.iters;
        D = cs.dangling;
        res = cs.residual;
        best = cs.best;
        stall = cs.stall;
        bprev = cs.bused;
        const bool fold = mode == kStepFinish || step > 1;
        if (fold && status == kColRunning) {
          double dsum = 0.0, rsum = 0.0;
          const double* ps = S->psum[prev];
          for (int32_t q = 0; q < S->nparts; ++q) {
            dsum += ps[(3 * q + 1) * kPprCols + tid];
            rsum += ps[(3 * q + 2) * kPprCols + tid];
          }
          D = dsum;
          res = rsum;
          iters += 1;
          const double d = cr.damping;
          if (rsum < best) {
            best = rsum;
            stall = 0;
          } else {
            ++stall;
          }
          if ((cr.tol > 0.f && ((d / (1.0 - d)) * rsum <= (double)cr.tol || stall >= kStallSteps)) ||
              iters >= cr.max_iters) {
            status = kColDone;
            newdone = 1;
          }
        }
      }
      s_status[tid] = status;
      s_iters[tid] = iters;
      s_D[tid] = D;
      s_newdone[tid] = newdone;
      s_bprev[tid] = bprev;
      // the seed coefficient this launch's step uses (as ColRegs computes it), if it runs one
      const float bnow = (mode == kStepRun && status == kColRunning)
                             ? (float)((1.0 - (double)cr.damping) + (double)cr.damping * D)
                             : bprev;
      if (item.part == 0) {
        if (mode == kStepFinish) {
          PprCol* w = S->rec + tid;
          w->status = status;
          w->iters = iters;
          w->dangling = D;
          w->residual = res;
          w->best = best;
          w->stall = stall;
          w->bused = bprev;
        } else {
          S->st[mode == kStepInit ? 0 : cur][tid] = ColState{status, iters, D, res, best, stall, bnow};
        }
      }
    }
    __syncthreads();

    // ---- fresh columns start at e_seed (X and the current contributions)
    if (mode == kStepInit) {
      // one pass over the part's rows: every fresh column of a row at once;
      // the other contribution buffer starts at 0 too (rows without in-edges
      // are skipped by the steps: their x stays 0 unless seeded there)
      T* Cc = (T*)S->C[S->parity];
      T* Co = (T*)S->C[S->parity ^ 1];
      const int k0 = 2 * lane, k1 = 2 * lane + 1;
      const bool f0 = S->rec[k0].status == kColFresh, f1 = S->rec[k1].status == kColFresh;
      const int32_t sr0 = s_seed[k0], sr1 = s_seed[k1];
      if (__any_sync(0xffffffffu, f0 || f1)) {
        for (int32_t p = r0 + warp; p < r1; p += kPprWarps) {
          const float idg = inv_deg[p];
          const int64_t o = (int64_t)p * kPprCols;
          if (f0) {
            const float v = p == sr0 ? 1.f : 0.f;
            if (X) X[o + k0] = v;
            st_one(Cc + o + k0, v * idg);
            st_one(Co + o + k0, 0.f);
          }
          if (f1) {
            const float v = p == sr1 ? 1.f : 0.f;
            if (X) X[o + k1] = v;
            st_one(Cc + o + k1, v * idg);
            st_one(Co + o + k1, 0.f);
          }
          if (YS) {  // running sums 0; sent sums = the first delta (the whole contribution)
            float4 r = YS[(int64_t)p * 32 + lane];
            if (f0) {
              r.x = 0.f;
              r.z = p == sr0 ? bf16_bits_to_float(bf16_bits_rn(idg)) : 0.f;
            }
            if (f1) {
              r.y = 0.f;
              r.w = p == sr1 ? bf16_bits_to_float(bf16_bits_rn(idg)) : 0.f;
            }
            YS[(int64_t)p * 32 + lane] = r;
          }
        }
      }
      __syncthreads();
    }

    // ---- columns finished by now: this part's rows go out by node id, in
    // one pass over the rows (a warp per row, two columns per lane)
    {
      const int k0 = 2 * lane, k1 = 2 * lane + 1;
      const bool d0 = s_newdone[k0] != 0, d1 = s_newdone[k1] != 0;
      if (__any_sync(0xffffffffu, d0 || d1)) {
        float* o0 = d0 ? S->rec[k0].out : nullptr;
        float* o1 = d1 ? S->rec[k1].out : nullptr;
        const int64_t l0 = d0 ? S->rec[k0].ldo : 0, l1 = d1 ? S->rec[k1].ldo : 0;
        for (int32_t p = r0 + warp; p < r1; p += kPprWarps) {
          const int64_t v = S->new2old[p];
          float2 x;
          if (kDelta)  // x of the column's last step from its running sums
            x = make_float2(x_from_ys(YS, p, k0, s_d[k0], s_seed[k0], s_bprev[k0]),
                            x_from_ys(YS, p, k1, s_d[k1], s_seed[k1], s_bprev[k1]));
          else
            x = ld_state(X, p, lane);
          if (d0) o0[v * l0] = x.x;
          if (d1) o1[v * l1] = x.y;
        }
      }
    }

    if (mode == kStepRun) {
      const T* __restrict__ Cin = (const T*)S->C[(S->parity + step - 1) & 1];
      T* __restrict__ Cout = (T*)S->C[(S->parity + step) & 1];
      const int32_t* __restrict__ col_ptr = S->col_ptr;
      const int32_t* __restrict__ row_idx = S->row_idx;
      ColRegs c;
      {
        const int k0 = 2 * lane, k1 = 2 * lane + 1;
        c.l0 = s_status[k0] == kColRunning;
        c.l1 = s_status[k1] == kColRunning;
        c.a0 = s_d[k0];
        c.a1 = s_d[k1];
        c.b0 = (float)((1.0 - (double)s_d[k0]) + (double)s_d[k0] * s_D[k0]);
        c.b1 = (float)((1.0 - (double)s_d[k1]) + (double)s_d[k1] * s_D[k1]);
        c.s0 = s_seed[k0];
        c.s1 = s_seed[k1];
        c.bp0 = s_bprev[k0];
        c.bp1 = s_bprev[k1];
      }
      float acc[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
      const int32_t heavy_deg = S->heavy_deg;
      int32_t wr0, wr1;
      warp_rows(col_ptr, r0, r1, warp, wr0, wr1);
      // (a lane whose two columns are not running reads and writes nothing:
      // a part-filled slot moves only the sectors of its running columns)
      const bool on = c.l0 || c.l1;
      for (int32_t p = wr0; p < wr1; ++p) {
        const int32_t e0 = col_ptr[p], e1 = col_ptr[p + 1];
        if (e1 - e0 > heavy_deg) continue;
        // a row without in-edges keeps x = 0 (and contributions 0) unless it
        // is a running column's seed
        if (e0 == e1 && !__any_sync(0xffffffffu, (c.l0 && p == c.s0) || (c.l1 && p == c.s1))) continue;
        const float2 xo = on && X ? ld_state(X, p, lane) : make_float2(0.f, 0.f);
        const float4 ys = on ? ld_ys(YS, p, lane) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float2 y = gather_row(row_idx, Cin, e0, e1, lane, on);
        if (on) finish_ppr_row(p, y, xo, ys, c, X, YS, Cout, inv_deg, lane, acc);
      }
      // long rows: their chunk sums (this step's chunk launch), in chunk
      // order, a warp per row
      const int32_t h0 = lower_bound_i32(S->heavy_rows, S->n_heavy, r0);
      const int32_t h1 = lower_bound_i32(S->heavy_rows, S->n_heavy, r1);
      for (int32_t hi = h0 + warp; on && hi < h1; hi += kPprWarps) {
        const int32_t p = S->heavy_rows[hi];
        const int32_t sp = S->heavy_split0 + hi;
        float yx = 0.f, yy = 0.f;
        for (int pass = 0; pass < 2; ++pass) {
          const int32_t c0 = pass == 0 ? S->split_hbeg[sp] : S->split_cbeg[sp];
          const int32_t c1 = pass == 0 ? S->split_hend[sp] : S->split_cend[sp];
          for (int32_t c = c0; c < c1; ++c) {
            const float2 v = __ldcg(reinterpret_cast<const float2*>(S->chunk_sum + (int64_t)c * kPprCols) + lane);
            yx += v.x;
            yy += v.y;
          }
        }
        finish_ppr_row(p, make_float2(yx, yy), X ? ld_state(X, p, lane) : make_float2(0.f, 0.f), ld_ys(YS, p, lane),
                       c, X, YS, Cout, inv_deg, lane, acc);
      }
      for (int v = 0; v < 3; ++v) {
        s_wpart[warp][v][2 * lane] = acc[0][v];
        s_wpart[warp][v][2 * lane + 1] = acc[1][v];
      }
      __syncthreads();
      if (tid < 3 * kPprCols) {
        const int v = tid / kPprCols, k = tid % kPprCols;
        double sum = 0.0;
        for (int w = 0; w < kPprWarps; ++w) sum += (double)s_wpart[w][v][k];
        S->psum[cur][(3 * (int64_t)item.part + v) * kPprCols + k] = sum;
      }
    }
    __syncthreads();  // shared state is reused by the next item
  }
}

// Long-row chunk sums of one step: item (slot, q) covers chunks
// [q * kChunksPerItem, (q + 1) * kChunksPerItem) of the slot's plan; a warp
// gathers a chunk's edges for all 64 columns.
template <typename T>
__global__ void __launch_bounds__(kPprThreads, 1) ppr_chunk_kernel(const SlotDesc* __restrict__ slots,
                                                                  const StepItem* __restrict__ items, int32_t nitems,
                                                                  int32_t step) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int32_t ii = blockIdx.x; ii < nitems; ii += gridDim.x) {
    const StepItem item = items[ii];
    const SlotDesc* S = slots + item.slot;
    const T* __restrict__ Cin = (const T*)S->C[(S->parity + step - 1) & 1];
    const int32_t c_end = min(S->nchunks, (item.part + 1) * kChunksPerItem);
    // columns running after the previous step (the step launch may still stop
    // some of them; their sums then go unused)
    const ColState* stp = S->st[(step - 1) & 1];
    const bool on = stp[2 * lane].status == kColRunning || stp[2 * lane + 1].status == kColRunning;
    for (int32_t ch = item.part * kChunksPerItem + warp; ch < c_end; ch += kPprWarps) {
      const float2 y = gather_row(S->row_idx, Cin, S->chunk_begin[ch], S->chunk_end[ch], lane, on);
      reinterpret_cast<float2*>(S->chunk_sum + (int64_t)ch * kPprCols)[lane] = y;
    }
  }
}

__global__ void part_bounds_kernel(const int32_t* __restrict__ col_ptr, int32_t n, int64_t m, int32_t nparts,
                                   int32_t* __restrict__ part_rows) {
  for (int32_t i = blockIdx.x * blockDim.x + threadIdx.x; i <= nparts; i += gridDim.x * blockDim.x) {
    if (i == 0) {
      part_rows[i] = 0;
    } else if (i == nparts) {
      part_rows[i] = n;
    } else {
      const int64_t work = m + kRowWeight * n;  // edges + kRowWeight * rows
      const int64_t target = (work * i + nparts - 1) / nparts;
      part_rows[i] = min(n, lower_bound_work(col_ptr, n, target));
    }
  }
}

// ---- host side ----------------------------------------------------------------

template <typename T>
static int max_clusters_for(int cluster) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(cluster * 64, 1, 1);
  cfg.blockDim = dim3(kPprThreads, 1, 1);
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int num = 0;
  if (cudaOccupancyMaxActiveClusters(&num, ppr_kernel<T>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return num;
}

void ppr_part_bounds(const int32_t* col_ptr, int32_t n, int64_t m, int32_t nparts, int32_t* part_rows,
                     cudaStream_t s) {
  part_bounds_kernel<<<std::max(1, (nparts + 256) / 256), 256, 0, s>>>(col_ptr, n, m, nparts, part_rows);
  GPR_CUDA(cudaGetLastError());
  count_launches(1);
}

template <typename T>
static int step_grid(int32_t nitems) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ppr_step_kernel<T>, kPprThreads, 0);
  return std::max(1, std::min(nitems, num_sms() * std::max(per_sm, 1)));
}

void ppr_step_launch(const SlotDesc* slots_dev, const StepItem* items_dev, int32_t nitems, int mode, int32_t step,
                     gpr_dtype dt, cudaStream_t s) {
  if (nitems <= 0) return;
  if (dt == GPR_BF16)
    ppr_step_kernel<__nv_bfloat16><<<step_grid<__nv_bfloat16>(nitems), kPprThreads, 0, s>>>(slots_dev, items_dev,
                                                                                          nitems, mode, step);
  else if (dt == GPR_FP16)
    ppr_step_kernel<__half><<<step_grid<__half>(nitems), kPprThreads, 0, s>>>(slots_dev, items_dev, nitems, mode, step);
  else
    ppr_step_kernel<float><<<step_grid<float>(nitems), kPprThreads, 0, s>>>(slots_dev, items_dev, nitems, mode, step);
  GPR_CUDA(cudaGetLastError());
  count_launches(1);
}

template <typename T>
static int chunk_grid(int32_t nitems) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ppr_chunk_kernel<T>, kPprThreads, 0);
  return std::max(1, std::min(nitems, num_sms() * std::max(per_sm, 1)));
}

void ppr_chunk_launch(const SlotDesc* slots_dev, const StepItem* items_dev, int32_t nitems, int32_t step,
                      gpr_dtype dt, cudaStream_t s) {
  if (nitems <= 0) return;
  if (dt == GPR_BF16)
    ppr_chunk_kernel<__nv_bfloat16><<<chunk_grid<__nv_bfloat16>(nitems), kPprThreads, 0, s>>>(slots_dev, items_dev,
                                                                                            nitems, step);
  else if (dt == GPR_FP16)
    ppr_chunk_kernel<__half><<<chunk_grid<__half>(nitems), kPprThreads, 0, s>>>(slots_dev, items_dev, nitems, step);
  else
    ppr_chunk_kernel<float><<<chunk_grid<float>(nitems), kPprThreads, 0, s>>>(slots_dev, items_dev, nitems, step);
  GPR_CUDA(cudaGetLastError());
  count_launches(1);
}


static int max_clusters(gpr_dtype dt, int cluster) {
  if (dt == GPR_BF16) return max_clusters_for<__nv_bfloat16>(cluster);
  if (dt == GPR_FP16) return max_clusters_for<__half>(cluster);
  return max_clusters_for<float>(cluster);
}

static void ppr_launch(PprJob* jobs_dev, const int32_t* order_dev, int32_t njobs, uint32_t* queue_dev, char* ws,
                       int64_t ws_stride, int clusters, int cluster, gpr_dtype dt, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(clusters * cluster), 1, 1);
  cfg.blockDim = dim3(kPprThreads, 1, 1);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e;
  if (dt == GPR_BF16)
    e = cudaLaunchKernelEx(&cfg, ppr_kernel<__nv_bfloat16>, jobs_dev, order_dev, njobs, queue_dev, ws, ws_stride,
                           cluster);
  else if (dt == GPR_FP16)
    e = cudaLaunchKernelEx(&cfg, ppr_kernel<__half>, jobs_dev, order_dev, njobs, queue_dev, ws, ws_stride, cluster);
  else
    e = cudaLaunchKernelEx(&cfg, ppr_kernel<float>, jobs_dev, order_dev, njobs, queue_dev, ws, ws_stride, cluster);
  if (e != cudaSuccess) throw CudaFail{e, "cudaLaunchKernelEx(ppr_kernel)"};
  count_launches(1);
}

// ---- graph-size classes and the cluster-shape autotuner ---------------------
// A job's graph falls in class k by ceil(log2 n): <= 11, 12-13, 14-15, 16-17,
// >= 18.  Each class present in a call runs as its own persistent launch with
// its own number of CTAs per cluster: one CTA suits a small graph (its steps
// need no cluster barrier and its rows fill one CTA), eight a large one.
// ppr_tune times the shapes of a (class, storage type) on a sample of the
// class's jobs and keeps the fastest for the process; an untuned class takes
// kDefaultShape.  A column's bits depend on its class's shape (the row split
// among a cluster's CTAs orders the FP64 partial sums), not on the other
// columns or jobs of the call.
constexpr int kPprClasses = 5;
constexpr int kClusterCands[] = {1, 2, 4, 8};
constexpr int kDefaultCluster = 8;
constexpr int kDefaultShape[kPprClasses] = {4, 4, 8, 4, 4};  // measured on GB300 (R-MAT batch, FP32 and BF16)
constexpr int32_t kTuneSampleJobs = 64;
constexpr int64_t kWorkspaceBudget = (int64_t)16 << 30;  // per launch: clusters x stride at most

static int ceil_log2_n(int32_t n) {
  int lg = 0;
  while (((int64_t)1 << lg) < n) ++lg;
  return lg;
}
static int ppr_class_of(int32_t n) { return std::min(kPprClasses - 1, std::max(0, (ceil_log2_n(n) - 10) / 2)); }
static int class_log2n_max(int k) { return k == kPprClasses - 1 ? 31 : 11 + 2 * k; }

static std::mutex g_ppr_tune_mu;
static std::map<std::pair<int, int>, int> g_ppr_tuned;  // (class, dtype) -> CTAs per cluster

// GPR_PPR_CLUSTER=k (1, 2, 4 or 8) forces the shape of every class.
static int env_cluster() {
  const char* e = getenv("GPR_PPR_CLUSTER");
  if (!e) return 0;
  const int k = atoi(e);
  return (k == 1 || k == 2 || k == 4 || k == 8) ? k : 0;
}

// Bytes per workspace row (64 columns): the rank state and two contribution
// buffers, or with BF16 deltas two delta buffers and the running and sent sums.
static int64_t ws_row_bytes(gpr_dtype dt) {
  if (dt == GPR_BF16) return (int64_t)kPprCols * (2 * 2 + 8);  // two delta buffers, running and sent sums
  const int64_t tsz = dt == GPR_FP16 ? 2 : 4;
  return (int64_t)kPprCols * (4 + 2 * tsz);  // x and two contribution buffers
}

// One persistent launch over jobs_dev[order[i]], i < order.size(), whose
// graphs have at most n_cap rows; device temporaries through `alloc`.
template <typename A>
static void launch_set(PprJob* jobs_dev, const std::vector<int32_t>& order, int32_t n_cap, gpr_dtype dt,
                       int cluster, cudaStream_t s, A alloc) {
  const int32_t nj = (int32_t)order.size();
  if (nj == 0) return;
  int clusters = max_clusters(dt, cluster);
  if (clusters <= 0) throw StatusFail{GPR_ECUDA, "no thread-block cluster of the PPR kernel fits on this GPU"};
  const int64_t stride = ((int64_t)std::max(n_cap, 1) * ws_row_bytes(dt) + 255) & ~(int64_t)255;
  clusters = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)clusters, (int64_t)nj, kWorkspaceBudget / stride}));
  int32_t* order_dev = (int32_t*)alloc((size_t)nj * 4);
  uint32_t* queue = (uint32_t*)alloc(16);
  char* ws = (char*)alloc((size_t)stride * clusters);
  GPR_CUDA(cudaMemcpyAsync(order_dev, order.data(), (size_t)nj * 4, cudaMemcpyHostToDevice, s));
  GPR_CUDA(cudaMemsetAsync(queue, 0, 16, s));
  ppr_launch(jobs_dev, order_dev, nj, queue, ws, stride, clusters, cluster, dt, s);
}

// Times each cluster shape on up to kTuneSampleJobs jobs of one class
// (trial_steps steps from fresh columns) and returns the fastest; ms_out[i]
// gets candidate i's time.  The trial writes into the jobs' outputs, which
// the call's real run then overwrites.
template <typename A>
static int tune_class(const std::vector<PprJob>& dj, const std::vector<std::vector<PprCol>>& cols,
                      const std::vector<int32_t>& members, int32_t n_cap, gpr_dtype dt, int32_t trial_steps,
                      cudaStream_t s, A alloc, double* ms_out) {
  std::vector<int32_t> pick;
  const int32_t step = std::max<int32_t>(1, (int32_t)members.size() / kTuneSampleJobs);
  for (size_t i = 0; i < members.size() && (int32_t)pick.size() < kTuneSampleJobs; i += step) pick.push_back(members[i]);
  const int32_t nt = (int32_t)pick.size();
  PprCol* tcols = (PprCol*)alloc((size_t)nt * kPprCols * sizeof(PprCol));
  PprJob* tjobs = (PprJob*)alloc((size_t)nt * sizeof(PprJob));
  std::vector<PprCol> flat((size_t)nt * kPprCols);
  std::vector<PprJob> tj(nt);
  for (int32_t i = 0; i < nt; ++i) {
    tj[i] = dj[pick[i]];
    tj[i].iters = trial_steps;
    tj[i].cols = tcols + (size_t)i * kPprCols;
    for (int k = 0; k < kPprCols; ++k) {
      PprCol c = cols[pick[i]][k];
      c.max_iters = std::min(c.max_iters, trial_steps);
      c.tol = 0.f;
      flat[(size_t)i * kPprCols + k] = c;
    }
  }
  GPR_CUDA(cudaMemcpyAsync(tjobs, tj.data(), (size_t)nt * sizeof(PprJob), cudaMemcpyHostToDevice, s));
  std::vector<int32_t> order(nt);
  std::iota(order.begin(), order.end(), 0);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  GPR_CUDA(cudaEventCreate(&e0));
  GPR_CUDA(cudaEventCreate(&e1));
  int best = kDefaultCluster;
  float best_ms = 0.f;
  try {
    for (int ci = 0; ci < 4; ++ci) {
      const int cl = kClusterCands[ci];
      float ms = 0.f;
      for (int rep = 0; rep < 2; ++rep) {  // the first run warms the caches
        GPR_CUDA(cudaMemcpyAsync(tcols, flat.data(), flat.size() * sizeof(PprCol), cudaMemcpyHostToDevice, s));
        GPR_CUDA(cudaEventRecord(e0, s));
        launch_set(tjobs, order, n_cap, dt, cl, s, alloc);
        GPR_CUDA(cudaEventRecord(e1, s));
        GPR_CUDA(cudaStreamSynchronize(s));
        GPR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      }
      ms_out[ci] = ms;
      if (ci == 0 || ms < best_ms) {
        best = cl;
        best_ms = ms;
      }
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

// The batch: one device job per 64 columns, grouped by class, each class
// one launch with its shape; with tune_all, each class's shape is timed and
// kept instead (nothing else runs).
static gpr_status run_ppr(const gpr_ppr_job* jobs, int32_t num_jobs, int32_t max_iters, double tol, gpr_dtype dt,
                          cudaStream_t s, bool tune_all, int32_t trial_steps, gpr_ppr_tune_result* tres) {
  std::vector<void*> tmp;
  auto T = [&](size_t bytes) {
    void* p = dalloc(bytes, s);
    tmp.push_back(p);
    return p;
  };
  try {
    std::vector<PprJob> dj;
    std::vector<std::vector<PprCol>> cols;
    std::vector<std::pair<int32_t, int32_t>> src;  // (request, first column)
    for (int32_t j = 0; j < num_jobs; ++j) {
      const gpr_graph* g = jobs[j].graph;
      for (int32_t k0 = 0; k0 < jobs[j].num_seeds; k0 += kPprCols) {
        PprJob J{};
        J.inv_deg = g->plan.inv_deg;
        J.old2new = g->plan.old2new;
        J.n = g->n;
        J.col_ptr = g->col_ptr;
        J.row_idx = g->row_idx;
        J.heavy_rows = g->plan.rows;
        J.n_heavy = 0;
        J.heavy_deg = INT_MAX;
        for (int b = 0; b < g->plan.nbuckets; ++b)
          if (g->plan.bucket[b].lanes == 0) {
            J.heavy_rows = g->plan.rows + g->plan.bucket[b].row_begin;
            J.n_heavy = g->plan.bucket[b].row_end - g->plan.bucket[b].row_begin;
            J.heavy_deg = b > 0 ? g->plan.deg_threshold[b - 1] : -1;  // bucket 0 holds every degree from 0
          }
        J.iters = max_iters;
        std::vector<PprCol> cc(kPprCols);
        for (int k = 0; k < kPprCols; ++k) {
          PprCol c{};
          const int32_t kk = k0 + k;
          if (kk < jobs[j].num_seeds) {
            c.status = kColFresh;
            c.seed = jobs[j].seeds[kk];
            c.damping = jobs[j].damping[kk];
            c.tol = (float)tol;
            c.max_iters = max_iters;
            c.out = jobs[j].x_out + kk;
            c.ldo = jobs[j].num_seeds;
          } else {
            c.status = kColEmpty;
            c.seed = 0;
            c.damping = 0.5f;
          }
          cc[k] = c;
        }
        dj.push_back(J);
        cols.push_back(cc);
        src.emplace_back(j, k0);
      }
    }
    const int32_t nj = (int32_t)dj.size();
    if (tres) *tres = gpr_ppr_tune_result{};
    if (nj == 0) return GPR_OK;
    // classes: members (largest work first) and row capacity
    std::vector<std::vector<int32_t>> members(kPprClasses);
    std::vector<int32_t> ncap(kPprClasses, 1);
    {
      std::vector<int32_t> order(nj);
      std::iota(order.begin(), order.end(), 0);
      std::vector<int64_t> work(nj);
      for (int32_t i = 0; i < nj; ++i) {
        const gpr_graph* g = jobs[src[i].first].graph;
        work[i] = g->m + g->n;
      }
      std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return work[a] > work[b]; });
      for (int32_t i : order) {
        const int k = ppr_class_of(dj[i].n);
        members[k].push_back(i);
        ncap[k] = std::max(ncap[k], dj[i].n);
      }
    }
    for (int32_t i = 0; i < nj; ++i) dj[i].n_cap = ncap[ppr_class_of(dj[i].n)];
    PprCol* cols_dev = (PprCol*)T((size_t)nj * kPprCols * sizeof(PprCol));
    std::vector<PprCol> flat((size_t)nj * kPprCols);
    for (int32_t i = 0; i < nj; ++i)
      std::copy(cols[i].begin(), cols[i].end(), flat.begin() + (size_t)i * kPprCols);
    for (int32_t i = 0; i < nj; ++i) dj[i].cols = cols_dev + (size_t)i * kPprCols;
    PprJob* jobs_dev = (PprJob*)T((size_t)nj * sizeof(PprJob));
    GPR_CUDA(cudaMemcpyAsync(jobs_dev, dj.data(), (size_t)nj * sizeof(PprJob), cudaMemcpyHostToDevice, s));
    // the shape of each class
    const int forced = env_cluster();
    int shape[kPprClasses];
    for (int k = 0; k < kPprClasses; ++k) {
      shape[k] = kDefaultShape[k];
      if (members[k].empty()) continue;
      const std::pair<int, int> key(k, (int)dt);
      {
        std::lock_guard<std::mutex> lk(g_ppr_tune_mu);
        auto it = g_ppr_tuned.find(key);
        if (it != g_ppr_tuned.end()) shape[k] = it->second;
      }
      if (tune_all) {
        double ms[4] = {0, 0, 0, 0};
        shape[k] = tune_class(dj, cols, members[k], ncap[k], dt, std::max(1, trial_steps), s, T, ms);
        {
          std::lock_guard<std::mutex> lk(g_ppr_tune_mu);
          g_ppr_tuned[key] = shape[k];
        }
        if (tres) {
          const int c = tres->classes++;
          tres->log2n_max[c] = class_log2n_max(k);
          tres->jobs[c] = (int32_t)members[k].size();
          tres->cluster[c] = shape[k];
          for (int ci = 0; ci < 4; ++ci) {
            if (kClusterCands[ci] == shape[k]) tres->ms[c] = ms[ci];
            if (kClusterCands[ci] == 8) tres->ms_cluster8[c] = ms[ci];
          }
        }
      }
      if (forced) shape[k] = forced;
    }
    if (tune_all) {
      GPR_CUDA(cudaStreamSynchronize(s));
      for (void* p : tmp) dfree(p, s);
      return GPR_OK;
    }
    GPR_CUDA(cudaMemcpyAsync(cols_dev, flat.data(), flat.size() * sizeof(PprCol), cudaMemcpyHostToDevice, s));
    for (int k = 0; k < kPprClasses; ++k) launch_set(jobs_dev, members[k], ncap[k], dt, shape[k], s, T);
    // per-column results back to the caller
    GPR_CUDA(cudaMemcpyAsync(flat.data(), cols_dev, flat.size() * sizeof(PprCol), cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    for (int32_t i = 0; i < nj; ++i) {
      const gpr_ppr_job& rq = jobs[src[i].first];
      for (int k = 0; k < kPprCols; ++k) {
        const int32_t kk = src[i].second + k;
        if (kk >= rq.num_seeds) break;
        const PprCol& c = flat[(size_t)i * kPprCols + k];
        if (rq.iters_out) rq.iters_out[kk] = c.iters;
        if (rq.residual_out) rq.residual_out[kk] = c.residual;
      }
    }
    for (void* p : tmp) dfree(p, s);
    return GPR_OK;
  } catch (const StatusFail& f) {
    for (void* p : tmp) dfree(p, s);
    set_error("%s: %s", tres ? "ppr_tune" : "ppr_batch", f.msg.c_str());
    return f.st;
  } catch (const CudaFail& f) {
    cudaGetLastError();
    for (void* p : tmp) dfree(p, s);
    set_error("%s: %s failed: %s", tres ? "ppr_tune" : "ppr_batch", f.what, cudaGetErrorString(f.err));
    return GPR_ECUDA;
  }
}

gpr_status run_ppr_batch(const gpr_ppr_job* jobs, int32_t num_jobs, int32_t max_iters, double tol, gpr_dtype dt,
                         cudaStream_t s) {
  return run_ppr(jobs, num_jobs, max_iters, tol, dt, s, false, 8, nullptr);
}

gpr_status run_ppr_tune(const gpr_ppr_job* jobs, int32_t num_jobs, gpr_dtype dt, int32_t trial_steps,
                        gpr_ppr_tune_result* out, cudaStream_t s) {
  gpr_ppr_tune_result local{};
  return run_ppr(jobs, num_jobs, trial_steps, 0.0, dt, s, true, trial_steps, out ? out : &local);
}

}  // namespace gpr
