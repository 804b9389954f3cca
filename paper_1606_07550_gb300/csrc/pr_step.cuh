// Device pieces of one PageRank step shared by the pull schedule
// (pagerank.cu) and the blocked schedule (blocked.cu): the step
// coefficients, the finishing of a row, per-block partial sums and the
// deterministic fold of those partials (section 4 Table "snap_methods").
//
// A step maps the row sums y[v] = sum over in-neighbours u of c[u] to
//   x'[v] = coefB + coefA * y[v],   c'[v] = x'[v] * inv_outdeg[v]
// with coefA = d / S and coefB = (1 - d)/N + d D / (N S), where S = sum(x)
// and D = the dangling mass of x, both FP64: the step
//   x'[v] = (1 - d)/N + d (sum_{u->v} x[u]/outdeg(u) + D/N)
// applied to x / S.
#pragma once

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
__device__ __forceinline__ void store_rank(T* p, int64_t i, float v);
template <>
__device__ __forceinline__ void store_rank<float>(float* p, int64_t i, float v) {
  p[i] = v;
}
template <>
__device__ __forceinline__ void store_rank<__nv_bfloat16>(__nv_bfloat16* p, int64_t i, float v) {
  p[i] = __float2bfloat16_rn(v);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block partial of three per-thread FP32 sums: FP32 within each warp, FP64
// across warps in warp order, written to out[0..2].  Call with all threads
// of the block (at most 1024).
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
  __syncthreads();
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

// Run by every thread of the one block that arrived last in a step: folds
// the step's `npartials` block partials (mass, dangling mass, residual) in
// a fixed order (thread-strided, then a shuffle tree, then warps in order),
// logs them in log_row[0..2] and writes the next step's coefficients.
__device__ __forceinline__ void fold_step(const double* partials, int32_t npartials, StepParams* prm,
                                          double* log_row) {
  __shared__ double s[3][32];
  double a = 0, b = 0, c = 0;
  for (int32_t i = threadIdx.x; i < npartials; i += blockDim.x) {
    a += __ldcg(partials + 3 * (int64_t)i);
    b += __ldcg(partials + 3 * (int64_t)i + 1);
    c += __ldcg(partials + 3 * (int64_t)i + 2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    s[0][w] = a;
    s[1][w] = b;
    s[2][w] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
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
    // (mass is positive for PageRank; a zero vector, possible for the
    // centralities that share these kernels, stays zero)
    prm->coefA = mass > 0.0 ? (float)(d / mass) : 0.f;
    prm->coefB = (float)((1.0 - d) / n + (mass > 0.0 ? d * dang / (n * mass) : 0.0));
  }
}

}  // namespace gpr
