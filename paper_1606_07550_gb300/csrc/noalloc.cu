// pagerank_csc_noalloc: PageRank on a CSC the caller already holds in device
// memory, for callers that cannot allocate device memory -- code that runs
// under a fixed, pre-planned memory budget (an embedded or real-time host
// that must not grow its footprint after start-up), inside allocator-free
// regions of a larger runtime, or next to an allocator it does not own.  It
// calls no cudaMalloc, cudaFree or any other allocating routine.
//
// Its scratch (the two contribution vectors, a second rank vector, per-block
// partial sums and the step coefficients) is one file-scope device array of
// kScratchBytes, which every GPU that loads the library holds until the
// process exits.  Host code cannot use the array's name as a device address:
// on the first call on each device the entry point looks the address up with
// cudaGetSymbolAddress, with that device current, and passes it to the
// kernels.  Do that first call before any stream capture.  All calls share
// the one array and it keeps the last call's contents: each call clears what
// must start at zero, and calls whose kernels overlap on the GPU race.
#include <algorithm>
#include <mutex>

#include "gpr_internal.cuh"

namespace gpr {
namespace {

constexpr int32_t kNoallocMaxNodes = 1 << 21;
constexpr int kNoallocMaxBlocks = 2048;
constexpr int kNoallocThreads = 256;

struct NoallocState {
  float coefA, coefB;
  double d, n;
  unsigned int arrive;
  unsigned int pad;
};

// c[2][kNoallocMaxNodes] floats | x[kNoallocMaxNodes] floats | partials (mass,
// dangling mass per block) | state
constexpr size_t kVecBytes = (size_t)kNoallocMaxNodes * 4;
constexpr size_t kPartialBytes = (size_t)kNoallocMaxBlocks * 2 * sizeof(double);
constexpr size_t kScratchBytes = 3 * kVecBytes + kPartialBytes + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

__device__ __forceinline__ float nz_warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One step (mode 1) or the initial vector (mode 0) with one warp per row;
// the last block to finish folds the block partials in index order and
// writes the next step's coefficients.  The mass and dangling-mass partials
// are summed in FP64 throughout (per warp, per block, then across blocks),
// as the FP64 reductions of the main PageRank step are.
__global__ void __launch_bounds__(kNoallocThreads) noalloc_step_kernel(
    const int32_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx, const int32_t* __restrict__ outdeg,
    int32_t n, int mode, const float* __restrict__ c_in, float* __restrict__ c_out, float* __restrict__ x_out,
    double* __restrict__ partials, NoallocState* __restrict__ st) {
  __shared__ double s[2][kNoallocThreads / 32];
  __shared__ bool s_last;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const float A = st->coefA, B = st->coefB;
  double mass = 0.0, dang = 0.0;  // lane 0 of each warp finishes its rows
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t r = warp; r < n; r += nwarps) {
    float xs;
    if (mode == 0) {
      xs = 1.0f / (float)n;
    } else {
      float y = 0.f;
      for (int32_t e = col_ptr[r] + lane; e < col_ptr[r + 1]; e += 32) y += c_in[row_idx[e]];
      xs = fmaf(A, nz_warp_sum(y), B);
    }
    if (lane == 0) {
      const int32_t od = outdeg[r];
      x_out[r] = xs;
      c_out[r] = od > 0 ? xs / (float)od : 0.f;
      mass += (double)xs;
      if (od == 0) dang += (double)xs;
    }
  }
  if (lane == 0) {
    s[0][w] = mass;
    s[1][w] = dang;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int i = 0; i < kNoallocThreads / 32; ++i) {
      a += s[0][i];
      b += s[1][i];
    }
    partials[2 * blockIdx.x] = a;
    partials[2 * blockIdx.x + 1] = b;
    __threadfence();
    s_last = atomicAdd(&st->arrive, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last || threadIdx.x != 0) return;
  __threadfence();
  double total = 0, dsum = 0;
  for (unsigned int i = 0; i < gridDim.x; ++i) {
    total += __ldcg(partials + 2 * i);
    dsum += __ldcg(partials + 2 * i + 1);
  }
  st->coefA = (float)(st->d / total);
  st->coefB = (float)((1.0 - st->d) / st->n + st->d * dsum / (st->n * total));
  st->arrive = 0;
}

__global__ void noalloc_reset_kernel(NoallocState* st, double d, int32_t n) {
  st->coefA = 0.f;
  st->coefB = 0.f;
  st->d = d;
  st->n = (double)n;
  st->arrive = 0;
}

__global__ void noalloc_copy_kernel(const float* __restrict__ src, float* __restrict__ dst, int32_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {nullptr};

}  // namespace
}  // namespace gpr

using namespace gpr;

extern "C" gpr_status pagerank_csc_noalloc(const int32_t* col_ptr, const int32_t* row_idx, const int32_t* outdeg,
                                           int32_t n, double damping, int32_t iters, float* x_out, void* stream) {
  clear_error();
  if (!col_ptr || !row_idx || !outdeg || !x_out) {
    set_error("pagerank_csc_noalloc: NULL argument");
    return GPR_EINVAL;
  }
  if (n < 1 || n > kNoallocMaxNodes) {
    set_error("pagerank_csc_noalloc: n = %d outside [1, %d], the size of the static scratch", (int)n,
              (int)kNoallocMaxNodes);
    return GPR_EINVAL;
  }
  if (!(damping > 0.0 && damping < 1.0) || iters < 0 || iters > (1 << 20)) {
    set_error("pagerank_csc_noalloc: damping %g or iters %d out of range", damping, (int)iters);
    return GPR_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 64) {
    set_error("pagerank_csc_noalloc: no usable current device");
    return GPR_ECUDA;
  }
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      // the symbol's device address on the current device (first call only)
      e = cudaGetSymbolAddress(&g_noalloc_addr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_noalloc_addr[dev] = nullptr;
        set_error("pagerank_csc_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return GPR_ECUDA;
      }
    }
    base = g_noalloc_addr[dev];
  }
  unsigned char* b = (unsigned char*)base;
  float* c[2] = {(float*)b, (float*)(b + kVecBytes)};
  float* x_tmp = (float*)(b + 2 * kVecBytes);
  double* partials = (double*)(b + 3 * kVecBytes);
  NoallocState* st = (NoallocState*)(b + 3 * kVecBytes + kPartialBytes);
  float* x[2] = {x_out, x_tmp};
  cudaStream_t s = (cudaStream_t)stream;
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>({((int64_t)n * 32 + kNoallocThreads - 1) / kNoallocThreads, (int64_t)num_sms() * 8,
                            (int64_t)kNoallocMaxBlocks}));
  noalloc_reset_kernel<<<1, 1, 0, s>>>(st, damping, n);
  noalloc_step_kernel<<<grid, kNoallocThreads, 0, s>>>(col_ptr, row_idx, outdeg, n, 0, c[1], c[0], x[0], partials,
                                                       st);
  int launches = 2;
  for (int32_t it = 0; it < iters; ++it) {
    const int a = it & 1, bb = a ^ 1;
    noalloc_step_kernel<<<grid, kNoallocThreads, 0, s>>>(col_ptr, row_idx, outdeg, n, 1, c[a], c[bb], x[bb],
                                                         partials, st);
    ++launches;
  }
  if (iters & 1) {  // the last step wrote the scratch copy
    noalloc_copy_kernel<<<grid, kNoallocThreads, 0, s>>>(x_tmp, x_out, n);
    ++launches;
  }
  e = cudaGetLastError();
  count_launches(launches);
  if (e != cudaSuccess) {
    set_error("pagerank_csc_noalloc: launch failed: %s", cudaGetErrorString(e));
    return GPR_ECUDA;
  }
  return GPR_OK;
}
