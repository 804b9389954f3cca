// CUDA twin of the seeded input generators (see gen.h): one thread per edge
// slot, the same counter-based bits as the host loop, so the device-made COO
// equals the host-made COO element for element.
#include <cuda_runtime.h>

#include "gen.h"
#include "rng.h"

namespace {

__global__ void uniform_kernel(uint64_t key, uint32_t n, int64_t m_raw, int32_t* src, int32_t* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m_raw;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t u, v;
    gen_uniform_edge(key, (uint64_t)i, n, &u, &v);
    src[i] = u;
    dst[i] = v;
  }
}

__global__ void rmat_kernel(uint64_t key, int scale, uint32_t n, uint32_t ta, uint32_t tab,
                            uint32_t tabc, const int32_t* perm, int64_t m_raw, int32_t* src,
                            int32_t* dst) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m_raw;
       i += (int64_t)gridDim.x * blockDim.x) {
    int32_t u, v;
    gen_rmat_edge(key, (uint64_t)i, scale, n, ta, tab, tabc, &u, &v);
    if (perm) {
      u = perm[u];
      v = perm[v];
    }
    src[i] = u;
    dst[i] = v;
  }
}

int grid_for(int64_t m) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t want = (m + 255) / 256;
  int64_t cap = (int64_t)sms * 16;
  if (want > cap) want = cap;
  if (want < 1) want = 1;
  return (int)want;
}

}  // namespace

extern "C" int gen_uniform_coo_dev(int32_t n, int64_t m_raw, uint64_t seed, int32_t* src_dev,
                                   int32_t* dst_dev, void* stream) {
  if (n <= 0 || m_raw < 0) return -1;
  if (m_raw == 0) return 0;
  uint64_t key = gen_stream_key(seed, GEN_STREAM_UNIFORM);
  uniform_kernel<<<grid_for(m_raw), 256, 0, (cudaStream_t)stream>>>(key, (uint32_t)n, m_raw,
                                                                      src_dev, dst_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : -4;
}

extern "C" int gen_rmat_coo_dev(int scale, int32_t n, int64_t m_raw, double a, double b, double c,
                                uint64_t seed, const int32_t* perm_dev, int32_t* src_dev,
                                int32_t* dst_dev, void* stream) {
  if (scale < 1 || scale > 31 || n <= 0 || m_raw < 0) return -1;
  if ((int64_t)n > ((int64_t)1 << scale)) return -1;
  uint32_t ta, tab, tabc;
  if (gen_rmat_thresholds(a, b, c, &ta, &tab, &tabc)) return -1;
  if (m_raw == 0) return 0;
  uint64_t key = gen_stream_key(seed, GEN_STREAM_RMAT);
  rmat_kernel<<<grid_for(m_raw), 256, 0, (cudaStream_t)stream>>>(
      key, scale, (uint32_t)n, ta, tab, tabc, perm_dev, m_raw, src_dev, dst_dev);
  return cudaGetLastError() == cudaSuccess ? 0 : -4;
}
