// Weakly connected components (section 4 Table "snap_methods": connected
// components; section 6 Table "exp_algs" times WCC on LiveJournal).
//
// Hook and compress on the relabelled CSC, edge directions ignored:
//   parent[p] = p;  repeat
//     hook:     for every edge (u, p): a = root(u), b = root(p); if a != b,
//               atomicMin(parent[max(a, b)], min(a, b))
//     compress: parent[p] = root(p)
//   until a hook round changes nothing.
// Parents only decrease (a node is hooked under a smaller id), so every chain
// of parents strictly decreases and every root search ends.  At the end each
// tree is one component; its label is the smallest caller id among its nodes
// (an atomicMin, order-free), so the output does not depend on the schedule.
// Edges are walked with the execution plan's layout: G lanes per row by
// in-degree bucket, and long rows as edge chunks.
#include <algorithm>

#include "gpr_internal.cuh"

namespace gpr {

__device__ __forceinline__ int32_t wcc_root(const int32_t* parent, int32_t v) {
  int32_t p = __ldcg(parent + v);
  while (p != v) {  // strictly decreasing: ends within v steps
    v = p;
    p = __ldcg(parent + v);
  }
  return v;
}

__device__ __forceinline__ bool wcc_hook(int32_t* parent, int32_t u, int32_t p) {
  const int32_t a = wcc_root(parent, u), b = wcc_root(parent, p);
  if (a == b) return false;
  atomicMin(parent + max(a, b), min(a, b));
  return true;
}

// G lanes per row over rows[i0, i1).
template <int G>
__global__ void __launch_bounds__(256) wcc_rows_kernel(const int32_t* __restrict__ col_ptr,
                                                       const int32_t* __restrict__ row_idx,
                                                       const int32_t* __restrict__ rows, int32_t i0, int32_t i1,
                                                       int32_t* __restrict__ parent, int* __restrict__ changed) {
  const int lane = threadIdx.x & 31, sub = lane & (G - 1);
  constexpr int kRowsPerWarp = 32 / G;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  bool any = false;
  for (int64_t wi = i0 + warp * kRowsPerWarp; wi < i1; wi += nwarps * kRowsPerWarp) {
    const int64_t i = wi + lane / G;
    if (i >= i1) continue;
    const int32_t p = rows[i];
    for (int32_t e = col_ptr[p] + sub; e < col_ptr[p + 1]; e += G) any |= wcc_hook(parent, row_idx[e], p);
  }
  if (__any_sync(0xffffffffu, any) && lane == 0) *changed = 1;
}

// Warp per long-row edge chunk.
__global__ void __launch_bounds__(256) wcc_chunks_kernel(const int32_t* __restrict__ row_idx,
                                                         const int32_t* __restrict__ chunk_row,
                                                         const int32_t* __restrict__ chunk_begin,
                                                         const int32_t* __restrict__ chunk_end, int32_t nchunks,
                                                         int32_t* __restrict__ parent, int* __restrict__ changed) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  bool any = false;
  for (int64_t ch = warp; ch < nchunks; ch += nwarps) {
    const int32_t p = chunk_row[ch];
    for (int32_t e = chunk_begin[ch] + lane; e < chunk_end[ch]; e += 32) any |= wcc_hook(parent, row_idx[e], p);
  }
  if (__any_sync(0xffffffffu, any) && lane == 0) *changed = 1;
}

__global__ void wcc_init_kernel(int32_t* __restrict__ parent, int32_t* __restrict__ minid, int32_t n) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    parent[v] = (int32_t)v;
    minid[v] = INT32_MAX;
  }
}

__global__ void wcc_compress_kernel(int32_t* __restrict__ parent, int32_t n) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    parent[v] = wcc_root(parent, (int32_t)v);
}

// minid[root] = the smallest caller id of the component; count the roots.
__global__ void wcc_min_kernel(const int32_t* __restrict__ parent, const int32_t* __restrict__ new2old, int32_t n,
                               int32_t* __restrict__ minid, int32_t* __restrict__ roots) {
  int32_t local = 0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t r = parent[v];  // compressed: the root
    atomicMin(minid + r, new2old[v]);
    local += r == (int32_t)v;
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  if ((threadIdx.x & 31) == 0 && local) atomicAdd(roots, local);
}

// out[caller id v] = minid[root of old2new[v]]
__global__ void wcc_label_kernel(const int32_t* __restrict__ parent, const int32_t* __restrict__ old2new,
                                 const int32_t* __restrict__ minid, int32_t n, int32_t* __restrict__ out) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    out[v] = minid[parent[old2new[v]]];
}

static int wcc_grid(int64_t items) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, (int64_t)num_sms() * 8));
}

gpr_status run_wcc(gpr_graph* g, int32_t* labels_out, int32_t* num_components, int flags, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g->mu);
  const int32_t n = g->n;
  int32_t* parent = nullptr;
  int32_t* minid = nullptr;
  int32_t* flagbuf = nullptr;  // [0] changed, [1] roots
  int32_t* out_tmp = nullptr;
  try {
    parent = (int32_t*)dalloc((size_t)n * 4, s);
    minid = (int32_t*)dalloc((size_t)n * 4, s);
    flagbuf = (int32_t*)dalloc(16, s);
    wcc_init_kernel<<<wcc_grid(n), 256, 0, s>>>(parent, minid, n);
    GPR_CUDA(cudaGetLastError());
    count_launches(1);
    const Plan& P = g->plan;
    int32_t hflag[2] = {1, 0};
    int rounds = 0;
    // at most ~log2(n) rounds in practice; the cap turns a fault in the
    // reasoning above into an error instead of a hang
    while (hflag[0] != 0 && g->m > 0) {
      if (++rounds > 4096) throw StatusFail{GPR_ETIMEOUT, "wcc: no convergence after 4096 rounds"};
      GPR_CUDA(cudaMemsetAsync(flagbuf, 0, 8, s));
      for (int bi = 0; bi < P.nbuckets; ++bi) {
        const Bucket& b = P.bucket[bi];
        const int64_t rows = b.row_end - b.row_begin;
        if (b.lanes == 0) {
          if (P.nchunks > 0) {
            wcc_chunks_kernel<<<wcc_grid((int64_t)P.nchunks * 32), 256, 0, s>>>(
                g->row_idx, P.chunk_row, P.chunk_begin, P.chunk_end, P.nchunks, parent, flagbuf);
            count_launches(1);
          }
          continue;
        }
        if (rows <= 0) continue;
        const int grid = wcc_grid(rows * b.lanes);
#define GPR_WCC_ROWS(GL)                                                                                       \
  wcc_rows_kernel<GL><<<grid, 256, 0, s>>>(g->col_ptr, g->row_idx, P.rows, b.row_begin, b.row_end, parent, \
                                           flagbuf)
        switch (b.lanes) {
          case 1: GPR_WCC_ROWS(1); break;
          case 2: GPR_WCC_ROWS(2); break;
          case 4: GPR_WCC_ROWS(4); break;
          case 8: GPR_WCC_ROWS(8); break;
          case 16: GPR_WCC_ROWS(16); break;
          default: GPR_WCC_ROWS(32); break;
        }
#undef GPR_WCC_ROWS
        count_launches(1);
      }
      wcc_compress_kernel<<<wcc_grid(n), 256, 0, s>>>(parent, n);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
      GPR_CUDA(cudaMemcpyAsync(hflag, flagbuf, 8, cudaMemcpyDeviceToHost, s));
      GPR_CUDA(cudaStreamSynchronize(s));
    }
    GPR_CUDA(cudaMemsetAsync(flagbuf + 1, 0, 4, s));
    wcc_min_kernel<<<wcc_grid(n), 256, 0, s>>>(parent, P.new2old, n, minid, flagbuf + 1);
    int32_t* dst = labels_out;
    if (flags & GPR_PTR_HOST) {
      out_tmp = (int32_t*)dalloc((size_t)n * 4, s);
      dst = out_tmp;
    }
    wcc_label_kernel<<<wcc_grid(n), 256, 0, s>>>(parent, P.old2new, minid, n, dst);
    GPR_CUDA(cudaGetLastError());
    count_launches(2);
    int32_t roots = 0;
    GPR_CUDA(cudaMemcpyAsync(&roots, flagbuf + 1, 4, cudaMemcpyDeviceToHost, s));
    if (flags & GPR_PTR_HOST)
      GPR_CUDA(cudaMemcpyAsync(labels_out, out_tmp, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    if (num_components) *num_components = roots;
    dfree(parent, s);
    dfree(minid, s);
    dfree(flagbuf, s);
    dfree(out_tmp, s);
    return GPR_OK;
  } catch (const StatusFail& f) {
    dfree(parent, s);
    dfree(minid, s);
    dfree(flagbuf, s);
    dfree(out_tmp, s);
    set_error("wcc: %s", f.msg.c_str());
    return f.st;
  } catch (const CudaFail& f) {
    cudaGetLastError();
    dfree(parent, s);
    dfree(minid, s);
    dfree(flagbuf, s);
    dfree(out_tmp, s);
    set_error("wcc: %s failed: %s", f.what, cudaGetErrorString(f.err));
    return GPR_ECUDA;
  }
}

}  // namespace gpr
