// Weakly connected components (section 4 Table "snap_methods": connected
// components; section 6 Table "exp_algs" times WCC on LiveJournal).
//
// Union-find over the relabelled CSC, edge directions ignored, in the manner
// of Afforest (Sutton, Hsiao, Pan and Owens, 2018):
//   1. parent[v] = v; for r = 0, 1: every node links with its r-th
//      in-neighbour; compress (parent[v] = root(v)).
//   2. c = the most frequent root among 1,024 sampled nodes (the giant
//      component when there is one).  From here c ranks below every other
//      root, so it is never hooked under another and stays the giant's root.
//   3. Link every in-edge (u, v) unless both u and v were in c's tree after
//      step 2 (a 1-bit-per-node map of parent[x] == c, small enough to stay in
//      L2): a stream over all edges links those whose source is outside c
//      (the row of such an edge is found by binary search: they are rare), and
//      a pass over the rows outside c links all of their edges; compress.
// link(u, v) finds both roots and sets parent[hi] = lo by compare-and-swap,
// hi being the root of larger rank (rank: c lowest, then ascending id);
// when the swap fails another thread moved hi and the search repeats.  When
// it returns, u and v are in one tree, and trees only merge, so one pass over
// the edges suffices.  Every parent has a lower rank than its child, so every
// root search ends.  Each tree is one component; its label is the smallest
// caller id among its nodes (an atomicMin, order-free), so the output does
// not depend on the schedule.
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "gpr_internal.cuh"

namespace cg = cooperative_groups;

namespace gpr {

constexpr uint32_t kLinkRetries = 1u << 20;  // a bound that turns a fault in the reasoning above into an error

__device__ __forceinline__ int32_t wcc_root(const int32_t* parent, int32_t v) {
  int32_t p = __ldcg(parent + v);
  while (p != v) {  // ranks strictly decrease along a chain: ends within n steps
    v = p;
    p = __ldcg(parent + v);
  }
  return v;
}

// true when a ranks above b (c ranks lowest)
__device__ __forceinline__ bool wcc_above(int32_t a, int32_t b, int32_t c) {
  return b == c || (a != c && a > b);
}

__device__ __forceinline__ void wcc_link(int32_t* parent, int32_t u, int32_t v, int32_t c, int* err) {
  int32_t a = wcc_root(parent, u), b = wcc_root(parent, v);
  for (uint32_t k = 0; a != b; ++k) {
    if (k == kLinkRetries) {
      atomicOr(err, DERR_TIMEOUT);
      return;
    }
    const int32_t hi = wcc_above(a, b, c) ? a : b, lo = hi == a ? b : a;
    if (atomicCAS(parent + hi, hi, lo) == hi) return;
    a = wcc_root(parent, hi);
    b = wcc_root(parent, lo);
  }
}

// Step 1: every node links with its first two in-neighbours.
__global__ void wcc_sample_kernel(const int32_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx,
                                  int32_t n, int32_t* __restrict__ parent, int* __restrict__ err) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e0 = col_ptr[v], e1 = col_ptr[v + 1];
    for (int32_t e = e0; e < e1 && e < e0 + 2; ++e) wcc_link(parent, row_idx[e], (int32_t)v, -1, err);
  }
}

__device__ __forceinline__ bool wcc_in(const uint32_t* __restrict__ inc, int32_t x) {
  return (__ldg(inc + (x >> 5)) >> (x & 31)) & 1u;
}

// inc bit x = (parent[x] == c), one word per 32 nodes.
__global__ void wcc_bitmap_kernel(const int32_t* __restrict__ parent, int32_t n, int32_t c,
                                  uint32_t* __restrict__ inc) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); v0 < n; v0 += stride) {
    const int64_t v = v0 + lane;
    const unsigned bits = __ballot_sync(0xffffffffu, v < n && parent[v] == c);
    if (lane == 0) inc[v0 >> 5] = bits;
  }
}

// The row holding edge e: the last p with col_ptr[p] <= e.
__device__ __forceinline__ int32_t wcc_row_of(const int32_t* __restrict__ col_ptr, int32_t n, int64_t e) {
  int32_t lo = 0, hi = n;  // col_ptr[lo] <= e < col_ptr[hi]
  while (hi - lo > 1) {
    const int32_t mid = lo + (hi - lo) / 2;
    if (col_ptr[mid] <= e)
      lo = mid;
    else
      hi = mid;
  }
  return lo;
}

// Step 3, all edges: four per thread and trip (16-byte loads).  An edge
// whose source is outside c goes to the pending list (its index), to be
// linked by wcc_pending_kernel with every lane busy; when the list is full it
// is linked here.
__device__ __forceinline__ void wcc_defer(int64_t e, int32_t u, const int32_t* __restrict__ col_ptr, int32_t n,
                                          int32_t c, int32_t* __restrict__ parent, int64_t* __restrict__ pending,
                                          unsigned long long* __restrict__ npending, int64_t cap,
                                          int* __restrict__ err) {
  cg::coalesced_group grp = cg::coalesced_threads();
  unsigned long long k = 0;
  if (grp.thread_rank() == 0) k = atomicAdd(npending, (unsigned long long)grp.size());
  k = grp.shfl(k, 0) + grp.thread_rank();
  if ((int64_t)k < cap)
    pending[k] = e;
  else
    wcc_link(parent, u, wcc_row_of(col_ptr, n, e), c, err);
}

__global__ void __launch_bounds__(256) wcc_edges_kernel(const int32_t* __restrict__ col_ptr,
                                                        const int32_t* __restrict__ row_idx, int64_t m, int32_t n,
                                                        int32_t c, const uint32_t* __restrict__ inc,
                                                        int32_t* __restrict__ parent, int64_t* __restrict__ pending,
                                                        unsigned long long* __restrict__ npending, int64_t cap,
                                                        int* __restrict__ err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t m4 = m / 4;
  const int4* rows4 = reinterpret_cast<const int4*>(row_idx);  // device allocations are 256-byte aligned
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < m4; q += stride) {
    const int4 u = __ldcs(rows4 + q);
    if (!wcc_in(inc, u.x)) wcc_defer(4 * q, u.x, col_ptr, n, c, parent, pending, npending, cap, err);
    if (!wcc_in(inc, u.y)) wcc_defer(4 * q + 1, u.y, col_ptr, n, c, parent, pending, npending, cap, err);
    if (!wcc_in(inc, u.z)) wcc_defer(4 * q + 2, u.z, col_ptr, n, c, parent, pending, npending, cap, err);
    if (!wcc_in(inc, u.w)) wcc_defer(4 * q + 3, u.w, col_ptr, n, c, parent, pending, npending, cap, err);
  }
  for (int64_t e = 4 * m4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += stride) {
    const int32_t u = row_idx[e];
    if (!wcc_in(inc, u)) wcc_defer(e, u, col_ptr, n, c, parent, pending, npending, cap, err);
  }
}

// Step 3, the pending edges: each linked with its row.
__global__ void __launch_bounds__(256) wcc_pending_kernel(const int32_t* __restrict__ col_ptr,
                                                          const int32_t* __restrict__ row_idx, int32_t n, int32_t c,
                                                          const int64_t* __restrict__ pending,
                                                          const unsigned long long* __restrict__ npending,
                                                          int64_t cap, int32_t* __restrict__ parent,
                                                          int* __restrict__ err) {
  const int64_t k = min((int64_t)*npending, cap);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = pending[i];
    wcc_link(parent, row_idx[e], wcc_row_of(col_ptr, n, e), c, err);
  }
}

// Step 3, rows outside c: 32 rows per warp trip, each such row's edges taken
// by the whole warp.
__global__ void __launch_bounds__(256) wcc_rows_out_kernel(const int32_t* __restrict__ col_ptr,
                                                           const int32_t* __restrict__ row_idx, int32_t n,
                                                           int32_t c, const uint32_t* __restrict__ inc,
                                                           int32_t* __restrict__ parent, int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
    const int64_t p = base + lane;
    const bool out = p < n && !wcc_in(inc, (int32_t)p) && col_ptr[p + 1] > col_ptr[p];
    for (unsigned mask = __ballot_sync(0xffffffffu, out); mask; mask &= mask - 1) {
      const int32_t row = (int32_t)(base + __ffs(mask) - 1);
      const int32_t e1 = col_ptr[row + 1];
      for (int32_t e = col_ptr[row] + lane; e < e1; e += 32) wcc_link(parent, row_idx[e], row, c, err);
    }
  }
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

// the roots of k sampled nodes (node i * stride mod n)
__global__ void wcc_sample_roots_kernel(const int32_t* __restrict__ parent, int32_t n, int32_t k, int64_t stride,
                                        int32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < k) out[i] = parent[(int64_t)i * stride % n];
}

// minid[root] = the smallest caller id of the component; count the roots.
// Lanes of a warp in the giant component c take their minimum first, so one
// atomic per warp reaches minid[c]; an isolated node stores its own id;
// other lanes go straight to memory with an atomic.  c = -1: no giant.
__global__ void wcc_min_kernel(const int32_t* __restrict__ parent, const int32_t* __restrict__ new2old,
                               const int32_t* __restrict__ col_ptr, const int32_t* __restrict__ outdeg, int32_t n,
                               int32_t c, int32_t* __restrict__ minid, int32_t* __restrict__ roots) {
  int32_t local = 0;
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); v0 < n; v0 += stride) {
    const int64_t v = v0 + lane;
    const bool live = v < n;
    const int32_t r = live ? parent[v] : -1;  // compressed: the root
    const uint32_t id = live ? (uint32_t)new2old[v] : 0xFFFFFFFFu;
    const unsigned in_c = __ballot_sync(0xffffffffu, live && r == c);
    if (live && r == c) {
      const uint32_t lo = __reduce_min_sync(in_c, id);
      if (lane == __ffs(in_c) - 1) atomicMin(minid + c, (int32_t)lo);
    } else if (live) {
      if (outdeg[v] == 0 && col_ptr[v + 1] == col_ptr[v])
        minid[v] = (int32_t)id;  // an isolated node: its own component, nobody else writes here
      else
        atomicMin(minid + r, (int32_t)id);
    }
    local += live && r == (int32_t)v;
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
  int32_t* flagbuf = nullptr;  // [0] error bits, [1] roots, [2 ..] sampled roots
  int32_t* out_tmp = nullptr;
  uint32_t* inc = nullptr;
  int64_t* pending = nullptr;  // edge indices to link, then their count
  constexpr int kSample = 1024;
  try {
    parent = (int32_t*)dalloc((size_t)n * 4, s);
    minid = (int32_t*)dalloc((size_t)n * 4, s);
    flagbuf = (int32_t*)dalloc((2 + kSample) * 4, s);
    int* err = (int*)flagbuf;
    GPR_CUDA(cudaMemsetAsync(flagbuf, 0, 8, s));
    wcc_init_kernel<<<wcc_grid(n), 256, 0, s>>>(parent, minid, n);
    GPR_CUDA(cudaGetLastError());
    count_launches(1);
    const Plan& P = g->plan;
    int32_t c = -1;  // the giant component's root (-1: none)
    if (g->m > 0) {
      // 1. two sampled in-neighbours per node
      wcc_sample_kernel<<<wcc_grid(n), 256, 0, s>>>(g->col_ptr, g->row_idx, n, parent, err);
      count_launches(1);
      wcc_compress_kernel<<<wcc_grid(n), 256, 0, s>>>(parent, n);
      // 2. the most frequent root of a sample
      const int k = (int)std::min<int64_t>(kSample, n);
      const int64_t stride = std::max<int64_t>(1, (int64_t)n / k) | 1;  // odd: spreads over [0, n)
      wcc_sample_roots_kernel<<<(k + 255) / 256, 256, 0, s>>>(parent, n, k, stride, flagbuf + 2);
      GPR_CUDA(cudaGetLastError());
      count_launches(2);
      std::vector<int32_t> roots(k);
      GPR_CUDA(cudaMemcpyAsync(roots.data(), flagbuf + 2, (size_t)k * 4, cudaMemcpyDeviceToHost, s));
      GPR_CUDA(cudaStreamSynchronize(s));
      std::sort(roots.begin(), roots.end());
      c = roots[0];
      for (int a = 0, best = 0; a < k;) {
        int b = a;
        while (b < k && roots[b] == roots[a]) ++b;
        if (b - a > best) {
          best = b - a;
          c = roots[a];
        }
        a = b;
      }
      // 3. every edge not already inside c
      inc = (uint32_t*)dalloc(((size_t)n + 31) / 32 * 4, s);
      wcc_bitmap_kernel<<<wcc_grid(n), 256, 0, s>>>(parent, n, c, inc);
      count_launches(1);
      const int64_t cap = std::max<int64_t>(1 << 20, std::min<int64_t>(g->m / 16, (int64_t)1 << 26));
      pending = (int64_t*)dalloc((size_t)cap * 8 + 8, s);
      unsigned long long* npending = (unsigned long long*)(pending + cap);
      GPR_CUDA(cudaMemsetAsync(npending, 0, 8, s));
      wcc_edges_kernel<<<wcc_grid(g->m / 4 + 1), 256, 0, s>>>(g->col_ptr, g->row_idx, g->m, n, c, inc, parent,
                                                                 pending, npending, cap, err);
      wcc_pending_kernel<<<num_sms() * 8, 256, 0, s>>>(g->col_ptr, g->row_idx, n, c, pending, npending, cap,
                                                        parent, err);
      wcc_rows_out_kernel<<<wcc_grid(n), 256, 0, s>>>(g->col_ptr, g->row_idx, n, c, inc, parent, err);
      count_launches(3);
      wcc_compress_kernel<<<wcc_grid(n), 256, 0, s>>>(parent, n);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
    }
    GPR_CUDA(cudaMemsetAsync(flagbuf + 1, 0, 4, s));
    wcc_min_kernel<<<wcc_grid(n), 256, 0, s>>>(parent, P.new2old, g->col_ptr, g->outdeg, n, c, minid, flagbuf + 1);
    int32_t* dst = labels_out;
    if (flags & GPR_PTR_HOST) {
      out_tmp = (int32_t*)dalloc((size_t)n * 4, s);
      dst = out_tmp;
    }
    wcc_label_kernel<<<wcc_grid(n), 256, 0, s>>>(parent, P.old2new, minid, n, dst);
    GPR_CUDA(cudaGetLastError());
    count_launches(2);
    int32_t hb[2] = {0, 0};
    GPR_CUDA(cudaMemcpyAsync(hb, flagbuf, 8, cudaMemcpyDeviceToHost, s));
    if (flags & GPR_PTR_HOST)
      GPR_CUDA(cudaMemcpyAsync(labels_out, out_tmp, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    if (hb[0] & DERR_TIMEOUT) throw StatusFail{GPR_ETIMEOUT, "a link gave up after 2^20 retries"};
    const int32_t roots = hb[1];
    if (num_components) *num_components = roots;
    dfree(parent, s);
    dfree(minid, s);
    dfree(flagbuf, s);
    dfree(out_tmp, s);
    dfree(inc, s);
    dfree(pending, s);
    return GPR_OK;
  } catch (const StatusFail& f) {
    dfree(parent, s);
    dfree(minid, s);
    dfree(flagbuf, s);
    dfree(out_tmp, s);
    dfree(inc, s);
    dfree(pending, s);
    set_error("wcc: %s", f.msg.c_str());
    return f.st;
  } catch (const CudaFail& f) {
    cudaGetLastError();
    dfree(parent, s);
    dfree(minid, s);
    dfree(flagbuf, s);
    dfree(out_tmp, s);
    dfree(inc, s);
    dfree(pending, s);
    set_error("wcc: %s failed: %s", f.what, cudaGetErrorString(f.err));
    return GPR_ECUDA;
  }
}

}  // namespace gpr
