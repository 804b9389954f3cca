// Single-target personalised PageRank, bidirectional (section 4.3, "Fast
// Random Walk Algorithms"): a backward phase from the target t finds the
// nodes near it, then random walks forward from the sources meet that set.
//
// pi_s is the personalised PageRank of the library's reading (restart
// a = 1 - d to s, the mass of dangling nodes back to s).  Q_s(t), the chance
// that an excursion from s (stop with probability a; absorbed at a dangling
// node) stops at t, satisfies Q_s = a e_s + d Q_s P (P: 1/outdeg along each
// edge, zero rows at dangling nodes), and pi_s = (c_s / a) Q_s with
// c_s = a + d pi_s(dangling set).
//
// Backward phase (reverse push, in the relabelled ids of the CSC): p = 0,
// r = e_t; a push at v moves r(v) into p(v) += a r(v) and
// r(u) += d r(v) / outdeg(u) for each in-neighbour u.  Every push keeps
//   pi_s(t) = (c_s / a) p(s) + sum_v pi_s(v) r(v).
// The push runs in rounds: a round pushes every node whose residual exceeded
// r_max when the previous round ended (the frontier), all at once.  A push
// takes r(v) with an atomic exchange, so additions racing with it stay in
// r(v) for a later round and the invariant holds for any interleaving; a node
// joins the next frontier when an atomic add carries its residual across
// r_max, which happens at most once per node and round.  The push ends when
// every residual is at most r_max.
//
// Forward phase: W PageRank walks from each source s (stop with probability
// a; at a dangling node go back to s; else a uniform out-neighbour), over the
// out-adjacency in the caller's ids, neighbours ascending.  With endpoints
// V_1..V_W the estimate
//   pi^_s(t) = p(s) (1 + (d/a) #{V_i dangling} / W) + sum_i r(V_i) / W
// is unbiased.  Walk w of the i-th source draws from the SplitMix64 stream
// (Steele, Lea and Flood, 2014) whose state starts at
// seed ^ ((i << 32 | w) * 0xD6E8FEB86659FD93): one draw x per step stops the
// walk when (x >> 11) 2^-53 < a, tested exactly in integers as
// (x >> 11) < ceil(a 2^53); a second draw x' picks out-neighbour
// floor((x' >> 11) k / 2^53) of a node of out-degree k, as the high word of
// (x' with its low 11 bits cleared) * k.  A walk is cut after 2^20 steps.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "gpr_internal.cuh"

namespace cg = cooperative_groups;

namespace gpr {

namespace {

constexpr int kBlock = 256;
constexpr int kItemEdges = 16;           // in-edges of one frontier node per work item
constexpr int kRoundsPerCheck = 8;       // rounds launched between host reads of the frontier size
constexpr int32_t kMaxRounds = 1 << 16;  // a push that needs more is reported as an error
constexpr int kMaxWalkSteps = 1 << 20;

struct PushCtl {
  uint32_t fcount[2];  // frontier sizes by round parity
  uint32_t icount[2];  // work items by round parity
  unsigned long long pushes;
  int32_t overflow;
  int32_t pad;
};

__device__ __forceinline__ double take_double(double* p) {
  return __longlong_as_double((long long)atomicExch((unsigned long long*)p, 0ull));
}

// Round `cur`: take the residual of every frontier node, add a * amount to
// its p, keep d * amount per frontier entry, and cut its in-edges into work
// items of kItemEdges.  Clears the counters the next round fills.
__global__ void __launch_bounds__(kBlock) push_take_kernel(const int32_t* __restrict__ col_ptr,
                                                           const int32_t* __restrict__ frontier, PushCtl* ctl,
                                                           int cur, double a, double d, double* __restrict__ p,
                                                           double* __restrict__ r, double* __restrict__ famt,
                                                           int32_t* __restrict__ item_f, int32_t* __restrict__ item_e,
                                                           int32_t n, uint32_t item_cap) {
  const int nxt = cur ^ 1;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->fcount[nxt] = 0;
    ctl->icount[nxt] = 0;
  }
  const uint32_t F = min(ctl->fcount[cur], (uint32_t)n);  // a frontier holds each node at most once
  const int lane = threadIdx.x & 31;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < F; i0 += stride) {
    const uint32_t i = i0 + lane;
    int32_t nit = 0, e0 = 0;
    if (i < F) {
      const int32_t v = frontier[i];
      const double amt = take_double(r + v);
      p[v] += a * amt;
      famt[i] = d * amt;
      e0 = col_ptr[v];
      nit = (col_ptr[v + 1] - e0 + kItemEdges - 1) / kItemEdges;
    }
    int32_t incl = nit;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int32_t total = __shfl_sync(0xffffffffu, incl, 31);
    uint32_t base = 0;
    if (lane == 31 && total > 0) {
      base = atomicAdd(&ctl->icount[cur], (uint32_t)total);
      if (base + (uint32_t)total > item_cap) ctl->overflow = 1;
    }
    base = __shfl_sync(0xffffffffu, base, 31) + (uint32_t)(incl - nit);
    const unsigned live = __ballot_sync(0xffffffffu, nit > 0);
    for (unsigned rest = live; rest; rest &= rest - 1) {  // lane L's items, written by the whole warp
      const int L = __ffs(rest) - 1;
      const int32_t cnt = __shfl_sync(0xffffffffu, nit, L);
      const uint32_t b0 = __shfl_sync(0xffffffffu, base, L);
      const int32_t ee = __shfl_sync(0xffffffffu, e0, L);
      for (int32_t j = lane; j < cnt && b0 + j < item_cap; j += 32) {  // items per round <= n + m / kItemEdges
        item_f[b0 + j] = (int32_t)(i0 + L);
        item_e[b0 + j] = ee + j * kItemEdges;
      }
    }
    const unsigned took = __ballot_sync(0xffffffffu, i < F);
    if (lane == 0) atomicAdd(&ctl->pushes, (unsigned long long)__popc(took));
  }
}

// Round `cur`: spread each item's amount over its in-edges; a node whose
// residual crosses r_max joins the next frontier.
__global__ void __launch_bounds__(kBlock) push_scatter_kernel(
    const int32_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx, const int32_t* __restrict__ outdeg,
    const int32_t* __restrict__ frontier, const int32_t* __restrict__ item_f, const int32_t* __restrict__ item_e,
    const double* __restrict__ famt, PushCtl* ctl, int cur, double r_max, double* __restrict__ r,
    int32_t* __restrict__ next, int32_t n, uint32_t item_cap) {
  const int nxt = cur ^ 1;
  const uint32_t I = min(ctl->icount[cur], item_cap);
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < I; j += stride) {
    const int32_t f = item_f[j];
    const int32_t e0 = item_e[j];
    const int32_t e1 = min(e0 + kItemEdges, col_ptr[frontier[f] + 1]);
    const double amt = famt[f];
    for (int32_t e = e0; e < e1; ++e) {
      const int32_t u = row_idx[e];
      const double inc = amt / (double)outdeg[u];
      const double old = atomicAdd(r + u, inc);
      if (old <= r_max && old + inc > r_max) {
        cg::coalesced_group grp = cg::coalesced_threads();
        uint32_t pos = 0;
        if (grp.thread_rank() == 0) pos = atomicAdd(&ctl->fcount[nxt], grp.size());
        pos = grp.shfl(pos, 0) + grp.thread_rank();
        if (pos < (uint32_t)n)
          next[pos] = u;
        else
          ctl->overflow = 1;  // not expected: a node crosses at most once per round
      }
    }
  }
}

__global__ void set_residual_kernel(double* __restrict__ r, int32_t v, int32_t* __restrict__ frontier,
                                    PushCtl* ctl, int above) {
  r[v] = 1.0;
  frontier[0] = v;
  ctl->fcount[0] = above ? 1u : 0u;
}

// out[v] = x[old2new[v]] for the caller's ids.
__global__ void to_caller_kernel(const double* __restrict__ x, const int32_t* __restrict__ old2new, int32_t n,
                                 double* __restrict__ out) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    out[v] = x[old2new[v]];
}

__global__ void check_sources_kernel(const int32_t* __restrict__ src, int32_t k, int32_t n, int* __restrict__ err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
    if ((uint32_t)src[i] >= (uint32_t)n) atomicOr(err, DERR_BAD_ID);
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t& state) {
  uint64_t z = (state += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// One thread per walk; blocks of `bps` per source.  Per source: the sum of
// r at the endpoints (relabelled r, looked up through old2new) and the count
// of dangling endpoints.
__global__ void __launch_bounds__(kBlock) walk_kernel(const int32_t* __restrict__ wptr,
                                                      const int32_t* __restrict__ wadj,
                                                      const int32_t* __restrict__ old2new,
                                                      const double* __restrict__ r,
                                                      const int32_t* __restrict__ sources, int32_t walks, int32_t bps,
                                                      uint64_t seed, uint64_t stop_below,
                                                      double* __restrict__ sum_r,
                                                      unsigned long long* __restrict__ n_dang) {
  const int32_t i = blockIdx.x / bps;
  const int32_t w = (blockIdx.x % bps) * kBlock + threadIdx.x;
  double val = 0.0;
  unsigned dang = 0;
  if (w < walks) {
    const int32_t s = sources[i];
    uint64_t st = seed ^ ((((uint64_t)(uint32_t)i << 32) | (uint32_t)w) * 0xD6E8FEB86659FD93ull);
    int32_t u = s;
    int32_t b = wptr[u], k = wptr[u + 1] - b;
    for (int step = 0; step < kMaxWalkSteps; ++step) {
      if ((splitmix64(st) >> 11) < stop_below) break;
      if (k == 0) {
        u = s;
      } else {
        const uint64_t j = __umul64hi(splitmix64(st) & ~0x7FFull, (uint64_t)k);
        u = wadj[b + (int32_t)j];
      }
      b = wptr[u];
      k = wptr[u + 1] - b;
    }
    val = r[old2new[u]];
    dang = k == 0;
  }
  for (int o = 16; o > 0; o >>= 1) {
    val += __shfl_xor_sync(0xffffffffu, val, o);
    dang += __shfl_xor_sync(0xffffffffu, dang, o);
  }
  __shared__ double s_val[kBlock / 32];
  __shared__ unsigned s_dang[kBlock / 32];
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_val[wid] = val;
    s_dang[wid] = dang;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tv = 0.0;
    unsigned td = 0;
    for (int q = 0; q < kBlock / 32; ++q) {
      tv += s_val[q];
      td += s_dang[q];
    }
    if (tv != 0.0) atomicAdd(sum_r + i, tv);
    if (td) atomicAdd(n_dang + i, (unsigned long long)td);
  }
}

__global__ void estimate_kernel(const double* __restrict__ p, const int32_t* __restrict__ old2new,
                                const int32_t* __restrict__ sources, int32_t k, int32_t walks, double coef,
                                const double* __restrict__ sum_r, const unsigned long long* __restrict__ n_dang,
                                double* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = p[old2new[sources[i]]] * (1.0 + coef * ((double)n_dang[i] / walks)) + sum_r[i] / walks;
}

int grid_items(int64_t items, int per_sm = 8) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((items + kBlock - 1) / kBlock, (int64_t)num_sms() * per_sm));
}

struct Buffers {
  cudaStream_t s;
  std::vector<void*> ptrs;
  void* get(size_t bytes) {
    void* q = dalloc(std::max<size_t>(bytes, 16), s);
    ptrs.push_back(q);
    return q;
  }
  ~Buffers() {
    for (void* q : ptrs) dfree(q, s);
  }
};

// Reverse push from relabelled node tn into p, r (relabelled, n each).
// Returns the number of pushes.
int64_t reverse_push(const gpr_graph* g, int32_t tn, double d, double r_max, double* p, double* r, Buffers& buf,
                     cudaStream_t s) {
  const int32_t n = g->n;
  const int64_t item_cap = (int64_t)n + g->m / kItemEdges + 32;
  int32_t* front[2] = {(int32_t*)buf.get((size_t)n * 4), (int32_t*)buf.get((size_t)n * 4)};
  double* famt = (double*)buf.get((size_t)n * 8);
  int32_t* item_f = (int32_t*)buf.get((size_t)item_cap * 4);
  int32_t* item_e = (int32_t*)buf.get((size_t)item_cap * 4);
  PushCtl* ctl = (PushCtl*)buf.get(sizeof(PushCtl));
  GPR_CUDA(cudaMemsetAsync(p, 0, (size_t)n * 8, s));
  GPR_CUDA(cudaMemsetAsync(r, 0, (size_t)n * 8, s));
  GPR_CUDA(cudaMemsetAsync(ctl, 0, sizeof(PushCtl), s));
  set_residual_kernel<<<1, 1, 0, s>>>(r, tn, front[0], ctl, 1.0 > r_max ? 1 : 0);
  GPR_CUDA(cudaGetLastError());
  count_launches(1);
  const double a = 1.0 - d;
  const int gt = grid_items(n), gs = grid_items(item_cap);
  int32_t round = 0;
  PushCtl h{};
  for (;;) {
    for (int q = 0; q < kRoundsPerCheck; ++q, ++round) {
      const int cur = round & 1;
      push_take_kernel<<<gt, kBlock, 0, s>>>(g->col_ptr, front[cur], ctl, cur, a, d, p, r, famt, item_f, item_e, n,
                                             (uint32_t)item_cap);
      push_scatter_kernel<<<gs, kBlock, 0, s>>>(g->col_ptr, g->row_idx, g->outdeg, front[cur], item_f, item_e, famt,
                                                ctl, cur, r_max, r, front[cur ^ 1], n, (uint32_t)item_cap);
    }
    GPR_CUDA(cudaGetLastError());
    count_launches(2 * kRoundsPerCheck);
    GPR_CUDA(cudaMemcpyAsync(&h, ctl, sizeof h, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    if (h.overflow) throw StatusFail{GPR_ECUDA, "reverse push: frontier or work list overflow"};
    if (h.fcount[round & 1] == 0) break;
    if (round >= kMaxRounds) throw StatusFail{GPR_ETIMEOUT, "reverse push: no end after 65536 rounds"};
  }
  return (int64_t)h.pushes;
}

void check_args(const gpr_graph* g, int32_t target, double d, double r_max) {
  if (target < 0 || target >= g->n) throw StatusFail{GPR_EINVAL, "target out of range"};
  if (!(d > 0.0 && d < 1.0)) throw StatusFail{GPR_EINVAL, "damping outside (0, 1)"};
  if (!(r_max > 0.0) || !std::isfinite(r_max)) throw StatusFail{GPR_EINVAL, "r_max must be positive and finite"};
}

int32_t relabelled(const gpr_graph* g, int32_t v, cudaStream_t s) {
  int32_t tn = 0;
  GPR_CUDA(cudaMemcpyAsync(&tn, g->plan.old2new + v, 4, cudaMemcpyDeviceToHost, s));
  GPR_CUDA(cudaStreamSynchronize(s));
  return tn;
}

}  // namespace

gpr_status run_reverse_push(gpr_graph* g, int32_t target, double d, double r_max, double* p_out, double* r_out,
                            int64_t* pushes, int flags, cudaStream_t s) {
  try {
    check_args(g, target, d, r_max);
    const int32_t n = g->n;
    Buffers buf{s, {}};
    double* p = (double*)buf.get((size_t)n * 8);
    double* r = (double*)buf.get((size_t)n * 8);
    const int64_t k = reverse_push(g, relabelled(g, target, s), d, r_max, p, r, buf, s);
    double* outs[2] = {p_out, r_out};
    const double* ins[2] = {p, r};
    for (int q = 0; q < 2; ++q) {
      if (!outs[q]) continue;
      double* dst = (flags & GPR_PTR_HOST) ? (double*)buf.get((size_t)n * 8) : outs[q];
      to_caller_kernel<<<grid_items(n), kBlock, 0, s>>>(ins[q], g->plan.old2new, n, dst);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
      if (flags & GPR_PTR_HOST) GPR_CUDA(cudaMemcpyAsync(outs[q], dst, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    }
    GPR_CUDA(cudaStreamSynchronize(s));
    if (pushes) *pushes = k;
    return GPR_OK;
  } catch (const StatusFail& f) {
    set_error("ppr_reverse_push: %s", f.msg.c_str());
    return f.st;
  } catch (const CudaFail& f) {
    cudaGetLastError();
    set_error("ppr_reverse_push: %s failed: %s", f.what, cudaGetErrorString(f.err));
    return GPR_ECUDA;
  }
}

gpr_status run_ppr_target(gpr_graph* g, int32_t target, double d, double r_max, const int32_t* sources, int32_t k,
                          int32_t walks, uint64_t seed, double* est_out, int flags, cudaStream_t s) {
  try {
    check_args(g, target, d, r_max);
    if (k < 0 || walks < 1) throw StatusFail{GPR_EINVAL, "need k >= 0 sources and walks >= 1"};
    const int64_t bps = (walks + kBlock - 1) / kBlock;
    if ((int64_t)k * bps > INT32_MAX) throw StatusFail{GPR_EINVAL, "too many walks in one call"};
    if (k == 0) return GPR_OK;
    const int32_t n = g->n;
    {
      std::lock_guard<std::mutex> lock(g->mu);
      if (!g->walk_ptr) build_caller_out_adjacency(g, s, &g->walk_ptr, &g->walk_adj);
    }
    Buffers buf{s, {}};
    const int32_t* src = sources;
    if (flags & GPR_PTR_HOST) {
      int32_t* dsrc = (int32_t*)buf.get((size_t)k * 4);
      GPR_CUDA(cudaMemcpyAsync(dsrc, sources, (size_t)k * 4, cudaMemcpyHostToDevice, s));
      src = dsrc;
    }
    int* err = (int*)buf.get(8);
    GPR_CUDA(cudaMemsetAsync(err, 0, 8, s));
    check_sources_kernel<<<grid_items(k), kBlock, 0, s>>>(src, k, n, err);
    GPR_CUDA(cudaGetLastError());
    count_launches(1);
    double* p = (double*)buf.get((size_t)n * 8);
    double* r = (double*)buf.get((size_t)n * 8);
    int32_t tn = 0;
    int herr = 0;
    GPR_CUDA(cudaMemcpyAsync(&tn, g->plan.old2new + target, 4, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    if (herr) throw StatusFail{GPR_EINVAL, "a source id is out of range"};
    reverse_push(g, tn, d, r_max, p, r, buf, s);
    double* sum_r = (double*)buf.get((size_t)k * 8);
    unsigned long long* n_dang = (unsigned long long*)buf.get((size_t)k * 8);
    GPR_CUDA(cudaMemsetAsync(sum_r, 0, (size_t)k * 8, s));
    GPR_CUDA(cudaMemsetAsync(n_dang, 0, (size_t)k * 8, s));
    const double a = 1.0 - d;
    const uint64_t stop_below = (uint64_t)std::ceil(std::ldexp(a, 53));
    walk_kernel<<<(unsigned)(k * bps), kBlock, 0, s>>>(g->walk_ptr, g->walk_adj, g->plan.old2new, r, src,
                                                       walks, (int32_t)bps, seed, stop_below, sum_r, n_dang);
    double* out = (flags & GPR_PTR_HOST) ? (double*)buf.get((size_t)k * 8) : est_out;
    estimate_kernel<<<grid_items(k), kBlock, 0, s>>>(p, g->plan.old2new, src, k, walks, d / a, sum_r, n_dang, out);
    GPR_CUDA(cudaGetLastError());
    count_launches(2);
    if (flags & GPR_PTR_HOST) GPR_CUDA(cudaMemcpyAsync(est_out, out, (size_t)k * 8, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    return GPR_OK;
  } catch (const StatusFail& f) {
    set_error("ppr_target: %s", f.msg.c_str());
    return f.st;
  } catch (const CudaFail& f) {
    cudaGetLastError();
    set_error("ppr_target: %s failed: %s", f.what, cudaGetErrorString(f.err));
    return GPR_ECUDA;
  }
}

}  // namespace gpr
