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
#include <map>
#include <mutex>

#include "gpr_internal.cuh"

namespace cg = cooperative_groups;

namespace gpr {

namespace {

constexpr int kBlock = 256;
constexpr int kItemEdges = 16;           // in-edges of one frontier node per work item
constexpr int kRoundsPerCheck = 8;       // rounds launched between host reads of the frontier size (4 at first)
constexpr int32_t kMaxRounds = 1 << 16;  // a push that needs more is reported as an error
constexpr int kMaxWalkSteps = 1 << 20;

struct PushCtl {
  uint32_t fcount[2];  // frontier sizes by round parity
  uint32_t icount[2];  // work items by round parity
  unsigned long long pushes;
  unsigned long long edges;  // in-edges scanned
  uint32_t rounds;           // rounds with a non-empty frontier
  int32_t overflow;
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
  if (blockIdx.x == 0 && threadIdx.x == 0 && F > 0) ctl->rounds += 1;
  const int lane = threadIdx.x & 31;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < F; i0 += stride) {
    const uint32_t i = i0 + lane;
    int32_t nit = 0, e0 = 0, deg = 0;
    if (i < F) {
      const int32_t v = frontier[i];
      const double amt = take_double(r + v);
      p[v] += a * amt;
      famt[i] = d * amt;
      e0 = col_ptr[v];
      deg = col_ptr[v + 1] - e0;
      nit = (deg + kItemEdges - 1) / kItemEdges;
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
    for (int o = 16; o > 0; o >>= 1) deg += __shfl_xor_sync(0xffffffffu, deg, o);
    if (lane == 0) {
      atomicAdd(&ctl->pushes, (unsigned long long)__popc(took));
      atomicAdd(&ctl->edges, (unsigned long long)(uint32_t)deg);
    }
  }
}

// Round `cur`: spread each item's amount over its in-edges; a node whose
// residual crosses r_max joins the next frontier.
__global__ void __launch_bounds__(kBlock) push_scatter_kernel(
    const int32_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx, const int32_t* __restrict__ outdeg,
    const int32_t* __restrict__ frontier, const int32_t* __restrict__ item_f, const int32_t* __restrict__ item_e,
    const double* __restrict__ famt, PushCtl* ctl, int cur, double r_max, double* __restrict__ r,
    int32_t* __restrict__ next, int32_t n, uint32_t item_cap, uint32_t* __restrict__ dirty) {
  const int nxt = cur ^ 1;
  const uint32_t I = min(ctl->icount[cur], item_cap);
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < I; j += stride) {
    const int32_t f = item_f[j];
    const int32_t e0 = item_e[j];
    const int32_t cnt = min(kItemEdges, col_ptr[frontier[f] + 1] - e0);
    const double amt = famt[f];
    // all of the item's loads and atomics in flight at once; the crossing
    // tests only after every add has returned
    int32_t u[kItemEdges];
    double inc[kItemEdges], old[kItemEdges];
#pragma unroll
    for (int q = 0; q < kItemEdges; ++q) u[q] = q < cnt ? row_idx[e0 + q] : -1;
#pragma unroll
    for (int q = 0; q < kItemEdges; ++q) inc[q] = u[q] >= 0 ? amt / (double)outdeg[u[q]] : 0.0;
#pragma unroll
    for (int q = 0; q < kItemEdges; ++q) old[q] = u[q] >= 0 ? atomicAdd(r + u[q], inc[q]) : 1.0;
#pragma unroll
    for (int q = 0; q < kItemEdges; ++q)  // first touch since zero: to be cleared after the call
      if (old[q] == 0.0) atomicOr(dirty + (u[q] >> 5), 1u << (u[q] & 31));
#pragma unroll
    for (int q = 0; q < kItemEdges; ++q) {
      if (u[q] >= 0 && old[q] <= r_max && old[q] + inc[q] > r_max) {
        cg::coalesced_group grp = cg::coalesced_threads();
        uint32_t pos = 0;
        if (grp.thread_rank() == 0) pos = atomicAdd(&ctl->fcount[nxt], grp.size());
        pos = grp.shfl(pos, 0) + grp.thread_rank();
        if (pos < (uint32_t)n)
          next[pos] = u[q];
        else
          ctl->overflow = 1;  // not expected: a node crosses at most once per round
      }
    }
  }
}

__global__ void set_residual_kernel(double* __restrict__ r, int32_t v, int32_t* __restrict__ frontier,
                                    PushCtl* ctl, int above, uint32_t* __restrict__ dirty) {
  r[v] = 1.0;
  dirty[v >> 5] |= 1u << (v & 31);
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

// Each adjacency entry's target with its own out-list: nbr[e] = (offset,
// out-degree) of adj[e], so that a walk step is one 8-byte load; then the
// entry itself becomes the target's relabelled id, the index of the push's
// residuals (the order of each list, by caller id, stays).
__global__ void walk_nbr_kernel(const int32_t* __restrict__ wptr, int32_t* __restrict__ wadj,
                                const int32_t* __restrict__ old2new, int64_t m, int2* __restrict__ nbr) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = wadj[e];
    const int32_t b = wptr[v];
    nbr[e] = make_int2(b, wptr[v + 1] - b);
    wadj[e] = old2new[v];
  }
}

// Walks of the flattened (source index i, walk w) order, idx = i W + w.  A
// warp owns the range [w0, w0 + per_warp); each lane runs one walk, and a
// lane whose walk ends takes the next index of the range, so the lanes stay
// busy although walk lengths are geometric.  The state of a walk is the
// (offset, out-degree) of its node and the last edge taken; its endpoint is
// written as the relabelled id, with bit 31 set when that node is dangling.
__global__ void __launch_bounds__(kBlock) walk_kernel(const int32_t* __restrict__ wptr,
                                                      const int2* __restrict__ wnbr,
                                                      const int32_t* __restrict__ wadj,
                                                      const int32_t* __restrict__ old2new,
                                                      const int32_t* __restrict__ sources, int32_t walks,
                                                      int64_t total, int32_t per_warp, uint64_t seed,
                                                      uint64_t stop_below, int32_t* __restrict__ end,
                                                      unsigned long long* __restrict__ steps_total) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * per_warp;
  const int64_t w1 = min(w0 + per_warp, total);
  if (w0 >= w1) return;  // warp-uniform
  int64_t next = w0 + 32;
  int64_t idx = w0 + lane < w1 ? w0 + lane : -1;
  uint64_t st = 0;
  int32_t src = 0, s_new = 0, s_off = 0, s_deg = 0, off = 0, deg = 0, last_e = -1, moves = 0;
  unsigned long long steps = 0;
  auto start = [&]() {
    const uint32_t i = (uint32_t)idx / (uint32_t)walks;  // idx < 2^31
    const uint32_t w = (uint32_t)idx - i * (uint32_t)walks;
    st = seed ^ ((((uint64_t)i << 32) | w) * 0xD6E8FEB86659FD93ull);
    src = sources[i];
    s_new = old2new[src];
    s_off = wptr[src];
    s_deg = wptr[src + 1] - s_off;
    off = s_off;
    deg = s_deg;
    last_e = -1;
    moves = 0;
  };
  if (idx >= 0) start();
  for (;;) {
    bool done = false;
    if (idx >= 0) {
      if (moves == kMaxWalkSteps || (splitmix64(st) >> 11) < stop_below) {
        done = true;
      } else {
        ++moves;
        if (deg == 0) {  // dangling: back to the source
          off = s_off;
          deg = s_deg;
          last_e = -1;
        } else {
          last_e = off + (int32_t)__umul64hi(splitmix64(st) & ~0x7FFull, (uint64_t)deg);
          const int2 nb = __ldg(wnbr + last_e);
          off = nb.x;
          deg = nb.y;
        }
      }
    }
    if (done) {
      const int32_t id = last_e < 0 ? s_new : wadj[last_e];
      end[idx] = (int32_t)((uint32_t)id | (deg == 0 ? 0x80000000u : 0u));
      steps += (unsigned long long)moves;
    }
    const unsigned dm = __ballot_sync(0xffffffffu, done);
    if (dm) {
      if (done) {
        const int64_t q = next + __popc(dm & ((1u << lane) - 1u));
        idx = q < w1 ? q : -1;
        if (idx >= 0) start();
      }
      next += __popc(dm);
    }
    if (!__any_sync(0xffffffffu, idx >= 0)) break;
  }
  for (int o = 16; o > 0; o >>= 1) steps += __shfl_xor_sync(0xffffffffu, steps, o);
  if (lane == 0 && steps) atomicAdd(steps_total, steps);
}

// One block per source: the estimate from its W endpoints (relabelled ids,
// bit 31 = dangling), summed in a fixed
// order (so the result does not depend on the schedule):
//   p(s) (1 + (d/a) #dangling / W) + sum r(V) / W.
__global__ void __launch_bounds__(kBlock) estimate_kernel(const double* __restrict__ p,
                                                          const double* __restrict__ r,
                                                          const int32_t* __restrict__ old2new,
                                                          const int32_t* __restrict__ sources,
                                                          const int32_t* __restrict__ end, int32_t walks,
                                                          double coef, double* __restrict__ out) {
  const int32_t i = blockIdx.x;
  const int32_t* e = end + (int64_t)i * walks;
  double val = 0.0;
  uint32_t dang = 0;
  for (int32_t w = threadIdx.x; w < walks; w += kBlock) {
    const uint32_t u = (uint32_t)e[w];
    val += r[u & 0x7FFFFFFFu];
    dang += u >> 31;
  }
  for (int o = 16; o > 0; o >>= 1) {
    val += __shfl_xor_sync(0xffffffffu, val, o);
    dang += __shfl_xor_sync(0xffffffffu, dang, o);
  }
  __shared__ double s_val[kBlock / 32];
  __shared__ uint32_t s_dang[kBlock / 32];
  if ((threadIdx.x & 31) == 0) {
    s_val[threadIdx.x >> 5] = val;
    s_dang[threadIdx.x >> 5] = dang;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tv = 0.0;
    uint32_t td = 0;
    for (int q = 0; q < kBlock / 32; ++q) {
      tv += s_val[q];
      td += s_dang[q];
    }
    out[i] = p[old2new[sources[i]]] * (1.0 + coef * ((double)td / walks)) + tv / walks;
  }
}

// A high-priority stream per device for the push, so that its short rounds
// get SMs ahead of the walks running beside them on the caller's stream.
cudaStream_t push_stream() {
  static std::mutex mu;
  static std::map<int, cudaStream_t> streams;
  std::lock_guard<std::mutex> lock(mu);
  const int dev = device_ordinal();
  auto it = streams.find(dev);
  if (it != streams.end()) return it->second;
  int lo = 0, hi = 0;
  GPR_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  cudaStream_t st = nullptr;
  GPR_CUDA(cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, hi));
  streams[dev] = st;
  return st;
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

// The reverse push's device workspace, one per graph, kept between calls.
// p and r are zero between calls: a call marks in `dirty` (one bit per node)
// every node whose residual it touches first, and wipe_kernel clears exactly
// those entries (and the bits) at its end, instead of two n-sized memsets.
struct PushWork {
  int32_t n = 0;
  int64_t item_cap = 0;
  double* p = nullptr;
  double* r = nullptr;
  uint32_t* dirty = nullptr;
  int32_t* front[2] = {nullptr, nullptr};
  double* famt = nullptr;
  int32_t* item_f = nullptr;
  int32_t* item_e = nullptr;
  PushCtl* ctl = nullptr;
};

std::mutex g_work_mu;
std::map<const gpr_graph*, PushWork*> g_work;

void free_work(PushWork* w, cudaStream_t s) {
  for (void* q : {(void*)w->p, (void*)w->r, (void*)w->dirty, (void*)w->front[0], (void*)w->front[1],
                  (void*)w->famt, (void*)w->item_f, (void*)w->item_e, (void*)w->ctl})
    dfree(q, s);
  delete w;
}

// The graph's workspace, made on first use; the work lists grow with m
// (edge updates).  Callers hold g->mu.
PushWork* push_work(const gpr_graph* g, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g_work_mu);
  PushWork*& w = g_work[g];
  const int32_t n = g->n;
  const int64_t cap = (int64_t)n + g->m / kItemEdges + 32;
  if (!w) {
    w = new PushWork();
    try {
      w->n = n;
      w->p = (double*)dalloc((size_t)n * 8, s);
      w->r = (double*)dalloc((size_t)n * 8, s);
      w->dirty = (uint32_t*)dalloc(((size_t)n + 31) / 32 * 4, s);
      w->front[0] = (int32_t*)dalloc((size_t)n * 4, s);
      w->front[1] = (int32_t*)dalloc((size_t)n * 4, s);
      w->famt = (double*)dalloc((size_t)n * 8, s);
      w->ctl = (PushCtl*)dalloc(sizeof(PushCtl), s);
      GPR_CUDA(cudaMemsetAsync(w->p, 0, (size_t)n * 8, s));
      GPR_CUDA(cudaMemsetAsync(w->r, 0, (size_t)n * 8, s));
      GPR_CUDA(cudaMemsetAsync(w->dirty, 0, ((size_t)n + 31) / 32 * 4, s));
    } catch (...) {
      free_work(w, s);
      g_work.erase(g);
      throw;
    }
  }
  if (w->item_cap < cap) {
    dfree(w->item_f, s);
    dfree(w->item_e, s);
    w->item_f = w->item_e = nullptr;
    w->item_cap = 0;
    w->item_f = (int32_t*)dalloc((size_t)cap * 4, s);
    w->item_e = (int32_t*)dalloc((size_t)cap * 4, s);
    w->item_cap = cap;
  }
  return w;
}

// After a failed call the workspace may hold residue: drop it.
void drop_work(const gpr_graph* g, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g_work_mu);
  auto it = g_work.find(g);
  if (it == g_work.end()) return;
  cudaDeviceSynchronize();  // the push may have been running on another stream
  free_work(it->second, s);
  g_work.erase(it);
}

// p[v] = r[v] = 0 for every node marked in dirty; the marks cleared.
__global__ void wipe_kernel(double* __restrict__ p, double* __restrict__ r, uint32_t* __restrict__ dirty,
                            int32_t n) {
  const int64_t words = ((int64_t)n + 31) / 32;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < words; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t bits = dirty[i];
    if (!bits) continue;
    dirty[i] = 0;
    for (; bits; bits &= bits - 1) {
      const int64_t v = i * 32 + __ffs(bits) - 1;
      p[v] = 0.0;
      r[v] = 0.0;
    }
  }
}

void wipe(PushWork* w, cudaStream_t s) {
  wipe_kernel<<<grid_items((w->n + 31) / 32), kBlock, 0, s>>>(w->p, w->r, w->dirty, w->n);
  GPR_CUDA(cudaGetLastError());
  count_launches(1);
}

// Reverse push from relabelled node tn into the workspace's p, r
// (relabelled, zero on entry) on stream s; its counters into st (pushes,
// edges, rounds).
void reverse_push(const gpr_graph* g, int32_t tn, double d, double r_max, PushWork* W, cudaStream_t s,
                  gpr_target_stats* st) {
  const int32_t n = g->n;
  const int64_t item_cap = W->item_cap;
  int32_t* const* front = W->front;
  double* famt = W->famt;
  int32_t* item_f = W->item_f;
  int32_t* item_e = W->item_e;
  PushCtl* ctl = W->ctl;
  double* p = W->p;
  double* r = W->r;
  GPR_CUDA(cudaMemsetAsync(ctl, 0, sizeof(PushCtl), s));
  set_residual_kernel<<<1, 1, 0, s>>>(r, tn, front[0], ctl, 1.0 > r_max ? 1 : 0, W->dirty);
  GPR_CUDA(cudaGetLastError());
  count_launches(1);
  const double a = 1.0 - d;
  const int gt = grid_items(n), gs = grid_items(item_cap);
  int32_t round = 0;
  PushCtl h{};
  for (int batch = kRoundsPerCheck / 2;; batch = kRoundsPerCheck) {
    for (int q = 0; q < batch; ++q, ++round) {
      const int cur = round & 1;
      push_take_kernel<<<gt, kBlock, 0, s>>>(g->col_ptr, front[cur], ctl, cur, a, d, p, r, famt, item_f, item_e, n,
                                             (uint32_t)item_cap);
      push_scatter_kernel<<<gs, kBlock, 0, s>>>(g->col_ptr, g->row_idx, g->outdeg, front[cur], item_f, item_e, famt,
                                                ctl, cur, r_max, r, front[cur ^ 1], n, (uint32_t)item_cap, W->dirty);
    }
    GPR_CUDA(cudaGetLastError());
    count_launches(2 * batch);
    GPR_CUDA(cudaMemcpyAsync(&h, ctl, sizeof h, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    if (h.overflow) throw StatusFail{GPR_ECUDA, "reverse push: frontier or work list overflow"};
    if (h.fcount[round & 1] == 0) break;
    if (round >= kMaxRounds) throw StatusFail{GPR_ETIMEOUT, "reverse push: no end after 65536 rounds"};
  }
  st->pushes = (int64_t)h.pushes;
  st->edges = (int64_t)h.edges;
  st->rounds = (int32_t)h.rounds;
}

struct Events {
  cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
  Events() {
    for (auto& x : e) GPR_CUDA(cudaEventCreate(&x));
  }
  ~Events() {
    for (auto& x : e)
      if (x) cudaEventDestroy(x);
  }
  double ms(int a, int b) const {
    float t = 0.f;
    GPR_CUDA(cudaEventElapsedTime(&t, e[a], e[b]));
    return t;
  }
};

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

// Frees the push workspace of g, if it has one (called when g is freed).
void target_work_free(const gpr_graph* g, cudaStream_t s) {
  std::lock_guard<std::mutex> lock(g_work_mu);
  auto it = g_work.find(g);
  if (it == g_work.end()) return;
  free_work(it->second, s);
  g_work.erase(it);
}

gpr_status run_reverse_push(gpr_graph* g, int32_t target, double d, double r_max, double* p_out, double* r_out,
                            gpr_target_stats* stats, int flags, cudaStream_t s) {
  try {
    check_args(g, target, d, r_max);
    const int32_t n = g->n;
    std::lock_guard<std::mutex> lock(g->mu);
    Buffers buf{s, {}};
    Events ev;
    gpr_target_stats st{};
    PushWork* W = push_work(g, s);
    const int32_t tn = relabelled(g, target, s);
    GPR_CUDA(cudaEventRecord(ev.e[0], s));
    reverse_push(g, tn, d, r_max, W, s, &st);
    GPR_CUDA(cudaEventRecord(ev.e[1], s));
    double* outs[2] = {p_out, r_out};
    const double* ins[2] = {W->p, W->r};
    for (int q = 0; q < 2; ++q) {
      if (!outs[q]) continue;
      double* dst = (flags & GPR_PTR_HOST) ? (double*)buf.get((size_t)n * 8) : outs[q];
      to_caller_kernel<<<grid_items(n), kBlock, 0, s>>>(ins[q], g->plan.old2new, n, dst);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
      if (flags & GPR_PTR_HOST) GPR_CUDA(cudaMemcpyAsync(outs[q], dst, (size_t)n * 8, cudaMemcpyDeviceToHost, s));
    }
    wipe(W, s);
    GPR_CUDA(cudaStreamSynchronize(s));
    st.push_ms = ev.ms(0, 1);
    st.total_ms = st.push_ms;
    if (stats) *stats = st;
    return GPR_OK;
  } catch (const StatusFail& f) {
    drop_work(g, s);
    set_error("ppr_reverse_push: %s", f.msg.c_str());
    return f.st;
  } catch (const CudaFail& f) {
    cudaGetLastError();
    drop_work(g, s);
    set_error("ppr_reverse_push: %s failed: %s", f.what, cudaGetErrorString(f.err));
    return GPR_ECUDA;
  }
}

gpr_status run_ppr_target(gpr_graph* g, int32_t target, double d, double r_max, const int32_t* sources, int32_t k,
                          int32_t walks, uint64_t seed, double* est_out, gpr_target_stats* stats, int flags,
                          cudaStream_t s) {
  bool pushed = false;
  try {
    check_args(g, target, d, r_max);
    if (k < 0 || walks < 1) throw StatusFail{GPR_EINVAL, "need k >= 0 sources and walks >= 1"};
    if ((int64_t)k * walks > INT32_MAX) throw StatusFail{GPR_EINVAL, "k * walks must stay below 2^31"};
    if (k == 0) {
      if (stats) *stats = gpr_target_stats{};
      return GPR_OK;
    }
    const int32_t n = g->n;
    std::lock_guard<std::mutex> lock(g->mu);  // the walk arrays and the push workspace are the graph's
    if (!g->walk_ptr) {
      build_caller_out_adjacency(g, s, &g->walk_ptr, &g->walk_adj);
      g->walk_nbr = (int2*)dalloc((size_t)std::max<int64_t>(g->m, 1) * sizeof(int2), s);
      walk_nbr_kernel<<<grid_items(g->m), kBlock, 0, s>>>(g->walk_ptr, g->walk_adj, g->plan.old2new, g->m,
                                                           g->walk_nbr);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
    }
    Buffers buf{s, {}};
    Events ev;
    gpr_target_stats st{};
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
    const int64_t total = (int64_t)k * walks;
    int32_t* end = (int32_t*)buf.get((size_t)total * 4);
    unsigned long long* steps_dev = (unsigned long long*)buf.get(8);
    PushWork* W = push_work(g, s);
    GPR_CUDA(cudaMemsetAsync(steps_dev, 0, 8, s));
    int32_t tn = 0;
    int herr = 0;
    GPR_CUDA(cudaMemcpyAsync(&tn, g->plan.old2new + target, 4, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    if (herr) throw StatusFail{GPR_EINVAL, "a source id is out of range"};
    // the push on a high-priority stream, the walks beside it on s; they meet
    // at the estimate
    cudaStream_t ps = push_stream();
    GPR_CUDA(cudaEventRecord(ev.e[0], s));
    GPR_CUDA(cudaStreamWaitEvent(ps, ev.e[0], 0));
    // about two resident waves of warps, each with a pool of >= 64 walks
    const int64_t resident_warps = (int64_t)num_sms() * 64;
    const int32_t per_warp = (int32_t)std::max<int64_t>(64, std::min<int64_t>(4096, total / (2 * resident_warps)));
    const int64_t warps = (total + per_warp - 1) / per_warp;
    const double a = 1.0 - d;
    const uint64_t stop_below = (uint64_t)std::ceil(std::ldexp(a, 53));
    walk_kernel<<<(unsigned)((warps * 32 + kBlock - 1) / kBlock), kBlock, 0, s>>>(
        g->walk_ptr, g->walk_nbr, g->walk_adj, g->plan.old2new, src, walks, total, per_warp, seed, stop_below, end,
        steps_dev);
    GPR_CUDA(cudaGetLastError());
    count_launches(1);
    GPR_CUDA(cudaEventRecord(ev.e[2], s));
    pushed = true;
    reverse_push(g, tn, d, r_max, W, ps, &st);
    GPR_CUDA(cudaEventRecord(ev.e[1], ps));
    GPR_CUDA(cudaStreamWaitEvent(s, ev.e[1], 0));
    double* out = (flags & GPR_PTR_HOST) ? (double*)buf.get((size_t)k * 8) : est_out;
    estimate_kernel<<<k, kBlock, 0, s>>>(W->p, W->r, g->plan.old2new, src, end, walks, d / a, out);
    GPR_CUDA(cudaGetLastError());
    count_launches(1);
    GPR_CUDA(cudaEventRecord(ev.e[3], s));
    wipe(W, s);
    unsigned long long steps = 0;
    GPR_CUDA(cudaMemcpyAsync(&steps, steps_dev, 8, cudaMemcpyDeviceToHost, s));
    if (flags & GPR_PTR_HOST) GPR_CUDA(cudaMemcpyAsync(est_out, out, (size_t)k * 8, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    st.walk_steps = (int64_t)steps;
    st.push_ms = ev.ms(0, 1);
    st.walk_ms = ev.ms(0, 2);
    st.total_ms = ev.ms(0, 3);
    if (stats) *stats = st;
    return GPR_OK;
  } catch (const StatusFail& f) {
    if (pushed) drop_work(g, s);
    set_error("ppr_target: %s", f.msg.c_str());
    return f.st;
  } catch (const CudaFail& f) {
    cudaGetLastError();
    if (pushed) drop_work(g, s);
    set_error("ppr_target: %s failed: %s", f.what, cudaGetErrorString(f.err));
    return GPR_ECUDA;
  }
}

}  // namespace gpr
