// Blocked schedule of the PageRank step (section 4 Table "snap_methods"),
// host side: the edge layout in bin-major order (one stable sort of the CSC
// edges by bin, then dense source or source block), the expand and
// accumulate work units, and the recording of steps.  The kernels and the
// layout's description are in blocked_kernels.cuh.
#include <algorithm>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "blocked_kernels.cuh"

namespace gpr {

// ---- layout construction --------------------------------------------------

// The sort index of an edge: bin b, then its dense source u (u < n_dense),
// or n_dense + (its source block - D); kb_bits bits per bin.
__device__ __forceinline__ uint64_t bk_index(uint64_t b, uint32_t u, int sb_bits, int32_t n_dense, int32_t D,
                                             int kb_bits) {
  const uint64_t j = u < (uint32_t)n_dense ? (uint64_t)u : (uint64_t)n_dense + ((u >> sb_bits) - (uint32_t)D);
  return (b << kb_bits) | j;
}
// The segment (b, s) of a sort index.
__device__ __forceinline__ int64_t bk_segment(uint64_t kidx, int sb_bits, int32_t n_dense, int32_t D, int kb_bits,
                                              int32_t S) {
  const int64_t b = (int64_t)(kidx >> kb_bits);
  const uint64_t j = kidx & ((1ull << kb_bits) - 1);
  const int64_t s = j < (uint64_t)n_dense ? (int64_t)(j >> sb_bits) : (int64_t)D + (int64_t)(j - (uint64_t)n_dense);
  return b * S + s;
}

// key = row-in-bin | source-in-block | sort index, one per CSC edge, in CSC
// order (256 threads per block).
__global__ void __launch_bounds__(256) bk_keys_kernel(const int32_t* __restrict__ col_ptr,
                                                      const int32_t* __restrict__ row_idx, int32_t n, int sb_bits,
                                                      int w_bits, int kbits, int32_t n_dense, int32_t D, int kb_bits,
                                                      uint64_t* __restrict__ keys) {
  __shared__ int32_t s_rows[8][kMarkStride];
  const uint32_t sb_mask = (1u << sb_bits) - 1;
  for_each_edge_with_row_marked(col_ptr, n, s_rows[threadIdx.x >> 5], [&](int64_t e, int32_t p) {
    const uint64_t b = (uint64_t)(p >> w_bits);
    const uint64_t hi = (uint64_t)(p & ((1 << w_bits) - 1)) << (sb_bits + kbits);
    const uint32_t u = (uint32_t)row_idx[e];
    keys[e] = hi | ((uint64_t)(u & sb_mask) << kbits) | bk_index(b, u, sb_bits, n_dense, D, kb_bits);
  });
}

// From the keys sorted (stably) on their low kbits bits, in bin-major edge
// order: the packed word of every dense-source edge, the local ids of every
// other edge, and seg[k] = first edge of segment k (seg[nseg] = m).  A thread
// takes four consecutive edges; a bin's dense edges precede its others, so
// four are nearly always of one kind and go out as one vector store.
__global__ void bk_extract_kernel(const uint64_t* __restrict__ keys, int64_t m, int sb_bits, int kbits,
                                  int32_t n_dense, int32_t D, int kb_bits, int dense_bits, int32_t S, int64_t nseg,
                                  uint16_t* __restrict__ src_lo, uint16_t* __restrict__ dst_lo,
                                  uint32_t* __restrict__ vals, int32_t* __restrict__ seg) {
  const uint64_t kmask = (1ull << kbits) - 1;
  const uint64_t jmask = (1ull << kb_bits) - 1;
  const uint32_t smask = (1u << sb_bits) - 1;
  const int64_t nq = (m + 3) / 4;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = 4 * q;
    const bool full = i0 + 4 <= m;
    uint64_t key[4];
    if (full) {
      const ulonglong2 a = *reinterpret_cast<const ulonglong2*>(keys + i0);
      const ulonglong2 b = *reinterpret_cast<const ulonglong2*>(keys + i0 + 2);
      key[0] = a.x;
      key[1] = a.y;
      key[2] = b.x;
      key[3] = b.y;
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) key[j] = i0 + j < m ? keys[i0 + j] : 0ull;
    }
    int64_t prev = i0 > 0 ? bk_segment(keys[i0 - 1] & kmask, sb_bits, n_dense, D, kb_bits, S) : -1;
    uint32_t v[4];
    uint16_t sl[4], dl[4];
    int ndense = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const uint64_t kidx = key[j] & kmask;
      const uint64_t jj = kidx & jmask;
      const uint32_t r = (uint32_t)(key[j] >> (kbits + sb_bits));
      const bool dn = jj < (uint64_t)n_dense;
      ndense += dn;
      v[j] = (uint32_t)jj | (r << dense_bits);
      sl[j] = (uint16_t)((key[j] >> kbits) & smask);
      dl[j] = (uint16_t)r;
      if (i0 + j < m) {
        const int64_t k = bk_segment(kidx, sb_bits, n_dense, D, kb_bits, S);
        for (int64_t kk = prev + 1; kk <= k; ++kk) seg[kk] = (int32_t)(i0 + j);
        prev = k;
        if (i0 + j == m - 1)
          for (int64_t kk = k + 1; kk <= nseg; ++kk) seg[kk] = (int32_t)m;
        if (!full) {
          if (dn) {
            vals[i0 + j] = v[j];
          } else {
            src_lo[i0 + j] = sl[j];
            dst_lo[i0 + j] = dl[j];
          }
        }
      }
    }
    if (!full) continue;
    if (ndense == 4) {
      *reinterpret_cast<uint4*>(vals + i0) = make_uint4(v[0], v[1], v[2], v[3]);
    } else if (ndense == 0) {
      *reinterpret_cast<uint2*>(src_lo + i0) =
          make_uint2((uint32_t)sl[0] | ((uint32_t)sl[1] << 16), (uint32_t)sl[2] | ((uint32_t)sl[3] << 16));
      *reinterpret_cast<uint2*>(dst_lo + i0) =
          make_uint2((uint32_t)dl[0] | ((uint32_t)dl[1] << 16), (uint32_t)dl[2] | ((uint32_t)dl[3] << 16));
    } else {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (((key[j] & kmask) & jmask) < (uint64_t)n_dense) {
          vals[i0 + j] = v[j];
        } else {
          src_lo[i0 + j] = sl[j];
          dst_lo[i0 + j] = dl[j];
        }
      }
    }
  }
}

// xseg[s * B + b] = edges of segment (b, s).
__global__ void bk_transpose_kernel(const int32_t* __restrict__ seg, int32_t S, int32_t B, int2* __restrict__ xseg) {
  const int64_t nseg = (int64_t)S * B;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nseg; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = k / S, s = k - b * S;
    xseg[s * B + b] = make_int2(seg[k], seg[k + 1]);
  }
}

// ---- host side --------------------------------------------------------------

static int bits_to_hold(uint64_t v) {
  int b = 0;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

// Key bits of the sort index: the radix sort orders whole 8-bit digits, so
// the index takes whole digits and the payload above it stays out of them.
static int segment_key_bits(int64_t nidx) {
  const int b = std::max(1, bits_to_hold((uint64_t)(nidx - 1)));
  return (b + 7) & ~7;
}

// Geometry of the sort index for n_dense dense sources: kb_bits bits per bin
// (room for n_dense dense sources and S - D other source blocks), kbits in
// all (whole digits).
struct KeyGeom {
  int kb_bits, kbits;
};
static KeyGeom key_geom(int64_t S, int64_t B, int32_t n_dense, int sb_bits) {
  const int64_t per_bin = (int64_t)n_dense + S - ((int64_t)n_dense >> sb_bits);
  KeyGeom k;
  k.kb_bits = bits_to_hold((uint64_t)std::max<int64_t>(per_bin - 1, 0));
  k.kbits = segment_key_bits(B << k.kb_bits);
  return k;
}

static int smem_optin() {
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device_ordinal());
  return optin;
}

static size_t expand_smem(int sb_bits) { return expand_ids_offset(sb_bits) + kExpandStageBytes; }
static size_t accum_smem(int w_bits) { return ((size_t)8 << w_bits) + kAccumStageBytes; }

static bool geometry_fits(const gpr_graph* g, int sb_bits, int w_bits, int32_t n_dense) {
  const int64_t S = ((int64_t)g->n + (1 << sb_bits) - 1) >> sb_bits;
  const int64_t B = ((int64_t)g->n + (1 << w_bits) - 1) >> w_bits;
  const KeyGeom kg = key_geom(S, B, n_dense, sb_bits);
  return kg.kbits + sb_bits + w_bits <= 64;
}

bool blocked_eligible(const gpr_graph* g, int sb_bits, int w_bits) {
  if (sb_bits < 4 || sb_bits > 16 || w_bits < 4 || w_bits > 16) return false;
  if (g->n < 1 || g->m > (int64_t)INT32_MAX - 2 * kChunk) return false;
  const int64_t S = ((int64_t)g->n + (1 << sb_bits) - 1) >> sb_bits;
  const int64_t B = ((int64_t)g->n + (1 << w_bits) - 1) >> w_bits;
  const int64_t nseg = S * B;
  if (nseg > ((int64_t)1 << 26)) return false;  // segment tables of at most 2^26 entries
  if (!geometry_fits(g, sb_bits, w_bits, 0)) return false;
  const size_t optin = (size_t)smem_optin();
  // static shared memory of the kernels is below 2 KB
  return expand_smem(sb_bits) + 2048 <= optin && accum_smem(w_bits) + 2048 <= optin;
}

int32_t blocked_max_dense(const gpr_graph* g, int sb_bits, int w_bits) {
  if (!blocked_eligible(g, sb_bits, w_bits)) return 0;
  const int dense_bits = 32 - w_bits;
  int64_t d = std::min<int64_t>((int64_t)1 << dense_bits, g->n);
  d = (d >> sb_bits) << sb_bits;  // whole source blocks
  while (d > 0 && !geometry_fits(g, sb_bits, w_bits, (int32_t)d)) d = ((d >> 1) >> sb_bits) << sb_bits;
  return (int32_t)d;
}

void blocked_free(Blocked* k, cudaStream_t s) {
  if (!k) return;
  dfree(k->src_lo, s);
  dfree(k->dst_lo, s);
  dfree(k->vals, s);
  dfree(k->xseg, s);
  dfree(k->xu, s);
  dfree(k->au, s);
  dfree(k->acc_g, s);
  dfree(k->bin_arrive, s);
  dfree(k->ctr, s);
  dfree(k->partials, s);
  delete k;
}

template <typename K>
static int persistent_grid(K kernel, size_t smem) {
  GPR_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  GPR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kBkThreads, smem));
  return num_sms() * std::max(per_sm, 1);
}

Blocked* blocked_build(const gpr_graph* g, int sb_bits, int w_bits, int32_t n_dense_req, int64_t unit_edges,
                       cudaStream_t s) {
  const int64_t unit = std::max<int64_t>(unit_edges, 1 << 12);
  const int64_t xunit = std::min<int64_t>(1 << 20, 4 * unit);  // expand units stage a source block each
  if (!blocked_eligible(g, sb_bits, w_bits))
    throw StatusFail{GPR_EINVAL, "the blocked schedule does not fit this graph"};
  Blocked* k = new Blocked();
  k->sb_bits = sb_bits;
  k->w_bits = w_bits;
  k->unit_edges = unit;
  k->dense_bits = 32 - w_bits;
  {
    const int32_t cap = blocked_max_dense(g, sb_bits, w_bits);
    int32_t nd = std::max<int32_t>(0, std::min(n_dense_req, cap));
    k->n_dense = (nd >> sb_bits) << sb_bits;
    k->D = k->n_dense >> sb_bits;
  }
  {
    int lg = 0;
    while (((int64_t)1 << lg) < g->n) ++lg;  // ceil(log2 n)
    k->ubits = std::min(60, 28 + lg);
  }
  const int32_t n = g->n;
  const int64_t m = g->m;
  k->S = (int32_t)(((int64_t)n + (1 << sb_bits) - 1) >> sb_bits);
  k->B = (int32_t)(((int64_t)n + (1 << w_bits) - 1) >> w_bits);
  const int32_t S = k->S, B = k->B, D = k->D;
  const int64_t nseg = (int64_t)S * B;
  const KeyGeom kg = key_geom(S, B, k->n_dense, sb_bits);
  std::unique_ptr<SortScratch> sc;  // the sort's two key buffers, until the segment table is read
  int32_t* seg = nullptr;
  int* derr = nullptr;
  try {
    trace_phase(nullptr, s);
    // whole 256-edge chunks are copied: kPad entries past the end, zeroed
    const size_t me = (size_t)m + kPad;
    k->src_lo = (uint16_t*)dalloc(me * 2, s);
    k->dst_lo = (uint16_t*)dalloc(me * 2, s);
    k->vals = (uint32_t*)dalloc(me * 4, s);
    GPR_CUDA(cudaMemsetAsync(k->src_lo + m, 0, kPad * 2, s));
    GPR_CUDA(cudaMemsetAsync(k->dst_lo + m, 0, kPad * 2, s));
    GPR_CUDA(cudaMemsetAsync(k->vals + m, 0, kPad * 4, s));
    seg = (int32_t*)dalloc((size_t)(nseg + 1) * 4, s);
    derr = (int*)dalloc(sizeof(int) * 2, s);
    GPR_CUDA(cudaMemsetAsync(derr, 0, sizeof(int) * 2, s));
    const int grid = num_sms() * 8;
    if (m > 0) {
      sc.reset(new SortScratch((size_t)m, s));
      uint64_t* keys = sc->a;
      uint64_t* alt = sc->b;
      trace_phase("layout: allocations", s);
      static const int keys_per_sm = [] {  // resident blocks: the chunks are dealt out statically
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, bk_keys_kernel, 256, 0);
        return std::max(b, 1);
      }();
      bk_keys_kernel<<<num_sms() * keys_per_sm, 256, 0, s>>>(g->col_ptr, g->row_idx, n, sb_bits, w_bits, kg.kbits,
                                                             k->n_dense, D, kg.kb_bits, keys);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
      trace_phase("layout: keys", s);
      const uint64_t* sorted = radix_sort_u64(keys, alt, m, kg.kbits, s, derr);
      trace_phase("layout: sort", s);
      bk_extract_kernel<<<grid, 256, 0, s>>>(sorted, m, sb_bits, kg.kbits, k->n_dense, D, kg.kb_bits, k->dense_bits,
                                             S, nseg, k->src_lo, k->dst_lo, k->vals, seg);
      GPR_CUDA(cudaGetLastError());
      count_launches(1);
    } else {
      GPR_CUDA(cudaMemsetAsync(seg, 0, (size_t)(nseg + 1) * 4, s));
    }
    k->xseg = (int2*)dalloc((size_t)nseg * sizeof(int2), s);
    bk_transpose_kernel<<<grid, 256, 0, s>>>(seg, S, B, k->xseg);
    GPR_CUDA(cudaGetLastError());
    count_launches(1);
    // the segment table on the host, source-block major (contiguous per
    // block), in pinned staging memory kept for the process (one layout
    // build at a time uses it)
    static std::mutex stage_mu;
    static int2* stage = nullptr;
    static size_t stage_cap = 0;
    std::lock_guard<std::mutex> stage_lk(stage_mu);
    const size_t need = (size_t)std::max<int64_t>(nseg, 1);
    if (stage_cap < need) {
      if (stage) cudaFreeHost(stage);
      stage = nullptr;
      stage_cap = 0;
      GPR_CUDA(cudaMallocHost((void**)&stage, need * sizeof(int2)));
      stage_cap = need;
    }
    int2* const X = stage;
    int herr = 0;
    GPR_CUDA(cudaMemcpyAsync(X, k->xseg, (size_t)nseg * sizeof(int2), cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    sc.reset();
    dfree(seg, s);
    dfree(derr, s);
    seg = nullptr;
    derr = nullptr;
    if (herr & DERR_TIMEOUT) throw StatusFail{GPR_ETIMEOUT, "blocked layout: a look-back wait of the sort timed out"};
    trace_phase("layout: extract + tables", s);

    // expand units (source blocks past the dense ones): per source block,
    // runs of consecutive bins' segments of at most unit edges and
    // kMaxUnitSegs segments; a longer segment is cut into pieces of its own.
    // Source blocks are independent: a few host threads take a range each
    // and the lists are joined in block order.
    auto expand_units = [&](int32_t sb0, int32_t sb1, std::vector<ExpandUnit>& xu) {
      for (int32_t sb = sb0; sb < sb1; ++sb) {
        int32_t first = -1, last = -1, clo = 0, chi = 0;
        int64_t edges = 0;
        auto flush = [&]() {
          if (first >= 0 && edges > 0) xu.push_back(ExpandUnit{sb, first, last + 1, clo, chi});
          first = -1;
          edges = 0;
        };
        const int2* Xs = X + (size_t)sb * B;
        for (int32_t b = 0; b < B; ++b) {
          const int32_t lo = Xs[b].x, hi = Xs[b].y;
          const int64_t len = hi - lo;
          if (len == 0) continue;
          if (len > xunit) {
            flush();
            for (int64_t o = 0; o < len; o += xunit)
              xu.push_back(
                  ExpandUnit{sb, b, b + 1, (int32_t)(lo + o), (int32_t)std::min<int64_t>(hi, lo + o + xunit)});
            continue;
          }
          if (first >= 0 && (edges + len > xunit || b - first >= kMaxUnitSegs)) flush();
          if (first < 0) {
            first = b;
            clo = lo;
          }
          last = b;
          chi = hi;
          edges += len;
        }
        flush();
      }
    };
    const int32_t nblk = S - D;
    const int nth = (int)std::max<int64_t>(1, std::min<int64_t>(8, (int64_t)nblk * B / (1 << 18)));
    std::vector<std::vector<ExpandUnit>> xparts(nth);
    {
      std::vector<std::thread> pool;
      for (int t = 1; t < nth; ++t)
        pool.emplace_back(expand_units, D + (int32_t)((int64_t)nblk * t / nth),
                          D + (int32_t)((int64_t)nblk * (t + 1) / nth), std::ref(xparts[t]));
      expand_units(D, D + (int32_t)((int64_t)nblk / nth), xparts[0]);
      for (std::thread& th : pool) th.join();
    }
    std::vector<ExpandUnit> xu;
    for (const auto& v : xparts) xu.insert(xu.end(), v.begin(), v.end());
    // accumulate units: each bin whole, or cut into near-equal edge ranges;
    // each knows where the bin's dense-source edges end
    std::vector<AccumUnit> au;
    int32_t n_split = 0;
    int64_t dense_edges = 0;
    const int2* X0 = X;                    // tiles (b, 0)
    const int2* XD = X + (size_t)D * B;     // tiles (b, D), the first after the dense ones
    const int2* XL = X + (size_t)(S - 1) * B;  // tiles (b, S - 1), the last of each bin
    for (int32_t b = 0; b < B; ++b) {
      const int64_t lo = X0[b].x, hi = XL[b].y;
      const int64_t mid = D < S ? XD[b].x : hi;
      dense_edges += mid - lo;
      const int64_t e = hi - lo;
      const int32_t parts = (int32_t)std::max<int64_t>(1, (e + unit - 1) / unit);
      const int32_t split = parts > 1 ? n_split++ : -1;
      for (int32_t q = 0; q < parts; ++q) {
        const int64_t pl = lo + e * q / parts, ph = lo + e * (q + 1) / parts;
        const int64_t pm = std::min(std::max(mid, pl), ph);
        au.push_back(AccumUnit{b, (int32_t)pl, (int32_t)pm, (int32_t)ph, parts, split});
      }
    }
    k->dense_edges = dense_edges;
    trace_phase("layout: units (host)", s);
    // largest first: the dynamic queues then end with small units
    std::stable_sort(xu.begin(), xu.end(),
                     [](const ExpandUnit& a, const ExpandUnit& b) { return a.hi - a.lo > b.hi - b.lo; });
    std::stable_sort(au.begin(), au.end(),
                     [](const AccumUnit& a, const AccumUnit& b) { return a.hi - a.lo > b.hi - b.lo; });
    k->n_xu = (int32_t)xu.size();
    k->n_au = (int32_t)au.size();
    k->n_split = n_split;
    k->xu = (ExpandUnit*)dalloc(std::max<size_t>(xu.size(), 1) * sizeof(ExpandUnit), s);
    k->au = (AccumUnit*)dalloc(au.size() * sizeof(AccumUnit), s);
    if (!xu.empty())
      GPR_CUDA(cudaMemcpyAsync(k->xu, xu.data(), xu.size() * sizeof(ExpandUnit), cudaMemcpyHostToDevice, s));
    GPR_CUDA(cudaMemcpyAsync(k->au, au.data(), au.size() * sizeof(AccumUnit), cudaMemcpyHostToDevice, s));
    const size_t W = (size_t)1 << w_bits;
    if (n_split > 0) {
      k->acc_g = (unsigned long long*)dalloc((size_t)n_split * W * 8, s);
      k->bin_arrive = (unsigned int*)dalloc((size_t)n_split * 4, s);
      GPR_CUDA(cudaMemsetAsync(k->acc_g, 0, (size_t)n_split * W * 8, s));
      GPR_CUDA(cudaMemsetAsync(k->bin_arrive, 0, (size_t)n_split * 4, s));
    }
    k->ctr = (unsigned int*)dalloc(16, s);
    GPR_CUDA(cudaMemsetAsync(k->ctr, 0, 16, s));
    k->partials = (double*)dalloc((size_t)B * 3 * sizeof(double), s);
    k->xgrid = persistent_grid(bk_expand_kernel, expand_smem(sb_bits));
    k->agrid = std::max(persistent_grid(bk_accum_kernel<float>, accum_smem(w_bits)),
                        persistent_grid(bk_accum_kernel<__nv_bfloat16>, accum_smem(w_bits)));
    trace_phase("layout: upload", s);
    k->bytes = (int64_t)me * 8 + nseg * (int64_t)sizeof(int2) + (int64_t)xu.size() * sizeof(ExpandUnit) +
               (int64_t)au.size() * sizeof(AccumUnit) + (int64_t)n_split * (int64_t)W * 8 + (int64_t)B * 24;
    return k;
  } catch (...) {
    sc.reset();
    dfree(seg, s);
    dfree(derr, s);
    blocked_free(k, s);
    throw;
  }
}

void blocked_record_reset(Blocked* k, cudaStream_t s) { GPR_CUDA(cudaMemsetAsync(k->ctr, 0, 16, s)); }

template <typename T>
void blocked_record_codes(Blocked* k, const gpr_graph* g, const float* x, const float* inv_deg, uint32_t* c,
                          cudaStream_t s) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(((int64_t)g->n + 255) / 256, num_sms() * 8));
  bk_codes_kernel<T><<<grid, 256, 0, s>>>(x, inv_deg, g->n, k->ubits, c);
  GPR_CUDA(cudaGetLastError());
}

template <typename T>
void blocked_record_step(Blocked* k, const gpr_graph* g, const uint32_t* c_in, const float* x_in, float* x_out,
                         uint32_t* c_out, const float* inv_deg, StepParams* prm, double* log_row, int32_t it,
                         cudaStream_t s) {
  // every CTA of a launch takes units until one fetch fails: a launch moves
  // a counter by exactly (units + grid)
  const unsigned int ex = (unsigned int)((int64_t)it * (k->n_xu + k->xgrid));
  const unsigned int ea = (unsigned int)((int64_t)it * (k->n_au + k->agrid));
  bk_expand_kernel<<<k->xgrid, kBkThreads, expand_smem(k->sb_bits), s>>>(
      c_in, g->n, k->sb_bits, k->B, k->xseg, k->xu, k->n_xu, k->src_lo, k->vals, k->ctr, ex);
  bk_accum_kernel<T><<<k->agrid, kBkThreads, accum_smem(k->w_bits), s>>>(
      k->vals, k->dst_lo, c_in, k->dense_bits, g->n, k->w_bits, k->ubits, k->au, k->n_au, k->ctr, ea, k->acc_g,
      k->bin_arrive, x_in, inv_deg, x_out, c_out, prm, k->partials, k->B, log_row);
  GPR_CUDA(cudaGetLastError());
}

template void blocked_record_codes<float>(Blocked*, const gpr_graph*, const float*, const float*, uint32_t*,
                                          cudaStream_t);
template void blocked_record_codes<__nv_bfloat16>(Blocked*, const gpr_graph*, const float*, const float*, uint32_t*,
                                                  cudaStream_t);
template void blocked_record_step<float>(Blocked*, const gpr_graph*, const uint32_t*, const float*, float*,
                                         uint32_t*, const float*, StepParams*, double*, int32_t, cudaStream_t);
template void blocked_record_step<__nv_bfloat16>(Blocked*, const gpr_graph*, const uint32_t*, const float*, float*,
                                                 uint32_t*, const float*, StepParams*, double*, int32_t,
                                                 cudaStream_t);

}  // namespace gpr
