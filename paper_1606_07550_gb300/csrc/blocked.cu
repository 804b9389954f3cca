// Blocked schedule of the PageRank step (section 4 Table "snap_methods"),
// host side: the edge layout in bin-major order (one stable sort of the CSC
// edges by bin, then dense source or source block), the expand and
// accumulate work units, and the recording of steps.  The kernels and the
// layout's description are in blocked_kernels.cuh.
#include <algorithm>
#include <memory>
#include <mutex>
#include <vector>

#include "blocked_kernels.cuh"

namespace gpr {

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
      bk_keys_kernel<<<grid, 256, 0, s>>>(g->col_ptr, g->row_idx, n, sb_bits, w_bits, kg.kbits, k->n_dense, D,
                                          kg.kb_bits, keys);
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
    // kMaxUnitSegs segments; a longer segment is cut into pieces of its own
    std::vector<ExpandUnit> xu;
    for (int32_t sb = D; sb < S; ++sb) {
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
            xu.push_back(ExpandUnit{sb, b, b + 1, (int32_t)(lo + o), (int32_t)std::min<int64_t>(hi, lo + o + xunit)});
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
