// Blocked schedule of the PageRank step (section 4 Table "snap_methods"):
// the same step as the pull kernels of pagerank.cu, with the per-edge random
// gather c[u] replaced by streaming phases.
//
// Sources are cut into blocks of 2^sb_bits relabelled ids and rows
// (destinations) into bins of 2^w_bits.  Relabelled ids run by descending
// out-degree, so the first sources hold a large share of the edges (at R-MAT
// scale 25 the first 2^18 of 2^25 sources hold about 60%).  The first
// n_dense sources (whole blocks, n_dense < 2^(32 - w_bits)) are "dense".  The
// edges are stored once in bin-major order: in bin b, first the edges of the
// dense sources, ordered by source then row, each as one packed 32-bit word
// source | row << (32 - w_bits); then, for each other source block s, the
// edges of segment (b, s) in CSC order (row, then source) as 16-bit local
// source and row ids.  The contributions c are held as 32-bit codes (below).
// Per step:
//   expand      for each non-dense source block s, its codes are copied into
//               shared memory and every edge of its segments gets
//               vals[e] = code[u], reading 16-bit local source ids: a read
//               stream and a write stream, with the random reads served by
//               shared memory;
//   accumulate  for each bin, the packed words of its dense-source edges are
//               streamed and each edge's code read straight from c (the dense
//               sources' codes, at most 1 MB, stay in cache, and a run of
//               edges shares few consecutive sources), then the codes and
//               16-bit rows of its other edges are streamed; all are added
//               into one accumulator per row in shared memory; the bin's rows
//               are then finished (x', c', partial sums) as in the pull
//               schedule.
// Sums are exact integers.  With a unit of 2^-U (U = min(60, 28 +
// ceil(log2 n))), contribution c is the integer q = floor(c * 2^U), and each
// row's accumulator holds the exact 64-bit sum of its q, so y[v] does not
// depend on the order of the additions, nor on which sources are dense: runs
// are bitwise reproducible however units are scheduled.  The 32-bit code of
// c is q itself when q < 2^31 (c < 2^(31-U), about 8 / n: nearly every
// contribution), else the bits of c with the top bit set, converted again
// where it is added.  Truncation costs less than 2^-U per edge (at most
// m * 2^-U in L1, 1.2e-7 for 2^25 nodes and 2^30 edges); y[v] is rounded
// to the nearest float.  With BF16 storage c is rounded to BF16 before it is
// coded.
//
// Streamed bytes per edge: 4 (packed word) for a dense source's edge;
// 2 (source id) + 4 (code written) in expand and 4 (code) + 2 (row id) in
// accumulate, 12, for the others.  The dense sources' codes are read from
// cache once per bin and source; the others' once per expand unit.
// Long rows need no special case: runs of one row are summed in registers
// before they reach shared memory (a warp step inside one row is added
// once), and a bin with many edges is cut into units whose sums meet in a
// global accumulator.
//
// This header holds the device side of a step: the expand and accumulate
// kernels and the code conversions; blocked.cu builds the layout (with its
// construction kernels) and records the steps.
#pragma once

#include "blocked.cuh"

namespace gpr {

constexpr int kBkThreads = 1024;
constexpr int kMaxUnitSegs = 1024;  // segments of one expand unit (one per thread in the prefix scan)
constexpr int kChunk = 256;         // edges per warp step: two runs of 4 consecutive edges per lane
constexpr int kMaxUnitChunks = (1 << 20) / kChunk + kMaxUnitSegs;  // chunks of one expand unit
constexpr int kPad = kChunk;        // entries after the end of the edge arrays (whole chunks are copied)
static_assert(kBkThreads == kMaxUnitSegs, "the segment scan gives one segment to each thread");

// floor(v * 2^U) from the bits of v (v >= 0, v * 2^U < 2^63), integer
// operations only (a float-to-64-bit conversion instruction would run on the
// FP64 pipe, which GB300 keeps slow).
__device__ __forceinline__ uint64_t fixed_of(float v, int U) {
  const uint32_t b = __float_as_uint(v);
  const int e = (int)(b >> 23);
  const int sh = e - 150 + U;  // v * 2^U = m * 2^sh
  const uint64_t m = (b & 0x7FFFFFu) | 0x800000u;
  if (e == 0 || sh < -24) return 0ull;  // zero, subnormal, or below one unit
  return sh >= 0 ? m << sh : m >> -sh;
}

// The 32-bit code of contribution c, and the integer value of a code.
__device__ __forceinline__ uint32_t code_of(float c, int U) {
  const uint64_t q = fixed_of(c, U);
  return q < 0x80000000ull ? (uint32_t)q : 0x80000000u | __float_as_uint(c);
}
__device__ __forceinline__ uint64_t value_of(uint32_t w, int U) {
  return (w >> 31) ? fixed_of(__uint_as_float(w & 0x7FFFFFFFu), U) : (uint64_t)w;
}

// a * 2^-U rounded to the nearest float (ties to even), integer operations only.
__device__ __forceinline__ float from_fixed(unsigned long long a, int U) {
  if (a == 0ull) return 0.f;
  const int msb = 63 - __clzll((long long)a);
  uint64_t m;
  int ex = msb;
  if (msb <= 23) {
    m = a << (23 - msb);
  } else {
    const int sh = msb - 23;
    m = a >> sh;
    const uint64_t rem = a & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) ++m;
    if (m >> 24) {  // rounded up to the next power of two
      m >>= 1;
      ++ex;
    }
  }
  return __uint_as_float((uint32_t)(ex - U + 127) << 23 | ((uint32_t)m & 0x7FFFFFu));
}

// Exact 64-bit addition into an accumulator held as two 32-bit words in
// shared memory, with 32-bit atomics: the low word takes the low half, and
// the high word the high half plus the carry out of the low word, seen in
// the value the low atomic returns.  Whatever the order of the additions,
// the number of carries is floor(sum of low halves / 2^32), so hi:lo ends
// as the exact sum.  (A 64-bit shared-memory atomic measured about twice as
// slow on GB300: four times the shared-memory wavefronts.)
// qh plus the carry out of old + ql.
__device__ __forceinline__ uint32_t carry_into(uint32_t old, uint32_t ql, uint32_t qh) {
  uint32_t up;
  asm("{\n\t.reg .u32 t;\n\tadd.cc.u32 t, %1, %2;\n\taddc.u32 %0, %3, 0;\n\t}" : "=r"(up) : "r"(old), "r"(ql), "r"(qh));
  return up;
}
__device__ __forceinline__ uint32_t atom_add(uint32_t addr, uint32_t v) {
  uint32_t old;
  asm volatile("atom.shared.add.u32 %0, [%1], %2;" : "=r"(old) : "r"(addr), "r"(v) : "memory");
  return old;
}
// Shared-memory addition of a non-zero amount (predicated: no branch).
__device__ __forceinline__ void red_add_nonzero(uint32_t addr, uint32_t v) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %1, 0;\n\t@p red.shared.add.u32 [%0], %1;\n\t}" ::"r"(addr),
               "r"(v)
               : "memory");
}

// ---- asynchronous copies to shared memory (cp.async) ------------------------
// Each lane copies exactly the bytes it later reads, so a wait on its own
// copy groups is the only synchronisation the staged data needs.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---- expand ---------------------------------------------------------------

// Shared memory of the expand kernel: codes (4 << sb_bits bytes), segment
// tables, the chunk map, then 16-byte-aligned per-warp staging slots.
__host__ __device__ constexpr size_t expand_ids_offset(int sb_bits) {
  return (((size_t)4 << sb_bits) + (size_t)(3 * kMaxUnitSegs + 1) * 4 + (size_t)kMaxUnitChunks * 2 + 15) & ~(size_t)15;
}
constexpr size_t kExpandStageBytes = (size_t)(kBkThreads / 32) * 128 * 8;
// Shared memory of the accumulate kernel: two 32-bit words per row of the
// bin, then per-warp staging slots (2 x (256 codes + 256 row ids)).
constexpr size_t kAccumSlotBytes = kChunk * 4 + kChunk * 2;
constexpr size_t kAccumStageBytes = (size_t)(kBkThreads / 32) * 2 * kAccumSlotBytes;

// Contributions as stored: FP32, or rounded to BF16 (nearest, ties to even).
__device__ __forceinline__ float round_store(float v, float*) { return v; }
__device__ __forceinline__ float round_store(float v, __nv_bfloat16*) {
  return __bfloat162float(__float2bfloat16_rn(v));
}

__global__ void __launch_bounds__(kBkThreads, 1) bk_expand_kernel(
    const uint32_t* __restrict__ c_in, int32_t n, int sb_bits, int32_t B, const int2* __restrict__ xseg,
    const ExpandUnit* __restrict__ units, int32_t nunits, const uint16_t* __restrict__ src_lo,
    uint32_t* __restrict__ vals, unsigned int* __restrict__ ctr, unsigned int epoch) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int32_t SB = 1 << sb_bits;
  uint32_t* s_code = reinterpret_cast<uint32_t*>(smem);
  int32_t* s_pref = reinterpret_cast<int32_t*>(smem + (size_t)SB * 4);  // kMaxUnitSegs + 1
  int32_t* s_lo = s_pref + kMaxUnitSegs + 1;
  int32_t* s_hi = s_lo + kMaxUnitSegs;
  uint16_t* s_map = reinterpret_cast<uint16_t*>(s_hi + kMaxUnitSegs);  // chunk -> segment, kMaxUnitChunks
  uint2* s_ids = reinterpret_cast<uint2*>(smem + expand_ids_offset(sb_bits));  // per warp: 2 slots x 64 x 8 bytes
  __shared__ int32_t s_unit;
  __shared__ int32_t s_wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  uint2* w_ids = s_ids + warp * 128;
  for (;;) {
    __syncthreads();  // the previous unit is done with s_code and the segment tables
    if (tid == 0) s_unit = (int32_t)(atomicAdd(ctr, 1u) - epoch);
    __syncthreads();
    const int32_t u = s_unit;
    if (u < 0 || u >= nunits) return;
    const ExpandUnit eu = units[u];
    // the block's codes: 16-byte loads, four in flight per thread
    const int64_t v0 = (int64_t)eu.s << sb_bits;
    const int32_t nb = (int32_t)(n - v0 < SB ? n - v0 : SB);
    {
      const int32_t nvec = nb / 4;
      const uint4* src = reinterpret_cast<const uint4*>(c_in + v0);
      uint4* dst = reinterpret_cast<uint4*>(s_code);
      for (int32_t i0 = tid; i0 < nvec; i0 += 4 * blockDim.x) {
        uint4 r[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (i0 + k * (int32_t)blockDim.x < nvec) r[k] = __ldg(src + i0 + k * blockDim.x);
#pragma unroll
        for (int k = 0; k < 4; ++k)
          if (i0 + k * (int32_t)blockDim.x < nvec) dst[i0 + k * blockDim.x] = r[k];
      }
      for (int32_t i = nvec * 4 + tid; i < nb; i += blockDim.x) s_code[i] = __ldg(c_in + v0 + i);
    }
    // clipped segment ranges and the prefix of their chunk counts
    const int nseg = eu.b_hi - eu.b_lo;
    int32_t chunks = 0;
    if (tid < nseg) {
      const int2 r = xseg[(int64_t)eu.s * B + eu.b_lo + tid];
      const int32_t lo = max(r.x, eu.lo), hi = min(r.y, eu.hi);
      s_lo[tid] = lo;
      s_hi[tid] = hi;
      chunks = hi > lo ? (hi - 1) / kChunk - lo / kChunk + 1 : 0;
    }
    int32_t v = chunks;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane == 31) s_wsum[warp] = v;
    __syncthreads();
    if (warp == 0) {
      int32_t t = lane < nwarps ? s_wsum[lane] : 0;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      s_wsum[lane] = t;
    }
    __syncthreads();
    const int32_t excl = v - chunks + (warp > 0 ? s_wsum[warp - 1] : 0);
    s_pref[tid] = excl;
    if (tid == blockDim.x - 1) s_pref[blockDim.x] = excl + chunks;
    __syncthreads();
    const int32_t total = s_pref[nseg];
    // the segment of every chunk, found once per chunk by all threads
    for (int32_t c = tid; c < total; c += blockDim.x) {
      int k0 = 0, k1 = nseg - 1;  // the last segment whose first chunk is <= c
      while (k0 < k1) {
        const int mid = (k0 + k1 + 1) >> 1;
        if (s_pref[mid] <= c)
          k0 = mid;
        else
          k1 = mid - 1;
      }
      s_map[c] = (uint16_t)k0;
    }
    __syncthreads();
    // a warp takes chunks warp, warp + nwarps, ...; lane l handles edges
    // 4l..4l+3 and 128+4l..128+4l+3 of a chunk, whose 16-bit source ids it
    // copies into its slot while the previous chunk is expanded
    int32_t base = 0, lo = 0, hi = 0;
    auto locate = [&](int32_t c, int32_t& b, int32_t& l, int32_t& h) {
      const int k = s_map[c];
      l = s_lo[k];
      h = s_hi[k];
      b = (l / kChunk + (c - s_pref[k])) * kChunk;
    };
    auto stage = [&](int slot, int32_t b) {
      cp_async8(w_ids + slot * 64 + lane, src_lo + b + 4 * lane);
      cp_async8(w_ids + slot * 64 + 32 + lane, src_lo + b + 128 + 4 * lane);
    };
    if (warp < total) {
      locate(warp, base, lo, hi);
      stage(0, base);
    }
    cp_async_commit();
    int slot = 0;
    for (int32_t ch = warp; ch < total; ch += nwarps, slot ^= 1) {
      int32_t nbase = 0, nlo = 0, nhi = 0;
      if (ch + nwarps < total) {
        locate(ch + nwarps, nbase, nlo, nhi);
        stage(slot ^ 1, nbase);
      }
      cp_async_commit();
      cp_async_wait<1>();  // this lane's copies for the current chunk are in
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const uint2 q = w_ids[slot * 64 + h * 32 + lane];
        const int32_t g = base + h * 128 + 4 * lane;
        const uint32_t id[4] = {q.x & 0xFFFFu, q.x >> 16, q.y & 0xFFFFu, q.y >> 16};
        if (g >= lo && g + 4 <= hi) {
          *reinterpret_cast<uint4*>(vals + g) = make_uint4(s_code[id[0]], s_code[id[1]], s_code[id[2]], s_code[id[3]]);
        } else {
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (g + j >= lo && g + j < hi) vals[g + j] = s_code[id[j]];
        }
      }
      base = nbase;
      lo = nlo;
      hi = nhi;
    }
    cp_async_wait<0>();
  }
}

// ---- accumulate -----------------------------------------------------------

// Values of 8 codes: codes below 2^31 are the value; the rest are converted
// (once any lane of the warp holds one).
__device__ __forceinline__ void codes_to_values(const uint32_t (&w)[8], int U, unsigned long long (&q)[8]) {
  const uint32_t any = (w[0] | w[1] | w[2] | w[3]) | (w[4] | w[5] | w[6] | w[7]);
#pragma unroll
  for (int j = 0; j < 8; ++j) q[j] = w[j];
  if (__any_sync(0xffffffffu, any >> 31)) {
#pragma unroll
    for (int j = 0; j < 8; ++j) q[j] = value_of(w[j], U);
  }
}

// Adds q[j] into row d[j] of the two-word accumulators (low words at a_lo,
// high words hw bytes above): the low words with independent atomics, then
// the high halves and carries, issued only when some lane of the warp has
// one (most steps carry nothing: codes are far below 2^32).
__device__ __forceinline__ void acc_add8(uint32_t a_lo, uint32_t hw, const uint32_t (&d)[8],
                                         const unsigned long long (&q)[8]) {
  uint32_t up[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) up[j] = atom_add(a_lo + 4u * d[j], (uint32_t)q[j]);
#pragma unroll
  for (int j = 0; j < 8; ++j) up[j] = carry_into(up[j], (uint32_t)q[j], (uint32_t)(q[j] >> 32));
  const uint32_t any = (up[0] | up[1] | up[2] | up[3]) | (up[4] | up[5] | up[6] | up[7]);
  if (__any_sync(0xffffffffu, any != 0u)) {
#pragma unroll
    for (int j = 0; j < 8; ++j) red_add_nonzero(a_lo + hw + 4u * d[j], up[j]);
  }
}

// Edge index of slot j of this lane in a 256-edge chunk at `base`: lane l
// holds edges 4l..4l+3 and 128+4l..128+4l+3.
__device__ __forceinline__ int32_t chunk_edge(int32_t base, int lane, int j) {
  return base + (j < 4 ? 4 * lane + j : 128 + 4 * lane + j - 4);
}

template <typename T>
__global__ void __launch_bounds__(kBkThreads, 1) bk_accum_kernel(
    const uint32_t* __restrict__ vals, const uint16_t* __restrict__ dst_lo, const uint32_t* __restrict__ c_in,
    int dense_bits, int32_t n, int w_bits, int U, const AccumUnit* __restrict__ units, int32_t nunits,
    unsigned int* __restrict__ ctr, unsigned int epoch, unsigned long long* __restrict__ acc_g,
    unsigned int* __restrict__ bin_arrive, const float* __restrict__ x_in, const float* __restrict__ inv_deg,
    float* __restrict__ x_out, uint32_t* __restrict__ c_out, StepParams* __restrict__ prm,
    double* __restrict__ partials, int32_t nbins, double* __restrict__ log_row) {
  extern __shared__ __align__(16) uint32_t s_acc32[];
  __shared__ int32_t s_unit;
  __shared__ int s_flag;
  const int32_t W = 1 << w_bits;
  uint32_t* s_lo = s_acc32;      // low words of the row accumulators
  uint32_t* s_hi = s_acc32 + W;  // high words
  const uint32_t a_lo = (uint32_t)__cvta_generic_to_shared(s_lo), hw = 4u * (uint32_t)W;
  const uint32_t dmask = (1u << dense_bits) - 1;  // dense_bits = 32 - w_bits <= 28
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  // this warp's two staging slots: 256 codes or packed words, then 256 row ids
  unsigned char* w_stage = reinterpret_cast<unsigned char*>(s_acc32 + 2 * W) + (size_t)warp * 2 * kAccumSlotBytes;
  for (;;) {
    __syncthreads();
    if (tid == 0) s_unit = (int32_t)(atomicAdd(ctr + 1, 1u) - epoch);
    __syncthreads();
    const int32_t u = s_unit;
    if (u < 0 || u >= nunits) return;
    const AccumUnit un = units[u];
    const int32_t v0 = un.b << w_bits;
    const int32_t nv = min(W, n - v0);
    for (int32_t i = tid; i < nv; i += blockDim.x) s_lo[i] = s_hi[i] = 0u;
    __syncthreads();
    // Lane l handles edges 4l..4l+3 and 128+4l..128+4l+3 of each 256-edge
    // chunk; it copies exactly those words (and row ids) into its slot while
    // the previous chunk is added.  An edge outside the unit's range (in a
    // chunk at either end) adds 0 to row 0.
    //
    // Dense sources, edges [lo, mid): each word packs the source and the row;
    // the source's code is read from c_in (at most 1 MB of codes, kept in
    // cache: a chunk's edges come from few, consecutive sources).
    {
      auto stage = [&](int slot, int32_t b) {
        unsigned char* st = w_stage + slot * kAccumSlotBytes;
        cp_async16(st + 16 * lane, vals + b + 4 * lane);
        cp_async16(st + 512 + 16 * lane, vals + b + 128 + 4 * lane);
      };
      const int32_t first = (un.lo & ~(kChunk - 1)) + warp * kChunk;
      if (first < un.mid) stage(0, first);
      cp_async_commit();
      int slot = 0;
      for (int32_t base = first; base < un.mid; base += nwarps * kChunk, slot ^= 1) {
        if (base + nwarps * kChunk < un.mid) stage(slot ^ 1, base + nwarps * kChunk);
        cp_async_commit();
        cp_async_wait<1>();
        const unsigned char* st = w_stage + slot * kAccumSlotBytes;
        const uint4 wa = *reinterpret_cast<const uint4*>(st + 16 * lane);
        const uint4 wb = *reinterpret_cast<const uint4*>(st + 512 + 16 * lane);
        uint32_t w[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
        uint32_t offm = 0;  // edges outside the range: word 0 (source 0, row 0), value 0
        if (base < un.lo || base + kChunk > un.mid) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int32_t e = chunk_edge(base, lane, j);
            if (e < un.lo || e >= un.mid) {
              w[j] = 0u;
              offm |= 1u << j;
            }
          }
        }
        uint32_t cw[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) cw[j] = __ldg(c_in + (w[j] & dmask));
        unsigned long long q[8];
        codes_to_values(cw, U, q);
        if (offm) {
#pragma unroll
          for (int j = 0; j < 8; ++j)
            if ((offm >> j) & 1u) q[j] = 0ull;
        }
        uint32_t d[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) d[j] = w[j] >> dense_bits;
        acc_add8(a_lo, hw, d, q);
      }
      cp_async_wait<0>();
    }
    // Other sources, edges [mid, hi): codes written by the expand phase and
    // 16-bit rows.
    {
      auto stage = [&](int slot, int32_t b) {
        unsigned char* st = w_stage + slot * kAccumSlotBytes;
        cp_async16(st + 16 * lane, vals + b + 4 * lane);
        cp_async16(st + 512 + 16 * lane, vals + b + 128 + 4 * lane);
        cp_async8(st + 1024 + 8 * lane, dst_lo + b + 4 * lane);
        cp_async8(st + 1280 + 8 * lane, dst_lo + b + 128 + 4 * lane);
      };
      const int32_t first = (un.mid & ~(kChunk - 1)) + warp * kChunk;
      if (first < un.hi) stage(0, first);
      cp_async_commit();
      int slot = 0;
      for (int32_t base = first; base < un.hi; base += nwarps * kChunk, slot ^= 1) {
        if (base + nwarps * kChunk < un.hi) stage(slot ^ 1, base + nwarps * kChunk);
        cp_async_commit();
        cp_async_wait<1>();  // this lane's copies for the current chunk are in
        const unsigned char* st = w_stage + slot * kAccumSlotBytes;
        const uint4 wa = *reinterpret_cast<const uint4*>(st + 16 * lane);
        const uint4 wb = *reinterpret_cast<const uint4*>(st + 512 + 16 * lane);
        const uint2 ra = *reinterpret_cast<const uint2*>(st + 1024 + 8 * lane);
        const uint2 rb = *reinterpret_cast<const uint2*>(st + 1280 + 8 * lane);
        uint32_t w[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
        uint32_t d[8] = {ra.x & 0xFFFFu, ra.x >> 16, ra.y & 0xFFFFu, ra.y >> 16,
                         rb.x & 0xFFFFu, rb.x >> 16, rb.y & 0xFFFFu, rb.y >> 16};
        if (base < un.mid || base + kChunk > un.hi) {
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const int32_t e = chunk_edge(base, lane, j);
            if (e < un.mid || e >= un.hi) {
              w[j] = 0u;  // adds 0 to row 0
              d[j] = 0u;
            }
          }
        }
        unsigned long long q[8];
        codes_to_values(w, U, q);
        // a warp step inside one row (a long row): one shared-memory addition
        const uint32_t r0 = __shfl_sync(0xffffffffu, d[0], 0);
        bool one = true;
#pragma unroll
        for (int j = 0; j < 8; ++j) one = one && d[j] == r0;
        if (__all_sync(0xffffffffu, one)) {
          unsigned long long r = ((q[0] + q[1]) + (q[2] + q[3])) + ((q[4] + q[5]) + (q[6] + q[7]));
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
          if (lane == 0) {
            const uint32_t up = carry_into(atom_add(a_lo + 4u * r0, (uint32_t)r), (uint32_t)r, (uint32_t)(r >> 32));
            red_add_nonzero(a_lo + hw + 4u * r0, up);
          }
          continue;
        }
        // runs of equal rows within each group of 4 consecutive edges are
        // folded into their first edge (backward, so a head holds its whole
        // run; the rest add 0): consecutive edges of one row would otherwise
        // meet in one atomic instruction
#pragma unroll
        for (int j = 6; j >= 0; --j) {
          if (j != 3 && d[j] == d[j + 1]) {
            q[j] += q[j + 1];
            q[j + 1] = 0ull;
          }
        }
        acc_add8(a_lo, hw, d, q);
      }
      cp_async_wait<0>();
    }
    __syncthreads();
    if (un.nparts > 1) {
      unsigned long long* g = acc_g + (int64_t)un.split * W;
      for (int32_t i = tid; i < nv; i += blockDim.x) {
        const unsigned long long a = ((unsigned long long)s_hi[i] << 32) | s_lo[i];
        if (a) atomicAdd(g + i, a);
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) s_flag = atomicAdd(bin_arrive + un.split, 1u) == (unsigned)(un.nparts - 1);
      __syncthreads();
      if (!s_flag) continue;
      __threadfence();
      // the last unit of the bin takes the totals and clears them for the next step
      for (int32_t i = tid; i < nv; i += blockDim.x) {
        const unsigned long long a = atomicExch(g + i, 0ull);
        s_lo[i] = (uint32_t)a;
        s_hi[i] = (uint32_t)(a >> 32);
      }
      if (tid == 0) bin_arrive[un.split] = 0;
      __syncthreads();
    }
    // finish the bin's rows: x' = coefB + coefA y, c' = code(T(x' / outdeg))
    const float A = prm->coefA, Bc = prm->coefB;
    float mass = 0.f, dang = 0.f, res = 0.f;
    for (int32_t i = tid; i < nv; i += blockDim.x) {
      const float y = from_fixed(((unsigned long long)s_hi[i] << 32) | s_lo[i], U);
      const int32_t r = v0 + i;
      const float idg = inv_deg[r];
      const float xs = fmaf(A, y, Bc);
      x_out[r] = xs;
      c_out[r] = code_of(round_store(xs * idg, (T*)nullptr), U);
      mass += xs;
      res += fabsf(xs - x_in[r]);
      if (idg == 0.0f) dang += xs;
    }
    block_partials3(mass, dang, res, partials + 3 * (int64_t)un.b);
    if (tid == 0) {
      __threadfence();
      s_flag = atomicAdd(ctr + 2, 1u) == (unsigned)(nbins - 1);
    }
    __syncthreads();
    if (s_flag) {
      // every bin of the step is finished: fold them, in bin order
      __threadfence();
      fold_step(partials, nbins, prm, log_row);
      if (tid == 0) ctr[2] = 0;
    }
  }
}

// c = code(T(x * inv_deg)): the codes of a start vector.
template <typename T>
__global__ void bk_codes_kernel(const float* __restrict__ x, const float* __restrict__ inv_deg, int32_t n, int U,
                                uint32_t* __restrict__ c) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
    c[v] = code_of(round_store(x[v] * inv_deg[v], (T*)nullptr), U);
}

}  // namespace gpr
