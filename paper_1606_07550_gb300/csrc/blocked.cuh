// The blocked schedule of a PageRank step (blocked.cu): host interface.
#pragma once

#include "pr_step.cuh"

namespace gpr {

// Schedules of the PageRank step.
enum : int { kSchedPull = 0, kSchedBlocked = 1 };

// Edges [lo, hi) of segments (b, s), b in [b_lo, b_hi), of source block s.
struct ExpandUnit {
  int32_t s, b_lo, b_hi, lo, hi;
};

// Edges [lo, hi) of bin b: [lo, mid) from dense sources (packed words),
// [mid, hi) from the other source blocks (codes written by the expand phase).
// A bin cut into nparts > 1 units adds its sums into global accumulator
// `split`; the unit that arrives last finishes it.
struct AccumUnit {
  int32_t b, lo, mid, hi, nparts, split;
};

struct Blocked {
  int sb_bits = 0, w_bits = 0;  // source blocks of 2^sb_bits nodes, bins of 2^w_bits rows
  int32_t n_dense = 0;          // sources [0, n_dense) are dense: a multiple of 2^sb_bits, below 2^dense_bits
  int32_t D = 0;                // dense source blocks: n_dense >> sb_bits
  int dense_bits = 0;           // bits of a dense source id in a packed word (32 - w_bits)
  int64_t unit_edges = 0;       // edges per expand / accumulate unit (at most, but for whole segments)
  int32_t S = 0, B = 0;         // source blocks, bins
  uint16_t* src_lo = nullptr;   // m: source id within its block (other sources), bin-major edge order
  uint16_t* dst_lo = nullptr;   // m: destination row within its bin (other sources)
  // m: dense sources: the packed word source | row << dense_bits, fixed;
  // other sources: the code of c[u], written each step by the expand phase
  uint32_t* vals = nullptr;
  int ubits = 60;               // fixed-point unit 2^-ubits of the sums
  int2* xseg = nullptr;         // S x B: segment (b, s) is edges [x, y) of xseg[s * B + b]
  ExpandUnit* xu = nullptr;
  int32_t n_xu = 0;
  AccumUnit* au = nullptr;
  int32_t n_au = 0;
  int32_t n_split = 0;
  unsigned long long* acc_g = nullptr;  // n_split x 2^w_bits
  unsigned int* bin_arrive = nullptr;   // n_split
  unsigned int* ctr = nullptr;          // [0] expand units, [1] accumulate units, [2] bins finished
  double* partials = nullptr;           // B x 3
  int xgrid = 1, agrid = 1;
  int64_t dense_edges = 0;  // edges from dense sources
  int64_t bytes = 0;        // device bytes held
};

// The largest dense-source count a layout of these sizes can take on g: whole
// source blocks, ids below 2^(32 - w_bits).
int32_t blocked_max_dense(const gpr_graph* g, int sb_bits, int w_bits);

// Can the blocked layout be made for this graph with these block sizes?
bool blocked_eligible(const gpr_graph* g, int sb_bits, int w_bits);

// Builds the layout (one stable sort of the edges by bin, then dense source
// or source block), with work units of about unit_edges edges and
// n_dense dense sources (rounded down to whole blocks and capped by
// blocked_max_dense).  Throws StatusFail / CudaFail.
Blocked* blocked_build(const gpr_graph* g, int sb_bits, int w_bits, int32_t n_dense, int64_t unit_edges,
                       cudaStream_t s);
void blocked_free(Blocked* k, cudaStream_t s);

// Records the unit-counter reset that precedes a run of steps.
void blocked_record_reset(Blocked* k, cudaStream_t s);

// The blocked schedule keeps the contributions c = x * inv_deg as 32-bit
// fixed-point codes (n entries).  Records c = code(T(x * inv_deg)) for a
// start vector x (T = FP32 or BF16 storage).
template <typename T>
void blocked_record_codes(Blocked* k, const gpr_graph* g, const float* x, const float* inv_deg, uint32_t* c,
                          cudaStream_t s);

// Records step `it` (0-based within the run): y from the codes c_in, finish
// into x_out / c_out = code(T(x_out * inv_deg)), fold into prm and log_row.
template <typename T>
void blocked_record_step(Blocked* k, const gpr_graph* g, const uint32_t* c_in, const float* x_in, float* x_out,
                         uint32_t* c_out, const float* inv_deg, StepParams* prm, double* log_row, int32_t it,
                         cudaStream_t s);

}  // namespace gpr
