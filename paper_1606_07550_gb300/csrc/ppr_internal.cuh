// Device-side records of the batched personalised-PageRank kernel, shared by
// the one-shot batch call (ppr.cu) and the continuous-batching server
// (serve.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace gpr {

constexpr int kPprCols = 64;  // columns per job: 32 lanes x 2

enum : int32_t { kColEmpty = 0, kColFresh = 1, kColRunning = 2, kColDone = 3 };

// One personalised-PageRank column (one seed).
struct PprCol {
  int32_t status;
  int32_t seed;       // original node id
  float damping;
  float tol;          // stop when d/(1-d) * ||x_k - x_{k-1}||_1 <= tol (0: never)
  int32_t max_iters;  // stop after this many steps in total
  int32_t iters;      // steps run so far
  double dangling;    // dangling mass of the current iterate
  double residual;    // last ||x_k - x_{k-1}||_1
  double best;        // smallest residual so far
  float* out;         // where the finished column goes: out[v * ldo], v = node id
  int32_t ldo;
  int32_t stall;      // steps since the residual last reached a new minimum
  float bused;        // seed coefficient (1 - d) + d D of the latest step (BF16 deltas recompute x from it)
};

// A column with tol > 0 also stops once its residual has not reached a new
// minimum for this many steps: the update contracts L1 distances by d per
// step, so a residual that stops shrinking has met the floor of the storage
// precision, and no further step brings the iterate closer.
constexpr int32_t kStallSteps = 8;

// One ppr_batch job: a graph and 64 column places; its state lives in the
// workspace of the cluster that runs it.
struct PprJob {
  const int32_t* col_ptr;  // relabelled CSC (execution layout)
  const int32_t* row_idx;
  const float* inv_deg;
  const int32_t* old2new;
  const int32_t* heavy_rows;  // ascending ids of the long rows (in-degree > heavy_deg)
  int32_t n_heavy;
  int32_t heavy_deg;
  int32_t n;
  int32_t n_cap;        // rows of the per-cluster workspace
  int32_t iters;        // steps to run at most
  PprCol* cols;         // 64 records
};

// ---- step-major execution for the server --------------------------------
// A slot's rows are split into parts of about equal edge count; one launch
// runs one step of every (slot, part) item, so a large graph is spread over
// every SM.  The per-column sums of a step are folded, in part order, at the
// start of the next launch; column state is double-buffered by step parity.
struct ColState {
  int32_t status, iters;
  double dangling, residual, best;
  int32_t stall;
  float bused;  // seed coefficient used by the step of the launch that wrote this state (1 before the first)
};

struct SlotDesc {
  const int32_t* col_ptr;
  const int32_t* row_idx;
  const float* inv_deg;
  const int32_t* old2new;
  const int32_t* new2old;
  const int32_t* heavy_rows;
  int32_t n_heavy, heavy_deg;
  int32_t n, nparts;
  const int32_t* part_rows;  // nparts + 1 row boundaries
  float* X;
  void* C[2];
  float4* YS;                // BF16 deltas: per row and lane the running and sent sums (null otherwise)
  int32_t parity;            // C buffer holding the contributions at the start of the tick
  int32_t pad;
  PprCol* rec;               // 64 host-visible records
  ColState* st[2];           // 64 each, by step parity
  double* psum[2];           // nparts x 3 x 64 each, by step parity
  // long rows (heavy_rows) as edge chunks of the graph's plan: long row i
  // sums chunks [hbeg, hend) then [cbeg, cend) of split entry heavy_split0 + i
  const int32_t* chunk_begin;
  const int32_t* chunk_end;
  const int32_t* split_hbeg;
  const int32_t* split_hend;
  const int32_t* split_cbeg;
  const int32_t* split_cend;
  int32_t nchunks, heavy_split0;
  float* chunk_sum;          // nchunks x 64: the chunk's sums of this step
};

struct StepItem {
  int32_t slot, part;
};

// 64 consecutive long-row chunks of one slot.
constexpr int32_t kChunksPerItem = 64;

enum : int { kStepInit = 0, kStepRun = 1, kStepFinish = 2 };

void ppr_step_launch(const SlotDesc* slots_dev, const StepItem* items_dev, int32_t nitems, int mode, int32_t step,
                     gpr_dtype dt, cudaStream_t s);
// The long-row chunk sums of step `step` for chunk items (slot, first chunk / kChunksPerItem).
void ppr_chunk_launch(const SlotDesc* slots_dev, const StepItem* items_dev, int32_t nitems, int32_t step,
                      gpr_dtype dt, cudaStream_t s);
void ppr_part_bounds(const int32_t* col_ptr, int32_t n, int64_t m, int32_t nparts, int32_t* part_rows,
                     cudaStream_t s);


}  // namespace gpr
