// Device-side records of the batched personalised-PageRank kernel, shared by
// the one-shot batch call (ppr.cu) and the continuous-batching server
// (serve.cu).
#pragma once

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
  float* out;         // where the finished column goes: out[v * ldo], v = node id
  int32_t ldo;
  int32_t pad;
};

// One job: a graph and 64 column slots.
struct PprJob {
  const int32_t* col_ptr;  // relabelled CSC (execution layout)
  const int32_t* row_idx;
  const float* inv_deg;
  const int32_t* old2new;
  const int32_t* heavy_rows;  // ascending ids of the long rows (in-degree > heavy_deg)
  int32_t n_heavy;
  int32_t heavy_deg;
  int32_t n;
  int32_t n_cap;        // rows of the per-cluster workspace (batch mode)
  int32_t iters;        // steps to run in this launch at most
  float* X;             // n x 64 FP32 state, or null: use the cluster workspace
  void* C0;             // n x 64 contributions (FP32 or BF16), double-buffered
  void* C1;
  int32_t parity;       // which C buffer holds the current contributions
  int32_t pad;
  PprCol* cols;         // 64 records
};

int ppr_max_clusters(gpr_dtype dt);
int ppr_cluster_size();
void ppr_launch(PprJob* jobs_dev, const int32_t* order_dev, int32_t njobs, uint32_t* queue_dev, char* ws,
                int64_t ws_stride, int clusters, gpr_dtype dt, cudaStream_t s);

}  // namespace gpr
