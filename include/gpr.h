/* gpr: GB300-native graph build and PageRank — the C-ABI boundary.
 *
 * The paper (SNAP, Leskovec and Sosic) treats a graph as a set of nodes with
 * non-negative integer ids and edges as (source, destination) pairs
 * (section 3, "SNAP Foundations"); its simple directed graph container keeps
 * no multi-edges and stores each node's neighbours in sorted vectors
 * (section 5, "Representation of Graphs and Networks").  Its methods table
 * lists PageRank and personalised PageRank among the analytics (section 4,
 * Table "snap_methods"); section 6 times 10 PageRank iterations on
 * LiveJournal (Table "exp_algs") and per-iteration PageRank on Twitter2010
 * (Table "exp_parallel").  Every entry point below computes one of those
 * operations on the GPU.  No torch types cross this boundary: pointers are
 * plain host or device addresses, streams are cudaStream_t passed as void*.
 *
 * Conventions for every function:
 *  - Return value: a gpr_status.  Nothing aborts or exits.  On any status
 *    other than GPR_OK, gpr_last_error() holds a one-line message for the
 *    calling thread, outputs are unspecified, and no resource the call made
 *    is left allocated.
 *  - Invalid arguments are reported as GPR_EINVAL before any device work.
 *  - `stream` may be NULL (the legacy default stream).  Work is ordered on
 *    it; functions that return values on the host synchronise it.
 *  - Device memory a gpr_graph owns is released by graph_free only.
 */
#ifndef GPR_H
#define GPR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GPR_OK = 0,
  GPR_EINVAL = 1,    /* bad argument: id out of range, n <= 0, damping outside (0, 1), ... */
  GPR_ENOMEM = 2,    /* device allocation failed, or a request can never fit its budget */
  GPR_ECUDA = 3,     /* a CUDA runtime call failed */
  GPR_ETIMEOUT = 4,  /* a bounded device-side wait gave up (the kernel returned, nothing hung) */
  GPR_EBUSY = 5,     /* queue full */
  GPR_ENOTREADY = 6, /* result not ready within the poll timeout */
  GPR_ENOTFOUND = 7  /* unknown ticket or graph id */
} gpr_status;

/* Storage type of the gathered contribution vector c = x / outdeg (the
 * bytes the pull step reads once per edge).  The rank vector x itself is
 * always FP32; accumulation is always FP32; the per-step mass,
 * dangling-mass and residual reductions are FP64.
 *   GPR_BF16: 8-bit significand.  pagerank rounds to nearest.  ppr_batch
 *             and the server send error-feedback deltas: a node keeps the
 *             FP32 sum s of what it has sent and stores bf16(c - s) (round to
 *             nearest), a row keeps the FP32 running sum of what it gathers,
 *             so each step's rounding is corrected by the next.
 *   GPR_FP16: ppr_batch only: 11-bit significand, values stored times 2^10
 *             (a personalised column lies in [0, 1]). */
typedef enum { GPR_FP32 = 0, GPR_BF16 = 1, GPR_FP16 = 2 } gpr_dtype;

/* Pointer-space flags */
#define GPR_PTR_DEVICE 0 /* arrays are device (or managed) memory */
#define GPR_PTR_HOST 1   /* arrays are host memory; the library copies them */
/* Schedule of the PageRank step (pagerank only; neither: the library's choice) */
#define GPR_SPMV_PULL 0x10    /* one gather per edge, rows by in-degree bucket */
#define GPR_SPMV_BLOCKED 0x20 /* two streaming phases over a bin-major edge copy */
/* pagerank only: start from the vector in x_out (n floats by node id, e.g. the
 * result before a graph_update) instead of the uniform vector */
#define GPR_WARM_START 0x40

/* A directed simple graph resident in device memory: the CSC (in-adjacency,
 * sources ascending within each destination), out-degrees, and an execution
 * layout for the PageRank kernels.  Opaque. */
typedef struct gpr_graph gpr_graph;

typedef struct {
  int32_t n;             /* nodes (ids 0..n-1; isolated nodes included) */
  int64_t m_raw;         /* COO length given to graph_build */
  int64_t m;             /* distinct non-loop edges */
  int32_t n_dangling;    /* nodes with out-degree 0 */
  int32_t max_in_degree;
  int32_t max_out_degree;
  int64_t device_bytes;  /* device memory the graph holds */
} gpr_graph_info;

typedef struct {
  int32_t iters_run;
  double residual_l1; /* ||x_k - x_{k-1}||_1 of the last step, FP64 sum of FP32 terms */
  double mass;        /* sum of x_k, FP64 */
  double dangling;    /* dangling mass of x_k, FP64 */
  double t_setup_ms;  /* host time this call spent making the workspace, the blocked edge
                         layout and the CUDA graph (0 when all were reused) */
  double t_iter_ms;   /* device time of the iteration loop (CUDA events on `stream`) */
  int32_t schedule;   /* the step's schedule: GPR_SPMV_PULL or GPR_SPMV_BLOCKED */
} gpr_stats;

/* ---- graph construction ------------------------------------------------
 * graph_build: the simple directed graph of a raw COO edge stream (section
 * 3, the directed graph container; section 5, sorted adjacency vectors).
 *   src, dst : m_raw int32 node ids each (structure of arrays), in host
 *              memory if flags has GPR_PTR_HOST, else device memory.  Not
 *              modified; the caller keeps ownership.
 *   m_raw    : >= 0 and < 2^31.   n : number of nodes, 1 <= n < 2^30.
 * Duplicate pairs collapse to one edge; self-loops are dropped; nodes
 * without edges are kept.  The result is bit-identical to sorting the
 * distinct non-loop pairs by (destination, source).
 * Errors: GPR_EINVAL if any id is outside [0, n) (detected on the device
 * during the build; everything allocated is freed before return), or for
 * bad sizes; GPR_ENOMEM; GPR_ECUDA; GPR_ETIMEOUT.
 * On success *out owns its device memory until graph_free.  Synchronises
 * `stream` once (to read the edge count and the error flag). */
gpr_status graph_build(const int32_t* src, const int32_t* dst, int64_t m_raw, int32_t n, int flags,
                       void* stream, gpr_graph** out);

/* Releases everything the graph owns.  NULL is accepted.  The caller must
 * not free a graph while work using it is still queued on a stream. */
gpr_status graph_free(gpr_graph* g);

gpr_status graph_info(const gpr_graph* g, gpr_graph_info* info);

/* Copies the CSC to caller-owned HOST arrays: col_ptr (n + 1), row_idx (m),
 * outdeg (n); any pointer may be NULL to skip it.  Synchronous. */
gpr_status graph_export(const gpr_graph* g, int32_t* col_ptr, int32_t* row_idx, int32_t* outdeg);

/* Binary save and load (section 3, Table "exp_basic": graphs are saved to
 * and loaded from a binary format).  graph_save writes the graph as the
 * library holds it (relabelled CSC and its permutation, little-endian) to
 * `path`; synchronous, GPR_EINVAL if the file cannot be written.  graph_load
 * reads such a file, checks it (header, sizes, offsets, sorted in-range
 * sources without self-loops, the permutation) and builds the graph with no
 * sort; GPR_ENOTFOUND if the file cannot be opened, GPR_EINVAL if it is not
 * a well-formed graph file.  A loaded graph is bit-identical to the saved one:
 * graph_export and every computation on it give the same bits. */
/* graph_update: edge insertions and deletions in place (section 5: SNAP's
 * graphs are dynamic; section 6 Table "exp_del" times deletions).  The new
 * edge set is E' = (E \ D) u I, with D the pairs (del_src[i], del_dst[i])
 * and I the pairs (ins_src[i], ins_dst[i]) (node ids in [0, n); n stays;
 * self-loops in I are dropped, deleting a missing edge does nothing, repeats
 * count once).  Arrays are device memory, or host memory with GPR_PTR_HOST;
 * either batch may be empty (count 0, NULL arrays).  The graph keeps its
 * internal numbering; its workspaces are dropped and rebuilt on next use.
 * Synchronous.  GPR_EINVAL (graph unchanged) if an id is out of range. */
gpr_status graph_update(gpr_graph* g, const int32_t* ins_src, const int32_t* ins_dst, int64_t n_ins,
                        const int32_t* del_src, const int32_t* del_dst, int64_t n_del, int flags, void* stream);

gpr_status graph_save(const gpr_graph* g, const char* path);
gpr_status graph_load(const char* path, void* stream, gpr_graph** out);

/* ---- PageRank ------------------------------------------------------------
 * pagerank: `iters` steps of PageRank power iteration (section 4 Table
 * "snap_methods"; the fixed iteration count follows section 6 Table
 * "exp_algs", which times 10 iterations):
 *   x_0 = 1/N;   D_k = sum of x_k over nodes with out-degree 0;
 *   x_{k+1}[v] = (1 - d)/N + d (sum_{u -> v} x_k[u] / outdeg(u) + D_k / N)
 * with each step applied to x_k / sum(x_k) (FP64 mass normalisation).
 *   damping : d in (0, 1).   iters : >= 0.
 *   dt      : storage of the contribution vector (GPR_FP32 or GPR_BF16).
 *   x_out   : n floats (FP32 even for BF16 storage), indexed by node id;
 *             device memory, or host memory if flags has GPR_PTR_HOST.
 *   st      : optional; filled if non-NULL (this synchronises `stream`).
 * Calls on one graph must not overlap in time (the graph holds the
 * iteration workspace); order them on one stream. */
gpr_status pagerank(const gpr_graph* g, double damping, int32_t iters, gpr_dtype dt, int flags,
                    float* x_out, gpr_stats* st, void* stream);

/* ---- autotuner for the PageRank step ---------------------------------------
 * pagerank_tune: times trial_steps steps (>= 1) of the pull schedule and of
 * several shapes of the blocked schedule (source-block bits, bin bits,
 * edges per work unit) on g, and keeps the fastest: later pagerank calls on
 * g, and on graphs of the same shape (ceil log2 n, ceil log2 m, dt) in this
 * process, use it unless flags force a schedule.  A pagerank call on a graph
 * of at least 2^22 edges with no tuned choice for its shape runs this first,
 * with 5 trial steps.  The workspace's rank vectors are overwritten.
 * Synchronous.  out may be NULL. */
typedef struct {
  int32_t schedule;         /* GPR_SPMV_PULL or GPR_SPMV_BLOCKED */
  int32_t sb_bits, w_bits;  /* blocked: log2 of the source-block and bin sizes (else 0) */
  int64_t unit_edges;       /* blocked: edges per work unit (else 0) */
  double ms_per_step;       /* the winner's device time per step */
  double pull_ms_per_step;  /* the pull schedule's */
  int32_t candidates;       /* schedules timed */
  int32_t dense_sources;    /* blocked: sources (highest out-degree first) whose edges read their
                               contribution directly instead of through the expand phase (else 0) */
} gpr_tune_result;

gpr_status pagerank_tune(const gpr_graph* g, gpr_dtype dt, int32_t trial_steps, gpr_tune_result* out,
                         void* stream);

/* ---- HITS and eigenvector centrality -----------------------------------------
 * Section 4 Table "snap_methods" names HITS and eigen-centrality among the
 * library's centralities; the paper prints no formula.  With A[u][v] = 1 for
 * each edge u -> v (the simple graph g holds) and h_0 = x_0 uniform:
 *   hits:             a_t = A^T h_{t-1} / ||A^T h_{t-1}||_2,  h_t = A a_t / ||A a_t||_2
 *   eigen_centrality: x_t = A^T x_{t-1} / ||A^T x_{t-1}||_2
 * for `iters` >= 0 steps; a vector whose norm is 0 stays 0.  Outputs are n
 * floats each, unit L2 norm, indexed by node id; device memory, or host
 * memory with GPR_PTR_HOST (then the call is synchronous).  FP32 products,
 * FP64 norms.  hits builds the graph's out-adjacency on its first call and
 * keeps it with the graph.  The products take the pull schedule, or the
 * blocked one (GPR_SPMV_BLOCKED, the default for graphs of 2^22 or more
 * edges; GPR_SPMV_PULL forces the pull schedule), with the vectors
 * L1-normalised between products.  Calls on one graph must not overlap in time (they
 * share the graph's workspace with pagerank). */
gpr_status hits(const gpr_graph* g, int32_t iters, float* hub_out, float* auth_out, int flags, void* stream);
gpr_status eigen_centrality(const gpr_graph* g, int32_t iters, float* x_out, int flags, void* stream);

/* ---- weakly connected components ------------------------------------------
 * wcc: the components of g with edge directions ignored (section 4 Table
 * "snap_methods": connected components; section 6 Table "exp_algs" times
 * WCC).  labels_out (n int32, by node id; device memory, or host memory with
 * GPR_PTR_HOST) receives for each node the smallest node id of its
 * component, so the output does not depend on scheduling; num_components
 * (host, nullable) receives the number of components (isolated nodes count).
 * Synchronous.  Union-find in the manner of Afforest: two sampled
 * in-neighbours per node, then one pass over the in-edges not already inside
 * the largest sampled component.  GPR_ETIMEOUT if a link gives up after 2^20
 * compare-and-swap retries (not expected: a bound that turns a fault into an
 * error). */
gpr_status wcc(const gpr_graph* g, int32_t* labels_out, int32_t* num_components, int flags, void* stream);

/* ---- single-target personalised PageRank (bidirectional) --------------------
 * Section 4.3, "Fast Random Walk Algorithms": the personalised PageRank from
 * sources to one target t, found by working backwards from t to the nodes
 * near it and then walking forwards from the sources.  pi_s is the
 * personalised PageRank of ppr_batch (restart a = 1 - d to s, dangling mass
 * back to s).
 *
 * ppr_reverse_push: the backward phase.  From p = 0, r = e_t, pushes every
 * node v with r(v) > r_max: p(v) += a r(v); r(u) += d r(v) / outdeg(u) for
 * each in-neighbour u of v; r(v) = 0; until every r(v) <= r_max.  Then for
 * every s, Q_s(t) = p(s) + sum_v Q_s(v) r(v), where Q_s(v) is the chance
 * that a walk from s, stopping with probability a at each node and absorbed
 * at a dangling node, stops at v; so 0 <= Q_s(t) - p(s) <= r_max.  Nodes are
 * pushed in rounds (all nodes above r_max at once), so p and r depend on the
 * schedule in their last digits and in which nodes ended below r_max; the
 * invariant and the bound do not.
 *   target  : node id in [0, n).   damping : d in (0, 1).   r_max : > 0.
 *   p_out, r_out : n doubles each by node id (either may be NULL); device
 *             memory, or host memory with GPR_PTR_HOST.
 *   stats   : host, nullable: pushes, edges scanned, rounds, device time.
 * Synchronous.  GPR_EINVAL for a bad argument, GPR_ETIMEOUT if the push
 * needs more than 65536 rounds.
 *
 * ppr_target: estimates pi_s(t) for k sources.  After the backward phase,
 * `walks` PageRank walks from each source s (stop with probability a; from a
 * dangling node go back to s; else to a uniform out-neighbour) end at
 * V_1..V_W, and
 *   est[i] = p(s) (1 + (d/a) #{V_j dangling} / W) + sum_j r(V_j) / W,
 * an unbiased estimate of pi_s(t) whose terms lie in [0, p(s) d/a + r_max].
 * The walks are reproducible: walk w of sources[i] draws from the SplitMix64
 * stream with state seed ^ ((i << 32 | w) * 0xD6E8FEB86659FD93); a step stops
 * when the draw's top 53 bits X satisfy X 2^-53 < a, else moves to
 * out-neighbour floor(X' k / 2^53) (next draw X', out-degree k, neighbours by
 * ascending id).  A walk is cut after 2^20 steps.
 *   sources : k node ids; est_out : k doubles (device memory, or host memory
 *             with GPR_PTR_HOST for both).  k >= 0, walks >= 1,
 *             k * walks < 2^31.   stats : host, nullable.
 * The walks run on `stream` beside the push, which takes a high-priority
 * stream of the library's and joins `stream` before the estimates; the sum
 * over each source's walks is taken in a fixed order, so a call's result
 * depends only on its arguments and the push's rounding. 
 * The first call on a graph builds the out-adjacency in node-id order and
 * a push workspace and keeps them with the graph; calls on one graph take
 * turns (a per-graph lock).  Synchronous.  GPR_EINVAL for a bad argument
 * (including a source id out of range), GPR_ETIMEOUT as above. */
typedef struct {
  int64_t pushes;     /* pushes taken by the backward phase */
  int64_t edges;      /* in-edges those pushes scanned */
  int32_t rounds;     /* push rounds with a non-empty frontier */
  int64_t walk_steps; /* steps of all walks (ppr_target; 0 for ppr_reverse_push) */
  double push_ms;     /* device time of the backward phase (CUDA events) */
  double walk_ms;     /* device time of the walks (ppr_target: they run beside the push) */
  double total_ms;    /* device time of the whole call after its argument checks */
} gpr_target_stats;
gpr_status ppr_reverse_push(const gpr_graph* g, int32_t target, double damping, double r_max, double* p_out,
                            double* r_out, gpr_target_stats* stats, int flags, void* stream);
gpr_status ppr_target(const gpr_graph* g, int32_t target, double damping, double r_max, const int32_t* sources,
                      int32_t k, int32_t walks, uint64_t seed, double* est_out, gpr_target_stats* stats, int flags,
                      void* stream);

/* ---- batched personalised PageRank ---------------------------------------
 * Personalised PageRank (section 4 Table "snap_methods"; section 4,
 * "Fast Random Walk Algorithms": scores from the point of view of a given
 * node), one column per seed s, teleport vector e_s, dangling mass returned
 * to the seed:
 *   x_0 = e_s;  x_{k+1}[v] = (1 - d) e_s[v] + d (sum_{u->v} x_k[u]/outdeg(u) + D_k e_s[v])
 * A column stops after max_iters steps, or, if tol > 0, after the first step
 * k with d/(1-d) * ||x_k - x_{k-1}||_1 <= tol (an a-posteriori bound on the
 * L1 distance to the fixed point).  One call runs every column of every job
 * in one persistent launch; a column's result does not depend on the other
 * columns or jobs in the call. */
typedef struct {
  const gpr_graph* graph;
  int32_t num_seeds;     /* K >= 1 columns */
  const int32_t* seeds;  /* host: K node ids in [0, n) (repeats allowed) */
  const float* damping;  /* host: K values in (0, 1) */
  float* x_out;          /* device: n x K FP32, node-major: x_out[v * K + k] */
  int32_t* iters_out;    /* host, optional: steps each column ran */
  double* residual_out;  /* host, optional: last ||x_k - x_{k-1}||_1 per column */
} gpr_ppr_job;

/* jobs: host array of num_jobs >= 0 jobs (graphs may repeat).  max_iters in
 * [0, 2^20]; tol >= 0 (0: run exactly max_iters steps).  dt: storage of the
 * gathered contributions (the rank state and accumulation stay FP32).
 * Synchronises `stream`.  Errors: GPR_EINVAL for a bad argument (nothing
 * launched), GPR_ENOMEM, GPR_ECUDA. */
gpr_status ppr_batch(const gpr_ppr_job* jobs, int32_t num_jobs, int32_t max_iters, double tol, gpr_dtype dt,
                     void* stream);

/* ---- autotuner for the batched launch (no counterpart in the paper) -------
 * ppr_batch groups its 64-column jobs by graph size, class k holding graphs
 * with ceil(log2 n) <= log2n_max[k] (11, 13, 15, 17, then all larger), and
 * runs each class as one persistent launch of thread-block clusters, each
 * cluster one job at a time, its rows split among the cluster's CTAs.  The
 * CTAs per cluster (1, 2, 4 or 8) of a (class, dt): ppr_tune times each on
 * up to 64 of the class's jobs in `jobs` (trial_steps in [1, 1000] steps per
 * trial; the jobs' outputs are overwritten) and keeps the fastest for later
 * ppr_batch calls in this process; a class never tuned takes 4 CTAs (8 for
 * ceil log2 n in 14..15, the choice measured on GB300 for R-MAT graphs).  The
 * environment variable GPR_PPR_CLUSTER=1|2|4|8 forces one shape for every
 * class.  A column's bits depend on its class's shape (the row split orders
 * the FP64 partial sums), never on the other columns or jobs of a call.
 * Synchronous.  out may be NULL. */
typedef struct {
  int32_t classes;         /* classes present in the jobs (entries below) */
  int32_t log2n_max[5];    /* the class's largest ceil(log2 n) (31: unbounded) */
  int32_t jobs[5];         /* 64-column jobs of the class */
  int32_t cluster[5];      /* CTAs per cluster chosen */
  double ms[5];            /* trial time with the chosen shape */
  double ms_cluster8[5];   /* trial time with 8 CTAs per cluster */
} gpr_ppr_tune_result;

gpr_status ppr_tune(const gpr_ppr_job* jobs, int32_t num_jobs, gpr_dtype dt, int32_t trial_steps,
                    gpr_ppr_tune_result* out, void* stream);

/* ---- serving: continuous batching of personalised-PageRank requests ------
 * A server keeps a pool of graphs resident on the device and answers
 * personalised-PageRank requests (the same operation as ppr_batch) that
 * arrive at any time.  A scheduler thread admits queued requests first come,
 * first served while the device-memory budget allows, packs their columns
 * into per-graph batches of 64 columns, and runs a few steps of every active
 * batch per launch; columns that finish free their place, and requests that
 * arrived meanwhile join the running batches at the next launch.  A
 * request's result does not depend on the requests it ran with. */
typedef struct gpr_server gpr_server;

typedef struct {
  int64_t budget_bytes;    /* device memory for the pool + batch state + results */
  int32_t max_queue;       /* queued (not yet admitted) requests before GPR_EBUSY; <= 0: 65536 */
  int32_t steps_per_tick;  /* steps between two admission rounds; <= 0: 8 */
  int64_t edges_per_part;  /* a batch's rows are split into parts of about this much work
                              (an edge counts 1, a row 3), each part one unit of work per
                              step, so large graphs spread over every SM; <= 0: 2^18 */
  int32_t fail_alloc_at;   /* test hook: the k-th batch allocation fails as if out of memory (0: off) */
} gpr_server_config;

typedef struct {
  int32_t graph_id;      /* index into the pool */
  int32_t num_seeds;     /* 1..64 */
  const int32_t* seeds;  /* host: node ids in [0, n); copied by serve_submit */
  float damping;         /* in (0, 1) */
  double tol;            /* >= 0; 0: run max_iters steps */
  int32_t max_iters;     /* >= 0 */
  gpr_dtype dt;          /* storage of the gathered contributions */
} gpr_request;

typedef struct {
  gpr_status status;    /* GPR_OK, or why the request failed (GPR_ENOMEM, GPR_ECUDA) */
  int32_t n;            /* nodes of the graph */
  int32_t num_seeds;
  int32_t iters_max;    /* steps run by the slowest column */
  double latency_ms;    /* submit to completion */
  const float* x;       /* device: n x num_seeds FP32, node-major; owned by the
                           server until serve_release */
} gpr_result;

typedef struct {
  int64_t submitted, admitted, completed, failed, rejected_busy, rejected_nomem;
  int64_t ticks, queued, active_columns, device_bytes_in_use;
} gpr_server_stats;

/* pool: num_graphs graphs that outlive the server.  Errors: GPR_EINVAL;
 * GPR_ENOMEM if the pool alone exceeds the budget; GPR_ECUDA. */
gpr_status serve_create(const gpr_graph* const* pool, int32_t num_graphs, const gpr_server_config* cfg,
                        gpr_server** out);
/* Non-blocking.  GPR_EINVAL for a bad request; GPR_ENOMEM if it could never
 * fit the budget; GPR_EBUSY if the queue is full. */
gpr_status serve_submit(gpr_server* s, const gpr_request* r, uint64_t* ticket);
/* Waits up to timeout_us (0: just look) for the request to finish.
 * GPR_ENOTREADY on timeout; GPR_ENOTFOUND for an unknown ticket. */
gpr_status serve_poll(gpr_server* s, uint64_t ticket, int64_t timeout_us, gpr_result* r);
/* Completion queue: waits up to timeout_us (0: just look) for requests to
 * finish (successfully or not) and writes up to cap of their tickets, each
 * reported once, to `tickets`; *count receives how many. */
gpr_status serve_completed(gpr_server* s, uint64_t* tickets, int32_t cap, int64_t timeout_us, int32_t* count);
/* Copies a finished result (n x num_seeds floats) to dst (device memory, or
 * host memory with GPR_PTR_HOST).  Synchronous. */
gpr_status serve_fetch(gpr_server* s, uint64_t ticket, float* dst, int flags);
/* Frees a finished result.  GPR_ENOTREADY if it is still running. */
gpr_status serve_release(gpr_server* s, uint64_t ticket);
gpr_status serve_stats(gpr_server* s, gpr_server_stats* st);
/* Stops the scheduler, cancels queued and running requests and frees all
 * server memory (not the pool).  No serve_* call may run concurrently. */
gpr_status serve_destroy(gpr_server* s);

/* ---- allocation-free variant (no counterpart in the paper) ----------------
 * pagerank_csc_noalloc: the iteration of `pagerank` (same update, same FP64
 * mass normalisation, FP32 contributions) on a CSC that the caller already
 * holds in device memory, for callers that cannot allocate device memory:
 * hosts that run on a fixed memory plan made at start-up, allocator-free
 * regions of a larger runtime, or code that shares the device with an
 * allocator it does not own.  It allocates nothing: its scratch is one
 * static device array of about 24 MiB that every GPU loading this library
 * holds until the process exits.
 *   col_ptr (n + 1), row_idx (m), outdeg (n): device int32 arrays of the
 *             in-adjacency (sources of node v are row_idx[col_ptr[v] ..
 *             col_ptr[v+1]), any order), as graph_export returns them.
 *   n       : 1 <= n <= 2^21 (the scratch size); larger n is GPR_EINVAL.
 *   x_out   : device, n floats, written by node id.
 * The first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream capture.
 * All calls share the one scratch array: calls whose work overlaps on the
 * GPU (on different streams, or from different threads) race.  Work is
 * queued on `stream`; the call does not synchronise it. */
gpr_status pagerank_csc_noalloc(const int32_t* col_ptr, const int32_t* row_idx, const int32_t* outdeg, int32_t n,
                                double damping, int32_t iters, float* x_out, void* stream);

/* Thread-local message for the last failing call on this thread ("" if none). */
const char* gpr_last_error(void);

/* Diagnostics (no counterpart in the paper): how many CUDA kernels this
 * library has launched in this process so far, counted on the host at each
 * launch (a CUDA graph launch adds its kernel nodes).  Thread-safe. */
int64_t gpr_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* GPR_H */
