/* CPU oracle for the graph-build and PageRank path.  TEST INFRASTRUCTURE ONLY:
 * tests, the smoke check and the benchmark's CPU-baseline leg use it; the
 * library never does.  Plain single-threaded C, FP64, no blocking, fusion or
 * reordering beyond the definitions below, and no code shared with the CUDA
 * path.
 *
 * What it computes (the paper names PageRank and personalised PageRank among
 * its graph methods, section 4 Table "snap_methods", and times them in
 * section 6, but prints no formula; the readings below are the standard
 * definition with the choices the benchmark configurations fix):
 *
 *   Graph: a simple directed graph (section 3, the TNGraph container, and
 *   section 5, "Representation of Graphs and Networks": no multi-edges,
 *   edges are (source, destination) pairs).  From a raw COO stream, E is the
 *   set of distinct pairs (u, v) with u != v.  The in-adjacency of each node
 *   is kept sorted (section 5: adjacency vectors are sorted), giving the CSC
 *   arrays col_ptr[n + 1], row_idx[m] (sources grouped by destination, each
 *   group ascending) and outdeg[n].
 *
 *   PageRank with damping d and teleport vector t (sum 1):
 *     D_k      = sum over u with outdeg(u) = 0 of x_k[u]
 *     x_{k+1}[v] = (1 - d) t[v] + d ( sum_{(u, v) in E} x_k[u] / outdeg(u) + D_k t[v] )
 *   Plain PageRank: t = x_0 = 1/N everywhere.  Personalised PageRank for seed
 *   s: t = x_0 = e_s (dangling mass returns to the seed).
 *
 * Parity pins for every function are in the repository's CPU test suite
 * (closed forms, brute force, dense solves, invariants).
 */
#ifndef GPR_ORACLE_H
#define GPR_ORACLE_H

#include <stdint.h>

/* Build the CSC of the simple directed graph of a raw COO stream.
 * row_idx needs room for m_raw entries.  Returns m (distinct non-loop
 * edges) or -1 if an id is outside [0, n) or n <= 0, -2 on allocation
 * failure. */
int64_t oracle_build_csc(int32_t n, int64_t m_raw, const int32_t* src, const int32_t* dst,
                         int32_t* col_ptr, int32_t* row_idx, int32_t* outdeg);

/* Power iteration from x0 with teleport t (both length n, FP64).
 * Runs max_iters steps, or stops after the first step k with
 * (d / (1 - d)) * ||x_{k+1} - x_k||_1 <= tol when tol > 0.
 * resid (nullable, length max_iters) receives ||x_{k+1} - x_k||_1 per step.
 * Returns the number of steps run, or -1 on bad arguments. */
int32_t oracle_pagerank(int32_t n, const int32_t* col_ptr, const int32_t* row_idx,
                        const int32_t* outdeg, double d, const double* t, const double* x0,
                        int32_t max_iters, double tol, double* x_out, double* resid);

/* Plain PageRank: t = x0 = 1/N, fixed iteration count. */
int32_t oracle_pagerank_uniform(int32_t n, const int32_t* col_ptr, const int32_t* row_idx,
                                const int32_t* outdeg, double d, int32_t iters, double* x_out,
                                double* resid);

/* Personalised PageRank for one seed node: t = x0 = e_seed. */
int32_t oracle_ppr(int32_t n, const int32_t* col_ptr, const int32_t* row_idx, const int32_t* outdeg,
                   double d, int32_t seed, int32_t max_iters, double tol, double* x_out);

/* Sampled rows of the CSC straight from the raw COO, for graphs too large to
 * sort on the host: for each of the k listed destination nodes, the sorted
 * distinct sources u != v.  rows must be distinct.  row_off has k + 1
 * entries; row_src has room for cap entries.  Returns the total number of
 * sources written, or -1 on bad arguments, -2 if cap is too small. */
int64_t oracle_sample_in_rows(int32_t n, int64_t m_raw, const int32_t* src, const int32_t* dst,
                              int32_t k, const int32_t* rows, int64_t* row_off, int32_t* row_src,
                              int64_t cap);

/* Out-degree (distinct destinations v != u) of each of the k listed nodes,
 * straight from the raw COO.  nodes must be distinct.  Returns 0, or -1 on
 * bad arguments, -2 on allocation failure. */
int32_t oracle_sample_outdeg(int32_t n, int64_t m_raw, const int32_t* src, const int32_t* dst,
                             int32_t k, const int32_t* nodes, int32_t* outdeg_out);

/* HITS (section 4 Table "snap_methods" names Hits among the centralities;
 * the paper prints no formula).  Reading: Kleinberg's hubs and authorities on
 * the directed graph, with A[u][v] = 1 for each edge u -> v:
 *   h_0 = 1/sqrt(n) everywhere;  for t = 1..iters:
 *     a_t = A^T h_{t-1} / ||A^T h_{t-1}||_2   (a_t[v] = sum over in-neighbours u of h[u])
 *     h_t = A a_t       / ||A a_t||_2         (h_t[u] = sum over out-neighbours v of a[v])
 * A vector whose norm is 0 stays 0.  iters = 0 gives a = h = 1/sqrt(n).
 * Returns 0, or -1 on bad arguments. */
int32_t oracle_hits(int32_t n, const int32_t* col_ptr, const int32_t* row_idx, int32_t iters, double* hub,
                    double* auth);

/* Eigenvector centrality (section 4 Table "snap_methods": eigen-centrality;
 * no formula printed).  Reading: the power iteration toward the Perron
 * vector of A^T, x_0 = 1/sqrt(n), x_t = A^T x_{t-1} / ||A^T x_{t-1}||_2
 * (a node is central when central nodes point to it); a vector whose norm
 * is 0 stays 0.  Returns 0, or -1 on bad arguments. */
int32_t oracle_eigen_centrality(int32_t n, const int32_t* col_ptr, const int32_t* row_idx, int32_t iters,
                                double* x);

/* Weakly connected components (section 4 Table "snap_methods": connected
 * components; section 6 Table "exp_algs" times WCC).  Reading: nodes u and v
 * are in one component when a path joins them with edge directions ignored;
 * labels[v] = the smallest node id of v's component (isolated nodes are
 * their own component).  Union-find over every edge of the CSC.  Returns the
 * number of components, or -1 on bad arguments / allocation failure. */
int32_t oracle_wcc(int32_t n, const int32_t* col_ptr, const int32_t* row_idx, int32_t* labels);

/* Single-target personalised PageRank, bidirectional (section 4.3 "Fast
 * Random Walk Algorithms": work backwards from the target to a set of
 * intermediate nodes, then walk forwards from the sources).  Reading, for
 * the personalised PageRank pi_s of oracle_ppr (restart a = 1 - d, dangling
 * mass back to the seed s):
 *   Q_s(t): the chance that an excursion from s (stop with probability a at
 *   each node; absorbed at a dangling node when it does not stop) stops at t;
 *   Q_s = a e_s + d Q_s P, P[u][v] = 1/outdeg(u) for u -> v, 0 rows at
 *   dangling nodes.  pi_s solves pi_s = c_s e_s + d pi_s P with
 *   c_s = a + d pi_s(dangling set), so pi_s = (c_s / a) Q_s.
 *   Reverse push from t (threshold r_max): p = 0, r = e_t; while some v has
 *   r(v) > r_max: p(v) += a r(v), r(u) += d r(v) / outdeg(u) for each
 *   in-neighbour u of v, r(v) = 0.  Each push keeps
 *     Q_s(t) = p(s) + sum_v Q_s(v) r(v)   and   pi_s(t) = (c_s / a) p(s) + sum_v pi_s(v) r(v).
 *   Estimate: W walks of the PageRank process from s (stop with probability
 *   a; from a dangling node go back to s; else to a uniform out-neighbour,
 *   out-neighbours in ascending id order), ending at V_1..V_W:
 *     pi^_s(t) = p(s) (1 + (d / a) #{i : V_i dangling} / W) + sum_i r(V_i) / W,
 *   an unbiased estimate (E[1{V dangling}] = pi_s(dangling set)).
 * oracle_reverse_push: p and r (n doubles each); returns the number of
 * pushes, or -1 on bad arguments.  Pushes in FIFO order. */
int64_t oracle_reverse_push(int32_t n, const int32_t* col_ptr, const int32_t* row_idx, const int32_t* outdeg,
                            int32_t target, double d, double r_max, double* p, double* r);

/* oracle_ppr_contrib: q(s) = Q_s(target) for every s, by iterating
 * q <- a e_target + (1 - a) P q  (P q)(s) = mean of q over the out-neighbours
 * of s, 0 at a dangling s; `iters` steps from q = 0 (error <= (1 - a)^iters).
 * Returns 0, or -1 on bad arguments / allocation failure. */
int32_t oracle_ppr_contrib(int32_t n, const int32_t* col_ptr, const int32_t* row_idx, const int32_t* outdeg,
                           int32_t target, double d, int32_t iters, double* q);

/* oracle_ppr_target: estimates for k sources (ids) into out (k doubles).
 * Walk w of source i draws from the SplitMix64 stream whose state starts at
 * seed ^ ((i << 32 | w) * 0xD6E8FEB86659FD93); each step takes one draw
 * u = (x >> 11) 2^-53 and stops if u < a; otherwise, at a node of out-degree
 * k > 0, a second draw x' picks out-neighbour floor((x' >> 11) k / 2^53)
 * (exact integer arithmetic).  A walk is cut (ending where it is) after 2^20
 * steps.  Returns 0, or -1 on bad
 * arguments / allocation failure. */
int32_t oracle_ppr_target(int32_t n, const int32_t* col_ptr, const int32_t* row_idx, const int32_t* outdeg,
                          int32_t target, double d, double r_max, const int32_t* sources, int32_t k,
                          int32_t walks, uint64_t seed, double* out);

#endif /* GPR_ORACLE_H */
