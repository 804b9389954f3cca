// C-ABI entry points (declared and documented in include/gpr.h).
#include <climits>

#include "gpr_internal.cuh"

namespace gpr {
const char* last_error_cstr();
gpr_status build_graph(const int32_t* src, const int32_t* dst, int64_t m_raw, int32_t n, int flags, cudaStream_t s,
                       gpr_graph** out);
gpr_status run_pagerank(gpr_graph* g, double damping, int32_t iters, gpr_dtype dt, int flags, float* x_out,
                        gpr_stats* st, cudaStream_t s);
gpr_status run_pagerank_tune(gpr_graph* g, gpr_dtype dt, int32_t trial_steps, gpr_tune_result* out, cudaStream_t s);
gpr_status run_centrality(gpr_graph* g, int kind, int32_t iters, float* out_x, float* out_hub, int flags,
                          cudaStream_t s);
gpr_status run_wcc(gpr_graph* g, int32_t* labels_out, int32_t* num_components, int flags, cudaStream_t s);
gpr_status save_graph(const gpr_graph* g, const char* path);
gpr_status load_graph(const char* path, cudaStream_t s, gpr_graph** out);
gpr_status update_graph(gpr_graph* g, const int32_t* ins_src, const int32_t* ins_dst, int64_t n_ins,
                        const int32_t* del_src, const int32_t* del_dst, int64_t n_del, int flags, cudaStream_t s);
gpr_status run_ppr_batch(const gpr_ppr_job* jobs, int32_t num_jobs, int32_t max_iters, double tol, gpr_dtype dt,
                         cudaStream_t s);
gpr_status run_ppr_tune(const gpr_ppr_job* jobs, int32_t num_jobs, gpr_dtype dt, int32_t trial_steps,
                        gpr_ppr_tune_result* out, cudaStream_t s);

gpr_status run_reverse_push(gpr_graph* g, int32_t target, double d, double r_max, double* p_out, double* r_out,
                            gpr_target_stats* st, int flags, cudaStream_t s);
gpr_status run_ppr_target(gpr_graph* g, int32_t target, double d, double r_max, const int32_t* sources, int32_t k,
                          int32_t walks, uint64_t seed, double* est_out, gpr_target_stats* st, int flags,
                          cudaStream_t s);

void target_work_free(const gpr_graph* g, cudaStream_t s);  // bippr.cu

void graph_free_device(gpr_graph* g, cudaStream_t s) {
  if (!g) return;
  target_work_free(g, s);
  if (g->transposed) {
    graph_free_device(g->transposed, s);
    delete g->transposed;
    g->transposed = nullptr;
  }
  dfree(g->walk_ptr, s);
  dfree(g->walk_adj, s);
  dfree(g->walk_nbr, s);
  g->walk_ptr = g->walk_adj = nullptr;
  g->walk_nbr = nullptr;
  if (g->work) {
    pagerank_work_free(g->work);
    g->work = nullptr;
  }
  plan_free(g->plan, s);
  dfree(g->col_ptr, s);
  dfree(g->row_idx, s);
  dfree(g->outdeg, s);
  g->col_ptr = g->row_idx = g->outdeg = nullptr;
}

static int64_t graph_bytes(const gpr_graph* g) {
  const int64_t n = g->n, m = g->m;
  // CSC (relabelled ids) + out-degrees + permutations + inverse degrees + row lists + chunks
  return (n + 1) * 4 + m * 4 + n * 4 + 2 * n * 4 + n * 4 + n * 4 + (int64_t)g->plan.nchunks * 16 +
         (int64_t)g->plan.nsplit * 12;
}
}  // namespace gpr

using namespace gpr;

extern "C" {

const char* gpr_last_error(void) { return last_error_cstr(); }

int64_t gpr_kernel_launches(void) { return launches_so_far(); }

gpr_status graph_build(const int32_t* src, const int32_t* dst, int64_t m_raw, int32_t n, int flags, void* stream,
                       gpr_graph** out) {
  clear_error();
  if (!out) {
    set_error("graph_build: out is NULL");
    return GPR_EINVAL;
  }
  *out = nullptr;
  if (n < 1 || n >= (1 << 30)) {
    set_error("graph_build: n = %d outside [1, 2^30)", (int)n);
    return GPR_EINVAL;
  }
  if (m_raw < 0 || m_raw >= ((int64_t)1 << 31)) {
    set_error("graph_build: m_raw = %lld outside [0, 2^31)", (long long)m_raw);
    return GPR_EINVAL;
  }
  if (m_raw > 0 && (!src || !dst)) {
    set_error("graph_build: src or dst is NULL");
    return GPR_EINVAL;
  }
  if (flags & ~GPR_PTR_HOST) {
    set_error("graph_build: unknown flags 0x%x", flags);
    return GPR_EINVAL;
  }
  gpr_status st = build_graph(src, dst, m_raw, n, flags, (cudaStream_t)stream, out);
  if (st == GPR_OK) (*out)->device_bytes = graph_bytes(*out);
  return st;
}

gpr_status graph_free(gpr_graph* g) {
  clear_error();
  if (!g) return GPR_OK;
  // work on any stream may still read the graph: drain the device first
  cudaError_t e = cudaDeviceSynchronize();
  graph_free_device(g, nullptr);
  cudaError_t e2 = cudaStreamSynchronize(nullptr);
  if (e == cudaSuccess) e = e2;
  delete g;
  if (e != cudaSuccess) {
    set_error("graph_free: %s", cudaGetErrorString(e));
    return GPR_ECUDA;
  }
  return GPR_OK;
}

gpr_status graph_update(gpr_graph* g, const int32_t* ins_src, const int32_t* ins_dst, int64_t n_ins,
                        const int32_t* del_src, const int32_t* del_dst, int64_t n_del, int flags, void* stream) {
  clear_error();
  if (!g) {
    set_error("graph_update: NULL graph");
    return GPR_EINVAL;
  }
  if (n_ins < 0 || n_del < 0 || n_ins >= ((int64_t)1 << 31) || n_del >= ((int64_t)1 << 31) ||
      (n_ins > 0 && (!ins_src || !ins_dst)) || (n_del > 0 && (!del_src || !del_dst))) {
    set_error("graph_update: bad batch sizes or NULL arrays");
    return GPR_EINVAL;
  }
  if (flags & ~GPR_PTR_HOST) {
    set_error("graph_update: unknown flags 0x%x", flags);
    return GPR_EINVAL;
  }
  gpr_status st = update_graph(g, ins_src, ins_dst, n_ins, del_src, del_dst, n_del, flags, (cudaStream_t)stream);
  if (st == GPR_OK) g->device_bytes = graph_bytes(g);
  return st;
}

gpr_status graph_save(const gpr_graph* g, const char* path) {
  clear_error();
  if (!g || !path) {
    set_error("graph_save: NULL graph or path");
    return GPR_EINVAL;
  }
  return save_graph(g, path);
}

gpr_status graph_load(const char* path, void* stream, gpr_graph** out) {
  clear_error();
  if (!path || !out) {
    set_error("graph_load: NULL path or out");
    return GPR_EINVAL;
  }
  *out = nullptr;
  gpr_status st = load_graph(path, (cudaStream_t)stream, out);
  if (st == GPR_OK) (*out)->device_bytes = graph_bytes(*out);
  return st;
}

gpr_status graph_info(const gpr_graph* g, gpr_graph_info* info) {
  clear_error();
  if (!g || !info) {
    set_error("graph_info: NULL argument");
    return GPR_EINVAL;
  }
  info->n = g->n;
  info->m_raw = g->m_raw;
  info->m = g->m;
  info->n_dangling = g->n_dangling;
  info->max_in_degree = g->max_in;
  info->max_out_degree = g->max_out;
  info->device_bytes = g->device_bytes;
  return GPR_OK;
}

gpr_status graph_export(const gpr_graph* g, int32_t* col_ptr, int32_t* row_idx, int32_t* outdeg) {
  clear_error();
  if (!g) {
    set_error("graph_export: NULL graph");
    return GPR_EINVAL;
  }
  return export_graph(g, col_ptr, row_idx, outdeg);
}

gpr_status pagerank(const gpr_graph* g, double damping, int32_t iters, gpr_dtype dt, int flags, float* x_out,
                    gpr_stats* st, void* stream) {
  clear_error();
  if (!g || !x_out) {
    set_error("pagerank: NULL graph or output");
    return GPR_EINVAL;
  }
  if (!(damping > 0.0 && damping < 1.0)) {
    set_error("pagerank: damping %g outside (0, 1)", damping);
    return GPR_EINVAL;
  }
  if (iters < 0 || iters > (1 << 20)) {
    set_error("pagerank: iters %d outside [0, 2^20]", (int)iters);
    return GPR_EINVAL;
  }
  if (dt != GPR_FP32 && dt != GPR_BF16) {
    set_error("pagerank: unknown dtype %d", (int)dt);
    return GPR_EINVAL;
  }
  if ((flags & ~(GPR_PTR_HOST | GPR_SPMV_PULL | GPR_SPMV_BLOCKED | GPR_WARM_START)) ||
      (flags & (GPR_SPMV_PULL | GPR_SPMV_BLOCKED)) == (GPR_SPMV_PULL | GPR_SPMV_BLOCKED)) {
    set_error("pagerank: unknown or conflicting flags 0x%x", flags);
    return GPR_EINVAL;
  }
  return run_pagerank(const_cast<gpr_graph*>(g), damping, iters, dt, flags, x_out, st, (cudaStream_t)stream);
}

gpr_status pagerank_tune(const gpr_graph* g, gpr_dtype dt, int32_t trial_steps, gpr_tune_result* out,
                         void* stream) {
  clear_error();
  if (!g) {
    set_error("pagerank_tune: NULL graph");
    return GPR_EINVAL;
  }
  if (dt != GPR_FP32 && dt != GPR_BF16) {
    set_error("pagerank_tune: unknown dtype %d", (int)dt);
    return GPR_EINVAL;
  }
  if (trial_steps < 1 || trial_steps > 1000) {
    set_error("pagerank_tune: trial_steps %d outside [1, 1000]", (int)trial_steps);
    return GPR_EINVAL;
  }
  return run_pagerank_tune(const_cast<gpr_graph*>(g), dt, trial_steps, out, (cudaStream_t)stream);
}

static gpr_status check_centrality(const char* what, const gpr_graph* g, int32_t iters, int flags) {
  if (!g) {
    set_error("%s: NULL graph", what);
    return GPR_EINVAL;
  }
  if (iters < 0 || iters > (1 << 20)) {
    set_error("%s: iters %d outside [0, 2^20]", what, (int)iters);
    return GPR_EINVAL;
  }
  if ((flags & ~(GPR_PTR_HOST | GPR_SPMV_PULL | GPR_SPMV_BLOCKED)) ||
      (flags & (GPR_SPMV_PULL | GPR_SPMV_BLOCKED)) == (GPR_SPMV_PULL | GPR_SPMV_BLOCKED)) {
    set_error("%s: unknown or conflicting flags 0x%x", what, flags);
    return GPR_EINVAL;
  }
  return GPR_OK;
}

gpr_status hits(const gpr_graph* g, int32_t iters, float* hub_out, float* auth_out, int flags, void* stream) {
  clear_error();
  gpr_status st = check_centrality("hits", g, iters, flags);
  if (st != GPR_OK) return st;
  if (!hub_out || !auth_out) {
    set_error("hits: NULL output");
    return GPR_EINVAL;
  }
  return run_centrality(const_cast<gpr_graph*>(g), 1, iters, auth_out, hub_out, flags, (cudaStream_t)stream);
}

gpr_status eigen_centrality(const gpr_graph* g, int32_t iters, float* x_out, int flags, void* stream) {
  clear_error();
  gpr_status st = check_centrality("eigen_centrality", g, iters, flags);
  if (st != GPR_OK) return st;
  if (!x_out) {
    set_error("eigen_centrality: NULL output");
    return GPR_EINVAL;
  }
  return run_centrality(const_cast<gpr_graph*>(g), 0, iters, x_out, nullptr, flags, (cudaStream_t)stream);
}

gpr_status wcc(const gpr_graph* g, int32_t* labels_out, int32_t* num_components, int flags, void* stream) {
  clear_error();
  if (!g || !labels_out) {
    set_error("wcc: NULL graph or output");
    return GPR_EINVAL;
  }
  if (flags & ~GPR_PTR_HOST) {
    set_error("wcc: unknown flags 0x%x", flags);
    return GPR_EINVAL;
  }
  return run_wcc(const_cast<gpr_graph*>(g), labels_out, num_components, flags, (cudaStream_t)stream);
}

gpr_status ppr_reverse_push(const gpr_graph* g, int32_t target, double damping, double r_max, double* p_out,
                            double* r_out, gpr_target_stats* stats, int flags, void* stream) {
  clear_error();
  if (!g) {
    set_error("ppr_reverse_push: NULL graph");
    return GPR_EINVAL;
  }
  if (flags & ~GPR_PTR_HOST) {
    set_error("ppr_reverse_push: unknown flags 0x%x", flags);
    return GPR_EINVAL;
  }
  return run_reverse_push(const_cast<gpr_graph*>(g), target, damping, r_max, p_out, r_out, stats, flags,
                          (cudaStream_t)stream);
}

gpr_status ppr_target(const gpr_graph* g, int32_t target, double damping, double r_max, const int32_t* sources,
                      int32_t k, int32_t walks, uint64_t seed, double* est_out, gpr_target_stats* stats, int flags,
                      void* stream) {
  clear_error();
  if (!g || (k > 0 && (!sources || !est_out))) {
    set_error("ppr_target: NULL graph, sources or output");
    return GPR_EINVAL;
  }
  if (flags & ~GPR_PTR_HOST) {
    set_error("ppr_target: unknown flags 0x%x", flags);
    return GPR_EINVAL;
  }
  return run_ppr_target(const_cast<gpr_graph*>(g), target, damping, r_max, sources, k, walks, seed, est_out, stats,
                        flags, (cudaStream_t)stream);
}

}  // extern "C"

// Validation shared by ppr_batch and ppr_tune; `who` names the entry point.
static gpr_status check_ppr_jobs(const char* who, const gpr_ppr_job* jobs, int32_t num_jobs, int32_t max_iters,
                                 double tol, gpr_dtype dt) {

  if (num_jobs < 0 || (num_jobs > 0 && !jobs)) {
    set_error("%s: bad job array", who);
    return GPR_EINVAL;
  }
  if (max_iters < 0 || max_iters > (1 << 20) || !(tol >= 0.0)) {
    set_error("%s: max_iters %d or tol %g out of range", who, (int)max_iters, tol);
    return GPR_EINVAL;
  }
  if (dt != GPR_FP32 && dt != GPR_BF16 && dt != GPR_FP16) {
    set_error("%s: unknown dtype %d", who, (int)dt);
    return GPR_EINVAL;
  }
  for (int32_t j = 0; j < num_jobs; ++j) {
    const gpr_ppr_job& q = jobs[j];
    if (!q.graph || q.num_seeds < 1 || !q.seeds || !q.damping || !q.x_out) {
      set_error("%s: job %d: missing graph, seeds, damping or output, or num_seeds < 1", who, (int)j);
      return GPR_EINVAL;
    }
    for (int32_t k = 0; k < q.num_seeds; ++k) {
      if (q.seeds[k] < 0 || q.seeds[k] >= q.graph->n) {
        set_error("%s: job %d: seed %d outside [0, %d)", who, (int)j, (int)q.seeds[k], (int)q.graph->n);
        return GPR_EINVAL;
      }
      if (!(q.damping[k] > 0.f && q.damping[k] < 1.f)) {
        set_error("%s: job %d: damping %g outside (0, 1)", who, (int)j, (double)q.damping[k]);
        return GPR_EINVAL;
      }
    }
  }
  return GPR_OK;
}

extern "C" {

gpr_status ppr_batch(const gpr_ppr_job* jobs, int32_t num_jobs, int32_t max_iters, double tol, gpr_dtype dt,
                     void* stream) {
  clear_error();
  const gpr_status st = check_ppr_jobs("ppr_batch", jobs, num_jobs, max_iters, tol, dt);
  if (st != GPR_OK) return st;
  return run_ppr_batch(jobs, num_jobs, max_iters, tol, dt, (cudaStream_t)stream);
}

gpr_status ppr_tune(const gpr_ppr_job* jobs, int32_t num_jobs, gpr_dtype dt, int32_t trial_steps,
                    gpr_ppr_tune_result* out, void* stream) {
  clear_error();
  if (trial_steps < 1 || trial_steps > 1000) {
    set_error("ppr_tune: trial_steps %d outside [1, 1000]", (int)trial_steps);
    return GPR_EINVAL;
  }
  const gpr_status st = check_ppr_jobs("ppr_tune", jobs, num_jobs, trial_steps, 0.0, dt);
  if (st != GPR_OK) return st;
  return run_ppr_tune(jobs, num_jobs, dt, trial_steps, out, (cudaStream_t)stream);
}

}  // extern "C"
