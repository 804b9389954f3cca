// Continuous-batching server for personalised-PageRank requests (the
// operation of ppr.cu; section 4 Table "snap_methods").
//
// A slot is one graph with 64 column places whose rank state (X) and
// contributions (C, double-buffered) stay on the device between launches.
// The scheduler thread loops:
//   1. admit queued requests first come, first served: a request takes
//      num_seeds free places of a slot of its graph and storage type (a new
//      slot if none has room) and an n x num_seeds result buffer, if the
//      device budget allows; otherwise it waits.  While the head waits (at
//      most kOvertakeMs), later requests may take free places of running
//      slots, which needs no new slot;
//   2. run steps_per_tick steps of every slot with live columns: each slot's
//      rows are split into parts of about edges_per_part units of work (an
//      edge counts 1, a row 3); per step, one launch gathers the long rows'
//      edge chunks of every slot and one runs every (slot, part) (ppr.cu,
//      ppr_step_kernel: new columns start at e_seed, finished ones freeze
//      and are written to their result buffer by node id);
//   3. read back the column records, complete requests whose columns are
//      all finished, free their places and slots that became empty.
// A column's arithmetic does not depend on the other columns, so a result
// is the same whether its request ran alone or in a mix.
#include <algorithm>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gpr_internal.cuh"
#include "ppr_internal.cuh"

namespace gpr {

using Clock = std::chrono::steady_clock;

// Later requests may fill free places of running slots while the queue head
// has waited less than this; they are looked for among this many queued ones.
constexpr int kOvertakeMs = 2000;
constexpr int kOvertakeScan = 4096;

struct Slot {
  int graph = -1;
  gpr_dtype dt = GPR_FP32;
  float* X = nullptr;
  void* C0 = nullptr;
  void* C1 = nullptr;
  float4* YS = nullptr;  // BF16 deltas: running and sent sums
  int32_t parity = 0;
  int64_t bytes = 0;
  int32_t nparts = 1;
  int32_t* part_rows = nullptr;  // device, nparts + 1
  PprCol* d_rec = nullptr;       // device, 64
  ColState* d_st = nullptr;      // device, 2 x 64
  double* d_psum = nullptr;      // device, 2 x nparts x 3 x 64
  float* chunk_sum = nullptr;    // device, nchunks x 64: long-row chunk sums of a step
  PprCol cols[kPprCols];         // host mirror of d_rec
  uint64_t owner[kPprCols];      // ticket holding each place (0: free)
  int used = 0;
};

enum ReqState { kQueued, kRunning, kDone, kFailed };

struct Req {
  uint64_t ticket = 0;
  int32_t graph = 0;
  std::vector<int32_t> seeds;
  float damping = 0.85f;
  double tol = 0.0;
  int32_t max_iters = 0;
  gpr_dtype dt = GPR_FP32;
  ReqState state = kQueued;
  gpr_status status = GPR_OK;
  float* result = nullptr;
  int64_t result_bytes = 0;
  int remaining = 0;
  int32_t iters_max = 0;
  Clock::time_point t_submit, t_done;
};

}  // namespace gpr

struct gpr_server {
  int device = 0;
  cudaStream_t stream = nullptr;
  std::vector<const gpr_graph*> pool;
  gpr_server_config cfg{};
  int64_t pool_bytes = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<uint64_t> queue;
  std::deque<uint64_t> finished;  // completion queue for serve_completed
  std::unordered_map<uint64_t, gpr::Req> reqs;
  std::vector<gpr::Slot*> slots;
  int64_t bytes_in_use = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread th;
  int alloc_attempts = 0;
  gpr_server_stats st{};
  // device staging for one tick
  gpr::SlotDesc* d_desc = nullptr;
  gpr::StepItem* d_items = nullptr;
  gpr::StepItem* d_citems = nullptr;
  int cap_desc = 0, cap_items = 0, cap_citems = 0;
};

namespace gpr {

static size_t elem_bytes(gpr_dtype dt) { return dt == GPR_FP32 ? 4 : 2; }

static int32_t parts_for(const gpr_server* S, const gpr_graph* g) {
  // parts of about edges_per_part units of work (an edge; a row counts as 3)
  const int64_t work = g->m + 3 * (int64_t)g->n;
  const int64_t p = (work + S->cfg.edges_per_part - 1) / std::max<int64_t>(S->cfg.edges_per_part, 1);
  return (int32_t)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(p, 1024), std::max(g->n, 1)));
}

static int64_t slot_bytes(const gpr_server* S, const gpr_graph* g, gpr_dtype dt) {
  const int64_t P = parts_for(S, g);
  // per row and column: x and two contribution buffers, or with BF16 deltas
  // two delta buffers and the running and sent sums
  return (int64_t)g->n * kPprCols * (dt == GPR_BF16 ? 2 * 2 + 8 : 4 + 2 * (int64_t)elem_bytes(dt)) + (P + 1) * 4 +
         kPprCols * (int64_t)(sizeof(PprCol) + 2 * sizeof(ColState)) + 2 * P * 3 * kPprCols * 8 +
         (int64_t)std::max(g->plan.nchunks, 1) * kPprCols * 4;
}

static void fill_desc(SlotDesc& D, const gpr_graph* g, const Slot* sl) {
  D = SlotDesc{};
  D.col_ptr = g->col_ptr;
  D.row_idx = g->row_idx;
  D.inv_deg = g->plan.inv_deg;
  D.old2new = g->plan.old2new;
  D.new2old = g->plan.new2old;
  D.n = g->n;
  D.heavy_rows = g->plan.rows;
  D.n_heavy = 0;
  D.heavy_deg = INT_MAX;
  // the long rows are the last chunked (lanes 0) bucket; the plan's split
  // entries list the rows of every chunked bucket in bucket order
  int32_t before = 0;
  for (int b = 0; b < g->plan.nbuckets; ++b)
    if (g->plan.bucket[b].lanes == 0) {
      D.heavy_split0 = before;
      D.heavy_rows = g->plan.rows + g->plan.bucket[b].row_begin;
      D.n_heavy = g->plan.bucket[b].row_end - g->plan.bucket[b].row_begin;
      D.heavy_deg = b > 0 ? g->plan.deg_threshold[b - 1] : -1;  // bucket 0 holds every degree from 0
      before += D.n_heavy;
    }
  D.chunk_begin = g->plan.chunk_begin;
  D.chunk_end = g->plan.chunk_end;
  D.split_hbeg = g->plan.split_hbeg;
  D.split_hend = g->plan.split_hend;
  D.split_cbeg = g->plan.split_cbeg;
  D.split_cend = g->plan.split_cend;
  D.nchunks = g->plan.nchunks;
  D.chunk_sum = sl->chunk_sum;
  D.nparts = sl->nparts;
  D.part_rows = sl->part_rows;
  D.X = sl->X;
  D.C[0] = sl->C0;
  D.C[1] = sl->C1;
  D.YS = sl->YS;
  D.parity = sl->parity;
  D.rec = sl->d_rec;
  D.st[0] = sl->d_st;
  D.st[1] = sl->d_st + kPprCols;
  D.psum[0] = sl->d_psum;
  D.psum[1] = sl->d_psum + (int64_t)sl->nparts * 3 * kPprCols;
}

static void free_slot(gpr_server* S, Slot* sl) {
  dfree(sl->X, S->stream);
  dfree(sl->C0, S->stream);
  dfree(sl->C1, S->stream);
  dfree(sl->YS, S->stream);
  dfree(sl->part_rows, S->stream);
  dfree(sl->d_rec, S->stream);
  dfree(sl->d_st, S->stream);
  dfree(sl->d_psum, S->stream);
  dfree(sl->chunk_sum, S->stream);
  S->bytes_in_use -= sl->bytes;
  delete sl;
}

// Place a queued request (lock held).  Returns false if it must wait.  With
// existing_only, only free places of an existing slot are considered.
static bool try_admit(gpr_server* S, Req& r, bool existing_only = false) {
  const gpr_graph* g = S->pool[r.graph];
  const int k = (int)r.seeds.size();
  Slot* target = nullptr;
  for (Slot* sl : S->slots)
    if (sl->graph == r.graph && sl->dt == r.dt && kPprCols - sl->used >= k) {
      target = sl;
      break;
    }
  if (existing_only && !target) return false;
  const int64_t need = (target ? 0 : slot_bytes(S, g, r.dt)) + (int64_t)g->n * k * 4;
  if (S->bytes_in_use + need > S->cfg.budget_bytes) return false;
  try {
    if (!target) {
      ++S->alloc_attempts;
      if (S->cfg.fail_alloc_at > 0 && S->alloc_attempts == S->cfg.fail_alloc_at)
        throw StatusFail{GPR_ENOMEM, "injected allocation failure"};
      Slot* sl = new Slot();
      sl->graph = r.graph;
      sl->dt = r.dt;
      sl->bytes = slot_bytes(S, g, r.dt);
      sl->nparts = parts_for(S, g);
      try {
        if (r.dt != GPR_BF16) sl->X = (float*)dalloc((size_t)g->n * kPprCols * 4, S->stream);
        sl->C0 = dalloc((size_t)g->n * kPprCols * elem_bytes(r.dt), S->stream);
        sl->C1 = dalloc((size_t)g->n * kPprCols * elem_bytes(r.dt), S->stream);
        if (r.dt == GPR_BF16) sl->YS = (float4*)dalloc((size_t)g->n * kPprCols * 8, S->stream);
        sl->part_rows = (int32_t*)dalloc(((size_t)sl->nparts + 1) * 4, S->stream);
        sl->d_rec = (PprCol*)dalloc(kPprCols * sizeof(PprCol), S->stream);
        sl->d_st = (ColState*)dalloc(2 * kPprCols * sizeof(ColState), S->stream);
        sl->d_psum = (double*)dalloc((size_t)2 * sl->nparts * 3 * kPprCols * 8, S->stream);
        sl->chunk_sum = (float*)dalloc((size_t)std::max(g->plan.nchunks, 1) * kPprCols * 4, S->stream);
        ppr_part_bounds(g->col_ptr, g->n, g->m, sl->nparts, sl->part_rows, S->stream);
      } catch (...) {
        dfree(sl->X, S->stream);
        dfree(sl->C0, S->stream);
        dfree(sl->C1, S->stream);
        dfree(sl->YS, S->stream);
        dfree(sl->part_rows, S->stream);
        dfree(sl->d_rec, S->stream);
        dfree(sl->d_st, S->stream);
        dfree(sl->d_psum, S->stream);
        dfree(sl->chunk_sum, S->stream);
        delete sl;
        throw;
      }
      for (int c = 0; c < kPprCols; ++c) {
        sl->cols[c] = PprCol{};
        sl->cols[c].status = kColEmpty;
        sl->cols[c].damping = 0.5f;
        sl->owner[c] = 0;
      }
      S->slots.push_back(sl);
      S->bytes_in_use += sl->bytes;
      target = sl;
    }
    r.result = (float*)dalloc((size_t)g->n * k * 4, S->stream);
  } catch (const CudaFail& f) {
    cudaGetLastError();
    r.state = kFailed;
    r.status = GPR_ECUDA;
    r.t_done = Clock::now();
    ++S->st.failed;
    S->finished.push_back(r.ticket);
    S->cv_done.notify_all();
    return true;
  } catch (const StatusFail& f) {
    r.state = kFailed;
    r.status = f.st;
    r.t_done = Clock::now();
    ++S->st.failed;
    S->finished.push_back(r.ticket);
    S->cv_done.notify_all();
    return true;  // consumed (failed), the queue moves on
  }
  r.result_bytes = (int64_t)g->n * k * 4;
  S->bytes_in_use += r.result_bytes;
  int placed = 0;
  for (int c = 0; c < kPprCols && placed < k; ++c) {
    if (target->owner[c]) continue;
    PprCol& col = target->cols[c];
    col = PprCol{};
    col.status = kColFresh;
    col.seed = r.seeds[placed];
    col.damping = r.damping;
    col.tol = (float)r.tol;
    col.max_iters = r.max_iters;
    col.out = r.result + placed;
    col.ldo = k;
    target->owner[c] = r.ticket;
    ++placed;
  }
  target->used += k;
  r.state = kRunning;
  r.remaining = k;
  ++S->st.admitted;
  return true;
}

template <typename V>
static V* grow(V* p, int& cap, int need, cudaStream_t s) {
  if (need <= cap) return p;
  dfree(p, s);
  cap = std::max(need, 2 * cap + 16);
  return (V*)dalloc((size_t)cap * sizeof(V), s);
}

// One tick: per storage type, kStepInit, steps_per_tick run launches and
// kStepFinish over every (slot, part) of the slots with live columns, then
// the records come back.  Runs without the lock: only the scheduler thread
// touches slots.
static void run_tick(gpr_server* S, const std::vector<Slot*>& live) {
  std::vector<SlotDesc> desc(live.size());
  for (size_t i = 0; i < live.size(); ++i) {
    Slot* sl = live[i];
    fill_desc(desc[i], S->pool[sl->graph], sl);
    GPR_CUDA(cudaMemcpyAsync(sl->d_rec, sl->cols, kPprCols * sizeof(PprCol), cudaMemcpyHostToDevice, S->stream));
  }
  S->d_desc = grow(S->d_desc, S->cap_desc, (int)desc.size(), S->stream);
  GPR_CUDA(cudaMemcpyAsync(S->d_desc, desc.data(), desc.size() * sizeof(SlotDesc), cudaMemcpyHostToDevice, S->stream));
  const int32_t T = S->cfg.steps_per_tick;
  for (gpr_dtype dt : {GPR_FP32, GPR_BF16, GPR_FP16}) {
    std::vector<StepItem> items;
    for (size_t i = 0; i < live.size(); ++i)
      if (live[i]->dt == dt)
        for (int32_t q = 0; q < live[i]->nparts; ++q) items.push_back(StepItem{(int32_t)i, q});
    if (items.empty()) continue;
    S->d_items = grow(S->d_items, S->cap_items, (int)items.size(), S->stream);
    GPR_CUDA(cudaMemcpyAsync(S->d_items, items.data(), items.size() * sizeof(StepItem), cudaMemcpyHostToDevice,
                             S->stream));
    std::vector<StepItem> citems;  // long-row chunk groups of the same slots
    for (size_t i = 0; i < live.size(); ++i)
      if (live[i]->dt == dt)
        for (int32_t q = 0; q * kChunksPerItem < desc[i].nchunks; ++q) citems.push_back(StepItem{(int32_t)i, q});
    const int32_t ni = (int32_t)items.size(), nci = (int32_t)citems.size();
    if (nci > 0) {
      S->d_citems = grow(S->d_citems, S->cap_citems, nci, S->stream);
      GPR_CUDA(cudaMemcpyAsync(S->d_citems, citems.data(), citems.size() * sizeof(StepItem),
                               cudaMemcpyHostToDevice, S->stream));
    }
    ppr_step_launch(S->d_desc, S->d_items, ni, kStepInit, 0, dt, S->stream);
    for (int32_t st = 1; st <= T; ++st) {
      ppr_chunk_launch(S->d_desc, S->d_citems, nci, st, dt, S->stream);
      ppr_step_launch(S->d_desc, S->d_items, ni, kStepRun, st, dt, S->stream);
    }
    ppr_step_launch(S->d_desc, S->d_items, ni, kStepFinish, T + 1, dt, S->stream);
    // the host copy of `items` must outlive the copy above
    GPR_CUDA(cudaStreamSynchronize(S->stream));
  }
  for (Slot* sl : live)
    GPR_CUDA(cudaMemcpyAsync(sl->cols, sl->d_rec, kPprCols * sizeof(PprCol), cudaMemcpyDeviceToHost, S->stream));
  GPR_CUDA(cudaStreamSynchronize(S->stream));
  for (Slot* sl : live) sl->parity = (sl->parity + T) & 1;
}

static void fail_running(gpr_server* S, gpr_status st) {
  for (Slot* sl : S->slots) {
    for (int c = 0; c < kPprCols; ++c) {
      if (!sl->owner[c]) continue;
      auto it = S->reqs.find(sl->owner[c]);
      if (it != S->reqs.end() && it->second.state == kRunning) {
        it->second.state = kFailed;
        it->second.status = st;
        it->second.t_done = Clock::now();
        ++S->st.failed;
        S->finished.push_back(it->first);
      }
      sl->owner[c] = 0;
      sl->cols[c].status = kColEmpty;
    }
    sl->used = 0;
  }
  S->cv_done.notify_all();
}

static void scheduler(gpr_server* S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  for (;;) {
    // 1. admission, first come first served
    while (!S->queue.empty()) {
      auto it = S->reqs.find(S->queue.front());
      if (it == S->reqs.end()) {
        S->queue.pop_front();
        continue;
      }
      if (!try_admit(S, it->second)) break;
      S->queue.pop_front();
    }
    // 1b. while the head waits for memory, later requests may take free
    // places of running slots of their graph (they need no new slot, only a
    // result buffer); bounded so the head cannot starve
    if (!S->queue.empty()) {
      auto head = S->reqs.find(S->queue.front());
      const bool head_fresh =
          head != S->reqs.end() && Clock::now() - head->second.t_submit < std::chrono::milliseconds(kOvertakeMs);
      if (head_fresh) {
        int scanned = 0;
        for (auto q = S->queue.begin() + 1; q != S->queue.end() && scanned < kOvertakeScan; ++scanned) {
          auto it = S->reqs.find(*q);
          if (it != S->reqs.end() && try_admit(S, it->second, /*existing_only=*/true)) {
            q = S->queue.erase(q);
          } else {
            ++q;
          }
        }
      }
    }
    std::vector<Slot*> live;
    for (Slot* sl : S->slots)
      if (sl->used > 0) live.push_back(sl);
    if (live.empty()) {
      if (S->stop) break;
      S->cv_work.wait_for(lk, std::chrono::milliseconds(2));
      continue;
    }
    if (S->stop) break;
    // 2. one tick on the device
    lk.unlock();
    bool ok = true;
    std::string err;
    try {
      run_tick(S, live);
    } catch (const CudaFail& f) {
      cudaGetLastError();
      ok = false;
      err = std::string(f.what) + ": " + cudaGetErrorString(f.err);
    } catch (const StatusFail& f) {
      ok = false;
      err = f.msg;
    }
    lk.lock();
    ++S->st.ticks;
    if (!ok) {
      fail_running(S, GPR_ECUDA);
      continue;
    }
    // 3. retire finished columns and requests
    const auto now = Clock::now();
    for (Slot* sl : live) {
      for (int c = 0; c < kPprCols; ++c) {
        if (!sl->owner[c] || sl->cols[c].status != kColDone) continue;
        auto it = S->reqs.find(sl->owner[c]);
        if (it != S->reqs.end()) {
          Req& r = it->second;
          r.iters_max = std::max(r.iters_max, sl->cols[c].iters);
          if (--r.remaining == 0 && r.state == kRunning) {
            r.state = kDone;
            r.status = GPR_OK;
            r.t_done = now;
            ++S->st.completed;
            S->finished.push_back(r.ticket);
          }
        }
        sl->owner[c] = 0;
        sl->cols[c] = PprCol{};
        sl->cols[c].status = kColEmpty;
        sl->cols[c].damping = 0.5f;
        --sl->used;
      }
    }
    for (size_t i = 0; i < S->slots.size();) {
      if (S->slots[i]->used == 0) {
        free_slot(S, S->slots[i]);
        S->slots.erase(S->slots.begin() + i);
      } else {
        ++i;
      }
    }
    S->cv_done.notify_all();
  }
}

}  // namespace gpr

using namespace gpr;

extern "C" {

gpr_status serve_create(const gpr_graph* const* pool, int32_t num_graphs, const gpr_server_config* cfg,
                        gpr_server** out) {
  clear_error();
  if (!out || !cfg || num_graphs < 1 || !pool) {
    set_error("serve_create: bad arguments");
    return GPR_EINVAL;
  }
  *out = nullptr;
  for (int32_t i = 0; i < num_graphs; ++i)
    if (!pool[i]) {
      set_error("serve_create: pool graph %d is NULL", (int)i);
      return GPR_EINVAL;
    }
  gpr_server* S = new gpr_server();
  S->device = device_ordinal();
  S->pool.assign(pool, pool + num_graphs);
  S->cfg = *cfg;
  if (S->cfg.max_queue <= 0) S->cfg.max_queue = 65536;
  if (S->cfg.steps_per_tick <= 0) S->cfg.steps_per_tick = 8;
  if (S->cfg.edges_per_part <= 0) S->cfg.edges_per_part = (int64_t)1 << 18;
  std::vector<const gpr_graph*> uniq(S->pool);
  std::sort(uniq.begin(), uniq.end());
  uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
  for (const gpr_graph* g : uniq) S->pool_bytes += g->device_bytes;
  S->bytes_in_use = S->pool_bytes;
  if (S->pool_bytes > S->cfg.budget_bytes) {
    set_error("serve_create: the pool alone (%lld bytes) exceeds the budget", (long long)S->pool_bytes);
    delete S;
    return GPR_ENOMEM;
  }
  try {
    GPR_CUDA(cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking));
  } catch (const StatusFail& f) {
    if (S->stream) cudaStreamDestroy(S->stream);
    delete S;
    set_error("serve_create: %s", f.msg.c_str());
    return f.st;
  } catch (const CudaFail& f) {
    cudaGetLastError();
    if (S->stream) cudaStreamDestroy(S->stream);
    delete S;
    set_error("serve_create: %s failed: %s", f.what, cudaGetErrorString(f.err));
    return GPR_ECUDA;
  }
  S->th = std::thread(scheduler, S);
  *out = S;
  return GPR_OK;
}

gpr_status serve_submit(gpr_server* S, const gpr_request* r, uint64_t* ticket) {
  clear_error();
  if (!S || !r || !ticket) {
    set_error("serve_submit: NULL argument");
    return GPR_EINVAL;
  }
  if (r->graph_id < 0 || r->graph_id >= (int32_t)S->pool.size()) {
    set_error("serve_submit: graph_id %d not in the pool", (int)r->graph_id);
    return GPR_EINVAL;
  }
  const gpr_graph* g = S->pool[r->graph_id];
  if (r->num_seeds < 1 || r->num_seeds > kPprCols || !r->seeds) {
    set_error("serve_submit: num_seeds %d outside [1, %d]", (int)r->num_seeds, kPprCols);
    return GPR_EINVAL;
  }
  for (int32_t k = 0; k < r->num_seeds; ++k)
    if (r->seeds[k] < 0 || r->seeds[k] >= g->n) {
      set_error("serve_submit: seed %d outside [0, %d)", (int)r->seeds[k], (int)g->n);
      return GPR_EINVAL;
    }
  if (!(r->damping > 0.f && r->damping < 1.f) || !(r->tol >= 0.0) || r->max_iters < 0 ||
      (r->dt != GPR_FP32 && r->dt != GPR_BF16 && r->dt != GPR_FP16)) {
    set_error("serve_submit: damping, tol, max_iters or dtype out of range");
    return GPR_EINVAL;
  }
  const int64_t alone = S->pool_bytes + slot_bytes(S, g, r->dt) + (int64_t)g->n * r->num_seeds * 4;
  std::lock_guard<std::mutex> lk(S->mu);
  ++S->st.submitted;
  if (alone > S->cfg.budget_bytes) {
    ++S->st.rejected_nomem;
    set_error("serve_submit: the request needs %lld bytes with the pool; the budget is %lld", (long long)alone,
              (long long)S->cfg.budget_bytes);
    return GPR_ENOMEM;
  }
  if ((int32_t)S->queue.size() >= S->cfg.max_queue) {
    ++S->st.rejected_busy;
    set_error("serve_submit: queue full");
    return GPR_EBUSY;
  }
  Req q;
  q.ticket = S->next_ticket++;
  q.graph = r->graph_id;
  q.seeds.assign(r->seeds, r->seeds + r->num_seeds);
  q.damping = r->damping;
  q.tol = r->tol;
  q.max_iters = r->max_iters;
  q.dt = r->dt;
  q.t_submit = Clock::now();
  *ticket = q.ticket;
  S->reqs.emplace(q.ticket, std::move(q));
  S->queue.push_back(*ticket);
  S->cv_work.notify_one();
  return GPR_OK;
}

gpr_status serve_poll(gpr_server* S, uint64_t ticket, int64_t timeout_us, gpr_result* out) {
  clear_error();
  if (!S || !out) {
    set_error("serve_poll: NULL argument");
    return GPR_EINVAL;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  auto ready = [&]() {
    auto it = S->reqs.find(ticket);
    return it == S->reqs.end() || it->second.state == kDone || it->second.state == kFailed;
  };
  if (timeout_us > 0) S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) {
    set_error("serve_poll: unknown ticket %llu", (unsigned long long)ticket);
    return GPR_ENOTFOUND;
  }
  Req& r = it->second;
  if (r.state != kDone && r.state != kFailed) return GPR_ENOTREADY;
  out->status = r.status;
  out->n = S->pool[r.graph]->n;
  out->num_seeds = (int32_t)r.seeds.size();
  out->iters_max = r.iters_max;
  out->latency_ms = std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count();
  out->x = r.state == kDone ? r.result : nullptr;
  return GPR_OK;
}

gpr_status serve_completed(gpr_server* S, uint64_t* tickets, int32_t cap, int64_t timeout_us, int32_t* count) {
  clear_error();
  if (!S || !tickets || cap < 1 || !count) {
    set_error("serve_completed: bad arguments");
    return GPR_EINVAL;
  }
  std::unique_lock<std::mutex> lk(S->mu);
  if (timeout_us > 0 && S->finished.empty())
    S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&]() { return !S->finished.empty(); });
  int32_t k = 0;
  while (k < cap && !S->finished.empty()) {
    tickets[k++] = S->finished.front();
    S->finished.pop_front();
  }
  *count = k;
  return GPR_OK;
}

gpr_status serve_fetch(gpr_server* S, uint64_t ticket, float* dst, int flags) {
  clear_error();
  if (!S || !dst) {
    set_error("serve_fetch: NULL argument");
    return GPR_EINVAL;
  }
  const float* src = nullptr;
  size_t bytes = 0;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) {
      set_error("serve_fetch: unknown ticket");
      return GPR_ENOTFOUND;
    }
    if (it->second.state != kDone) {
      set_error("serve_fetch: request not finished");
      return GPR_ENOTREADY;
    }
    src = it->second.result;
    bytes = (size_t)it->second.result_bytes;
  }
  cudaError_t e = cudaMemcpy(dst, src, bytes, (flags & GPR_PTR_HOST) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice);
  if (e != cudaSuccess) {
    set_error("serve_fetch: %s", cudaGetErrorString(e));
    return GPR_ECUDA;
  }
  return GPR_OK;
}

gpr_status serve_release(gpr_server* S, uint64_t ticket) {
  clear_error();
  if (!S) {
    set_error("serve_release: NULL server");
    return GPR_EINVAL;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) {
    set_error("serve_release: unknown ticket");
    return GPR_ENOTFOUND;
  }
  if (it->second.state != kDone && it->second.state != kFailed) {
    set_error("serve_release: request still queued or running");
    return GPR_ENOTREADY;
  }
  if (it->second.result) {
    dfree(it->second.result, S->stream);
    S->bytes_in_use -= it->second.result_bytes;
  }
  S->reqs.erase(it);
  S->cv_work.notify_one();
  return GPR_OK;
}

gpr_status serve_stats(gpr_server* S, gpr_server_stats* st) {
  clear_error();
  if (!S || !st) {
    set_error("serve_stats: NULL argument");
    return GPR_EINVAL;
  }
  std::lock_guard<std::mutex> lk(S->mu);
  *st = S->st;
  st->queued = (int64_t)S->queue.size();
  int64_t cols = 0;
  for (Slot* sl : S->slots) cols += sl->used;
  st->active_columns = cols;
  st->device_bytes_in_use = S->bytes_in_use;
  return GPR_OK;
}

gpr_status serve_destroy(gpr_server* S) {
  clear_error();
  if (!S) return GPR_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    S->cv_work.notify_all();
  }
  if (S->th.joinable()) S->th.join();
  cudaStreamSynchronize(S->stream);
  for (Slot* sl : S->slots) free_slot(S, sl);
  S->slots.clear();
  for (auto& kv : S->reqs)
    if (kv.second.result) dfree(kv.second.result, S->stream);
  dfree(S->d_desc, S->stream);
  dfree(S->d_items, S->stream);
  dfree(S->d_citems, S->stream);
  cudaError_t e = cudaStreamSynchronize(S->stream);
  cudaStreamDestroy(S->stream);
  delete S;
  if (e != cudaSuccess) {
    set_error("serve_destroy: %s", cudaGetErrorString(e));
    return GPR_ECUDA;
  }
  return GPR_OK;
}

}  // extern "C"
