// Binary save and load of a built graph (section 3, Table "exp_basic": the
// paper saves and loads graphs in SNAP's binary format and times both).
//
// The file holds the graph as the library keeps it, so a load needs no sort:
//   bytes 0-7    magic "GPRCSC\0\1"
//   int32        version (1), n, id_bits, reserved (0)
//   int64        m, m_raw
//   int32[n+1]   col_ptr   (relabelled ids: in-adjacency of row p is
//   int32[m]     row_idx    row_idx[col_ptr[p] .. col_ptr[p+1]), ascending)
//   int32[n]     new2old   (relabelled node p is the caller's node new2old[p])
// little-endian, as every machine this library runs on.  Out-degrees, the
// inverse permutation and the execution plan are rebuilt on load.  A load
// checks the header, the sizes and, on the device, every array: offsets
// that start at 0, never decrease and end at m; sources in [0, n), strictly
// ascending within a row, never the row itself; new2old a permutation.
#include <cstdio>
#include <cstring>
#include <vector>

#include "gpr_internal.cuh"

namespace gpr {

namespace {

constexpr char kMagic[8] = {'G', 'P', 'R', 'C', 'S', 'C', 0, 1};
constexpr int32_t kVersion = 1;

struct Header {
  char magic[8];
  int32_t version, n, id_bits, reserved;
  int64_t m, m_raw;
};
static_assert(sizeof(Header) == 40, "file header layout");

enum : int { IOERR_OFFSETS = 1, IOERR_ROWS = 2, IOERR_PERM = 4 };

__global__ void check_offsets_kernel(const int32_t* __restrict__ col_ptr, int32_t n, int64_t m, int* __restrict__ err) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = col_ptr[p], b = col_ptr[p + 1];
    if (a > b || (p == 0 && a != 0) || (p == n - 1 && b != m)) atomicOr(err, IOERR_OFFSETS);
  }
}

// One warp per row (offsets already checked), lanes over its edges: sources
// in range, strictly ascending, no self-loop; counts out-degrees.
__global__ void check_rows_kernel(const int32_t* __restrict__ col_ptr, const int32_t* __restrict__ row_idx, int32_t n,
                                  int32_t* __restrict__ outdeg, int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = warp; p < n; p += nwarps) {
    const int32_t e0 = col_ptr[p], e1 = col_ptr[p + 1];
    bool bad = false;
    for (int32_t e = e0 + lane; e < e1; e += 32) {
      const int32_t u = row_idx[e];
      if (u < 0 || u >= n || u == (int32_t)p || (e > e0 && u <= row_idx[e - 1])) {
        bad = true;
      } else {
        atomicAdd(outdeg + u, 1);
      }
    }
    if (bad) atomicOr(err, IOERR_ROWS);
  }
}

// old2new[new2old[p]] = p; a value out of range or met twice is an error.
__global__ void invert_perm_kernel(const int32_t* __restrict__ new2old, int32_t n, int32_t* __restrict__ old2new,
                                   int* __restrict__ err) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = new2old[p];
    if (v < 0 || v >= n || atomicCAS(old2new + v, -1, (int32_t)p) != -1) atomicOr(err, IOERR_PERM);
  }
}

int grid_for_n(int64_t items) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((items + 255) / 256, (int64_t)num_sms() * 8));
}

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

}  // namespace

gpr_status save_graph(const gpr_graph* g, const char* path) {
  try {
    File fl;
    fl.f = fopen(path, "wb");
    if (!fl.f) {
      set_error("graph_save: cannot open %s for writing", path);
      return GPR_EINVAL;
    }
    Header h{};
    memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.n = g->n;
    h.id_bits = g->id_bits;
    h.m = g->m;
    h.m_raw = g->m_raw;
    std::vector<int32_t> buf;
    auto put = [&](const int32_t* dev, size_t count) {
      buf.resize(std::max<size_t>(count, 1));
      if (count) GPR_CUDA(cudaMemcpy(buf.data(), dev, count * 4, cudaMemcpyDeviceToHost));
      if (fwrite(buf.data(), 4, count, fl.f) != count) throw StatusFail{GPR_EINVAL, "graph_save: write failed"};
    };
    GPR_CUDA(cudaDeviceSynchronize());  // work queued on any stream may still be writing the graph
    if (fwrite(&h, sizeof h, 1, fl.f) != 1) throw StatusFail{GPR_EINVAL, "graph_save: write failed"};
    put(g->col_ptr, (size_t)g->n + 1);
    put(g->row_idx, (size_t)g->m);
    put(g->plan.new2old, (size_t)g->n);
    if (fclose(fl.f) != 0) {
      fl.f = nullptr;
      throw StatusFail{GPR_EINVAL, "graph_save: write failed"};
    }
    fl.f = nullptr;
    return GPR_OK;
  } catch (const StatusFail& f) {
    set_error("%s (%s)", f.msg.c_str(), path);
    return f.st;
  } catch (const CudaFail& f) {
    cudaGetLastError();
    set_error("graph_save: %s failed: %s", f.what, cudaGetErrorString(f.err));
    return GPR_ECUDA;
  }
}

gpr_status load_graph(const char* path, cudaStream_t s, gpr_graph** out) {
  gpr_graph* g = nullptr;
  int* err = nullptr;
  try {
    File fl;
    fl.f = fopen(path, "rb");
    if (!fl.f) {
      set_error("graph_load: cannot open %s", path);
      return GPR_ENOTFOUND;
    }
    Header h{};
    if (fread(&h, sizeof h, 1, fl.f) != 1 || memcmp(h.magic, kMagic, 8) != 0 || h.version != kVersion)
      throw StatusFail{GPR_EINVAL, "graph_load: not a graph file of this library"};
    if (h.n < 1 || h.n >= (1 << 30) || h.m < 0 || h.m >= ((int64_t)1 << 31) || h.m_raw < h.m || h.id_bits < 1 ||
        h.id_bits > 30 || (int64_t)1 << h.id_bits < h.n)
      throw StatusFail{GPR_EINVAL, "graph_load: header sizes out of range"};
    const int64_t want = (int64_t)sizeof h + 4 * ((int64_t)h.n + 1 + h.m + h.n);
    if (fseek(fl.f, 0, SEEK_END) != 0 || (int64_t)ftell(fl.f) != want)
      throw StatusFail{GPR_EINVAL, "graph_load: file size does not match its header"};
    fseek(fl.f, sizeof h, SEEK_SET);
    g = new gpr_graph();
    g->n = h.n;
    g->m = h.m;
    g->m_raw = h.m_raw;
    g->id_bits = h.id_bits;
    g->device = device_ordinal();
    const int32_t n = h.n;
    std::vector<int32_t> buf;
    auto get = [&](int32_t* dev, size_t count) {
      buf.resize(std::max<size_t>(count, 1));
      if (fread(buf.data(), 4, count, fl.f) != count) throw StatusFail{GPR_EINVAL, "graph_load: read failed"};
      if (count) GPR_CUDA(cudaMemcpyAsync(dev, buf.data(), count * 4, cudaMemcpyHostToDevice, s));
      GPR_CUDA(cudaStreamSynchronize(s));  // buf is reused
    };
    g->col_ptr = (int32_t*)dalloc(((size_t)n + 1) * 4, s);
    g->row_idx = (int32_t*)dalloc((size_t)std::max<int64_t>(h.m, 1) * 4, s);
    g->outdeg = (int32_t*)dalloc((size_t)n * 4, s);
    g->plan.new2old = (int32_t*)dalloc((size_t)n * 4, s);
    g->plan.old2new = (int32_t*)dalloc((size_t)n * 4, s);
    get(g->col_ptr, (size_t)n + 1);
    get(g->row_idx, (size_t)h.m);
    get(g->plan.new2old, (size_t)n);
    err = (int*)dalloc(8, s);
    GPR_CUDA(cudaMemsetAsync(err, 0, 8, s));
    GPR_CUDA(cudaMemsetAsync(g->outdeg, 0, (size_t)n * 4, s));
    GPR_CUDA(cudaMemsetAsync(g->plan.old2new, 0xFF, (size_t)n * 4, s));  // -1: not yet seen
    check_offsets_kernel<<<grid_for_n(n), 256, 0, s>>>(g->col_ptr, n, h.m, err);
    int herr = 0;
    GPR_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    if (herr) throw StatusFail{GPR_EINVAL, "graph_load: column offsets are not a CSC of m edges"};
    check_rows_kernel<<<grid_for_n(n), 256, 0, s>>>(g->col_ptr, g->row_idx, n, g->outdeg, err);
    invert_perm_kernel<<<grid_for_n(n), 256, 0, s>>>(g->plan.new2old, n, g->plan.old2new, err);
    GPR_CUDA(cudaGetLastError());
    count_launches(3);
    GPR_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    if (herr & IOERR_ROWS) throw StatusFail{GPR_EINVAL, "graph_load: a row's sources are out of range or unsorted"};
    if (herr & IOERR_PERM) throw StatusFail{GPR_EINVAL, "graph_load: new2old is not a permutation"};
    GPR_CUDA(cudaMemsetAsync(err, 0, 8, s));
    plan_build(g, s, err);
    GPR_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s));
    GPR_CUDA(cudaStreamSynchronize(s));
    dfree(err, s);
    err = nullptr;
    if (herr & DERR_TIMEOUT) throw StatusFail{GPR_ETIMEOUT, "graph_load: a device-side wait timed out"};
    *out = g;
    return GPR_OK;
  } catch (const StatusFail& f) {
    dfree(err, s);
    if (g) {
      graph_free_device(g, s);
      cudaStreamSynchronize(s);
      delete g;
    }
    set_error("%s (%s)", f.msg.c_str(), path);
    return f.st;
  } catch (const CudaFail& f) {
    cudaGetLastError();
    dfree(err, s);
    if (g) {
      graph_free_device(g, s);
      cudaStreamSynchronize(s);
      delete g;
    }
    set_error("graph_load: %s failed: %s", f.what, cudaGetErrorString(f.err));
    return GPR_ECUDA;
  }
}

}  // namespace gpr
