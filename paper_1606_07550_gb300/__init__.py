"""gpr: GB300-native graph build and PageRank (Python binding).

Thin ctypes marshalling over the C-ABI library ``libgpr.so`` (declared in
``include/gpr.h``).  Every step of the computation runs in the library's CUDA
kernels; this module converts arguments only.  PyTorch supplies device memory
and streams.  There is no fallback: if the library is missing, calls raise.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_CSRC = os.path.join(_HERE, "csrc")
_OBJ = os.path.join(_HERE, "_build")
LIB_PATH = os.path.join(_HERE, "libgpr.so")

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo", "-O3", "-std=c++17",
              "-Xcompiler", "-fPIC", f"-I{os.path.join(_ROOT, 'include')}"]

# status codes (include/gpr.h)
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EBUSY, ENOTREADY, ENOTFOUND = range(8)
_NAMES = ["GPR_OK", "GPR_EINVAL", "GPR_ENOMEM", "GPR_ECUDA", "GPR_ETIMEOUT", "GPR_EBUSY", "GPR_ENOTREADY",
          "GPR_ENOTFOUND"]
FP32, BF16, FP16 = 0, 1, 2
PTR_DEVICE, PTR_HOST = 0, 1
SPMV_PULL, SPMV_BLOCKED = 0x10, 0x20
WARM_START = 0x40
_SPMV = {"auto": 0, "pull": SPMV_PULL, "blocked": SPMV_BLOCKED}


def _spmv_flag(spmv: str) -> int:
    if spmv not in _SPMV:
        raise ValueError(f"spmv must be one of {sorted(_SPMV)}, not {spmv!r}")
    return _SPMV[spmv]


def sources():
    return sorted(os.path.join(_CSRC, f) for f in os.listdir(_CSRC) if f.endswith(".cu"))


def build(verbose: bool = False) -> str:
    """Compile every CUDA source for sm_103a (in parallel) and link libgpr.so."""
    os.makedirs(_OBJ, exist_ok=True)
    srcs = sources()

    def compile_one(src):
        obj = os.path.join(_OBJ, os.path.basename(src)[:-3] + ".o")
        cmd = ["nvcc", *NVCC_FLAGS, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB_PATH + ".tmp"
    subprocess.check_call(["nvcc", "-shared", "-gencode", "arch=compute_103a,code=sm_103a", *objs, "-o", tmp,
                           "-lcudart"])
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


class GprError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_NAMES[status] if 0 <= status < len(_NAMES) else status}: {msg}")
        self.status = status


class GraphInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m_raw", ctypes.c_int64), ("m", ctypes.c_int64),
                ("n_dangling", ctypes.c_int32), ("max_in_degree", ctypes.c_int32),
                ("max_out_degree", ctypes.c_int32), ("device_bytes", ctypes.c_int64)]


class PprJob(ctypes.Structure):
    _fields_ = [("graph", ctypes.c_void_p), ("num_seeds", ctypes.c_int32), ("seeds", ctypes.c_void_p),
                ("damping", ctypes.c_void_p), ("x_out", ctypes.c_void_p), ("iters_out", ctypes.c_void_p),
                ("residual_out", ctypes.c_void_p)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("max_queue", ctypes.c_int32), ("steps_per_tick", ctypes.c_int32),
                ("edges_per_part", ctypes.c_int64), ("fail_alloc_at", ctypes.c_int32)]


class Request(ctypes.Structure):
    _fields_ = [("graph_id", ctypes.c_int32), ("num_seeds", ctypes.c_int32), ("seeds", ctypes.c_void_p),
                ("damping", ctypes.c_float), ("tol", ctypes.c_double), ("max_iters", ctypes.c_int32),
                ("dt", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("n", ctypes.c_int32), ("num_seeds", ctypes.c_int32),
                ("iters_max", ctypes.c_int32), ("latency_ms", ctypes.c_double), ("x", ctypes.c_void_p)]


class ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in ("submitted", "admitted", "completed", "failed", "rejected_busy",
                                               "rejected_nomem", "ticks", "queued", "active_columns",
                                               "device_bytes_in_use")]


class TargetStats(ctypes.Structure):
    """gpr_target_stats: counters and device times of ppr_reverse_push / ppr_target."""
    _fields_ = [("pushes", ctypes.c_int64), ("edges", ctypes.c_int64), ("rounds", ctypes.c_int32),
                ("walk_steps", ctypes.c_int64), ("push_ms", ctypes.c_double), ("walk_ms", ctypes.c_double),
                ("total_ms", ctypes.c_double)]


class TuneResult(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int32), ("sb_bits", ctypes.c_int32), ("w_bits", ctypes.c_int32),
                ("unit_edges", ctypes.c_int64), ("ms_per_step", ctypes.c_double),
                ("pull_ms_per_step", ctypes.c_double), ("candidates", ctypes.c_int32),
                ("dense_sources", ctypes.c_int32)]


class PprTuneResult(ctypes.Structure):
    _fields_ = [("classes", ctypes.c_int32), ("log2n_max", ctypes.c_int32 * 5), ("jobs", ctypes.c_int32 * 5),
                ("cluster", ctypes.c_int32 * 5), ("ms", ctypes.c_double * 5), ("ms_cluster8", ctypes.c_double * 5)]


class Stats(ctypes.Structure):
    _fields_ = [("iters_run", ctypes.c_int32), ("residual_l1", ctypes.c_double), ("mass", ctypes.c_double),
                ("dangling", ctypes.c_double), ("t_setup_ms", ctypes.c_double), ("t_iter_ms", ctypes.c_double),
                ("schedule", ctypes.c_int32)]


_lib = None
_VP = ctypes.c_void_p


def lib():
    """The loaded C-ABI library; raises if it was not built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgpr.so not built ({LIB_PATH}); run paper_1606_07550_gb300.build()")
        L = ctypes.CDLL(LIB_PATH)
        L.gpr_last_error.restype = ctypes.c_char_p
        L.graph_build.argtypes = [_VP, _VP, ctypes.c_int64, ctypes.c_int32, ctypes.c_int, _VP,
                                  ctypes.POINTER(_VP)]
        L.graph_free.argtypes = [_VP]
        L.graph_info.argtypes = [_VP, ctypes.POINTER(GraphInfo)]
        L.graph_export.argtypes = [_VP, _VP, _VP, _VP]
        L.pagerank.argtypes = [_VP, ctypes.c_double, ctypes.c_int32, ctypes.c_int, ctypes.c_int, _VP,
                               ctypes.POINTER(Stats), _VP]
        L.hits.argtypes = [_VP, ctypes.c_int32, _VP, _VP, ctypes.c_int, _VP]
        L.eigen_centrality.argtypes = [_VP, ctypes.c_int32, _VP, ctypes.c_int, _VP]
        L.graph_update.argtypes = [_VP, _VP, _VP, ctypes.c_int64, _VP, _VP, ctypes.c_int64, ctypes.c_int, _VP]
        L.graph_save.argtypes = [_VP, ctypes.c_char_p]
        L.graph_load.argtypes = [ctypes.c_char_p, _VP, ctypes.POINTER(_VP)]
        L.wcc.argtypes = [_VP, _VP, ctypes.POINTER(ctypes.c_int32), ctypes.c_int, _VP]
        L.ppr_reverse_push.argtypes = [_VP, ctypes.c_int32, ctypes.c_double, ctypes.c_double, _VP, _VP,
                                       ctypes.POINTER(TargetStats), ctypes.c_int, _VP]
        L.ppr_target.argtypes = [_VP, ctypes.c_int32, ctypes.c_double, ctypes.c_double, _VP, ctypes.c_int32,
                                 ctypes.c_int32, ctypes.c_uint64, _VP, ctypes.POINTER(TargetStats), ctypes.c_int, _VP]
        L.pagerank_tune.argtypes = [_VP, ctypes.c_int, ctypes.c_int32, ctypes.POINTER(TuneResult), _VP]
        L.ppr_batch.argtypes = [ctypes.POINTER(PprJob), ctypes.c_int32, ctypes.c_int32, ctypes.c_double,
                                ctypes.c_int, _VP]
        L.ppr_tune.argtypes = [ctypes.POINTER(PprJob), ctypes.c_int32, ctypes.c_int, ctypes.c_int32,
                               ctypes.POINTER(PprTuneResult), _VP]
        L.gpr_kernel_launches.restype = ctypes.c_int64
        L.serve_create.argtypes = [ctypes.POINTER(_VP), ctypes.c_int32, ctypes.POINTER(ServerConfig),
                                   ctypes.POINTER(_VP)]
        L.serve_submit.argtypes = [_VP, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
        L.serve_poll.argtypes = [_VP, ctypes.c_uint64, ctypes.c_int64, ctypes.POINTER(Result)]
        L.serve_fetch.argtypes = [_VP, ctypes.c_uint64, _VP, ctypes.c_int]
        L.serve_completed.argtypes = [_VP, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int32, ctypes.c_int64,
                                      ctypes.POINTER(ctypes.c_int32)]
        L.serve_release.argtypes = [_VP, ctypes.c_uint64]
        L.serve_stats.argtypes = [_VP, ctypes.POINTER(ServerStats)]
        L.serve_destroy.argtypes = [_VP]
        L.pagerank_csc_noalloc.argtypes = [_VP, _VP, _VP, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, _VP, _VP]
        L.pagerank_csc_noalloc.restype = ctypes.c_int
        for name in ("graph_build", "graph_free", "graph_info", "graph_export", "pagerank", "pagerank_tune", "hits",
                     "eigen_centrality", "wcc", "graph_save", "graph_load", "graph_update", "ppr_batch", "ppr_tune",
                     "ppr_reverse_push", "ppr_target",
                     "serve_create", "serve_submit", "serve_poll", "serve_fetch", "serve_release", "serve_stats",
                     "serve_destroy", "serve_completed"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(status: int):
    if status != OK:
        raise GprError(status, lib().gpr_last_error().decode())


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _ptr_and_flag(a):
    """(address, is_host) of a torch tensor or numpy array of int32/float32."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be contiguous")
        return a.ctypes.data, True
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr(), not a.is_cuda


class Graph:
    """A device-resident simple directed graph (owns its device memory)."""

    def __init__(self, handle: int):
        self._h = handle

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("graph already freed")
        return self._h

    def info(self) -> GraphInfo:
        inf = GraphInfo()
        _check(lib().graph_info(self.handle, ctypes.byref(inf)))
        return inf

    @property
    def n(self) -> int:
        return self.info().n

    @property
    def m(self) -> int:
        return self.info().m

    def export(self):
        """Host copies of (col_ptr, row_idx, outdeg)."""
        inf = self.info()
        cp = np.empty(inf.n + 1, np.int32)
        ri = np.empty(max(inf.m, 1), np.int32)
        od = np.empty(inf.n, np.int32)
        _check(lib().graph_export(self.handle, cp.ctypes.data, ri.ctypes.data, od.ctypes.data))
        return cp, ri[: inf.m], od

    def save(self, path: str):
        """Binary save (see graph_save in include/gpr.h)."""
        _check(lib().graph_save(self.handle, os.fsencode(path)))

    def free(self):
        if self._h:
            h, self._h = self._h, None
            _check(lib().graph_free(h))

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.graph_free(self._h)
                self._h = None
        except Exception:
            pass


def graph_build(src, dst, n: int, stream=None) -> Graph:
    """COO -> device CSC.  src/dst: int32 torch CUDA tensors, or host arrays
    (numpy or CPU tensors), which the library copies to the device."""
    if len(src) != len(dst):
        raise ValueError("src and dst differ in length")
    ps, hs = _ptr_and_flag(src)
    pd, hd = _ptr_and_flag(dst)
    if hs != hd:
        raise ValueError("src and dst must both be host or both be device arrays")
    h = _VP()
    _check(lib().graph_build(ps, pd, len(src), n, PTR_HOST if hs else PTR_DEVICE, _stream_ptr(stream),
                             ctypes.byref(h)))
    return Graph(h.value)


def graph_update(g: Graph, ins=None, dels=None, stream=None):
    """Insert the (src, dst) pairs `ins` and delete the pairs `dels` (each a
    pair of equal-length int32 arrays, CUDA tensors or host arrays; None for
    none): E' = (E minus dels) plus ins (see graph_update in include/gpr.h)."""
    def pair(p):
        if p is None or len(p[0]) == 0:
            return None, None, 0, None
        s_, d_ = p
        if len(s_) != len(d_):
            raise ValueError("src and dst differ in length")
        ps, hs = _ptr_and_flag(s_)
        pd, hd = _ptr_and_flag(d_)
        if hs != hd:
            raise ValueError("src and dst must both be host or both be device arrays")
        return ps, pd, len(s_), hs
    a, b, k1, h1 = pair(ins)
    c, d, k2, h2 = pair(dels)
    hosts = {h for h in (h1, h2) if h is not None}
    if len(hosts) > 1:
        raise ValueError("insertions and deletions must both be host or both be device arrays")
    host = hosts.pop() if hosts else False
    _check(lib().graph_update(g.handle, a, b, k1, c, d, k2, PTR_HOST if host else PTR_DEVICE, _stream_ptr(stream)))


def graph_load(path: str, stream=None) -> Graph:
    """A graph saved by Graph.save (see graph_load in include/gpr.h)."""
    h = _VP()
    _check(lib().graph_load(os.fsencode(path), _stream_ptr(stream), ctypes.byref(h)))
    return Graph(h.value)


def pagerank(g: Graph, out, damping: float = 0.85, iters: int = 50, dtype: int = FP32, stream=None,
             stats: bool = False, spmv: str = "auto", warm_start: bool = False):
    """Writes PageRank (n floats, by node id) into `out` (a CUDA tensor, or a
    host array / CPU tensor).  Returns a Stats if stats=True.  spmv picks the
    step's schedule: "pull", "blocked", or "auto" (the library's choice).
    warm_start: start from the vector `out` holds instead of uniform."""
    po, host = _ptr_and_flag(out)
    st = Stats() if stats else None
    flags = (PTR_HOST if host else PTR_DEVICE) | _spmv_flag(spmv) | (WARM_START if warm_start else 0)
    _check(lib().pagerank(g.handle, damping, iters, dtype, flags, po,
                          ctypes.byref(st) if st is not None else None, _stream_ptr(stream)))
    return st


def hits(g: Graph, hub_out, auth_out, iters: int = 50, stream=None, spmv: str = "auto"):
    """HITS hubs and authorities (unit L2 norm, by node id) into two CUDA
    tensors, or host arrays / CPU tensors.  spmv: "auto", "pull" or "blocked"."""
    sp = _spmv_flag(spmv)
    ph, host = _ptr_and_flag(hub_out)
    pa, host2 = _ptr_and_flag(auth_out)
    if host != host2:
        raise ValueError("hub_out and auth_out must both be on the device or both on the host")
    _check(lib().hits(g.handle, iters, ph, pa, (PTR_HOST if host else PTR_DEVICE) | sp, _stream_ptr(stream)))


def eigen_centrality(g: Graph, out, iters: int = 50, stream=None, spmv: str = "auto"):
    """Eigenvector centrality (unit L2 norm, by node id) into `out`."""
    sp = _spmv_flag(spmv)
    po, host = _ptr_and_flag(out)
    _check(lib().eigen_centrality(g.handle, iters, po, (PTR_HOST if host else PTR_DEVICE) | sp, _stream_ptr(stream)))


def wcc(g: Graph, out, stream=None) -> int:
    """Weakly connected components: out[v] (int32, by node id; CUDA tensor or
    host array) = the smallest node id of v's component.  Returns the number
    of components."""
    po, host = _ptr_and_flag(out)
    k = ctypes.c_int32(0)
    _check(lib().wcc(g.handle, po, ctypes.byref(k), PTR_HOST if host else PTR_DEVICE, _stream_ptr(stream)))
    return int(k.value)


def _dtype_name(a):
    return str(a.dtype).replace("torch.", "")


def ppr_reverse_push(g: Graph, target: int, r_max: float, p_out=None, r_out=None, damping: float = 0.85,
                     stream=None) -> "TargetStats":
    """Reverse push from `target` (section 4.3): p and r (float64, by node id)
    into CUDA tensors or host arrays, either may be None.  Returns the push's
    counters (pushes, edges, rounds, push_ms).  Q_s(target) = p(s) +
    sum_v Q_s(v) r(v) afterwards."""
    host = None
    ptrs = []
    for a in (p_out, r_out):
        if a is None:
            ptrs.append(None)
            continue
        if _dtype_name(a) != "float64":
            raise ValueError("p_out and r_out must be float64")
        pa, h = _ptr_and_flag(a)
        if host is not None and h != host:
            raise ValueError("p_out and r_out must both be on the device or both on the host")
        host = h
        ptrs.append(pa)
    st = TargetStats()
    _check(lib().ppr_reverse_push(g.handle, int(target), damping, r_max, ptrs[0], ptrs[1], ctypes.byref(st),
                                  PTR_HOST if host else PTR_DEVICE, _stream_ptr(stream)))
    return st


def ppr_target(g: Graph, target: int, sources, out, r_max: float, walks: int, seed: int = 1,
               damping: float = 0.85, stream=None) -> "TargetStats":
    """Bidirectional estimates of pi_s(target) (section 4.3) for each source:
    `sources` (int32) and `out` (float64, same length) both CUDA tensors or
    both host arrays.  Returns the call's counters and phase times."""
    if _dtype_name(sources) != "int32" or _dtype_name(out) != "float64":
        raise ValueError("sources must be int32 and out float64")
    if len(sources) != len(out):
        raise ValueError("sources and out differ in length")
    ps, h1 = _ptr_and_flag(sources)
    po, h2 = _ptr_and_flag(out)
    if h1 != h2:
        raise ValueError("sources and out must both be on the device or both on the host")
    st = TargetStats()
    _check(lib().ppr_target(g.handle, int(target), damping, r_max, ps, len(sources), int(walks),
                            int(seed) & (2 ** 64 - 1), po, ctypes.byref(st), PTR_HOST if h1 else PTR_DEVICE,
                            _stream_ptr(stream)))
    return st


def pagerank_tune(g: Graph, dtype: int = FP32, trial_steps: int = 5, stream=None) -> TuneResult:
    """Times the PageRank step's schedules on g and keeps the fastest for g
    and for graphs of its shape (see pagerank_tune in include/gpr.h)."""
    r = TuneResult()
    _check(lib().pagerank_tune(g.handle, dtype, trial_steps, ctypes.byref(r), _stream_ptr(stream)))
    return r


def _ppr_jobs(requests):
    n_req = len(requests)
    arr = (PprJob * max(n_req, 1))()
    keep = []
    results = []
    for i, (g, seeds, damping, out) in enumerate(requests):
        seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.int32))
        k = len(seeds)
        d = np.ascontiguousarray(np.broadcast_to(np.asarray(damping, dtype=np.float32), (k,)))
        it = np.zeros(k, np.int32)
        res = np.zeros(k, np.float64)
        if not out.is_cuda or not out.is_contiguous() or out.numel() != g.n * k:
            raise ValueError("out must be a contiguous CUDA tensor of n x len(seeds) floats")
        keep += [seeds, d, it, res]
        arr[i] = PprJob(g.handle, k, seeds.ctypes.data, d.ctypes.data, out.data_ptr(), it.ctypes.data,
                        res.ctypes.data)
        results.append((it, res))
    return arr, n_req, keep, results


def ppr_batch(requests, max_iters: int = 50, tol: float = 0.0, dtype: int = FP32, stream=None):
    """Personalised PageRank for many (graph, seeds) requests in one launch.

    requests: list of (graph, seeds, damping, out) with seeds an int sequence,
    damping a float or a per-seed sequence, out a CUDA float32 tensor of shape
    (n, len(seeds)) (node-major).  Returns [(iters, residual)] numpy arrays
    per request."""
    arr, n_req, keep, results = _ppr_jobs(requests)
    _check(lib().ppr_batch(arr, n_req, max_iters, tol, dtype, _stream_ptr(stream)))
    return results


def ppr_tune(requests, dtype: int = FP32, trial_steps: int = 8, stream=None):
    """Times the cluster shapes of the batched launch for each graph-size
    class of `requests` (as for ppr_batch; their outputs are overwritten) and
    keeps the fastest.  Returns one dict per class: log2n_max, jobs, cluster,
    ms, ms_cluster8."""
    arr, n_req, keep, _ = _ppr_jobs(requests)
    r = PprTuneResult()
    _check(lib().ppr_tune(arr, n_req, dtype, trial_steps, ctypes.byref(r), _stream_ptr(stream)))
    return [{"log2n_max": r.log2n_max[i], "jobs": r.jobs[i], "cluster": r.cluster[i], "ms": r.ms[i],
             "ms_cluster8": r.ms_cluster8[i]} for i in range(r.classes)]


class Server:
    """Continuous-batching personalised-PageRank server over a resident pool
    of graphs (see serve_* in include/gpr.h)."""

    def __init__(self, pool, budget_bytes: int, max_queue: int = 0, steps_per_tick: int = 0,
                 edges_per_part: int = 0, fail_alloc_at: int = 0):
        self.pool = list(pool)
        arr = (_VP * len(self.pool))(*[g.handle for g in self.pool])
        cfg = ServerConfig(budget_bytes, max_queue, steps_per_tick, edges_per_part, fail_alloc_at)
        h = _VP()
        _check(lib().serve_create(arr, len(self.pool), ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h.value

    def submit(self, graph_id: int, seeds, damping: float = 0.85, tol: float = 0.0, max_iters: int = 50,
               dtype: int = FP32) -> int:
        seeds = np.ascontiguousarray(np.asarray(seeds, dtype=np.int32))
        req = Request(graph_id, len(seeds), seeds.ctypes.data, damping, tol, max_iters, dtype)
        t = ctypes.c_uint64()
        _check(lib().serve_submit(self._h, ctypes.byref(req), ctypes.byref(t)))
        return t.value

    def poll(self, ticket: int, timeout_us: int = 0):
        """The Result once finished, or None on timeout."""
        r = Result()
        st = lib().serve_poll(self._h, ticket, timeout_us, ctypes.byref(r))
        if st == ENOTREADY:
            return None
        _check(st)
        return r

    def completed(self, timeout_us: int = 0, cap: int = 4096):
        """Tickets of requests that finished since the last call."""
        buf = (ctypes.c_uint64 * cap)()
        cnt = ctypes.c_int32()
        _check(lib().serve_completed(self._h, buf, cap, timeout_us, ctypes.byref(cnt)))
        return list(buf[: cnt.value])

    def fetch(self, ticket: int, out):
        """Copy a finished result into `out` (CUDA tensor or host array, n*k floats)."""
        po, host = _ptr_and_flag(out)
        _check(lib().serve_fetch(self._h, ticket, po, PTR_HOST if host else PTR_DEVICE))
        return out

    def release(self, ticket: int):
        _check(lib().serve_release(self._h, ticket))

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().serve_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            h, self._h = self._h, None
            _check(lib().serve_destroy(h))

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.serve_destroy(self._h)
                self._h = None
        except Exception:
            pass


def pagerank_csc_noalloc(col_ptr, row_idx, outdeg, n: int, out, damping: float = 0.85, iters: int = 50,
                         stream=None):
    """PageRank on a caller-held device CSC without any device allocation
    (int32 CUDA tensors col_ptr, row_idx, outdeg; float32 CUDA tensor out;
    row_idx holds col_ptr[n] entries).  The tensors' types and the sizes that
    n fixes are checked here, before the library reads or writes them."""
    import torch
    for name, t in (("col_ptr", col_ptr), ("row_idx", row_idx), ("outdeg", outdeg)):
        if t.dtype != torch.int32:
            raise ValueError(f"pagerank_csc_noalloc: {name} must be int32, not {t.dtype}")
    if out.dtype != torch.float32:
        raise ValueError(f"pagerank_csc_noalloc: out must be float32, not {out.dtype}")
    if n < 1:
        raise ValueError("pagerank_csc_noalloc: n must be at least 1")
    if col_ptr.numel() < n + 1 or outdeg.numel() < n or out.numel() < n:
        raise ValueError("pagerank_csc_noalloc: col_ptr needs n + 1 entries, outdeg and out n each")
    for t in (col_ptr, row_idx, outdeg, out):
        if not t.is_cuda or not t.is_contiguous():
            raise ValueError("pagerank_csc_noalloc takes contiguous CUDA tensors")
    _check(lib().pagerank_csc_noalloc(col_ptr.data_ptr(), row_idx.data_ptr(), outdeg.data_ptr(), n, damping, iters,
                                      out.data_ptr(), _stream_ptr(stream)))
