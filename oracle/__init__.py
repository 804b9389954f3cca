"""CPU oracle for the graph build and PageRank.  TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg may import this package; the library never does, and it shares
no code with the CUDA path.  The arithmetic lives in plain single-threaded C
(``oracle.c``, FP64); this module only marshals numpy arrays.  The definitions
and the paper passages they follow are stated in ``oracle.h``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")

_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)

DAMPING = 0.85


def build() -> None:
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                           os.path.join(_HERE, "oracle.c"), "-o", _SO, "-lm"])


_lib = None


def _L():
    global _lib
    if _lib is None:
        if not os.path.exists(_SO):
            build()
        lib = ctypes.CDLL(_SO)
        lib.oracle_build_csc.restype = ctypes.c_int64
        lib.oracle_build_csc.argtypes = [ctypes.c_int32, ctypes.c_int64, _i32p, _i32p, _i32p, _i32p, _i32p]
        lib.oracle_pagerank.restype = ctypes.c_int32
        lib.oracle_pagerank.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, ctypes.c_double, _f64p, _f64p,
                                        ctypes.c_int32, ctypes.c_double, _f64p, _f64p]
        lib.oracle_pagerank_uniform.restype = ctypes.c_int32
        lib.oracle_pagerank_uniform.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, ctypes.c_double,
                                                ctypes.c_int32, _f64p, _f64p]
        lib.oracle_ppr.restype = ctypes.c_int32
        lib.oracle_ppr.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, ctypes.c_double, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_double, _f64p]
        lib.oracle_sample_in_rows.restype = ctypes.c_int64
        lib.oracle_sample_in_rows.argtypes = [ctypes.c_int32, ctypes.c_int64, _i32p, _i32p, ctypes.c_int32,
                                              _i32p, _i64p, _i32p, ctypes.c_int64]
        lib.oracle_sample_outdeg.restype = ctypes.c_int32
        lib.oracle_sample_outdeg.argtypes = [ctypes.c_int32, ctypes.c_int64, _i32p, _i32p, ctypes.c_int32,
                                             _i32p, _i32p]
        lib.oracle_hits.restype = ctypes.c_int32
        lib.oracle_hits.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32, _f64p, _f64p]
        lib.oracle_eigen_centrality.restype = ctypes.c_int32
        lib.oracle_eigen_centrality.argtypes = [ctypes.c_int32, _i32p, _i32p, ctypes.c_int32, _f64p]
        lib.oracle_wcc.restype = ctypes.c_int32
        lib.oracle_wcc.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p]
        lib.oracle_reverse_push.restype = ctypes.c_int64
        lib.oracle_reverse_push.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, ctypes.c_int32, ctypes.c_double,
                                            ctypes.c_double, _f64p, _f64p]
        lib.oracle_ppr_contrib.restype = ctypes.c_int32
        lib.oracle_ppr_contrib.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, ctypes.c_int32, ctypes.c_double,
                                           ctypes.c_int32, _f64p]
        lib.oracle_ppr_target.restype = ctypes.c_int32
        lib.oracle_ppr_target.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, ctypes.c_int32, ctypes.c_double,
                                          ctypes.c_double, _i32p, ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64,
                                          _f64p]
        _lib = lib
    return _lib


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_i32p)


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_f64p)


class CSC:
    """In-adjacency of a simple directed graph: sources of node v are
    row_idx[col_ptr[v]:col_ptr[v+1]], ascending."""

    def __init__(self, n, col_ptr, row_idx, outdeg):
        self.n = int(n)
        self.col_ptr = col_ptr
        self.row_idx = row_idx
        self.outdeg = outdeg

    @property
    def m(self) -> int:
        return int(self.col_ptr[-1])


def build_csc(n: int, src, dst) -> CSC:
    src, ps = _i32(src)
    dst, pd = _i32(dst)
    m_raw = len(src)
    col_ptr = np.empty(n + 1, np.int32)
    row_idx = np.empty(max(m_raw, 1), np.int32)
    outdeg = np.empty(n, np.int32)
    m = _L().oracle_build_csc(n, m_raw, ps, pd, col_ptr.ctypes.data_as(_i32p), row_idx.ctypes.data_as(_i32p),
                              outdeg.ctypes.data_as(_i32p))
    if m < 0:
        raise ValueError(f"oracle_build_csc: invalid input ({m})")
    return CSC(n, col_ptr, row_idx[:m].copy(), outdeg)


def _csc_ptrs(g: CSC):
    cp, pcp = _i32(g.col_ptr)
    ri, pri = _i32(g.row_idx if len(g.row_idx) else np.zeros(1, np.int32))
    od, pod = _i32(g.outdeg)
    return (cp, ri, od), (pcp, pri, pod)


def pagerank(g: CSC, d: float = DAMPING, iters: int = 50, t=None, x0=None, tol: float = 0.0,
             with_resid: bool = False):
    """Power iteration; t and x0 default to the uniform 1/N vector.
    Returns x (and the per-step L1 change and the step count if with_resid)."""
    n = g.n
    keep, ptrs = _csc_ptrs(g)
    if t is None:
        t = np.full(n, 1.0 / n)
    if x0 is None:
        x0 = t
    t, pt = _f64(t)
    x0, px = _f64(x0)
    x = np.empty(n, np.float64)
    resid = np.zeros(max(iters, 1), np.float64)
    k = _L().oracle_pagerank(n, *ptrs, d, pt, px, iters, tol, x.ctypes.data_as(_f64p),
                             resid.ctypes.data_as(_f64p))
    if k < 0:
        raise ValueError("oracle_pagerank: invalid arguments")
    if with_resid:
        return x, resid[:k], k
    return x


def pagerank_uniform(g: CSC, d: float = DAMPING, iters: int = 50):
    keep, ptrs = _csc_ptrs(g)
    x = np.empty(g.n, np.float64)
    k = _L().oracle_pagerank_uniform(g.n, *ptrs, d, iters, x.ctypes.data_as(_f64p), None)
    if k < 0:
        raise ValueError("oracle_pagerank_uniform: invalid arguments")
    return x


def ppr(g: CSC, seed: int, d: float = DAMPING, max_iters: int = 50, tol: float = 0.0):
    """Personalised PageRank of one seed; returns (x, steps run)."""
    keep, ptrs = _csc_ptrs(g)
    x = np.empty(g.n, np.float64)
    k = _L().oracle_ppr(g.n, *ptrs, d, int(seed), max_iters, tol, x.ctypes.data_as(_f64p))
    if k < 0:
        raise ValueError("oracle_ppr: invalid arguments")
    return x, k


def sample_in_rows(n: int, src, dst, rows):
    """Sorted distinct non-loop sources of each listed destination, from the raw COO."""
    src, ps = _i32(src)
    dst, pd = _i32(dst)
    rows, pr = _i32(rows)
    k = len(rows)
    off = np.zeros(k + 1, np.int64)
    cap = 1 << 16
    while True:
        out = np.empty(cap, np.int32)
        tot = _L().oracle_sample_in_rows(n, len(src), ps, pd, k, pr, off.ctypes.data_as(_i64p),
                                         out.ctypes.data_as(_i32p), cap)
        if tot == -2:
            cap *= 4
            continue
        if tot < 0:
            raise ValueError("oracle_sample_in_rows: invalid arguments")
        return [out[off[j]:off[j + 1]].copy() for j in range(k)]


def sample_outdeg(n: int, src, dst, nodes):
    src, ps = _i32(src)
    dst, pd = _i32(dst)
    nodes, pn = _i32(nodes)
    out = np.empty(len(nodes), np.int32)
    rc = _L().oracle_sample_outdeg(n, len(src), ps, pd, len(nodes), pn, out.ctypes.data_as(_i32p))
    if rc != 0:
        raise ValueError("oracle_sample_outdeg failed")
    return out


def hits(g: CSC, iters: int = 50):
    """HITS hubs and authorities after `iters` steps, each L2-normalised
    (oracle_hits in oracle/oracle.h).  Returns (hub, auth)."""
    keep, ptrs = _csc_ptrs(g)
    hub = np.empty(g.n, np.float64)
    auth = np.empty(g.n, np.float64)
    if _L().oracle_hits(g.n, ptrs[0], ptrs[1], iters, hub.ctypes.data_as(_f64p), auth.ctypes.data_as(_f64p)) < 0:
        raise ValueError("oracle_hits: invalid arguments")
    return hub, auth


def eigen_centrality(g: CSC, iters: int = 50):
    """Eigenvector centrality after `iters` power steps on A^T, L2-normalised
    (oracle_eigen_centrality in oracle/oracle.h)."""
    keep, ptrs = _csc_ptrs(g)
    x = np.empty(g.n, np.float64)
    if _L().oracle_eigen_centrality(g.n, ptrs[0], ptrs[1], iters, x.ctypes.data_as(_f64p)) < 0:
        raise ValueError("oracle_eigen_centrality: invalid arguments")
    return x


def wcc(g: CSC):
    """Weakly connected components: (labels, count), labels[v] = the smallest
    node id of v's component (oracle_wcc in oracle/oracle.h)."""
    keep, ptrs = _csc_ptrs(g)
    labels = np.empty(g.n, np.int32)
    k = _L().oracle_wcc(g.n, ptrs[0], ptrs[1], labels.ctypes.data_as(_i32p))
    if k < 0:
        raise ValueError("oracle_wcc: invalid arguments")
    return labels, int(k)


def reverse_push(g: CSC, target: int, d: float = DAMPING, r_max: float = 1e-4):
    """Reverse push from `target` (oracle_reverse_push): (p, r, pushes)."""
    keep, ptrs = _csc_ptrs(g)
    p = np.empty(g.n, np.float64)
    r = np.empty(g.n, np.float64)
    k = _L().oracle_reverse_push(g.n, *ptrs, target, d, r_max, p.ctypes.data_as(_f64p), r.ctypes.data_as(_f64p))
    if k < 0:
        raise ValueError("oracle_reverse_push: invalid arguments")
    return p, r, int(k)


def ppr_contrib(g: CSC, target: int, d: float = DAMPING, iters: int = 250):
    """q(s) = Q_s(target) for every s: the absorbing walk's chance to stop at target."""
    keep, ptrs = _csc_ptrs(g)
    q = np.empty(g.n, np.float64)
    if _L().oracle_ppr_contrib(g.n, *ptrs, target, d, iters, q.ctypes.data_as(_f64p)) < 0:
        raise ValueError("oracle_ppr_contrib: invalid arguments")
    return q


def ppr_target(g: CSC, target: int, sources, d: float = DAMPING, r_max: float = 1e-4, walks: int = 1000,
               seed: int = 1):
    """Bidirectional estimates of pi_s(target) for each source (oracle_ppr_target)."""
    keep, ptrs = _csc_ptrs(g)
    src, ps = _i32(sources)
    out = np.empty(len(src), np.float64)
    if _L().oracle_ppr_target(g.n, *ptrs, target, d, r_max, ps, len(src), walks, seed,
                              out.ctypes.data_as(_f64p)) < 0:
        raise ValueError("oracle_ppr_target: invalid arguments")
    return out
