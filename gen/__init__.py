"""Seeded synthetic inputs shared by the oracle's tests and the GPU path's tests.

This module is the only code both sides use.  It holds none of the graph
method's arithmetic: it draws raw COO edge streams (duplicates and self-loops
left in) for the directed Erdos-Renyi G(n, m) and R-MAT models that the
paper's generator table (section 4, Table "snap_gen") lists, plus seed nodes
for personalised PageRank.  The host functions are plain C (``gen.c``); the
``*_dev`` functions are a CUDA twin (``gen_dev.cu``) that emits identical bits.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_HOST_SO = os.path.join(_HERE, "libgprgen.so")
_DEV_SO = os.path.join(_HERE, "libgprgen_dev.so")

RMAT_ABC = (0.57, 0.19, 0.19)  # d = 0.05

_i32p = ctypes.POINTER(ctypes.c_int32)


def build(device: bool = True) -> None:
    """Compile the host library with gcc and, if asked, the CUDA twin with nvcc."""
    src_c = os.path.join(_HERE, "gen.c")
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", src_c, "-o", _HOST_SO, "-lm"])
    if device:
        subprocess.check_call([
            "nvcc", "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
            "-Xcompiler", "-fPIC", "-shared", os.path.join(_HERE, "gen_dev.cu"), src_c,
            "-o", _DEV_SO,
        ])


_host = None
_dev = None


def _host_lib():
    global _host
    if _host is None:
        if not os.path.exists(_HOST_SO):
            build(device=False)
        lib = ctypes.CDLL(_HOST_SO)
        lib.gen_uniform_coo.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, _i32p, _i32p]
        lib.gen_er_gnm.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, _i32p, _i32p,
                                   ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
        lib.gen_permutation.argtypes = [ctypes.c_int32, ctypes.c_uint64, _i32p]
        lib.gen_rmat_coo.argtypes = [ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_uint64, _i32p, _i32p, _i32p]
        lib.gen_seed_nodes.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, _i32p]
        lib.gen_unit_draws.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64,
                                       ctypes.POINTER(ctypes.c_double)]
        _host = lib
    return _host


def _dev_lib():
    global _dev
    if _dev is None:
        if not os.path.exists(_DEV_SO):
            raise RuntimeError("gen: CUDA twin not built (call gen.build())")
        lib = ctypes.CDLL(_DEV_SO)
        lib.gen_uniform_coo_dev.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.gen_rmat_coo_dev.argtypes = [ctypes.c_int, ctypes.c_int32, ctypes.c_int64, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        _dev = lib
    return _dev


def _p(a: np.ndarray):
    return a.ctypes.data_as(_i32p)


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise ValueError(f"gen: {what} failed with code {rc}")


def scale_for(n: int) -> int:
    """Smallest scale with 2^scale >= n (at least 1)."""
    return max(1, int(n - 1).bit_length())


def uniform_coo(n: int, m_raw: int, seed: int):
    src = np.empty(m_raw, np.int32)
    dst = np.empty(m_raw, np.int32)
    _check(_host_lib().gen_uniform_coo(n, m_raw, seed, _p(src), _p(dst)), "uniform_coo")
    return src, dst


def er_gnm(n: int, m: int, seed: int):
    """Raw stream of directed G(n, m): draws until m distinct non-loop pairs."""
    cap = max(16, int(m * 1.5) + 1024)
    while True:
        src = np.empty(cap, np.int32)
        dst = np.empty(cap, np.int32)
        m_raw = ctypes.c_int64(0)
        rc = _host_lib().gen_er_gnm(n, m, seed, _p(src), _p(dst), cap, ctypes.byref(m_raw))
        if rc == -2:
            cap *= 2
            continue
        _check(rc, "er_gnm")
        return src[: m_raw.value].copy(), dst[: m_raw.value].copy()


def permutation(n: int, seed: int) -> np.ndarray:
    perm = np.empty(n, np.int32)
    _check(_host_lib().gen_permutation(n, seed, _p(perm)), "permutation")
    return perm


def rmat_coo(n: int, m_raw: int, seed: int, abc=RMAT_ABC, permute: bool = True, scale: int | None = None):
    """R-MAT raw COO over ids [0, n), scale = ceil(log2 n) unless given."""
    scale = scale_for(n) if scale is None else scale
    perm = permutation(n, seed) if permute else None
    src = np.empty(m_raw, np.int32)
    dst = np.empty(m_raw, np.int32)
    rc = _host_lib().gen_rmat_coo(scale, n, m_raw, abc[0], abc[1], abc[2], seed,
                                  _p(perm) if perm is not None else None, _p(src), _p(dst))
    _check(rc, "rmat_coo")
    return src, dst


def seed_nodes(n: int, count: int, seed: int) -> np.ndarray:
    out = np.empty(count, np.int32)
    _check(_host_lib().gen_seed_nodes(n, count, seed, _p(out)), "seed_nodes")
    return out


def uniform_coo_dev(n: int, m_raw: int, seed: int, src_ptr: int, dst_ptr: int, stream: int = 0) -> None:
    _check(_dev_lib().gen_uniform_coo_dev(n, m_raw, seed, src_ptr, dst_ptr, stream), "uniform_coo_dev")


def rmat_coo_dev(n: int, m_raw: int, seed: int, src_ptr: int, dst_ptr: int, perm_ptr: int | None,
                 stream: int = 0, abc=RMAT_ABC, scale: int | None = None) -> None:
    """CUDA twin of rmat_coo; perm_ptr points at permutation(n, seed) on the device (or None)."""
    scale = scale_for(n) if scale is None else scale
    rc = _dev_lib().gen_rmat_coo_dev(scale, n, m_raw, abc[0], abc[1], abc[2], seed, perm_ptr,
                                     src_ptr, dst_ptr, stream)
    _check(rc, "rmat_coo_dev")


def unit_draws(seed: int, stream: int, count: int) -> np.ndarray:
    """`count` doubles uniform on [0, 1) from stream `stream` of `seed`."""
    out = np.empty(count, np.float64)
    _check(_host_lib().gen_unit_draws(seed, stream, count, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "unit_draws")
    return out
