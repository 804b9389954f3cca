"""Helpers shared by the GPU parity tests (test code only)."""
import numpy as np

import gen


def l1(a, b):
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).sum())


def max_rel(x, ref):
    ref = np.asarray(ref, np.float64)
    x = np.asarray(x, np.float64)
    nz = ref > 0
    if not nz.any():
        return 0.0
    return float(np.max(np.abs(x[nz] - ref[nz]) / ref[nz]))


def coo_for(spec):
    if spec.kind == "er":
        return gen.er_gnm(spec.n, spec.m, spec.seed)
    if spec.kind == "uniform":
        return gen.uniform_coo(spec.n, spec.m, spec.seed)
    return gen.rmat_coo(spec.n, spec.m, spec.seed, abc=spec.abc)


def random_coo_with_dups(rng, n, m_raw, p_loop=0.05, p_dup=0.2):
    src = rng.integers(0, n, m_raw).astype(np.int32)
    dst = rng.integers(0, n, m_raw).astype(np.int32)
    k = int(m_raw * p_loop)
    if k:
        idx = rng.choice(m_raw, k, replace=False)
        dst[idx] = src[idx]
    k = int(m_raw * p_dup)
    if k and m_raw > 1:
        idx = rng.choice(m_raw, k, replace=False)
        j = rng.integers(0, m_raw, k)
        src[idx], dst[idx] = src[j], dst[j]
    return src, dst
