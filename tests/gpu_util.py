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


def load_rmat25_oracle():
    """The oracle's stored PageRank of the R-MAT scale-25 workload (written by
    tests/golden/make_rmat25_oracle.py): the committed summary, and the whole
    FP64 vector when its file is present and its sha256 matches (else None)."""
    import hashlib
    import json
    import os

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    js = os.path.join(root, "tests", "golden", "rmat-s25-ef32_pagerank100.json")
    if not os.path.exists(js):
        return None, None
    with open(js) as f:
        meta = json.load(f)
    path = os.path.join(root, meta["vector_file"])
    full = None
    if os.path.exists(path):
        raw = open(path, "rb").read()
        if hashlib.sha256(raw).hexdigest() == meta["vector_sha256"]:
            full = np.frombuffer(raw, np.float64)
    return meta, full


def sampled_errors(x, meta):
    """On the summary's sampled nodes: the L1 error relative to the sampled
    mass (an unbiased estimate of the full-vector L1, whose mass is 1) and
    the largest relative error."""
    nodes = np.asarray(meta["sample_nodes"], np.int64)
    ref = np.asarray(meta["sample_x"], np.float64)
    got = np.asarray(x, np.float64)[nodes]
    return float(np.abs(got - ref).sum() / ref.sum()), max_rel(got, ref)
